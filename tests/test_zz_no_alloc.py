"""wri_gradient_noalloc: the allocation-free gradient entry point.

Some callers cannot call cudaMalloc (their device memory belongs to another
allocator, or they run in a loop that must not synchronise the device to allocate).
This entry point serves them with a static device scratch array instead of a
caller workspace.  It must give the same gradient and objective as wri_gradient,
also on consecutive calls that reuse the same static array for different problems.
"""
import numpy as np
import pytest

import synth
from wri_cases import case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_18429_gb300 import wri
    return wri


def _problem(W, dtype, nphys, nsys, seed):
    from paper_2410_18429_gb300.problem import to_device
    G = case(nphys=nphys, npml=3, nsys=nsys, seed=seed)
    u = synth.random_complex((nsys, G.spec.n), seed + 1) * 1e-3
    spec = to_device(G, dtype, "cuda", u=u)
    alpha = torch.as_tensor(synth.random_complex(nsys, seed + 2)).cuda()
    return spec, alpha


def _both(W, dtype, specs, alpha):
    g_ref, f_ref = W.gradient(specs, dtype, alpha)
    grads = [torch.zeros_like(g) for g in g_ref]
    f = torch.zeros_like(f_ref)
    W.gradient_noalloc(specs, dtype, alpha, grads, f)
    torch.cuda.synchronize()
    return g_ref, f_ref, grads, f


@pytest.mark.parametrize("dtype,tol", [(1, 1e-12), (0, 1e-6)])
def test_noalloc_gradient_matches_workspace_gradient_twice(W, dtype, tol):
    # first call: two groups, five systems
    s1, a1 = _problem(W, dtype, (21, 13, 11), 3, 31)
    s2, a2 = _problem(W, dtype, (14, 17, 9), 2, 41)
    g_ref, f_ref, g, f = _both(W, dtype, [s1, s2], torch.cat([a1, a2]))
    for x, y in zip(g, g_ref):
        assert rel(x.cpu().numpy(), y.cpu().numpy()) < tol
    assert abs(f.item() - f_ref.item()) <= tol * abs(f_ref.item()) * 10
    # second call in a row: a different, smaller problem over the same static scratch
    s3, a3 = _problem(W, dtype, (12, 10, 8), 1, 51)
    g_ref, f_ref, g, f = _both(W, dtype, [s3], a3)
    assert rel(g[0].cpu().numpy(), g_ref[0].cpu().numpy()) < tol
    assert abs(f.item() - f_ref.item()) <= tol * abs(f_ref.item()) * 10


def test_noalloc_rejects_problems_beyond_its_scratch(W):
    s1, a1 = _problem(W, 0, (40, 40, 30), 1, 61)
    n = s1.n
    per = 30000
    nsys = (W.NOALLOC_SCRATCH_BYTES // (4 * per)) + 2
    s1.src = np.full(nsys, s1.src[0], dtype=np.int64)
    s1.rec_off = (np.arange(nsys + 1) * per).astype(np.int32)
    s1.rec_idx = np.tile(np.arange(per, dtype=np.int32) * (n // per), nsys)
    s1.d = torch.zeros(nsys * per, dtype=torch.complex64, device="cuda")
    s1.u = torch.zeros(nsys, n, dtype=torch.complex64, device="cuda")
    grads = [torch.zeros(s1.nz, s1.ny, s1.nx, dtype=torch.float64, device="cuda")]
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    alpha = torch.zeros(nsys, dtype=torch.complex128, device="cuda")
    with pytest.raises(W.WriError) as e:
        W.gradient_noalloc([s1], 0, alpha, grads, f)
    assert e.value.code == W.ESCRATCH
    assert float(grads[0].abs().max()) == 0.0
