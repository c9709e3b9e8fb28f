"""The reduced objective f4(m) as a torch.autograd.Function (Eqs. VarObj2 / VarG2).

Checks, through libwri's C ABI: the backward gradient against central finite differences
of the forward objective, f and g against the oracle's exact evaluation (complex128 and
complex64 with FP64 refinement), chunked evaluation (wavefields recomputed chunk by chunk)
against one resident batch, and the recompute mode against the stored-gradient mode.
"""
import numpy as np
import pytest

import oracle as O
import synth
from wri_cases import case, rel, seen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_18429_gb300 import objective, wri
    return wri, objective


def _groups(W, G, dtype, source_free=True):
    from paper_2410_18429_gb300.problem import to_device
    return [to_device(G, dtype, "cuda", source_free=source_free)]


def _m(G, dtype):
    t = torch.float64 if dtype == 1 else torch.float32
    return torch.as_tensor(G.m.reshape(G.spec.shape), dtype=t).cuda()


@pytest.mark.parametrize("source_free", [True, False])
def test_backward_matches_central_differences(W, source_free):
    """<g, dm> equals (f(m + eps dm) - f(m - eps dm)) / (2 eps) on three random directions."""
    wri, obj = W
    G = case(nphys=(13, 11, 9), npml=3, nsys=2, freq=14.0)
    groups = _groups(W, G, 1, source_free)
    opts = wri.make_opts(tol=1e-11, max_iter=400000, dtype=1)
    m = _m(G, 1).requires_grad_(True)
    f = obj.objective(m, groups, opts)
    f.backward()
    g = m.grad.clone()
    r = synth.rng(17)
    for _ in range(3):
        dm = torch.as_tensor(r.standard_normal(G.spec.shape) * G.m.reshape(G.spec.shape)).cuda()
        eps = 1e-4
        with torch.no_grad():
            fp = obj.objective(m + eps * dm, groups, opts).item()
            fm = obj.objective(m - eps * dm, groups, opts).item()
        fd = (fp - fm) / (2 * eps)
        an = float((g * dm).sum())
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_objective_and_gradient_match_oracle_c128(W):
    wri, obj = W
    G = case(nphys=(17, 12, 10), npml=3, nsys=3, freq=13.0)
    groups = _groups(W, G, 1)
    m = _m(G, 1).requires_grad_(True)
    stats = {}
    f = obj.objective(m, groups, wri.make_opts(tol=1e-11, max_iter=400000, dtype=1), stats=stats)
    f.backward()
    assert stats["status"].cpu().tolist() == [wri.SYS_OK] * 3
    _, _, f_ex, g_ex = O.evaluate(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.src, G.rec_off,
                                  G.rec_idx, G.d, G.lam)
    assert abs(f.item() - f_ex) <= 1e-9 * abs(f_ex)
    assert rel(m.grad.cpu().numpy().ravel(), g_ex) < 1e-7


def test_objective_and_gradient_match_oracle_c64_refined(W):
    """complex64 stencils with FP64 augmented-system refinement: wavefield-derived f and g
    within the target tolerances (gradient rel-L2 <= 1e-4) of the FP64 oracle fed the same
    float32 model and complex64 data."""
    wri, obj = W
    G = case(nphys=(17, 12, 10), npml=3, nsys=3, freq=13.0)
    m32, d32, _ = seen(G, True)
    groups = _groups(W, G, 0)
    m = _m(G, 0).requires_grad_(True)
    stats = {}
    opts = wri.make_opts(tol=1e-3, max_iter=400000, dtype=0, max_refine=20, refine_tol=1e-10, inner_tol=1e-3)
    f = obj.objective(m, groups, opts, stats=stats)
    f.backward()
    assert stats["status"].cpu().tolist() == [wri.SYS_OK] * 3
    _, _, f_ex, g_ex = O.evaluate(G.spec.shape, G.spec.h, G.omega, m32, G.spec.npml, G.v_max, G.src, G.rec_off,
                                  G.rec_idx, d32, G.lam)
    assert abs(f.item() - f_ex) <= 1e-5 * abs(f_ex)
    assert rel(m.grad.double().cpu().numpy().ravel(), g_ex) < 1e-4


def test_chunked_and_recomputed_evaluations_agree(W):
    """One system resident at a time (wavefields recomputed per chunk) gives the f and g of
    the whole batch resident; recompute mode gives the g of the stored-gradient mode."""
    wri, obj = W
    G = case(nphys=(15, 12, 9), npml=3, nsys=4, freq=12.0)
    groups = _groups(W, G, 1)
    opts = wri.make_opts(tol=1e-9, max_iter=400000, dtype=1)
    res = []
    for kw in (dict(), dict(max_resident=1), dict(max_resident=3, recompute=True)):
        m = _m(G, 1).requires_grad_(True)
        f = obj.objective(m, groups, opts, **kw)
        f.backward()
        res.append((f.item(), m.grad.cpu().numpy()))
    for f, g in res[1:]:
        assert abs(f - res[0][0]) <= 1e-12 * abs(res[0][0])
        assert rel(g, res[0][1]) < 1e-12


def _smooth_direction(shape, seed, sigma=2.0):
    """Unit-norm Gaussian perturbation smoothed over about sigma cells (seeded)."""
    from scipy.ndimage import gaussian_filter
    r = synth.rng(seed)
    v = gaussian_filter(r.standard_normal(shape), sigma)
    return v / np.linalg.norm(v)


def test_mixed_precision_objective_fd_and_oracle_with_recompute(W):
    """The differentiation pattern at reduced size: complex64 stencils with FP64 refinement,
    two systems resident at a time, wavefields recomputed in the backward pass.  The gradient
    matches central differences of f on smooth random perturbations (eps = 1e-3 relative)
    and the FP64 oracle's gradient to 1e-4."""
    wri, obj = W
    G = case(nphys=(18, 16, 14), npml=4, nsys=4, freq=10.0, nrec=9)
    m32, d32, _ = seen(G, True)
    groups = _groups(W, G, 0)
    opts = wri.make_opts(tol=1e-3, max_iter=400000, dtype=0, max_refine=20, refine_tol=1e-9, inner_tol=1e-2)
    m = _m(G, 0).double().requires_grad_(True)
    f = obj.objective(m, groups, opts, max_resident=2, recompute=True)
    f.backward()
    g = m.grad.clone()
    _, _, f_ex, g_ex = O.evaluate(G.spec.shape, G.spec.h, G.omega, m32, G.spec.npml, G.v_max, G.src, G.rec_off,
                                  G.rec_idx, d32, G.lam)
    assert abs(f.item() - f_ex) <= 1e-6 * abs(f_ex)
    assert rel(g.cpu().numpy().ravel(), g_ex) < 1e-4
    mm = m.detach()
    for k in range(3):
        dm = torch.as_tensor(_smooth_direction(G.spec.shape, 30 + k)).cuda()
        eps = 1e-3 * float(mm.norm())
        with torch.no_grad():
            fp = obj.objective(mm + eps * dm, groups, opts, max_resident=2).item()
            fm = obj.objective(mm - eps * dm, groups, opts, max_resident=2).item()
        fd = (fp - fm) / (2 * eps)
        an = float((g * dm).sum())
        assert abs(fd - an) <= 1e-3 * abs(an) + 1e-6 * abs(f_ex) / eps, (k, fd, an)
