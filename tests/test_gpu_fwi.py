"""Reduced FWI (Eqs. PDEsolve, FWI and FWI2) through libwri against the FWI oracle.

The general right-hand side of the solve (wri_group.q, lambda = 0) is checked against a sparse LU
solve of A u = q; the whole evaluation (forward solves, weights and adjoint sources, adjoint solves,
gradient) against ``oracle.fwi_evaluate``, which is pinned by central differences and by the
lambda -> 0 limit of the WRI oracle.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
import synth
from wri_cases import rel, seen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_18429_gb300 import fwi, wri
    return wri, fwi


def _case(nphys=(12, 10, 8), seed=4, nsys=2):
    G = synth.workload_small(nphys=nphys, npml=3, h=10.0, freq=14.0, nsys=nsys, seed=seed, nrec=6)
    d = O.forward_data(G.spec.shape, G.spec.h, G.omega, G.m * 1.05, G.spec.npml, G.v_max, G.src, G.rec_off,
                       G.rec_idx, G.alpha)
    r = synth.rng(seed + 3)
    G.d = d * (1 + 0.05 * (r.standard_normal(d.shape) + 1j * r.standard_normal(d.shape)))
    return G


# An FP32 solve of A u = q cannot beat a forward error of about kappa(A) * 2^-24: on the 20 x 16 x 14
# grid of these cases kappa(A) = 3.1e3 (power iterations on A^H A and on its inverse through the LU
# factors), i.e. 1.9e-4, and a CGLS with complex64 operator products and FP64 scalars, run to the same
# 1e-6 on the CPU, ends 0.9e-4 and 1.6e-4 from the LU solution.  The FP32 bounds below are about five
# times kappa(A) * 2^-24 for the wavefield; the FWI quantities of that emulation end 2.2e-4 (f),
# 4.5e-5 (weights) and 9.5e-4 (gradient, a product of two such fields) from the oracle.
C64_U_TOL = 1e-3


@pytest.mark.parametrize("dtype,kernel,tol", [(1, 0, 1e-9), (0, 0, C64_U_TOL), (0, 1, C64_U_TOL)])
def test_general_right_hand_side_solves_the_pde(W, dtype, kernel, tol):
    """lambda = 0 and b1 = q: the solve is min ||A u - q||, i.e. A u = q (complex128 and complex64,
    TMA phases (the x extent, 20, is a multiple of 4) and z-march kernels).  Complex64: to the
    accuracy of an FP32 solve (C64_U_TOL)."""
    wri, _ = W
    from paper_2410_18429_gb300.problem import to_device
    G = _case(nphys=(14, 10, 8))
    m, _, _ = seen(G, dtype == 0)
    A = O.helmholtz_matrix(G.spec.shape, G.spec.h, G.omega, m, G.spec.npml, G.v_max, G.pml_R)
    q = synth.random_complex((G.nsys, G.spec.n), 9) * 1e-3
    if dtype == 0:
        q = q.astype(np.complex64).astype(np.complex128)
    spec = to_device(G, dtype, "cuda")
    spec.lam = 0.0
    spec.q = torch.as_tensor(q, dtype=spec.u.dtype).cuda()
    it, rr, st = wri.solve([spec], wri.make_opts(tol=1e-12 if dtype == 1 else 1e-6, max_iter=400000, dtype=dtype,
                                                 kernel=kernel))
    assert st.cpu().tolist() == [wri.SYS_OK] * G.nsys
    lu = spla.splu(A.tocsc())
    u = spec.u.cpu().numpy()
    for s in range(G.nsys):
        assert rel(u[s], lu.solve(q[s])) < tol, rel(u[s], lu.solve(q[s]))


@pytest.mark.parametrize("source_free", [True, False])
def test_fwi_evaluation_matches_oracle_c128(W, source_free):
    wri, fwi = W
    from paper_2410_18429_gb300.problem import to_device
    G = _case()
    spec = to_device(G, wri.C128, "cuda")
    alpha = None if source_free else torch.as_tensor(G.alpha).cuda()
    stats = {}
    f, g, a = fwi.evaluate([spec], wri.make_opts(tol=1e-12, max_iter=400000, dtype=wri.C128), alpha=alpha,
                           stats=stats)
    assert stats["forward_status"].cpu().tolist() == [wri.SYS_OK] * G.nsys
    assert stats["adjoint_status"].cpu().tolist() == [wri.SYS_OK] * G.nsys
    _, a_ex, f_ex, g_ex = O.fwi_evaluate(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.src,
                                         G.rec_off, G.rec_idx, G.d, None if source_free else G.alpha, G.pml_R)
    assert abs(f.item() - f_ex) <= 1e-8 * f_ex
    assert rel(a.cpu().numpy(), a_ex) < 1e-8
    assert rel(g[0].cpu().numpy().ravel(), g_ex) < 1e-6


def test_fwi_evaluation_c64(W):
    """Complex64 solves (FP32 stencils, FP64 reductions) to 1e-6: f, weights and gradient of the
    oracle on the float32 model and complex64 data to the accuracy of an FP32 solve (the bounds
    are about twice and five times the errors of the FP32 emulation described at C64_U_TOL)."""
    wri, fwi = W
    from paper_2410_18429_gb300.problem import to_device
    G = _case(nphys=(14, 10, 8))
    m, d, _ = seen(G, True)
    spec = to_device(G, wri.C64, "cuda")
    f, g, a = fwi.evaluate([spec], wri.make_opts(tol=1e-6, max_iter=400000, dtype=wri.C64))
    _, a_ex, f_ex, g_ex = O.fwi_evaluate(G.spec.shape, G.spec.h, G.omega, m, G.spec.npml, G.v_max, G.src,
                                         G.rec_off, G.rec_idx, d, None, G.pml_R)
    assert abs(f.item() - f_ex) <= 1e-3 * f_ex
    assert rel(a.cpu().numpy(), a_ex) < 5e-4
    assert rel(g[0].cpu().numpy().ravel(), g_ex) < 5e-3
