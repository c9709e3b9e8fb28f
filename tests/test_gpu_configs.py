"""The stated workload configurations, at their stated sizes, through libwri against the oracle.

Configuration 1 (plain SF-AWRI, one solve + gradient): 24^3 physical nodes + 6-cell layer (36^3),
h = 10 m, homogeneous 2000 m/s inversion model, 5 Hz, one source at (12, 12, 2), 20 receivers at
x = y = 18, z = 2..21, lambda = 10, complex128, tolerance 1e-8.  The observed data come from an
exact forward solve (sparse LU) on the true model, a +10 % Gaussian anomaly of sigma 3 cells, with
the true weight -10 (the 5 Hz weight of Table SrcCam).  The oracle's exact (LU) evaluation of the
same problem is the reference: wavefield within 1e-5 and gradient within 1e-4 (relative L2).
"""
import numpy as np
import pytest

import oracle as O
import synth
from wri_cases import rel

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


def test_config1_solve_and_gradient_match_exact(W):
    from paper_2410_18429_gb300.problem import to_device
    G = synth.workload_c1()
    shp, h, npml = G.spec.shape, G.spec.h, G.spec.npml
    m_true = synth.to_m(synth.workload_c1_true_velocity())
    G.d = O.forward_data(shp, h, G.omega, m_true, npml, G.v_max, G.src, G.rec_off, G.rec_idx, G.alpha)
    spec = to_device(G, W.C128, "cuda")
    tol = 1e-8
    it, rr, st = W.solve([spec], W.make_opts(tol=tol, max_iter=500000, dtype=W.C128))
    assert st.cpu().tolist() == [W.SYS_OK]
    assert 0 < float(rr[0]) <= tol
    a = W.source_estimate([spec], W.C128)
    g, f = W.gradient([spec], W.C128, a)
    u_ex, a_ex, f_ex, g_ex = O.evaluate(shp, h, G.omega, G.m, npml, G.v_max, G.src, G.rec_off, G.rec_idx,
                                        G.d, G.lam)
    err_u = rel(spec.u.cpu().numpy(), u_ex)
    err_g = rel(g[0].cpu().numpy().ravel(), g_ex)
    assert err_u < 1e-5, err_u
    assert rel(a.cpu().numpy(), a_ex) < 1e-5
    assert err_g < 1e-4, err_g
    assert abs(f.item() - f_ex) <= 1e-4 * abs(f_ex)
    # the homogeneous model is not the true one: the data misfit and the gradient are not zero
    assert f_ex > 0 and np.linalg.norm(g_ex) > 0
