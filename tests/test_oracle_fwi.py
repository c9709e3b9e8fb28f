"""Pins of the reduced-FWI oracle (Eqs. PDEsolve and FWI2), the paper's comparison method.

``fwi_evaluate`` (forward LU solve, closed-form weight, adjoint LU solve) is pinned by
  * central finite differences of its f in m (exact solves), both modes;
  * the lambda -> 0 limit of the independent WRI oracle: f_WRI(lambda) / lambda^2 -> f_FWI and
    g_WRI(lambda) / lambda^2 -> g_FWI, with an error that falls like lambda^2;
  * the data-consistency invariant: noise-free data of the true model give f = 0, g = 0 and, source
    free, the true weight.
"""
import numpy as np
import pytest

import oracle as O
import synth


def _case(seed=4, nsys=2):
    G = synth.workload_small(nphys=(7, 6, 5), npml=3, h=10.0, freq=14.0, nsys=nsys, seed=seed, nrec=5)
    d = O.forward_data(G.spec.shape, G.spec.h, G.omega, G.m * 1.05, G.spec.npml, G.v_max, G.src, G.rec_off,
                       G.rec_idx, G.alpha)
    r = synth.rng(seed + 3)
    G.d = d * (1 + 0.05 * (r.standard_normal(d.shape) + 1j * r.standard_normal(d.shape)))
    return G


def _fwi(G, m, source_free):
    return O.fwi_evaluate(G.spec.shape, G.spec.h, G.omega, m, G.spec.npml, G.v_max, G.src, G.rec_off, G.rec_idx,
                          G.d, None if source_free else G.alpha, G.pml_R)


@pytest.mark.parametrize("source_free", [True, False])
def test_fwi_gradient_matches_central_differences(source_free):
    G = _case()
    m = G.m
    _, _, f0, g = _fwi(G, m, source_free)
    assert f0 > 0
    r = synth.rng(8)
    for _ in range(3):
        dm = r.standard_normal(m.shape) * m
        eps = 1e-6
        fp = _fwi(G, m + eps * dm, source_free)[2]
        fm = _fwi(G, m - eps * dm, source_free)[2]
        fd = (fp - fm) / (2 * eps)
        an = float(np.sum(g * dm.ravel()))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


@pytest.mark.parametrize("source_free", [True, False])
def test_fwi_is_the_small_lambda_limit_of_wri(source_free):
    G = _case()
    _, a_f, f_f, g_f = _fwi(G, G.m, source_free)
    errs = []
    for lam in (1e-3, 1e-4):
        _, a_w, f_w, g_w = O.evaluate(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.src, G.rec_off,
                                      G.rec_idx, G.d, lam, None if source_free else G.alpha, source_free)
        errs.append((abs(f_w / lam ** 2 - f_f) / f_f, np.linalg.norm(g_w / lam ** 2 - g_f) / np.linalg.norm(g_f),
                     np.linalg.norm(a_w - a_f) / np.linalg.norm(a_f)))
    (ef1, eg1, ea1), (ef2, eg2, ea2) = errs
    assert ef2 < 1e-4 and eg2 < 1e-4 and ea2 < 1e-4, errs
    for e1, e2 in ((ef1, ef2), (eg1, eg2)):
        assert 50 < e1 / e2 < 200, errs      # O(lambda^2)


def test_fwi_data_consistency():
    G = synth.workload_small(nphys=(7, 6, 5), npml=3, h=10.0, freq=14.0, nsys=2, seed=6, nrec=5)
    G.d = O.forward_data(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.src, G.rec_off, G.rec_idx,
                         G.alpha)
    for source_free in (True, False):
        _, a, f, g = _fwi(G, G.m, source_free)
        g_off = _fwi(G, G.m * 1.02, source_free)[3]       # the scale of a gradient away from the truth
        assert f <= 1e-24 * np.vdot(G.d, G.d).real
        assert np.linalg.norm(g) <= 1e-9 * np.linalg.norm(g_off)
        assert np.allclose(a, G.alpha, rtol=1e-10)
