"""Pins of the C++/OpenMP oracle CGLS (oracle/cpu_cgls.cpp), the timed CPU baseline.

It restates the operator and CGLS as plain loops (A^H by its definition, the conjugated
coefficient of each node in its neighbours' rows), so it is pinned against the numpy oracle,
whose operator and CGLS are pinned in test_oracle_pins.py: the same iterates to rounding, in
both modes, on a grid with the absorbing layer and a ragged shape, with 1 and several threads.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import cpu_cgls


def _case(nphys=(9, 7, 6), npml=3, nsys=2, seed=4):
    G = synth.workload_small(nphys=nphys, npml=npml, h=10.0, freq=14.0, nsys=nsys, seed=seed, nrec=5)
    r = synth.rng(seed + 7)
    nnz = int(G.rec_off[-1])
    G.d = (r.standard_normal(nnz) + 1j * r.standard_normal(nnz)) * 1e-3
    return G


def _oracle_S_b(G, s, source_free):
    A = O.helmholtz_matrix(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.pml_R)
    rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
    S = O.augmented_operator(A, O.restriction(G.spec.n, rec), G.src[s], G.lam, source_free)
    b = O.rhs(G.spec.n, G.src[s], G.d[G.rec_off[s]:G.rec_off[s + 1]], G.lam, G.alpha[s], source_free)
    return S, b


def _cpp(G, s, source_free, **kw):
    rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
    return cpu_cgls.cgls(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.src[s], rec,
                         G.d[G.rec_off[s]:G.rec_off[s + 1]], G.lam, G.alpha[s], source_free, R=G.pml_R, **kw)


@pytest.mark.parametrize("source_free", [True, False])
@pytest.mark.parametrize("threads", [1, 4])
def test_fixed_iterates_equal_numpy_oracle(source_free, threads):
    G = _case()
    k = 15
    for s in range(G.nsys):
        S, b = _oracle_S_b(G, s, source_free)
        x_ref, it_ref, rr_ref = O.cgls(S, b, tol=0.0, max_iter=k)
        x, it, rr = _cpp(G, s, source_free, tol=0.0, max_iter=k, nthreads=threads)
        assert it == it_ref == k
        assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
        assert abs(rr - rr_ref) <= 1e-10 * rr_ref


def test_converged_solve_equals_numpy_oracle():
    """Solved to 1e-8: thousands of iterations (many times the unknowns), where rounding decides
    the iteration count, so the two differ by a fraction of a percent; the solutions agree to 1e-9."""
    G = _case(nphys=(8, 6, 5), npml=2, nsys=1, seed=9)
    S, b = _oracle_S_b(G, 0, True)
    x_ref, it_ref, _ = O.cgls(S, b, tol=1e-8, max_iter=100000)
    x, it, rr = _cpp(G, 0, True, tol=1e-8, max_iter=100000)
    assert abs(it - it_ref) <= 0.02 * it_ref and rr <= 1e-8
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_rejects_invalid_arguments():
    G = _case(nsys=1)
    with pytest.raises(ValueError):
        cpu_cgls.cgls(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.spec.n, G.rec_idx, G.d, G.lam)
    assert cpu_cgls.threads() >= 1
