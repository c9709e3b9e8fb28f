"""Shared helpers of the GPU parity tests: seeded cases and their oracle view.

The GPU consumes the model and data at its own precision (float32 / complex64 for
the C64 path), so the oracle is fed exactly those rounded values.
"""
import numpy as np

import oracle as O
import synth


def case(nphys=(21, 13, 11), npml=4, h=10.0, freq=12.0, nsys=3, seed=5, nrec=7, lam=None, d_noise=0.05,
         with_data=True):
    G = synth.workload_small(nphys=nphys, npml=npml, h=h, freq=freq, nsys=nsys, seed=seed, nrec=nrec, lam=lam)
    if with_data:
        # data from a perturbed model so the problem is inconsistent (non-zero residual at the optimum)
        d = O.forward_data(G.spec.shape, h, G.omega, G.m * 1.04, npml, G.v_max, G.src, G.rec_off, G.rec_idx, G.alpha)
        r = synth.rng(seed + 99)
        G.d = d * (1 + d_noise * (r.standard_normal(d.shape) + 1j * r.standard_normal(d.shape)))
    return G


def seen(G, c64: bool):
    """(m, d, alpha) exactly as the GPU path sees them."""
    if c64:
        m = G.m.astype(np.float32).astype(np.float64)
        d = None if G.d is None else G.d.astype(np.complex64).astype(np.complex128)
    else:
        m, d = G.m, G.d
    return m, d, G.alpha


def oracle_A(G, m):
    return O.helmholtz_matrix(G.spec.shape, G.spec.h, G.omega, m, G.spec.npml, G.v_max, G.pml_R)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
