"""Writes config1_oracle.json: the oracle's CGLS on configuration 1 at the tolerances the GPU
test uses (iterations, and the wavefield and gradient errors against the oracle's exact LU
evaluation).  Calls only oracle/ and synth/.  Run from the repository root:

    python tests/golden/make_config1_oracle.py

Configuration 1: 24^3 physical nodes + 6-cell layer, h = 10 m, homogeneous 2000 m/s model, 5 Hz,
source (12, 12, 2), 20 receivers at x = y = 18, z = 2..21, lambda = 10, data from an exact
forward solve on the +10 % Gaussian anomaly model with the true weight -10.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402
from oracle import cpu_cgls  # noqa: E402


def main():
    G = synth.workload_c1()
    shp, h, npml = G.spec.shape, G.spec.h, G.spec.npml
    m_true = synth.to_m(synth.workload_c1_true_velocity())
    G.d = O.forward_data(shp, h, G.omega, m_true, npml, G.v_max, G.src, G.rec_off, G.rec_idx, G.alpha)
    u_ex, _, _, g_ex = O.evaluate(shp, h, G.omega, G.m, npml, G.v_max, G.src, G.rec_off, G.rec_idx, G.d, G.lam)
    A = O.helmholtz_matrix(shp, h, G.omega, G.m, npml, G.v_max, G.pml_R)
    w = O.stretch_weight(shp, h, G.omega, npml, G.v_max, G.pml_R)
    out = {"workload": "configuration 1 (24^3 + 6, 5 Hz, lambda 10, complex128)", "solves": []}
    for tol in (1e-8, 1e-13):
        x, it, rr = cpu_cgls.cgls(shp, h, G.omega, G.m, npml, G.v_max, G.src[0], G.rec_idx, G.d, G.lam, tol=tol,
                                  max_iter=2000000)
        a = O.source_estimate(A, x, G.src[0])
        g = O.gradient(A, x, G.src[0], a, G.omega, w)
        out["solves"].append({"tol": tol, "iterations": it, "relres": rr,
                              "u_err_vs_exact": float(np.linalg.norm(x - u_ex[0]) / np.linalg.norm(u_ex[0])),
                              "g_err_vs_exact": float(np.linalg.norm(g - g_ex) / np.linalg.norm(g_ex))})
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
