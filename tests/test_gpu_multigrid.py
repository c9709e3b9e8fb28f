"""One model over two frequency groups on grids of their own, through libwri.

f(m) = sum_j f_j(R_j m) and g = sum_j R_j^T g_j (the grids' relation is a reading; the paper
states none) with every f_j, g_j from libwri's complex128 solves, against the oracle's exact
evaluations of each group at the same resampled model.  R_j itself is pinned on the CPU.
"""
import numpy as np
import pytest

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
    from paper_2410_18429_gb300 import awri, grids, wri
    return wri, awri, grids


def multigrid_case():
    """A 160 m box: 8^3 cells of 20 m at 6 Hz and 16^3 cells of 10 m at 12 Hz (padding 3 each),
    seeded data, and a master model on the fine grid's 16^3 physical nodes (velocities around
    2000 m/s with a seeded 5 % perturbation)."""
    gc = synth.workload_small(nphys=8, npml=3, h=20.0, freq=6.0, nsys=2, seed=21, nrec=5)
    gf = synth.workload_small(nphys=16, npml=3, h=10.0, freq=12.0, nsys=2, seed=22, nrec=7)
    dc = synth.random_complex(len(gc.rec_idx), 24)
    df = synth.random_complex(len(gf.rec_idx), 25)
    v = 2000.0 * (1.0 + 0.05 * synth.rng(23).standard_normal((16, 16, 16)))
    return (gc, dc, (8, 8, 8), 20.0), (gf, df, (16, 16, 16), 10.0), synth.to_m(v)


def test_multigrid_objective_matches_oracle_c128(W):
    wri, awri, grids = W
    from oracle.awri_oracle import exact_evaluate
    from paper_2410_18429_gb300.problem import to_device
    *cases, m_master = multigrid_case()
    opts = wri.make_opts(tol=1e-11, max_iter=400000, dtype=wri.C128)
    parts, f_ref, g_ref = [], 0.0, np.zeros(m_master.shape)
    for G, d, nphys, h in cases:
        r = grids.Resample(m_master.shape, 10.0, nphys, 3, h)
        parts.append((r, awri.make_evaluate([to_device(G, wri.C128, "cuda", d=d)], opts)))
        mj = r(torch.as_tensor(m_master)).numpy()
        fj, gj = exact_evaluate(G, d)(mj, 1e-11)
        f_ref += fj
        g_ref += r.adjoint(torch.as_tensor(np.asarray(gj).reshape(r.shape))).numpy()
    f, g = grids.multigrid_evaluate(parts)(torch.as_tensor(m_master).cuda(), 1e-11)
    assert abs(f - f_ref) <= 1e-9 * abs(f_ref)
    # the gradient parity target is 1e-4; with this rough model, solves to 1e-11 leave about 1e-7
    assert rel(g.cpu().numpy(), g_ref) < 1e-6
