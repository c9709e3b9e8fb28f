"""Resampling between the master model grid and the groups' grids, pinned on the CPU.

Trilinear interpolation is fixed by two facts that these tests check independently of the code's
construction: it reproduces affine functions exactly at every point inside the master nodes'
hull (clamped positions outside it), and its transpose is the exact adjoint (a brute-force matrix
built column by column from unit vectors, and the dot-product test).
"""
import numpy as np
import pytest
import torch

from paper_2410_18429_gb300.grids import Resample, interp_1d, multigrid_evaluate


def _centres(n, h):
    return (np.arange(n) + 0.5) * h


def _affine(z, y, x):
    return 0.3 + 2e-3 * x - 5e-4 * y + 1.25e-3 * z


def _expected(master_n, master_h, nphys, npml, h):
    """The affine field at the clamped position of every computational node (padding copies the
    nearest physical node)."""
    axes = []
    for n_m, n_p in zip(master_n, nphys):
        lo, hi = 0.5 * master_h, (n_m - 0.5) * master_h
        c = np.clip(np.arange(n_p + 2 * npml) - npml, 0, n_p - 1)
        axes.append(np.clip(_centres(n_p, h)[c], lo, hi))
    x, y, z = axes
    return _affine(z[:, None, None], y[None, :, None], x[None, None, :])


@pytest.mark.parametrize("master_n,master_h,nphys,npml,h", [
    ((32, 24, 16), 10.0, (16, 12, 8), 3, 20.0),           # coarser group (every node inside the hull)
    ((16, 16, 16), 20.0, (24, 24, 24), 2, 40.0 / 3.0),    # finer group (outer nodes clamped)
    ((12, 9, 6), 30.0, (8, 6, 4), 0, 45.0),               # ratio 2/3, no padding
])
def test_affine_fields_are_reproduced(master_n, master_h, nphys, npml, h):
    xm, ym, zm = (_centres(n, master_h) for n in master_n)
    m = torch.as_tensor(_affine(zm[:, None, None], ym[None, :, None], xm[None, None, :]))
    r = Resample(m.shape, master_h, nphys, npml, h)
    out = r(m).numpy()
    assert out.shape == tuple(n + 2 * npml for n in nphys[::-1])
    assert np.allclose(out, _expected(master_n, master_h, nphys, npml, h), rtol=0, atol=1e-14)


def test_same_grid_is_the_padding_copy_bit_for_bit():
    rng = np.random.default_rng(3)
    m = rng.standard_normal((7, 9, 11))
    r = Resample(m.shape, 26.0 + 2.0 / 3.0, (11, 9, 7), 4, 26.0 + 2.0 / 3.0)
    assert np.array_equal(r(torch.as_tensor(m)).numpy(), np.pad(m, 4, mode="edge"))


def test_rows_are_convex_weights():
    for n_m, n_p, p in ((128, 64, 10), (128, 96, 10), (64, 128, 10), (5, 3, 0), (1, 4, 2), (4, 1, 1)):
        w = interp_1d(n_m, n_p, p)
        assert w.shape == (n_p + 2 * p, n_m)
        assert (w >= 0).all() and np.allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-15)
        assert ((w > 0).sum(axis=1) <= 2).all()


@pytest.mark.parametrize("nphys,h", [((4, 3, 2), 24.0), ((12, 9, 6), 8.0)])
def test_adjoint_is_the_transpose_brute_force(nphys, h):
    master = (4, 6, 8)                                             # extents 48 x 72 x 96 (z, y, x)
    r = Resample(master, 12.0, nphys, 1, h)
    n_in = int(np.prod(master))
    cols = []
    for k in range(n_in):
        e = torch.zeros(n_in, dtype=torch.float64)
        e[k] = 1.0
        cols.append(r(e.reshape(master)).ravel())
    dense = torch.stack(cols, dim=1)                               # [n_out, n_in]
    rows = []
    for k in range(dense.shape[0]):
        e = torch.zeros(dense.shape[0], dtype=torch.float64)
        e[k] = 1.0
        rows.append(r.adjoint(e.reshape(r.shape)).ravel())
    assert torch.equal(torch.stack(rows, dim=0), dense)


def test_dot_product_test_at_multigrid_sizes():
    rng = np.random.default_rng(4)
    for nphys in ((64, 64, 64), (96, 96, 96)):
        h = 2560.0 / nphys[0]
        r = Resample((128, 128, 128), 20.0, nphys, 10, h)
        m = torch.as_tensor(rng.standard_normal((128, 128, 128)))
        y = torch.as_tensor(rng.standard_normal(r.shape))
        lhs = float((r(m) * y).sum())
        rhs = float((m * r.adjoint(y)).sum())
        assert abs(lhs - rhs) <= 1e-12 * float(r(m).norm()) * float(y.norm())


def test_rejects_mismatched_grids():
    with pytest.raises(ValueError):
        Resample((16, 16, 16), 20.0, (16, 16, 16), 2, 21.0)
    r = Resample((8, 8, 8), 10.0, (4, 4, 4), 1, 20.0)
    with pytest.raises(ValueError):
        r(torch.zeros(8, 8, 9, dtype=torch.float64))
    with pytest.raises(ValueError):
        r.adjoint(torch.zeros(4, 4, 4, dtype=torch.float64))
    with pytest.raises(ValueError):
        interp_1d(0, 4)
    with pytest.raises(ValueError):
        multigrid_evaluate([])


def test_multigrid_objective_gradient_is_the_chain_rule():
    """Quadratic stand-ins f_j(m_j) = 1/2 ||m_j - t_j||^2 on two grids plus a master-grid term:
    the composed gradient equals central differences of the composed objective (exact for a
    quadratic up to rounding) and the closed form sum_j R_j^T (R_j m - t_j)."""
    rng = np.random.default_rng(5)
    master = (12, 12, 12)
    rs = [Resample(master, 10.0, (6, 6, 6), 2, 20.0), Resample(master, 10.0, (8, 8, 8), 3, 15.0)]
    ts = [torch.as_tensor(rng.standard_normal(r.shape)) for r in rs]
    t0 = torch.as_tensor(rng.standard_normal(master))

    def quad(t):
        return lambda mj, eps: (0.5 * float(((mj - t) ** 2).sum()), mj - t)

    ev = multigrid_evaluate([(rs[0], quad(ts[0])), (rs[1], quad(ts[1])), (None, quad(t0))])
    m = torch.as_tensor(rng.standard_normal(master))
    f, g = ev(m, 1e-3)
    closed = sum(r.adjoint(r(m) - t) for r, t in zip(rs, ts)) + (m - t0)
    assert torch.allclose(g, closed, rtol=0, atol=1e-12)
    for _ in range(4):
        dm = torch.as_tensor(rng.standard_normal(master))
        eps = 1e-3
        fd = (ev(m + eps * dm, 1e-3)[0] - ev(m - eps * dm, 1e-3)[0]) / (2 * eps)
        assert abs(fd - float((g * dm).sum())) <= 1e-8 * abs(fd)


def test_for_group_reads_the_group_grid():
    from types import SimpleNamespace
    spec = SimpleNamespace(nx=84, ny=84, nz=84, npml=10, h=40.0)    # 64^3 physical cells over 2560 m
    r = Resample.for_group((128, 128, 128), 20.0, spec)
    assert r.shape == (84, 84, 84) and r.master_shape == (128, 128, 128)
    m = torch.full((128, 128, 128), 2.5e-7, dtype=torch.float64)
    assert torch.allclose(r(m), torch.full((84, 84, 84), 2.5e-7, dtype=torch.float64), rtol=1e-15, atol=0)


def test_outer_loop_over_grids_reduces_the_objective():
    """Algorithm 2's loop on a master-grid model whose objective lives on a coarser grid and on
    the master grid's own: every accepted step decreases f and the model approaches the fit.  The
    evaluations are exact, so once a full step fails halving eps cannot help and the loop ends at
    eps_min (the documented reading of the outer loop)."""
    from paper_2410_18429_gb300.awri import awri
    rng = np.random.default_rng(6)
    master = (8, 8, 8)
    rs = [Resample(master, 10.0, (4, 4, 4), 1, 20.0), Resample(master, 10.0, (8, 8, 8), 2, 10.0)]
    m_true = torch.as_tensor(1.0 + 0.1 * rng.standard_normal(master))
    ts = [r(m_true) for r in rs]

    def quad(t):
        return lambda mj, eps: (0.5 * float(((mj - t) ** 2).sum()), mj - t)

    ev = multigrid_evaluate([(r, quad(t)) for r, t in zip(rs, ts)])
    m0 = torch.ones(master, dtype=torch.float64)
    res = awri(m0, ev, 1e-2, 30, eps_min=1e-12, first_step=0.05)
    fs = [h["f"] for h in res.history]
    assert res.status in ("n_iter", "eps_min") and len(fs) >= 5
    assert all(b <= a for a, b in zip(fs, fs[1:]))
    assert res.f < 1e-2 * ev(m0, 1e-2)[0]
    # the second grid equals the master grid, so the fit's minimiser is m_true
    assert float((res.m - m_true).norm()) < 0.1 * float((m0 - m_true).norm())
