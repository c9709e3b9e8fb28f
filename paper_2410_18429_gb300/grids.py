"""One model over frequency groups on grids of their own: trilinear resampling and its adjoint.

The multi-frequency inversion solves each frequency on its own grid, coarse for low frequencies and
fine for high ones, but updates a single model.  The paper does not say how the grids relate
(Sec. GPU1 only groups the systems), so this module takes the following reading:

  * every physical grid covers the same box; along an axis a grid of n cells of size h spans
    [0, n h) and its nodes sit at the cell centres (i + 1/2) h;
  * the model lives on a master grid (physical nodes only, [Nz, Ny, Nx]);
  * a group's model is m_j = R_j m: trilinear interpolation of the master nodes at the group's
    physical node positions, with positions outside the master's first and last node clamped to
    them (constant extension), followed by the copy of the nearest physical node into the
    ``npml`` padding nodes on every face (the convention of the synthetic models);
  * the objective is f(m) = sum_j f_j(R_j m) and, by the chain rule, its gradient is
    sum_j R_j^T g_j, with f_j and g_j the group's reduced objective and gradient (Eqs. VarObj2
    and VarG2).

R_j is separable, R = Rz (x) Ry (x) Rx, and each 1-D factor has at most two non-zeros per row.
With equal extents (n h = N H) a node's master coordinate is the rational ((2i+1) N - n) / (2n),
so the weights are formed from integers: when a group's physical grid equals the master grid the
weights are exactly 0 and 1 and R_j is the padding copy, bit for bit.  R^T applies the transposed
factors in the reverse order, so <R m, y> = <m, R^T y> up to rounding.

These are small tensor contractions (three matrix products with factors of a few hundred rows)
run once per model update, next to the solves' thousands of stencil passes per system: host-side
glue around libwri's calls, not a step of the per-system path.
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence, Tuple

import numpy as np
import torch

__all__ = ["interp_1d", "Resample", "multigrid_evaluate"]


def interp_1d(n_master: int, n_phys: int, npml: int = 0) -> np.ndarray:
    """The 1-D factor, float64 [n_phys + 2 npml, n_master]: row c interpolates the master nodes at
    the position of computational node c of a grid of n_phys cells over the same extent."""
    if n_master < 1 or n_phys < 1 or npml < 0:
        raise ValueError("n_master >= 1, n_phys >= 1 and npml >= 0 required")
    w = np.zeros((n_phys + 2 * npml, n_master))
    for c in range(n_phys + 2 * npml):
        i = min(max(c - npml, 0), n_phys - 1)          # padding nodes copy the nearest physical node
        num, den = (2 * i + 1) * n_master - n_phys, 2 * n_phys   # master coordinate t = num / den
        if num <= 0 or n_master == 1:
            w[c, 0] = 1.0
        elif num >= (n_master - 1) * den:
            w[c, n_master - 1] = 1.0
        else:
            k, rem = divmod(num, den)
            w[c, k] = (den - rem) / den
            w[c, k + 1] = rem / den
    return w


class Resample:
    """m_j = R m from the master grid ([Nz, Ny, Nx], cell size ``master_h``) onto a group's
    computational grid (``nphys`` = (nx, ny, nz) physical cells of size ``h`` plus ``npml`` padding
    nodes per face); ``adjoint`` applies R^T.  Raises ValueError unless every axis has the same
    extent on both grids (relative 1e-9)."""

    def __init__(self, master_shape: Sequence[int], master_h: float, nphys: Sequence[int], npml: int, h: float):
        nz_m, ny_m, nx_m = (int(v) for v in master_shape)
        nxp, nyp, nzp = (int(v) for v in nphys)
        for a, b in ((nx_m, nxp), (ny_m, nyp), (nz_m, nzp)):
            if abs(a * master_h - b * h) > 1e-9 * a * master_h:
                raise ValueError(f"extents differ: {a} x {master_h} != {b} x {h}")
        self.master_shape = (nz_m, ny_m, nx_m)
        self.shape = (nzp + 2 * npml, nyp + 2 * npml, nxp + 2 * npml)
        self._w = [torch.from_numpy(interp_1d(nz_m, nzp, npml)), torch.from_numpy(interp_1d(ny_m, nyp, npml)),
                   torch.from_numpy(interp_1d(nx_m, nxp, npml))]

    @classmethod
    def for_group(cls, master_shape: Sequence[int], master_h: float, spec) -> "Resample":
        """R onto the computational grid of a ``wri.GroupSpec`` (or anything with nx, ny, nz, npml, h)."""
        p = int(spec.npml)
        return cls(master_shape, master_h, (spec.nx - 2 * p, spec.ny - 2 * p, spec.nz - 2 * p), p, spec.h)

    def _factors(self, t: torch.Tensor):
        return [w.to(device=t.device, dtype=t.dtype) for w in self._w]

    def __call__(self, m: torch.Tensor) -> torch.Tensor:
        if tuple(m.shape) != self.master_shape:
            raise ValueError(f"model shape {tuple(m.shape)} != master grid {self.master_shape}")
        wz, wy, wx = self._factors(m)
        t = torch.matmul(m, wx.T)                                   # [Nz, Ny, nx]
        t = torch.matmul(wy, t)                                     # [Nz, ny, nx]
        return torch.matmul(wz, t.reshape(t.shape[0], -1)).reshape(self.shape)

    def adjoint(self, g: torch.Tensor) -> torch.Tensor:
        if tuple(g.shape) != self.shape:
            raise ValueError(f"gradient shape {tuple(g.shape)} != group grid {self.shape}")
        wz, wy, wx = self._factors(g)
        t = torch.matmul(wz.T, g.reshape(g.shape[0], -1)).reshape(self.master_shape[0], *g.shape[1:])
        t = torch.matmul(wy.T, t)                                   # [Nz, Ny, nx]
        return torch.matmul(t, wx)                                  # [Nz, Ny, Nx]


Evaluate = Callable[[torch.Tensor, float], Tuple[float, torch.Tensor]]


def multigrid_evaluate(parts: Sequence[Tuple[Optional[Resample], Evaluate]]) -> Evaluate:
    """evaluate(m, eps) -> (f, g) of f(m) = sum_j f_j(R_j m) for the outer loop, from one
    (R_j, evaluate_j) pair per grid (``awri.make_evaluate`` of the groups on that grid; R_j None
    for a term on the master grid itself); g = sum_j R_j^T g_j, float64 on m's device."""
    if not parts:
        raise ValueError("at least one part required")

    def evaluate(m: torch.Tensor, eps: float):
        m64 = m.detach().to(torch.float64)
        f, g = 0.0, torch.zeros_like(m64)
        for r, ev in parts:
            if r is None:
                fj, gj = ev(m64, eps)
                g += gj.to(torch.float64)
            else:
                fj, gj = ev(r(m64), eps)
                g += r.adjoint(gj.to(torch.float64))
            f += float(fj)
        return f, g

    return evaluate
