"""The reduced WRI objective f4(m) as a ``torch.autograd.Function``.

f4(m) = f3(m, x(m)) with x(m) = (u(m), a(m)) the variable-projection minimiser of the
augmented least-squares problem (Eqs. SimpObj and VarObj2).  Because x(m) minimises f3,
the gradient needs no adjoint solve (Eq. VarG2): the forward pass solves every
(source, frequency) system, estimates its weight and accumulates f and g with the
gradient kernel; the backward pass returns ``grad_output * g``.

With complex64 stencils and FP64 refinement (``opts.max_refine > 0``) the refined FP64
wavefields are kept (``u64``), and g and f come from the refinement's FP64 residual
(``wri.gradient_refined``, no extra stencil pass).

Systems are processed in chunks of at most ``max_resident`` systems per group, so the
wavefields of one chunk are the only ones held in HBM at any time: when the source batch
outgrows device memory the wavefields are recomputed chunk by chunk instead of stored.
With ``recompute=True`` the forward pass keeps nothing but f, and the backward pass solves
every chunk again (same tolerance, zero start, so the same wavefields) to form g.

Every numerical step runs in libwri's kernels; this module only sequences the calls.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import wri


@dataclass
class Problem:
    """Geometry and data of the systems whose objective is summed.

    groups: one ``wri.GroupSpec`` per frequency group, all on the grid of the model; their
    ``m`` and ``u`` fields are ignored (the model is the autograd input; wavefields are
    chunk buffers owned here).  opts: ``wri.make_opts(...)`` of every solve.
    """

    groups: Sequence[wri.GroupSpec]
    opts: object
    max_resident: int = 1 << 30
    recompute: bool = False
    stats: dict = field(default_factory=dict)


def chunks(nsys: int, max_resident: int) -> List[tuple]:
    """Contiguous [begin, end) chunks of at most ``max_resident`` systems covering nsys."""
    if nsys < 0 or max_resident < 1:
        raise ValueError("nsys >= 0 and max_resident >= 1 required")
    return [(b, min(b + max_resident, nsys)) for b in range(0, nsys, max_resident)]


def _sub(g: wri.GroupSpec, b: int, e: int, m, u, u64=None) -> wri.GroupSpec:
    """Systems [b, e) of a group, with the model m and the wavefield buffers u (and u64)."""
    off = np.asarray(g.rec_off, dtype=np.int64)
    r0, r1 = int(off[b]), int(off[e])
    alpha = None if g.alpha is None else g.alpha[b:e]
    return replace(g, m=m, src=np.asarray(g.src)[b:e], rec_off=(off[b:e + 1] - r0).astype(np.int32),
                   rec_idx=np.asarray(g.rec_idx)[r0:r1], d=g.d[r0:r1], u=u, alpha=alpha, u64=u64)


def _evaluate(m: torch.Tensor, prob: Problem, want_grad: bool):
    """f (and g when asked) summed over every system, chunk by chunk."""
    opts = prob.opts
    dtype = int(opts.dtype)
    cdt = torch.complex128 if dtype == wri.C128 else torch.complex64
    rdt = torch.float64 if dtype == wri.C128 else torch.float32
    mm = m.detach().to(rdt).contiguous()
    dev = mm.device
    f = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros(mm.shape, dtype=torch.float64, device=dev) if want_grad else None
    scratch_g = g if want_grad else torch.zeros(mm.shape, dtype=torch.float64, device=dev)
    if tuple(mm.shape) != (prob.groups[0].nz, prob.groups[0].ny, prob.groups[0].nx):
        raise ValueError("the model must have the shape [nz, ny, nx] of the groups' grid")
    iters, status, relres = [], [], []
    # complex64 with FP64 refinement: the FP64 solution feeds the estimate and the gradient
    wide = dtype == wri.C64 and int(opts.max_refine) > 0
    for grp in prob.groups:
        step = min(prob.max_resident, grp.nsys)
        u = torch.zeros(step, grp.n, dtype=cdt, device=dev)
        u64 = torch.zeros(step, grp.n, dtype=torch.complex128, device=dev) if wide else None
        for b, e in chunks(grp.nsys, prob.max_resident):
            spec = _sub(grp, b, e, mm, u[:e - b], None if u64 is None else u64[:e - b])
            spec.u.zero_()
            work = torch.empty(wri.workspace_size([spec], opts), dtype=torch.uint8, device=dev)
            it, rr, st = wri.solve([spec], opts, workspace=work)
            if bool((st == wri.SYS_NONFINITE).any()):
                raise FloatingPointError(f"non-finite values in the solves of systems {b}..{e}")
            iters.append(it)
            status.append(st)
            relres.append(rr)
            if wide:
                # the refinement's FP64 residual gives g and f without another stencil pass
                wri.gradient_refined([spec], opts, work, grads=[scratch_g], f=f)
            else:
                a = spec_alpha(spec, dtype)
                wri.gradient([spec], dtype, a, grads=[scratch_g], f=f)
    prob.stats["iters"] = torch.cat(iters)
    prob.stats["status"] = torch.cat(status)
    prob.stats["relres"] = torch.cat(relres)
    return f, g


def spec_alpha(spec: wri.GroupSpec, dtype: int):
    """The weight used in f and g: the estimate (source-free) or the known weight."""
    if spec.alpha is None:
        return wri.source_estimate([spec], dtype)
    return torch.view_as_complex(spec.alpha.contiguous())


class WRIObjective(torch.autograd.Function):
    """f4(m) for a real model tensor m ([nz, ny, nx], float32 or float64, on the GPU)."""

    @staticmethod
    def forward(ctx, m: torch.Tensor, prob: Problem):
        f, g = _evaluate(m, prob, want_grad=not prob.recompute)
        ctx.prob = prob
        ctx.m_dtype = m.dtype
        if prob.recompute:
            ctx.save_for_backward(m)
        else:
            ctx.g = g
        return f[0]

    @staticmethod
    def backward(ctx, grad_out):
        prob = ctx.prob
        if prob.recompute:
            (m,) = ctx.saved_tensors
            _, g = _evaluate(m, prob, want_grad=True)
        else:
            g = ctx.g
        return (grad_out.to(torch.float64) * g).to(ctx.m_dtype), None


def objective(m: torch.Tensor, groups: Sequence[wri.GroupSpec], opts, max_resident: int = 1 << 30,
              recompute: bool = False, stats: Optional[dict] = None) -> torch.Tensor:
    """f4(m) with autograd support; see WRIObjective."""
    prob = Problem(groups, opts, max_resident, recompute, stats if stats is not None else {})
    return WRIObjective.apply(m, prob)
