"""Reduced FWI, the paper's comparison method (Eqs. FWI, PDEsolve and FWI2), through libwri.

The reduced objective eliminates the wavefield by the PDE solve u_i = a_i A^{-1} e_i (Eq. PDEsolve):
    f(m) = 1/2 sum_i ||a_i P_i A^{-1} e_i - d_i||^2                        (Eq. FWI2)
with the weights a_i given, or (source-free) each the minimiser of its term.  Its gradient needs
an adjoint solve per system (adjoint-state method): with G_i = A^{-1} e_i, r_i = a_i P_i G_i - d_i
and v_i = A^{-H} P_i^T r_i,
    grad f = -omega^2 sum_i Re(w a_i G_i conj(v_i)),
(dA/dm_k = omega^2 w_k e_k e_k^T; the weight's own derivative vanishes at its optimum).

Every numerical step runs in libwri's kernels; this module only sequences the calls:
  1. forward solves A G_i = e_i: wri_solve_batch with weight 1 and lambda = 0 (the PDE least
     squares problem min ||A G - e||, CGLS on A);
  2. wri_fwi_adjoint_source: the weights, the residuals, f and the adjoint right-hand sides
     conj(P^T r_i);
  3. adjoint solves A w_i = conj(P^T r_i) (general right-hand side, lambda = 0); A is complex
     symmetric, so v_i = conj(w_i);
  4. wri_fwi_gradient.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Optional, Sequence

import torch

from . import wri


def evaluate(groups: Sequence[wri.GroupSpec], opts, alpha: Optional[torch.Tensor] = None, stats: Optional[dict] = None):
    """Reduced-FWI objective f (tensor [1]) and gradients (one float64 tensor per group, shaped like
    the group's model) at the groups' models, with the weights ``alpha`` (complex128 [sum nsys]) or,
    when None, the source-free weights, which are returned as the third value.

    groups: the frequency groups (grid, m, geometry, observed data d); their ``u``, ``alpha``,
    ``q`` and ``lam`` are not used.  opts: the options of the forward and adjoint solves (their
    tolerance decides the accuracy of f and g)."""
    dtype = int(opts.dtype)
    cdt = torch.complex128 if dtype == wri.C128 else torch.complex64
    dev = groups[0].m.device
    ones = [torch.tensor([[1.0, 0.0]], dtype=torch.float64, device=dev).repeat(g.nsys, 1) for g in groups]
    fwd = [replace(g, alpha=o, lam=0.0, q=None, u64=None, u=torch.zeros(g.nsys, g.n, dtype=cdt, device=dev))
           for g, o in zip(groups, ones)]
    it1, rr1, st1 = wri.solve(fwd, opts)
    q_adj = [torch.zeros(g.nsys, g.n, dtype=cdt, device=dev) for g in groups]
    a, f = wri.fwi_adjoint_source(fwd, dtype, q_adj, alpha=alpha)
    adj = [replace(g, alpha=None, lam=0.0, q=q, u64=None, u=torch.zeros(g.nsys, g.n, dtype=cdt, device=dev))
           for g, q in zip(groups, q_adj)]
    it2, rr2, st2 = wri.solve(adj, opts)
    grads = wri.fwi_gradient(fwd, dtype, a, [s.u for s in adj])
    if stats is not None:
        stats.update(forward_iters=it1, forward_status=st1, forward_relres=rr1, adjoint_iters=it2,
                     adjoint_status=st2, adjoint_relres=rr2)
    return f, grads, a
