"""Source-free adaptive WRI outer loop (Algorithm 2), with the TV term of Eq. TVAWRI optional.

Every outer iteration evaluates the reduced objective f4 and its gradient g4 (Eqs. VarObj2 and
VarG2) with the augmented systems solved to the current tolerance eps, takes the l-BFGS step
m~ = m - H g, and evaluates f4 at m~ with the same eps.  A step that does not decrease f4 is
not taken: eps is halved, f4 and g4 are evaluated again at the same model, and the step is
recomputed.  The objective and gradient come from ``objective.py`` (libwri's kernels); this
module is host-side control flow plus a few vector operations on the model.

Readings (the paper states none of these):
  * eps is the relative normal-equation residual of the CGLS solves (and the FP64 refinement's
    target when refinement is on);
  * l-BFGS keeps the last ``memory`` (s, y) pairs of accepted steps (curvature s.y > 0 only);
    H0 = (s.y / y.y) I from the newest pair; before the first pair H0 = eta I with eta such that
    the first step changes m by ``first_step`` times max |m| at most;
  * the step is taken in full (Algorithm 2 has no line search);
  * the evaluation at an accepted m~ is reused as the next iteration's first evaluation (it is
    the same solve at the same model and tolerance);
  * if a step fails with eps already below ``eps_min`` the loop stops (status "eps_min").

The loop's whole state between iterations (model, f, g, eps, the l-BFGS pairs, counters and
history) is an ``AwriState``; ``save_state`` / ``load_state`` write and read it with
``torch.save``, and ``awri(..., state=...)`` continues from it exactly as if never interrupted.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Tuple

import torch


class LBFGS:
    """Limited-memory BFGS inverse-Hessian product by the two-loop recursion."""

    def __init__(self, memory: int = 5, s: Optional[List[torch.Tensor]] = None,
                 y: Optional[List[torch.Tensor]] = None):
        if memory < 1:
            raise ValueError("memory >= 1")
        self.memory = memory
        self.s: List[torch.Tensor] = [] if s is None else s
        self.y: List[torch.Tensor] = [] if y is None else y

    def update(self, s: torch.Tensor, y: torch.Tensor) -> bool:
        """Store the pair if it satisfies the curvature condition; returns whether it was kept."""
        sy = float(torch.dot(s.ravel(), y.ravel()))
        if not sy > 1e-12 * float(s.norm()) * float(y.norm()):
            return False
        self.s.append(s.clone())
        self.y.append(y.clone())
        if len(self.s) > self.memory:
            self.s.pop(0)
            self.y.pop(0)
        return True

    def apply(self, g: torch.Tensor, h0: Optional[float] = None) -> torch.Tensor:
        """H g.  h0 scales the initial matrix when no pair is stored (required then)."""
        q = g.clone()
        if not self.s:
            if h0 is None:
                raise ValueError("h0 is needed before the first pair")
            return h0 * q
        rho = [1.0 / float(torch.dot(s.ravel(), y.ravel())) for s, y in zip(self.s, self.y)]
        a = [0.0] * len(self.s)
        for i in range(len(self.s) - 1, -1, -1):
            a[i] = rho[i] * float(torch.dot(self.s[i].ravel(), q.ravel()))
            q -= a[i] * self.y[i]
        sn, yn = self.s[-1], self.y[-1]
        r = (float(torch.dot(sn.ravel(), yn.ravel())) / float(torch.dot(yn.ravel(), yn.ravel()))) * q
        for i in range(len(self.s)):
            bcoef = rho[i] * float(torch.dot(self.y[i].ravel(), r.ravel()))
            r += (a[i] - bcoef) * self.s[i]
        return r


@dataclass
class AwriState:
    """The outer loop between two iterations: model m with its f and g at tolerance eps, the
    stored l-BFGS pairs (oldest first), the iterations and evaluations done, and the history."""

    m: torch.Tensor
    f: float
    g: torch.Tensor
    eps: float
    s: List[torch.Tensor] = field(default_factory=list)
    y: List[torch.Tensor] = field(default_factory=list)
    iteration: int = 0
    evaluations: int = 0
    history: List[dict] = field(default_factory=list)


def save_state(state: AwriState, path: str) -> None:
    """Write the state with ``torch.save`` (to a temporary file first, then renamed, so an
    interrupted write leaves the previous checkpoint intact)."""
    tmp = path + ".tmp"
    torch.save({"m": state.m, "f": state.f, "g": state.g, "eps": state.eps, "s": state.s, "y": state.y,
                "iteration": state.iteration, "evaluations": state.evaluations, "history": state.history}, tmp)
    os.replace(tmp, path)


def load_state(path: str, device=None) -> AwriState:
    """Read a state written by ``save_state``; tensors go to ``device`` (default: where they were)."""
    d = torch.load(path, map_location=device, weights_only=True)
    return AwriState(m=d["m"], f=float(d["f"]), g=d["g"], eps=float(d["eps"]), s=list(d["s"]), y=list(d["y"]),
                     iteration=int(d["iteration"]), evaluations=int(d["evaluations"]), history=list(d["history"]))


@dataclass
class AwriResult:
    m: torch.Tensor
    f: float
    status: str                                    # "n_iter" or "eps_min"
    history: List[dict] = field(default_factory=list)
    evaluations: int = 0
    state: Optional[AwriState] = None              # to continue the loop (``awri(..., state=...)``)


def awri(m0: Optional[torch.Tensor], evaluate: Callable[[torch.Tensor, float], Tuple[float, torch.Tensor]],
         eps0: float, n_iter: int, eps_min: float = 1e-12, memory: int = 5, first_step: float = 0.05,
         model_error: Optional[Callable[[torch.Tensor], float]] = None, state: Optional[AwriState] = None,
         checkpoint: Optional[str] = None) -> AwriResult:
    """Algorithm 2 (gamma = 0).  ``evaluate(m, eps) -> (f, g)`` gives f4 and g4 at m with the
    systems solved to tolerance eps (e.g. ``make_evaluate``).

    ``n_iter`` counts all iterations, those of a resumed ``state`` included; with ``state`` the
    loop continues from it (m0 and eps0 are then not used).  With ``checkpoint`` the state is
    saved there after every accepted iteration."""
    if not (eps0 > 0 and n_iter >= 0):
        raise ValueError("eps0 > 0 and n_iter >= 0 required")
    if state is None and m0 is None:
        raise ValueError("a starting model m0 or a state to resume from is required")
    if state is None:
        m = m0.detach().clone().to(torch.float64)
        eps = float(eps0)
        f, g = evaluate(m, eps)
        state = AwriState(m=m, f=f, g=g, eps=eps, evaluations=1)
    lb = LBFGS(memory, state.s, state.y)
    m, f, g, eps, evals = state.m, state.f, state.g, state.eps, state.evaluations
    status = "n_iter"
    for k in range(state.iteration, n_iter):
        while True:
            h0 = None
            if not lb.s:
                gmax = float(g.abs().max())
                h0 = first_step * float(m.abs().max()) / gmax if gmax > 0 else 0.0
            m_t = m - lb.apply(g, h0)
            f_t, g_t = evaluate(m_t, eps)
            evals += 1
            if f_t <= f:
                break
            if 0.5 * eps < eps_min:
                status = "eps_min"
                break
            eps *= 0.5                       # reduce the tolerance and recompute at m^(k)
            f, g = evaluate(m, eps)
            evals += 1
        if status == "eps_min":
            break
        lb.update(m_t - m, g_t - g)
        m, f, g = m_t, f_t, g_t
        rec = {"iteration": k + 1, "f": f, "eps": eps, "evaluations": evals}
        if model_error is not None:
            rec["model_error"] = float(model_error(m))
        state.history.append(rec)
        state.m, state.f, state.g, state.eps, state.iteration, state.evaluations = m, f, g, eps, k + 1, evals
        if checkpoint is not None:
            save_state(state, checkpoint)
    state.m, state.f, state.g, state.eps, state.evaluations = m, f, g, eps, evals
    return AwriResult(m=m, f=f, status=status, history=state.history, evaluations=evals, state=state)


def make_evaluate(groups, opts, max_resident: int = 1 << 30, stats: Optional[dict] = None, tv_gamma: float = 0.0,
                  tv_beta: float = 1e-9):
    """evaluate(m, eps) for ``awri`` on libwri: the solves of ``objective.objective`` with tolerance
    eps (and FP64 refinement target eps when ``opts`` refines), plus tv_gamma times the TV term
    of Eq. TVAWRI (``wri_tv``, smoothing tv_beta) when tv_gamma > 0; returns (f, g), g float64."""
    from . import objective as obj
    from . import wri

    def evaluate(m: torch.Tensor, eps: float):
        o = wri.WriSolveOpts.from_buffer_copy(opts)
        o.tol = float(eps)
        if int(o.max_refine) > 0:
            o.refine_tol = float(eps)
        mm = m.detach().clone().requires_grad_(True)
        st = {} if stats is None else stats
        f = obj.objective(mm, groups, o, max_resident=max_resident, stats=st)
        f.backward()
        fv, g = float(f.item()), mm.grad.detach().to(torch.float64)
        if tv_gamma > 0:
            tv, _ = wri.tv(groups[0], m, tv_beta, tv_gamma, grad=g)
            fv += float(tv.item())
        return fv, g

    return evaluate
