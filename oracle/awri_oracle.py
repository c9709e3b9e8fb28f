"""Oracle of the adaptive WRI outer loop (Algorithm 2 without the TV term), numpy, float64.

TEST INFRASTRUCTURE ONLY: used by tests/; never by the product path, and it shares no code
with it.  The objective and gradient come from exact (LU) solves of ``wri_oracle.evaluate``,
so the tolerance eps only steers the control flow (it is halved when a step fails), as in the
paper's listing.

Readings, the same as the product's (the paper states none of these): eps is the solve
tolerance; l-BFGS keeps the last ``memory`` accepted pairs with s.y > 0; the initial inverse
Hessian is (s.y / y.y) I from the newest pair, or eta I before the first pair with eta such that
the first step changes m by ``first_step`` max |m| at most; full steps (no line search); the loop
stops when a step fails with eps below ``eps_min``.
"""
from __future__ import annotations

import numpy as np

from .wri_oracle import evaluate as _evaluate
from .wri_oracle import total_variation as _total_variation

__all__ = ["two_loop", "bfgs_inverse", "awri", "exact_evaluate"]


def two_loop(g, S, Y, h0=None):
    """H g by the l-BFGS two-loop recursion over the pairs (S[i], Y[i]), oldest first."""
    g = np.asarray(g, dtype=np.float64).ravel()
    if not S:
        return h0 * g
    rho = [1.0 / (s @ y) for s, y in zip(S, Y)]
    q = g.copy()
    alpha = np.zeros(len(S))
    for i in reversed(range(len(S))):
        alpha[i] = rho[i] * (S[i] @ q)
        q = q - alpha[i] * Y[i]
    r = ((S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])) * q
    for i in range(len(S)):
        beta = rho[i] * (Y[i] @ r)
        r = r + (alpha[i] - beta) * S[i]
    return r


def bfgs_inverse(S, Y):
    """The dense inverse-Hessian approximation of BFGS built from H0 = (s.y / y.y) I (newest
    pair) by the update H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T, oldest pair first
    (small n only; pins ``two_loop``)."""
    n = len(S[0])
    H = ((S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])) * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


def exact_evaluate(G, d, lam=None, source_free=True, tv_gamma=0.0, tv_beta=1e-9):
    """evaluate(m, eps) -> (f4 + tv_gamma TV, g4 + tv_gamma dTV/dm) of one frequency group by
    exact solves (eps unused); TV is ``total_variation`` (Eq. TVAWRI, our reading)."""
    lam = G.lam if lam is None else lam

    def evaluate(m, eps):
        mm = np.asarray(m).reshape(G.spec.shape)
        _, _, f, g = _evaluate(G.spec.shape, G.spec.h, G.omega, mm, G.spec.npml,
                               G.v_max, G.src, G.rec_off, G.rec_idx, d, lam, alpha=None if source_free else G.alpha,
                               source_free=source_free)
        if tv_gamma > 0:
            tv, gtv = _total_variation(mm, tv_beta)
            f = f + tv_gamma * tv
            g = g + tv_gamma * gtv.ravel()
        return f, g

    return evaluate


def awri(m0, evaluate, eps0, n_iter, eps_min=1e-12, memory=5, first_step=0.05):
    """Algorithm 2 (gamma = 0) with full l-BFGS steps; returns (m, f, status, history)."""
    m = np.asarray(m0, dtype=np.float64).ravel().copy()
    eps = float(eps0)
    S, Y = [], []
    f, g = evaluate(m, eps)
    g = np.asarray(g, dtype=np.float64).ravel()
    history = []
    status = "n_iter"
    for k in range(n_iter):
        while True:
            h0 = None
            if not S:
                gm = np.abs(g).max()
                h0 = first_step * np.abs(m).max() / gm if gm > 0 else 0.0
            m_t = m - two_loop(g, S, Y, h0)
            f_t, g_t = evaluate(m_t, eps)
            g_t = np.asarray(g_t, dtype=np.float64).ravel()
            if f_t <= f:
                break
            if 0.5 * eps < eps_min:
                status = "eps_min"
                break
            eps *= 0.5
            f, g = evaluate(m, eps)
            g = np.asarray(g, dtype=np.float64).ravel()
        if status == "eps_min":
            break
        s, y = m_t - m, g_t - g
        if s @ y > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        m, f, g = m_t, f_t, g_t
        history.append({"iteration": k + 1, "f": f, "eps": eps})
    return m, f, status, history
