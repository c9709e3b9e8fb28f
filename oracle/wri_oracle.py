"""Oracle: complex128 restatement of the WRI augmented least-squares problem.

TEST INFRASTRUCTURE ONLY: used by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product path.

Notation follows the paper's Methodology section.
  * m        squared slowness on the grid (Sec. "3D Source free WRI", first paragraph)
  * A_j      discretised Helmholtz matrix omega_j^2 diag(m) + Laplacian (same paragraph),
             here with a stretched-coordinate absorbing layer (our reading, see ``stretch``)
  * P_i, e_i receiver restriction and source unit vector (same paragraph)
  * f2       penalty objective (Eq. ObjPen); S, b the compact form (Eqs. CmpctWRIobj, Sandb)
  * (u, a)   variable-projection minimiser (Eq. SimpObj), f4 = f2 at it (Eq. VarObj2)
  * g4       gradient (Eq. VarG2)

Readings (the paper is silent or garbled on these):
  * the penalty weight lambda multiplies the DATA term:
        f = 1/2 ||A u - a e||^2 + 1/2 lambda^2 ||P u - d||^2,
    the paper's lambda_p on the PDE term is lambda = 1/lambda_p, f_paper = lambda_p^2 f;
    the minimiser (u, a) is the same;
  * transposes of complex operators are conjugate transposes;
  * eliminating the source weight from the 2x2 block system of Eq. SimpObj gives
    a = e^H A u and the masked problem min 1/2 ||Z A u||^2 + 1/2 lambda^2 ||P u - d||^2
    with Z = I - e e^H ("source-free" mode);
  * LSQR (Algorithm 1, whose printed listing is inconsistent) is taken as CGLS,
    which has the same iterates in exact arithmetic; the stopping test is the
    relative normal-equation residual ||S^H (b - S x)|| / ||S^H b||;
  * the gradient uses the frequency of the system (omega_j) and takes the real part
    (m is real), with the stretch weight w multiplying m inside A.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "stretch", "helmholtz_matrix", "apply_helmholtz", "restriction", "unit_vector",
    "augmented_operator", "rhs", "solve_kkt", "solve_dataspace", "solve_dense", "stretch_weight", "cgls", "source_estimate",
    "objective", "gradient", "solve_system", "evaluate", "fwi_evaluate", "forward_data", "total_variation",
]


# --------------------------------------------------------------------------------------
# Step a1: absorbing-layer stretch factors (our reading; the paper states no boundary)
# --------------------------------------------------------------------------------------
def stretch(n: int, npml: int, h: float, omega: float, v_max: float, R: float = 1e-3):
    """Complex stretch factors of one axis.

    s(xi) = 1 + i sigma(xi)/omega with sigma(xi) = sigma_max (xi/L)^2,
    L = npml*h and sigma_max = 3 v_max ln(1/R) / (2 L); xi is the distance into
    the padding measured from the last physical node.

    Returns (s_node[n], s_half[n+1]); s_half[k] sits at position k - 1/2, so
    s_half[0] and s_half[n] are the half points just outside the grid.
    """
    pos_node = np.arange(n, dtype=np.float64)
    pos_half = np.arange(n + 1, dtype=np.float64) - 0.5

    def s_of(pos):
        if npml <= 0:
            return np.ones(pos.shape, dtype=np.complex128)
        L = npml * h
        smax = 3.0 * v_max * np.log(1.0 / R) / (2.0 * L)
        xi = np.zeros_like(pos)
        left = pos < npml
        right = pos > (n - 1 - npml)
        xi[left] = (npml - pos[left]) * h
        xi[right] = (pos[right] - (n - 1 - npml)) * h
        sigma = smax * (xi / L) ** 2
        return 1.0 + 1j * sigma / omega

    return s_of(pos_node), s_of(pos_half)


def _coeffs(shape, h, omega, npml, v_max, R):
    nz, ny, nx = shape
    sx, sxh = stretch(nx, npml, h, omega, v_max, R)
    sy, syh = stretch(ny, npml, h, omega, v_max, R)
    sz, szh = stretch(nz, npml, h, omega, v_max, R)
    return (sx, sxh), (sy, syh), (sz, szh)


# --------------------------------------------------------------------------------------
# The Helmholtz matrix A = omega^2 diag(w m) + L (paper: A = omega^2 diag(m) + Laplacian)
# --------------------------------------------------------------------------------------
def helmholtz_matrix(shape, h, omega, m, npml=0, v_max=1.0, R=1e-3) -> sp.csr_matrix:
    """Sparse complex-symmetric 7-point Helmholtz matrix with stretched coordinates.

    Row for node (i, j, k):
        omega^2 w m u + sum over axes of  c(+1/2) (u_next - u) - c(-1/2) (u - u_prev)
    with w = sx(i) sy(j) sz(k) and, for the x axis, c(i +- 1/2) = sy(j) sz(k) / (sx(i +- 1/2) h^2)
    (likewise for y and z).  Nodes outside the grid are zero (Dirichlet).
    With npml = 0 this is omega^2 diag(m) plus the textbook 7-point Laplacian.
    """
    nz, ny, nx = shape
    n = nx * ny * nz
    (sx, sxh), (sy, syh), (sz, szh) = _coeffs(shape, h, omega, npml, v_max, R)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    K, J, I = K.ravel(), J.ravel(), I.ravel()
    row = (K * ny + J) * nx + I
    m = np.asarray(m, dtype=np.float64).ravel()
    w = sx[I] * sy[J] * sz[K]
    h2 = h * h
    # coefficients on the six half points of every node
    cxp = sy[J] * sz[K] / (sxh[I + 1] * h2)
    cxm = sy[J] * sz[K] / (sxh[I] * h2)
    cyp = sx[I] * sz[K] / (syh[J + 1] * h2)
    cym = sx[I] * sz[K] / (syh[J] * h2)
    czp = sx[I] * sy[J] / (szh[K + 1] * h2)
    czm = sx[I] * sy[J] / (szh[K] * h2)
    diag = omega ** 2 * w * m - (cxp + cxm + cyp + cym + czp + czm)
    rows, cols, vals = [row], [row], [diag]
    for c, ok, off in ((cxp, I + 1 < nx, 1), (cxm, I - 1 >= 0, -1),
                       (cyp, J + 1 < ny, nx), (cym, J - 1 >= 0, -nx),
                       (czp, K + 1 < nz, nx * ny), (czm, K - 1 >= 0, -nx * ny)):
        rows.append(row[ok])
        cols.append(row[ok] + off)
        vals.append(c[ok])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    return A


def apply_helmholtz(shape, h, omega, m, u, npml=0, v_max=1.0, R=1e-3, adjoint=False):
    """y = A u (or A^H u) for one vector, through the sparse matrix."""
    A = helmholtz_matrix(shape, h, omega, m, npml, v_max, R)
    return (A.conj().T @ u) if adjoint else (A @ u)


def restriction(n: int, rec_idx) -> sp.csr_matrix:
    """P: picks the receiver nodes (one row per receiver)."""
    rec_idx = np.asarray(rec_idx, dtype=np.int64)
    nr = len(rec_idx)
    return sp.csr_matrix((np.ones(nr), (np.arange(nr), rec_idx)), shape=(nr, n), dtype=np.complex128)


def unit_vector(n: int, idx: int) -> np.ndarray:
    e = np.zeros(n, dtype=np.complex128)
    e[int(idx)] = 1.0
    return e


# --------------------------------------------------------------------------------------
# Compact least-squares form (Eqs. CmpctWRIobj / Sandb) in the data-weighted convention
# --------------------------------------------------------------------------------------
def augmented_operator(A, P, src, lam, source_free=True) -> sp.csr_matrix:
    """S = [Z A ; lam P] (source-free, Z = I - e e^H) or [A ; lam P] (known weight)."""
    n = A.shape[0]
    if source_free:
        z = np.ones(n)
        z[int(src)] = 0.0
        top = sp.diags(z) @ A
    else:
        top = A
    return sp.vstack([top, lam * P]).tocsr()


def rhs(n, src, d, lam, alpha=None, source_free=True) -> np.ndarray:
    """b = [0 ; lam d] (source-free) or [alpha e ; lam d] (known weight)."""
    top = np.zeros(n, dtype=np.complex128)
    if not source_free:
        top[int(src)] = alpha
    return np.concatenate([top, lam * np.asarray(d, dtype=np.complex128)])


# --------------------------------------------------------------------------------------
# Solvers of min ||S x - b||
# --------------------------------------------------------------------------------------
def solve_kkt(S, b) -> np.ndarray:
    """Exact least-squares solution through a sparse LU of [[I, S], [S^H, 0]]."""
    M, n = S.shape
    K = sp.bmat([[sp.identity(M, dtype=np.complex128, format="csr"), S],
                 [S.conj().T, None]], format="csc")
    rhs_ = np.concatenate([b, np.zeros(n, dtype=np.complex128)])
    lu = spla.splu(K, permc_spec="COLAMD", diag_pivot_thresh=1.0)
    sol = lu.solve(rhs_)
    return sol[M:]


def solve_dataspace(lu, n, src, rec, d, lam, alpha=None, source_free=True) -> np.ndarray:
    """Exact solution through one LU of A (the receiver-space form of the same problem).

    Write u = A^{-1}(a e + v).  Then A u - a e = v and the objective becomes
    1/2 ||v||^2 + 1/2 lam^2 ||G v - (d - a g)||^2 with G = P A^{-1}, g = P A^{-1} e.
    Its minimiser is v = lam^2 G^H W (d - a g), W = (I + lam^2 G G^H)^{-1}, and in
    source-free mode the weight minimising 1/2 lam^2 (d - a g)^H W (d - a g) is
    a = g^H W d / g^H W g.  ``lu`` is ``scipy.sparse.linalg.splu(A)``.
    """
    rec = np.asarray(rec, dtype=np.int64)
    d = np.asarray(d, dtype=np.complex128)
    nr = len(rec)
    e = unit_vector(n, src)
    GH = np.zeros((n, nr), dtype=np.complex128)           # A^{-H} P^T, one column per receiver
    for k in range(nr):
        GH[:, k] = lu.solve(unit_vector(n, rec[k]), trans="H")
    GGH = GH.conj().T @ GH
    W = np.linalg.inv(np.eye(nr) + lam ** 2 * GGH)
    g = lu.solve(e)[rec]
    a = (g.conj() @ (W @ d)) / (g.conj() @ (W @ g)) if source_free else alpha
    v = lam ** 2 * (GH @ (W @ (d - a * g)))
    return lu.solve(a * e + v)


def solve_dense(S, b) -> np.ndarray:
    """Exact least-squares solution by dense SVD-based lstsq (tiny grids only)."""
    x, *_ = np.linalg.lstsq(S.toarray(), b, rcond=None)
    return x


def cgls(S, b, tol=1e-12, max_iter=100000, x0=None, history=False):
    """CG on the normal equations S^H S x = S^H b in least-squares form (CGLS).

    Steps per iteration (Algorithm 1 read as CGLS):
        t = S p; alpha = gamma / ||t||^2; x += alpha p; r -= alpha t;
        s = S^H r; gamma' = ||s||^2; stop if sqrt(gamma')/||S^H b|| <= tol;
        beta = gamma'/gamma; p = s + beta p.
    Returns (x, iterations, relres[, relres history]).
    """
    SH = S.conj().T.tocsr()
    x = np.zeros(S.shape[1], dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - S @ x
    s = SH @ r
    ref = np.linalg.norm(SH @ b)
    p = s.copy()
    gamma = np.vdot(s, s).real
    hist = []
    it = 0
    relres = np.sqrt(gamma) / ref if ref > 0 else 0.0
    while it < max_iter and relres > tol:
        t = S @ p
        delta = np.vdot(t, t).real
        alpha = gamma / delta
        x = x + alpha * p
        r = r - alpha * t
        s = SH @ r
        gamma_new = np.vdot(s, s).real
        it += 1
        relres = np.sqrt(gamma_new) / ref
        hist.append(relres)
        if relres <= tol:
            break
        beta = gamma_new / gamma
        gamma = gamma_new
        p = s + beta * p
    if history:
        return x, it, relres, np.array(hist)
    return x, it, relres


# --------------------------------------------------------------------------------------
# Source estimate, objective, gradient (Eqs. SimpObj, VarObj2, VarG2)
# --------------------------------------------------------------------------------------
def source_estimate(A, u, src) -> complex:
    """a = e^H A u: the minimiser over the weight of 1/2 ||A u - a e||^2."""
    return complex((A @ u)[int(src)])


def objective(A, P, u, src, d, lam, alpha) -> float:
    """1/2 ||A u - alpha e||^2 + 1/2 lam^2 ||P u - d||^2 (Eq. ObjPen, data-weighted)."""
    r1 = A @ u
    r1[int(src)] -= alpha
    r2 = P @ u - d
    return 0.5 * np.vdot(r1, r1).real + 0.5 * lam ** 2 * np.vdot(r2, r2).real


def gradient(A, u, src, alpha, omega, w) -> np.ndarray:
    """omega^2 Re( conj(w u) * (A u - alpha e) ), the model gradient of one system (Eq. VarG2)."""
    r1 = A @ u
    r1[int(src)] -= alpha
    return omega ** 2 * np.real(np.conj(w * u) * r1)


def stretch_weight(shape, h, omega, npml, v_max, R=1e-3) -> np.ndarray:
    """w = sx sy sz on every node (the factor multiplying omega^2 m in A)."""
    (sx, _), (sy, _), (sz, _) = _coeffs(shape, h, omega, npml, v_max, R)
    return (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]).ravel()


def solve_system(A, n, src, rec, d, lam, alpha=None, source_free=True, method="kkt", tol=1e-12,
                 max_iter=200000):
    """Wavefield of one system: u = argmin of the (masked or known-weight) problem."""
    P = restriction(n, rec)
    S = augmented_operator(A, P, src, lam, source_free)
    b = rhs(n, src, d, lam, alpha, source_free)
    if method == "kkt":
        return solve_kkt(S, b)
    if method == "dense":
        return solve_dense(S, b)
    if method == "cgls":
        return cgls(S, b, tol=tol, max_iter=max_iter)[0]
    raise ValueError(method)


def evaluate(shape, h, omega, m, npml, v_max, srcs, rec_off, rec_idx, d, lam, alpha=None,
             source_free=True, method="dataspace", R=1e-3, tol=1e-12):
    """Solve every system of one frequency group and return (u[nsys, n], a[nsys], f, g[n]).

    f and g sum over the systems; a is the estimated weight (source-free) or the
    given one (known-weight mode).
    """
    n = int(np.prod(shape))
    A = helmholtz_matrix(shape, h, omega, m, npml, v_max, R)
    w = stretch_weight(shape, h, omega, npml, v_max, R)
    lu = spla.splu(A.tocsc()) if method == "dataspace" else None
    us, als = [], []
    f = 0.0
    g = np.zeros(n)
    for s in range(len(srcs)):
        rec = rec_idx[rec_off[s]:rec_off[s + 1]]
        ds = d[rec_off[s]:rec_off[s + 1]]
        a_in = None if alpha is None else alpha[s]
        if method == "dataspace":
            u = solve_dataspace(lu, n, srcs[s], rec, ds, lam, a_in, source_free)
        else:
            u = solve_system(A, n, srcs[s], rec, ds, lam, a_in, source_free, method, tol)
        a = source_estimate(A, u, srcs[s]) if source_free else a_in
        P = restriction(n, rec)
        f += objective(A, P, u, srcs[s], ds, lam, a)
        g += gradient(A, u, srcs[s], a, omega, w)
        us.append(u)
        als.append(a)
    return np.array(us), np.array(als), f, g


def fwi_evaluate(shape, h, omega, m, npml, v_max, srcs, rec_off, rec_idx, d, alpha=None, R=1e-3):
    """Reduced FWI, the paper's comparison method (Eqs. PDEsolve and FWI2), by exact LU solves.

    Per system: G = A^{-1} e, the weight a (given, or source-free the minimiser of
    ||a P G - d||: a = (P G)^H d / ||P G||^2), u = a G (Eq. PDEsolve), the data residual
    r = P u - d, f = 1/2 sum ||r||^2 (Eq. FWI2), and the adjoint-state gradient
    g = -omega^2 sum Re(w u conj(v)) with v = A^{-H} P^T r (dA/dm_k = omega^2 w_k e_k e_k^T; the
    weight's own derivative vanishes at its optimum).  Returns (u[nsys, n], a[nsys], f, g[n]).
    """
    n = int(np.prod(shape))
    A = helmholtz_matrix(shape, h, omega, m, npml, v_max, R)
    w = stretch_weight(shape, h, omega, npml, v_max, R)
    lu = spla.splu(A.tocsc())
    us, als = [], []
    f = 0.0
    g = np.zeros(n)
    for s in range(len(srcs)):
        rec = np.asarray(rec_idx[rec_off[s]:rec_off[s + 1]], dtype=np.int64)
        ds = np.asarray(d[rec_off[s]:rec_off[s + 1]], dtype=np.complex128)
        Ge = lu.solve(unit_vector(n, srcs[s]))
        PG = Ge[rec]
        a = (np.vdot(PG, ds) / np.vdot(PG, PG)) if alpha is None else complex(alpha[s])
        u = a * Ge
        r = u[rec] - ds
        rhs_adj = np.zeros(n, dtype=np.complex128)
        rhs_adj[rec] = r
        v = lu.solve(rhs_adj, trans="H")
        f += 0.5 * np.vdot(r, r).real
        g += -omega ** 2 * np.real(w * u * np.conj(v))
        us.append(u)
        als.append(a)
    return np.array(us), np.array(als), f, g


def forward_data(shape, h, omega, m_true, npml, v_max, srcs, rec_off, rec_idx, alpha, R=1e-3):
    """Noise-free data d = P A(m_true)^{-1} (alpha e) (the PDE solve of Eq. PDEsolve)."""
    n = int(np.prod(shape))
    A = helmholtz_matrix(shape, h, omega, m_true, npml, v_max, R).tocsc()
    lu = spla.splu(A)
    out = np.zeros(int(rec_off[-1]), dtype=np.complex128)
    for s in range(len(srcs)):
        u = lu.solve(alpha[s] * unit_vector(n, srcs[s]))
        out[rec_off[s]:rec_off[s + 1]] = u[rec_idx[rec_off[s]:rec_off[s + 1]]]
    return out


# --------------------------------------------------------------------------------------
# Total-variation term of Eq. TVAWRI (our reading of the paper's ||m||_TV)
# --------------------------------------------------------------------------------------
def total_variation(m, beta):
    """Smoothed isotropic TV of a model on its grid and its gradient.

    TV(m) = sum over nodes of sqrt(dx^2 + dy^2 + dz^2 + beta^2), with forward differences in
    grid units (dx = m[i+1] - m[i], zero on the last node of an axis).  The gradient is the
    derivative of that sum; the paper's weight gamma multiplies both.  Returns (TV, grad).
    """
    m = np.asarray(m, dtype=np.float64)
    d = []
    for ax in range(3):
        da = np.zeros_like(m)
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        da[tuple(sl_lo)] = m[tuple(sl_hi)] - m[tuple(sl_lo)]
        d.append(da)
    q = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + beta ** 2)
    grad = np.zeros_like(m)
    for ax in range(3):
        w = d[ax] / q                     # derivative of q with respect to the difference
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        grad[tuple(sl_lo)] -= w[tuple(sl_lo)]
        grad[tuple(sl_hi)] += w[tuple(sl_lo)]
    return float(q.sum()), grad
