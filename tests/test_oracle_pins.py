"""Pins of the CPU oracle against things other than itself (runs without a GPU).

Each test names what it pins: dense least squares, an independent Kronecker
construction of the textbook stencil, exact symmetry, the free-space Green's
function, the small/large penalty limits, the data-consistency invariant with the
paper's printed true source weights, the joint (u, a) block solve, the Krylov
characterisation of CGLS iterates, and central finite differences of f4(m).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(source_free=True, nphys=4, npml=2, freq=20.0, seed=11, nrec=4):
    G = synth.workload_small(nphys=nphys, npml=npml, h=10.0, freq=freq, nsys=1, seed=seed, nrec=nrec)
    shp, n = G.spec.shape, G.spec.n
    A = O.helmholtz_matrix(shp, G.spec.h, G.omega, G.m, npml, G.v_max)
    d = synth.random_complex(len(G.rec_idx), seed + 5)
    return G, shp, n, A, d


# ---------------------------------------------------------------- operator (step a1/a2)
def test_interior_is_textbook_stencil():
    """With no padding, A = omega^2 diag(m) + Laplacian built as a Kronecker sum of
    1-D second differences (Dirichlet), the paper's definition of A_j."""
    nx, ny, nz, h, om = 5, 4, 3, 7.0, 11.0
    m = synth.rng(3).uniform(1e-7, 4e-7, (nz, ny, nx))
    A = O.helmholtz_matrix((nz, ny, nx), h, om, m, npml=0)

    def d2(k):
        return sp.diags([np.ones(k - 1), -2 * np.ones(k), np.ones(k - 1)], [-1, 0, 1]) / h ** 2

    L = (sp.kron(sp.identity(nz), sp.kron(sp.identity(ny), d2(nx)))
         + sp.kron(sp.identity(nz), sp.kron(d2(ny), sp.identity(nx)))
         + sp.kron(d2(nz), sp.kron(sp.identity(ny), sp.identity(nx))))
    ref = (om ** 2 * sp.diags(m.ravel()) + L).toarray()
    assert np.allclose(A.toarray(), ref, rtol=0, atol=1e-15)


def test_operator_complex_symmetric_and_stretch_weight():
    """A^T = A exactly (so A^H = conj(A)); A(m1) - A(m2) = omega^2 diag(w (m1 - m2))."""
    G = synth.workload_small(nphys=5, npml=3, freq=12.0)
    shp = G.spec.shape
    A = O.helmholtz_matrix(shp, G.spec.h, G.omega, G.m, 3, G.v_max)
    assert abs(A - A.T).max() == 0.0
    assert abs(A.imag).max() > 0   # the padding makes it genuinely complex
    m2 = G.m * 1.3
    A2 = O.helmholtz_matrix(shp, G.spec.h, G.omega, m2, 3, G.v_max)
    w = O.stretch_weight(shp, G.spec.h, G.omega, 3, G.v_max)
    D = (A2 - A).tocsr()
    assert np.allclose(D.diagonal(), G.omega ** 2 * w * (m2 - G.m).ravel(), rtol=1e-12, atol=0)
    D.setdiag(0)
    D.eliminate_zeros()
    assert D.nnz == 0
    # interior nodes have w = 1
    z, y, x = (s // 2 for s in shp)
    assert w.reshape(shp)[z, y, x] == 1.0


def test_stretch_zero_padding_and_profile_shape():
    s, sh = O.stretch(12, 0, 10.0, 30.0, 2000.0)
    assert np.all(s == 1) and np.all(sh == 1) and len(sh) == 13
    s, sh = O.stretch(12, 3, 10.0, 30.0, 2000.0)
    assert np.all(s[3:9] == 1) and np.all(sh[4:9] == 1)
    # symmetric profile, increasing damping towards the faces, never decreasing real part
    assert np.allclose(s, s[::-1]) and np.allclose(sh, sh[::-1])
    assert np.all(np.diff(s.imag[:4]) < 0) and np.all(s.real == 1)


@pytest.mark.slow
def test_free_space_greens_function():
    """Homogeneous medium, point source: A^{-1}(a e) ~ -a h^3 exp(i k r)/(4 pi r) for
    3h <= r <= 8h (time convention exp(-i w t), outgoing waves); 16 points per
    wavelength, 8-cell padding.  A wrong sign in the stretch (incoming or growing
    waves), a missing 1/h^2 or a wrong padding weight all fail this."""
    h, v, npml, nph = 10.0, 2000.0, 8, 17
    freq = v / (16 * h)
    g = synth.grid(nph, npml, h)
    m = synth.to_m(synth.velocity_homogeneous(g, v))
    om = 2 * np.pi * freq
    A = O.helmholtz_matrix(g.shape, h, om, m, npml, v)
    c = nph // 2
    src = synth.node_index(g, c, c, c)
    u = spla.splu(A.tocsc()).solve(O.unit_vector(g.n, src) * 1.0)
    k = om / v
    errs = []
    for (dx, dy, dz) in [(3, 0, 0), (0, 4, 0), (0, 0, 5), (4, 3, 0), (6, 0, 0), (5, 5, 3), (0, 0, 8)]:
        r = h * np.sqrt(dx * dx + dy * dy + dz * dz)
        ref = -h ** 3 * np.exp(1j * k * r) / (4 * np.pi * r)
        num = u[synth.node_index(g, c + dx, c + dy, c + dz)]
        errs.append(abs(num - ref) / abs(ref))
    assert max(errs) < 0.05, errs


@pytest.mark.slow
def test_free_space_greens_function_converges_at_second_order():
    """Halving h at a fixed absorbing-layer thickness in metres (8 -> 16 points per wavelength)
    cuts the error against -h^3 exp(i k r)/(4 pi r) at fixed physical points by about 4: the
    7-point stencil is second order.  A misplaced half-node coefficient or a stretch applied on the
    wrong side leaves a first-order (or no) decrease and fails the window."""
    v = 2000.0
    freq = v / (8 * 20.0)
    om, k = 2 * np.pi * freq, 2 * np.pi * freq / v
    offsets_m = [(40, 0, 0), (0, 60, 0), (0, 0, 80), (40, 40, 0), (40, 40, 40), (60, 40, 0), (0, 80, 40)]
    rms = []
    for h, nph, npml in ((20.0, 11, 2), (10.0, 21, 4)):
        g = synth.grid(nph, npml, h)
        A = O.helmholtz_matrix(g.shape, h, om, synth.to_m(synth.velocity_homogeneous(g, v)), npml, v)
        c = nph // 2
        u = spla.splu(A.tocsc()).solve(O.unit_vector(g.n, synth.node_index(g, c, c, c)) * 1.0)
        e = []
        for off in offsets_m:
            di = [int(round(x / h)) for x in off]
            r = h * np.sqrt(sum(x * x for x in di))
            ref = -h ** 3 * np.exp(1j * k * r) / (4 * np.pi * r)
            e.append(abs(u[synth.node_index(g, c + di[0], c + di[1], c + di[2])] - ref) / abs(ref))
        rms.append(np.sqrt(np.mean(np.square(e))))
    assert rms[1] < 0.03, rms
    assert 3.0 <= rms[0] / rms[1] <= 6.0, rms


# ---------------------------------------------------------------- exact solves (step a3)
@pytest.mark.parametrize("source_free", [True, False])
def test_exact_solvers_agree_with_dense_lstsq(source_free):
    G, shp, n, A, d = _tiny()
    P = O.restriction(n, G.rec_idx)
    S = O.augmented_operator(A, P, G.src[0], G.lam, source_free)
    b = O.rhs(n, G.src[0], d, G.lam, G.alpha[0], source_free)
    x_dense = O.solve_dense(S, b)
    x_kkt = O.solve_kkt(S, b)
    x_ds = O.solve_dataspace(spla.splu(A.tocsc()), n, G.src[0], G.rec_idx, d, G.lam, G.alpha[0], source_free)
    x_cg, it, rr = O.cgls(S, b, tol=1e-13, max_iter=50000)
    nrm = np.linalg.norm(x_dense)
    assert np.linalg.norm(x_kkt - x_dense) / nrm < 1e-10
    assert np.linalg.norm(x_ds - x_dense) / nrm < 1e-10
    assert np.linalg.norm(x_cg - x_dense) / nrm < 1e-10
    assert rr <= 1e-13 and it > 0


def test_masked_problem_equals_joint_block_solve():
    """Eq. SimpObj: jointly minimising over (u, a) the matrix [[A, -e], [lam P, 0]]
    gives the same u as the masked problem, and a = (A u)[src]."""
    G, shp, n, A, d = _tiny()
    P = O.restriction(n, G.rec_idx)
    e = O.unit_vector(n, G.src[0])
    J = sp.bmat([[A, -sp.csr_matrix(e).T], [G.lam * P, None]]).toarray()
    bj = np.concatenate([np.zeros(n), G.lam * d])
    xj, *_ = np.linalg.lstsq(J, bj, rcond=None)
    u_j, a_j = xj[:n], xj[n]
    u = O.solve_system(A, n, G.src[0], G.rec_idx, d, G.lam, source_free=True, method="dense")
    assert np.linalg.norm(u - u_j) / np.linalg.norm(u_j) < 1e-10
    assert abs(O.source_estimate(A, u, G.src[0]) - a_j) / abs(a_j) < 1e-10


def test_objective_is_compact_form():
    """f = 1/2 ||S x - b||^2 with the weight eliminated (Eq. CmpctWRIobj)."""
    G, shp, n, A, d = _tiny()
    P = O.restriction(n, G.rec_idx)
    u = synth.random_complex(n, 4)
    a = O.source_estimate(A, u, G.src[0])
    S = O.augmented_operator(A, P, G.src[0], G.lam, True)
    b = O.rhs(n, G.src[0], d, G.lam)
    r = S @ u - b
    assert np.isclose(O.objective(A, P, u, G.src[0], d, G.lam, a), 0.5 * np.vdot(r, r).real, rtol=1e-12)


def test_cgls_iterates_minimise_over_krylov_space():
    """CGLS iterate k minimises ||b - S x|| over span{S^H b, (S^H S) S^H b, ...} (k terms)."""
    G, shp, n, A, d = _tiny()
    P = O.restriction(n, G.rec_idx)
    S = O.augmented_operator(A, P, G.src[0], G.lam, True)
    b = O.rhs(n, G.src[0], d, G.lam)
    Sd = S.toarray()
    N = Sd.conj().T @ Sd
    v = Sd.conj().T @ b
    basis = []
    for k in range(1, 7):
        basis.append(v / np.linalg.norm(v))
        v = N @ basis[-1]
        K = np.column_stack(basis)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(Sd @ Q, b, rcond=None)
        x_ref = Q @ y
        x_k, it, _ = O.cgls(S, b, tol=0.0, max_iter=k)
        assert it == k
        assert np.linalg.norm(x_k - x_ref) / np.linalg.norm(x_ref) < 1e-8, k


# ---------------------------------------------------------------- limits (step a3/a7)
def test_small_lambda_source_free_limit():
    """lam -> 0: u -> c A^{-1} e with c = (P G)^H d / ||P G||^2 (the reduced-FWI
    solution of Eq. FWI2 with the best weight); error shrinks like lam^2."""
    G, shp, n, A, d = _tiny()
    lu = spla.splu(A.tocsc())
    Ge = lu.solve(O.unit_vector(n, G.src[0]))
    PG = Ge[G.rec_idx]
    u0 = (np.vdot(PG, d) / np.vdot(PG, PG)) * Ge
    errs = []
    for lam in (1e-2 * G.lam, 1e-3 * G.lam):
        u = O.solve_dataspace(lu, n, G.src[0], G.rec_idx, d, lam)
        errs.append(np.linalg.norm(u - u0) / np.linalg.norm(u0))
    assert errs[1] < 1e-3
    assert 50 < errs[0] / errs[1] < 200     # O(lam^2)


def test_small_lambda_known_weight_limit():
    """lam -> 0 with a known weight: u -> A^{-1}(a e), the PDE solve of Eq. PDEsolve."""
    G, shp, n, A, d = _tiny()
    lu = spla.splu(A.tocsc())
    u0 = lu.solve(G.alpha[0] * O.unit_vector(n, G.src[0]))
    u = O.solve_dataspace(lu, n, G.src[0], G.rec_idx, d, 1e-4 * G.lam, G.alpha[0], source_free=False)
    assert np.linalg.norm(u - u0) / np.linalg.norm(u0) < 1e-5


def test_large_lambda_fits_data():
    """lam -> infinity: ||P u - d|| = O(lam^-2)."""
    G, shp, n, A, d = _tiny()
    lu = spla.splu(A.tocsc())
    res = []
    for lam in (1e2 * G.lam, 1e3 * G.lam):
        u = O.solve_dataspace(lu, n, G.src[0], G.rec_idx, d, lam)
        res.append(np.linalg.norm(u[G.rec_idx] - d) / np.linalg.norm(d))
    assert res[1] < 1e-3 and 50 < res[0] / res[1] < 200


def test_data_consistency_recovers_paper_weights():
    """Noise-free data from the true model and the paper's printed true weights
    (Table SrcCam): at the true model the source-free estimate returns the weight,
    u = a A^{-1} e, f = 0 and g = 0."""
    with open(os.path.join(GOLDEN, "paper_source_weights.json")) as fh:
        gold = json.load(fh)
    for key in ("5Hz", "6Hz"):
        a_t = complex(*gold["alpha_true"][key])
        G = synth.workload_small(nphys=6, npml=3, freq=float(key[:-2]) * 3, nsys=1, nrec=5)
        shp, n = G.spec.shape, G.spec.n
        d = O.forward_data(shp, G.spec.h, G.omega, G.m, 3, G.v_max, G.src, G.rec_off, G.rec_idx, np.array([a_t]))
        u, a, f, g = O.evaluate(shp, G.spec.h, G.omega, G.m, 3, G.v_max, G.src, G.rec_off, G.rec_idx, d, G.lam)
        A = O.helmholtz_matrix(shp, G.spec.h, G.omega, G.m, 3, G.v_max)
        u_t = spla.spsolve(A.tocsc(), a_t * O.unit_vector(n, G.src[0]))
        assert abs(a[0] - a_t) / abs(a_t) < 1e-9
        assert np.linalg.norm(u[0] - u_t) / np.linalg.norm(u_t) < 1e-9
        # away from the true model f and g are clearly non-zero
        _, _, f1, g1 = O.evaluate(shp, G.spec.h, G.omega, G.m * 1.05, 3, G.v_max, G.src, G.rec_off,
                                  G.rec_idx, d, G.lam)
        assert f < 1e-16 * max(f1, 1e-300) * 1e6 and f1 > 0
        assert np.linalg.norm(g) < 1e-8 * np.linalg.norm(g1)


def test_paper_initial_weight_error_formula():
    """The printed initial error 34.4 % of Table SrcCam equals ||a0 - at|| / ||at||
    over both frequencies (inputs are printed to 2-3 digits, hence 0.2 % slack)."""
    with open(os.path.join(GOLDEN, "paper_source_weights.json")) as fh:
        gold = json.load(fh)
    at = np.array([complex(*gold["alpha_true"][k]) for k in ("5Hz", "6Hz")])
    a0 = np.array([complex(*gold["alpha_initial"][k]) for k in ("5Hz", "6Hz")])
    err = 100 * np.linalg.norm(a0 - at) / np.linalg.norm(at)
    assert abs(err - gold["initial_relative_error_percent"]) < 0.2


# ---------------------------------------------------------------- gradient (step a8)
@pytest.mark.parametrize("source_free", [True, False])
def test_gradient_matches_central_differences(source_free):
    """g4 (Eq. VarG2) equals the central difference of f4(m) = f at the exact
    minimiser; no adjoint solve is involved (variable projection)."""
    G = synth.workload_small(nphys=5, npml=2, freq=15.0, nsys=2, nrec=5)
    shp, n = G.spec.shape, G.spec.n
    d = O.forward_data(shp, G.spec.h, G.omega, G.m * 1.03, 2, G.v_max, G.src, G.rec_off, G.rec_idx, G.alpha)
    alpha = None if source_free else G.alpha * 0.9

    def f_of(m):
        return O.evaluate(shp, G.spec.h, G.omega, m, 2, G.v_max, G.src, G.rec_off, G.rec_idx, d, G.lam,
                          alpha=alpha, source_free=source_free)

    _, _, f0, g = f_of(G.m)
    r = synth.rng(9)
    for _ in range(3):
        dm = r.standard_normal(shp) * G.m
        eps = 1e-4
        fp = f_of(G.m + eps * dm)[2]
        fm = f_of(G.m - eps * dm)[2]
        fd = (fp - fm) / (2 * eps)
        an = float(g @ dm.ravel())
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


# ---------------------------------------------------------------- outer loop (Algorithm 2)
def test_two_loop_recursion_equals_dense_bfgs_inverse():
    """The l-BFGS two-loop product equals the dense inverse-Hessian BFGS update applied to g."""
    from oracle.awri_oracle import bfgs_inverse, two_loop
    r = synth.rng(23)
    n = 9
    Q = r.standard_normal((n, n))
    Q = Q @ Q.T + n * np.eye(n)
    S = [r.standard_normal(n) for _ in range(4)]
    Y = [Q @ s for s in S]                       # curvature pairs of a convex quadratic (s.y > 0)
    g = r.standard_normal(n)
    assert np.allclose(two_loop(g, S, Y), bfgs_inverse(S, Y) @ g, rtol=1e-12, atol=1e-12)
    # with one pair the inverse Hessian maps y to s (secant condition)
    assert np.allclose(two_loop(Y[-1], S[-1:], Y[-1:]), S[-1], rtol=1e-12)


def test_awri_oracle_minimises_a_convex_quadratic():
    """With exact evaluations Algorithm 2 reduces to full-step l-BFGS: on a well-conditioned
    quadratic the first 10 steps all decrease f and close in on the minimiser, and eps is never
    halved.  (Without a line search a later full step can fail; halving eps cannot help exact
    evaluations, so the loop then ends at eps_min, as the adaptive rule prescribes.)"""
    from oracle.awri_oracle import awri
    r = synth.rng(5)
    n = 12
    U, _ = np.linalg.qr(r.standard_normal((n, n)))
    Q = U @ np.diag(np.linspace(1.0, 10.0, n)) @ U.T
    m_star = r.uniform(1.0, 2.0, n)

    def evaluate(m, eps):
        e = m - m_star
        return 0.5 * e @ Q @ e, Q @ e

    m0 = np.full(n, 1.5)
    m, f, status, hist = awri(m0, evaluate, 1e-2, 10, first_step=0.05)
    assert status == "n_iter" and len(hist) == 10
    assert np.linalg.norm(m - m_star) < 1e-3 * np.linalg.norm(m0 - m_star)
    assert all(h["eps"] == 1e-2 for h in hist)
    assert all(a["f"] > b["f"] for a, b in zip(hist, hist[1:]))


def test_awri_oracle_halves_eps_until_the_step_decreases_f():
    """The adaptive rule: a step whose objective (at the current eps) does not decrease is
    refused, eps is halved and f, g are evaluated again at the same model."""
    from oracle.awri_oracle import awri
    calls = []

    def evaluate(m, eps):
        calls.append(eps)
        # exact part 1/2 |m|^2, plus an eps-sized bias that grows away from the start point
        return 0.5 * m @ m + 50.0 * eps * abs(m[0] - 1.0), m.copy()

    m, f, status, hist = awri(np.array([1.0, 1.0]), evaluate, 0.1, 1, first_step=0.5)
    # eps 0.1: f~ = 0.25 + 2.5 > 1.0 -> halve; 0.05: 0.25 + 1.25 > 1.0 -> halve; 0.025: accept
    assert calls == [0.1, 0.1, 0.05, 0.05, 0.025, 0.025]
    assert hist == [{"iteration": 1, "f": 0.25 + 50.0 * 0.025 * 0.5, "eps": 0.025}]
    m, f, status, hist = awri(np.array([1.0, 1.0]), evaluate, 0.1, 1, first_step=0.5, eps_min=0.04)
    assert status == "eps_min" and hist == []


# ---------------------------------------------------------------- TV term (Eq. TVAWRI)
def test_total_variation_pins():
    """Constant model: TV = n beta, zero gradient.  One planar step of height c across a face
    of n_face nodes: TV = (n - n_face) beta + n_face sqrt(c^2 + beta^2).  Gradient: central
    differences on random directions."""
    shp = (5, 6, 7)
    n = 5 * 6 * 7
    tv, g = O.total_variation(np.full(shp, 3.0), 0.1)
    assert np.isclose(tv, n * 0.1, rtol=1e-14) and np.abs(g).max() == 0.0
    m = np.zeros(shp)
    m[:, :, 4:] = 2.0                       # step between x = 3 and x = 4
    tv, _ = O.total_variation(m, 0.1)
    n_face = 5 * 6
    assert np.isclose(tv, (n - n_face) * 0.1 + n_face * np.sqrt(4.0 + 0.01), rtol=1e-14)
    r = synth.rng(31)
    m = r.standard_normal(shp)
    tv, g = O.total_variation(m, 0.3)
    for _ in range(3):
        dm = r.standard_normal(shp)
        eps = 1e-6
        fd = (O.total_variation(m + eps * dm, 0.3)[0] - O.total_variation(m - eps * dm, 0.3)[0]) / (2 * eps)
        assert abs(fd - float((g * dm).sum())) <= 1e-7 * abs(fd)
