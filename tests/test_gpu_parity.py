"""GPU parity: libwri (through the C ABI) against the CPU oracle.

Tolerances: complex128 path to 1e-10 (rounding only); complex64 stencils to 1e-6
relative per application; converged wavefields to rel-L2 1e-5 and gradients to
1e-4 against the oracle's exact (LU) solution, as the target states.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
import synth
from wri_cases import case, oracle_A, rel, seen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_18429_gb300 import wri
    return wri


def _spec(W, G, dtype, source_free=True, u=None):
    from paper_2410_18429_gb300.problem import to_device
    return to_device(G, dtype, "cuda", source_free=source_free, u=u)


# ------------------------------------------------------------------ operator (a1, a2)
@pytest.mark.parametrize("dtype,tol", [(1, 1e-12), (0, 2e-6)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_apply_matches_sparse_operator(W, dtype, tol, adjoint):
    """Ragged grid spanning several 32 x 8 tiles in x and y, 3 vectors."""
    G = case(nphys=(45, 21, 9), npml=5, nsys=3, with_data=False)
    m, _, _ = seen(G, dtype == 0)
    A = oracle_A(G, m)
    x = synth.random_complex((3, G.spec.n), 7)
    if dtype == 0:
        x = x.astype(np.complex64).astype(np.complex128)
    spec = _spec(W, G, dtype)
    xt = torch.as_tensor(x, dtype=spec.u.dtype).cuda()
    y = W.apply_A(spec, xt, adjoint=adjoint).cpu().numpy()
    Aop = A.conj().T if adjoint else A
    for s in range(3):
        ref = Aop @ x[s]
        assert rel(y[s], ref) < tol
        # every entry, not just the norm (catches a wrong neighbour on one face)
        assert np.max(np.abs(y[s] - ref)) <= 10 * tol * np.max(np.abs(ref))


def test_adjoint_identity_on_gpu(W):
    G = case(nphys=(33, 17, 12), npml=4, nsys=1, with_data=False)
    spec = _spec(W, G, 1)
    x = torch.as_tensor(synth.random_complex((1, G.spec.n), 1)).cuda()
    y = torch.as_tensor(synth.random_complex((1, G.spec.n), 2)).cuda()
    Ax = W.apply_A(spec, x)
    AHy = W.apply_A(spec, y, adjoint=True)
    lhs = torch.vdot(y.ravel(), Ax.ravel())
    rhs = torch.vdot(AHy.ravel(), x.ravel())
    assert abs(lhs - rhs) / (Ax.norm() * y.norm()) < 1e-13


# ------------------------------------------------------------------ CGLS iterates (a3)
@pytest.mark.parametrize("dtype,tol", [(1, 1e-10), (0, 3e-4)])
@pytest.mark.parametrize("source_free", [True, False])
def test_fixed_iterations_match_oracle_cgls(W, dtype, tol, source_free):
    G = case(nphys=(37, 13, 10), npml=4, nsys=2)
    m, d, al = seen(G, dtype == 0)
    A = oracle_A(G, m)
    spec = _spec(W, G, dtype, source_free)
    k = 25
    it, rr, st = W.solve([spec], W.make_opts(tol=0.0, max_iter=k, dtype=dtype))
    u = spec.u.cpu().numpy()
    assert it.cpu().tolist() == [k, k]
    assert st.cpu().tolist() == [W.SYS_MAXITER] * 2
    for s in range(2):
        rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
        P = O.restriction(G.spec.n, rec)
        S = O.augmented_operator(A, P, G.src[s], G.lam, source_free)
        b = O.rhs(G.spec.n, G.src[s], d[G.rec_off[s]:G.rec_off[s + 1]], G.lam, al[s], source_free)
        x_k, _, rr_k = O.cgls(S, b, tol=0.0, max_iter=k)
        assert rel(u[s], x_k) < tol, rel(u[s], x_k)
        assert abs(rr.cpu().numpy()[s] - rr_k) <= max(tol, 1e-6) * rr_k * 10


@pytest.mark.parametrize("cfg", list(range(25)))
@pytest.mark.parametrize("source_free", [True, False])
def test_tma_phases_match_oracle_and_march(W, cfg, source_free):
    """TMA-pipelined phases (x extent a multiple of 4; configurations 9-24 are the
    warp-specialised kernels): ragged 32 x BY tiles, iterates of k CGLS steps equal the
    oracle's and the z-march kernels' (same tile height)."""
    G = case(nphys=(36, 13, 10), npml=4, nsys=3)
    m, d, al = seen(G, True)
    A = oracle_A(G, m)
    k = 25
    by = 16 if cfg in (2, 3, 4, 5, 12, 16) else 8
    s_t, s_m = _spec(W, G, 0, source_free), _spec(W, G, 0, source_free)
    it_t, rr_t, st_t = W.solve([s_t], W.make_opts(tol=0.0, max_iter=k, dtype=0, kernel=W.KERNEL_TMA(cfg)))
    it_m, rr_m, st_m = W.solve([s_m], W.make_opts(tol=0.0, max_iter=k, dtype=0, kernel=W.KERNEL_MARCH,
                                                 tile=3 if by == 16 else 2))
    assert it_t.cpu().tolist() == [k] * 3
    u_t, u_m = s_t.u.cpu().numpy(), s_m.u.cpu().numpy()
    assert rel(u_t, u_m) < 1e-5
    for s in range(3):
        rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
        S = O.augmented_operator(A, O.restriction(G.spec.n, rec), G.src[s], G.lam, source_free)
        b = O.rhs(G.spec.n, G.src[s], d[G.rec_off[s]:G.rec_off[s + 1]], G.lam, al[s], source_free)
        x_k, _, _ = O.cgls(S, b, tol=0.0, max_iter=k)
        assert rel(u_t[s], x_k) < 3e-4


def _oracle_iterates(G, m, d, al, source_free, k):
    """The oracle's k-th CGLS iterate and its residual ||S^H (b - S x_k)|| / ||S^H b|| per system."""
    A = oracle_A(G, m)
    out = []
    for s in range(G.nsys):
        rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
        S = O.augmented_operator(A, O.restriction(G.spec.n, rec), G.src[s], G.lam, source_free)
        b = O.rhs(G.spec.n, G.src[s], d[G.rec_off[s]:G.rec_off[s + 1]], G.lam, al[s], source_free)
        x_k, _, rr_k = O.cgls(S, b, tol=0.0, max_iter=k)
        out.append((x_k, rr_k))
    return out


def _interior_case():
    """80 x 32 x 18 computational nodes (72 x 24 x 10 + 4-cell layer): the x tile 32..63 and the y
    tiles 8..15 and 16..23 lie inside the layer's inner edge (nodes 5..74 in x, 5..26 in y), so the
    phase kernels take their plain 7-point variant there (planes 5..12), the layer variants on the
    other tiles, and a ragged 16-wide tail in x."""
    return case(nphys=(72, 24, 10), npml=4, nsys=3, seed=12)


@pytest.mark.parametrize("cfg", [9, 18])
@pytest.mark.parametrize("order", [0, 6])
@pytest.mark.parametrize("zsplit", [1, 0])
def test_interior_tiles_tma_match_oracle(W, cfg, order, zsplit):
    """Warp-specialised TMA phases (configuration 9, the default, and 18, early stage release) on a
    grid with interior tiles: k CGLS iterates and the reported residuals equal the oracle's, element
    by element, with one z-chunk per tile column and with the automatic z-split (4 chunks)."""
    G = _interior_case()
    m, d, al = seen(G, True)
    k = 25
    spec = _spec(W, G, 0)
    it, rr, st = W.solve([spec], W.make_opts(tol=0.0, max_iter=k, dtype=0, kernel=W.KERNEL_TMA(cfg),
                                             order=order, zsplit=zsplit))
    assert it.cpu().tolist() == [k] * 3 and st.cpu().tolist() == [W.SYS_MAXITER] * 3
    u, rr = spec.u.cpu().numpy(), rr.cpu().numpy()
    for s, (x_k, rr_k) in enumerate(_oracle_iterates(G, m, d, al, True, k)):
        assert rel(u[s], x_k) < 3e-4, (s, rel(u[s], x_k))
        # every node, not just the norm: a wrong coefficient on one tile variant shows here
        assert np.max(np.abs(u[s] - x_k)) <= 3e-3 * np.max(np.abs(x_k))
        assert 0 < rr[s] and abs(rr[s] - rr_k) <= 3e-3 * rr_k, (s, rr[s], rr_k)


@pytest.mark.parametrize("pair,single", [(22, 18), (23, 20), (24, 18)])
def test_pair_updates_equal_single_updates(W, pair, single):
    """Grouped-update configurations update the iterate every second (22, 23) or fourth (24)
    iteration, adding the older steps first, so they round exactly like one update per iteration.
    On the grid with interior tiles the wavefields, residuals and iteration counts equal the
    single-update configuration's bit for bit: after 24 to 27 iterations (every count of pending
    steps at the end), for solves stopped by their tolerance (systems ending on different
    iterations), and for the inner solves of an FP64 refinement."""
    import torch
    G = _interior_case()

    def run(cfg, **kw):
        spec = _spec(W, G, 0)
        if kw.pop("refined", False):
            spec.u64 = torch.zeros(G.nsys, G.spec.n, dtype=torch.complex128, device="cuda")
        it, rr, st = W.solve([spec], W.make_opts(dtype=0, kernel=W.KERNEL_TMA(cfg), order=6, **kw))
        u = (spec.u64 if spec.u64 is not None else spec.u).cpu().numpy()
        return u, rr.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()

    cases = [dict(tol=0.0, max_iter=k) for k in (24, 25, 26, 27)] + [dict(tol=1e-3, max_iter=100000),
             dict(tol=1e-6, max_iter=100000, max_refine=3, refine_tol=1e-6, inner_tol=1e-3, refined=True)]
    for kw in cases:
        a, b = run(pair, **dict(kw)), run(single, **dict(kw))
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3]), (kw, a[2], b[2], a[3], b[3])
        diff = np.flatnonzero(a[0].ravel() != b[0].ravel())
        assert diff.size == 0, (kw, diff.size, diff[:8], rel(a[0], b[0]))
        assert np.array_equal(a[1], b[1]), (kw, a[1], b[1])
        if kw["tol"] > 0 and "refined" not in kw:
            assert a[3].tolist() == [W.SYS_OK] * G.nsys, (kw, a[3])


@pytest.mark.parametrize("dtype,tol", [(1, 1e-10), (0, 3e-4)])
@pytest.mark.parametrize("source_free", [True, False])
def test_interior_tiles_march_match_oracle(W, dtype, tol, source_free):
    """The z-march phase kernels (phases 1 and 2, complex128 and complex64) on the grid with interior
    tiles: k CGLS iterates and residuals equal the oracle's."""
    G = _interior_case()
    m, d, al = seen(G, dtype == 0)
    k = 25
    spec = _spec(W, G, dtype, source_free)
    it, rr, st = W.solve([spec], W.make_opts(tol=0.0, max_iter=k, dtype=dtype, kernel=W.KERNEL_MARCH))
    assert it.cpu().tolist() == [k] * 3
    u, rr = spec.u.cpu().numpy(), rr.cpu().numpy()
    for s, (x_k, rr_k) in enumerate(_oracle_iterates(G, m, d, al, source_free, k)):
        assert rel(u[s], x_k) < tol, (s, rel(u[s], x_k))
        assert np.max(np.abs(u[s] - x_k)) <= 10 * tol * np.max(np.abs(x_k))
        assert 0 < rr[s] and abs(rr[s] - rr_k) <= max(tol, 1e-6) * rr_k * 10, (s, rr[s], rr_k)


@pytest.mark.parametrize("cfg", [0, 8, 9, 14, 17])
def test_tma_z_chunks_and_convergence(W, cfg):
    """TMA path with z-chunks and a real stopping test: same iterations (within 5 %) and
    wavefields as the z-march kernels at tolerance 1e-3."""
    G = case(nphys=(28, 16, 14), npml=4, nsys=2)
    s_t, s_m = _spec(W, G, 0), _spec(W, G, 0)
    it_t, rr_t, st_t = W.solve([s_t], W.make_opts(tol=1e-3, max_iter=100000, dtype=0, zsplit=3,
                                                 kernel=W.KERNEL_TMA(cfg)))
    it_m, rr_m, st_m = W.solve([s_m], W.make_opts(tol=1e-3, max_iter=100000, dtype=0, zsplit=3,
                                                 kernel=W.KERNEL_MARCH))
    assert st_t.cpu().tolist() == [0, 0]
    a, b = it_t.cpu().numpy(), it_m.cpu().numpy()
    assert np.all(np.abs(a - b) <= 0.05 * b + 2)
    assert rel(s_t.u.cpu().numpy(), s_m.u.cpu().numpy()) < 2e-2


# ------------------------------------------------------------------ converged solves (a3, a6)
def _exact(G, m, d, source_free, s):
    A = oracle_A(G, m)
    lu = spla.splu(A.tocsc())
    rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
    return O.solve_dataspace(lu, G.spec.n, G.src[s], rec, d[G.rec_off[s]:G.rec_off[s + 1]], G.lam,
                             G.alpha[s], source_free)


@pytest.mark.parametrize("source_free", [True, False])
def test_converged_c128_matches_exact(W, source_free):
    G = case(nphys=(15, 11, 9), npml=3, nsys=2, freq=15.0)
    spec = _spec(W, G, 1, source_free)
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-10, max_iter=300000, dtype=1))
    assert st.cpu().tolist() == [W.SYS_OK] * 2
    assert 0 < float(rr.min()) and float(rr.max()) <= 1e-10
    u = spec.u.cpu().numpy()
    for s in range(2):
        assert rel(u[s], _exact(G, G.m, G.d, source_free, s)) < 1e-5


@pytest.mark.parametrize("source_free", [True, False])
def test_converged_relres_is_the_true_residual(W, source_free):
    """A converged complex128 solve reports ||S^H (b - S u)|| / ||S^H b|| of the wavefield it
    returns: positive, at most tol, and within 1 % of the oracle's evaluation of that expression at
    the returned u (at tol 1e-8 the gap between CGLS's recurred residual and the true one, about
    eps kappa(S) sqrt(k) relative, is far below 1 %)."""
    G = case(nphys=(15, 11, 9), npml=3, nsys=2, freq=15.0)
    spec = _spec(W, G, 1, source_free)
    tol = 1e-8
    it, rr, st = W.solve([spec], W.make_opts(tol=tol, max_iter=300000, dtype=1))
    assert st.cpu().tolist() == [W.SYS_OK] * 2
    u, rr = spec.u.cpu().numpy(), rr.cpu().numpy()
    A = oracle_A(G, G.m)
    for s in range(2):
        rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
        S = O.augmented_operator(A, O.restriction(G.spec.n, rec), G.src[s], G.lam, source_free)
        b = O.rhs(G.spec.n, G.src[s], G.d[G.rec_off[s]:G.rec_off[s + 1]], G.lam, G.alpha[s], source_free)
        SH = S.conj().T
        true_rr = np.linalg.norm(SH @ (b - S @ u[s])) / np.linalg.norm(SH @ b)
        assert 0 < rr[s] <= tol
        assert abs(rr[s] - true_rr) <= 0.01 * true_rr, (s, rr[s], true_rr)


@pytest.mark.parametrize("source_free", [True, False])
def test_mixed_precision_refinement_matches_exact(W, source_free):
    """FP32 complex stencil + FP64 refinement reaches the FP64 solution of the problem
    defined by the float32 model and complex64 data."""
    G = case(nphys=(15, 11, 9), npml=3, nsys=2, freq=15.0)
    m, d, _ = seen(G, True)
    spec = _spec(W, G, 0, source_free)
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-3, max_iter=200000, dtype=0, max_refine=12,
                                             refine_tol=1e-10, inner_tol=1e-3))
    assert st.cpu().tolist() == [W.SYS_OK] * 2, (st, rr, it)
    assert 0 < float(rr.min()) and float(rr.max()) <= 1e-10
    u = spec.u.cpu().numpy()
    for s in range(2):
        assert rel(u[s], _exact(G, m, d, source_free, s)) < 1e-5


@pytest.mark.parametrize("source_free", [True, False])
def test_refinement_on_tma_phases_matches_exact(W, source_free):
    """x extent a multiple of 4 (24): the refinement's inner solves run on the warp-specialised TMA
    phases (phase 2 adds S^H r64); the FP64 wavefield reaches the exact solution of the float32
    model / complex64 data problem, and the same refinement on the z-march kernels agrees."""
    G = case(nphys=(16, 11, 9), npml=4, nsys=2, freq=15.0)
    m, d, _ = seen(G, True)
    out = []
    for kernel in (0, 1):
        spec = _spec(W, G, 0, source_free)
        spec.u64 = torch.zeros(G.nsys, G.spec.n, dtype=torch.complex128, device="cuda")
        it, rr, st = W.solve([spec], W.make_opts(tol=1e-3, max_iter=200000, dtype=0, max_refine=12,
                                                 refine_tol=1e-10, inner_tol=1e-2, kernel=kernel))
        assert st.cpu().tolist() == [W.SYS_OK] * 2, (kernel, st, rr, it)
        assert 0 < float(rr.min()) and float(rr.max()) <= 1e-10
        out.append(spec.u64.cpu().numpy())
    for s in range(2):
        ex = _exact(G, m, d, source_free, s)
        assert rel(out[0][s], ex) < 1e-8
        assert rel(out[1][s], ex) < 1e-8


@pytest.mark.parametrize("k", [5, 25])
def test_first_refinement_step_is_cgls(W, k):
    """The first outer step of the augmented-system refinement starts from r64 = 0, x64 = 0,
    so its inner solve is plain CGLS on b: k inner iterations give the k-th CGLS iterate, and
    the reported residual is the FP64 normal-equation residual of that iterate."""
    G = case(nphys=(15, 11, 9), npml=3, nsys=2, freq=15.0)
    m, d, al = seen(G, True)
    A = oracle_A(G, m)
    spec = _spec(W, G, 0)
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-3, max_iter=k, dtype=0, max_refine=1, refine_tol=1e-12,
                                             inner_tol=1e-12))
    u = spec.u.cpu().numpy()
    assert it.cpu().tolist() == [k, k]
    for s in range(2):
        rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
        P = O.restriction(G.spec.n, rec)
        S = O.augmented_operator(A, P, G.src[s], G.lam, True)
        b = O.rhs(G.spec.n, G.src[s], d[G.rec_off[s]:G.rec_off[s + 1]], G.lam)
        x_k, _, _ = O.cgls(S, b, tol=0.0, max_iter=k)
        assert rel(u[s], x_k) < 1e-3, rel(u[s], x_k)
        SH = S.conj().T
        true_rr = np.linalg.norm(SH @ (b - S @ x_k)) / np.linalg.norm(SH @ b)
        assert abs(float(rr[s]) - true_rr) <= 0.05 * true_rr


def test_c64_forward_error_matches_fp64_cgls(W):
    """Unrefined FP32 solve at tolerance 1e-4: its distance to the exact solution is
    that of FP64 CGLS stopped at the same tolerance (within 4x), in about as many
    iterations.  (The true normal-equation residual of any FP32-stored wavefield is
    dominated by storage rounding amplified by sigma_max(S)^2, so it is not the
    quantity to compare.)"""
    G = case(nphys=(23, 13, 10), npml=4, nsys=2)
    m, d, _ = seen(G, True)
    spec = _spec(W, G, 0)
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-4, max_iter=100000, dtype=0))
    assert st.cpu().tolist() == [W.SYS_OK] * 2
    assert 0 < float(rr.min()) and float(rr.max()) <= 1e-4
    A = oracle_A(G, m)
    u = spec.u.cpu().numpy().astype(np.complex128)
    for s in range(2):
        rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
        P = O.restriction(G.spec.n, rec)
        S = O.augmented_operator(A, P, G.src[s], G.lam, True)
        b = O.rhs(G.spec.n, G.src[s], d[G.rec_off[s]:G.rec_off[s + 1]], G.lam)
        x64, it64, _ = O.cgls(S, b, tol=1e-4, max_iter=100000)
        ex = _exact(G, m, d, True, s)
        assert rel(u[s], ex) <= 4 * rel(x64, ex) + 1e-6
        assert abs(int(it[s]) - it64) <= 0.15 * it64


# ------------------------------------------------------------------ source estimate, gradient (a7, a8)
@pytest.mark.parametrize("dtype,tol", [(1, 1e-11), (0, 2e-5)])
@pytest.mark.parametrize("source_free", [True, False])
def test_source_estimate_and_gradient_on_given_fields(W, dtype, tol, source_free):
    """Same wavefields and weights on both sides: isolates the kernels of a7/a8."""
    G = case(nphys=(35, 18, 20), npml=4, nsys=3)
    m, d, _ = seen(G, dtype == 0)
    u = synth.random_complex((3, G.spec.n), 21) * 1e-3
    if dtype == 0:
        u = u.astype(np.complex64).astype(np.complex128)
    spec = _spec(W, G, dtype, source_free, u=u)
    A = oracle_A(G, m)
    w = O.stretch_weight(G.spec.shape, G.spec.h, G.omega, G.spec.npml, G.v_max, G.pml_R)
    a_gpu = W.source_estimate([spec], dtype).cpu().numpy()
    a_ref = np.array([O.source_estimate(A, u[s], G.src[s]) for s in range(3)])
    assert rel(a_gpu, a_ref) < tol
    a_use = a_ref if source_free else G.alpha
    g, f = W.gradient([spec], dtype, torch.as_tensor(a_use).cuda())
    g_ref = np.zeros(G.spec.n)
    f_ref = 0.0
    for s in range(3):
        rec = G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]]
        P = O.restriction(G.spec.n, rec)
        g_ref += O.gradient(A, u[s], G.src[s], a_use[s], G.omega, w)
        f_ref += O.objective(A, P, u[s], G.src[s], d[G.rec_off[s]:G.rec_off[s + 1]], G.lam, a_use[s])
    assert rel(g[0].cpu().numpy().ravel(), g_ref) < 10 * tol
    assert abs(f.item() - f_ref) <= 10 * tol * abs(f_ref)


def test_pipeline_gradient_matches_oracle(W):
    """Solve + estimate + gradient (C64 with FP64 refinement) against the oracle's
    exact evaluation of f4 and g4."""
    G = case(nphys=(17, 12, 9), npml=3, nsys=3, freq=14.0)
    m, d, _ = seen(G, True)
    spec = _spec(W, G, 0)
    spec.u64 = torch.zeros(G.nsys, G.spec.n, dtype=torch.complex128, device="cuda")
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-3, max_iter=200000, dtype=0, max_refine=12,
                                             refine_tol=1e-10, inner_tol=1e-3))
    assert st.cpu().tolist() == [W.SYS_OK] * 3
    assert rel(spec.u.cpu().numpy(), spec.u64.cpu().numpy()) < 1e-7   # u is the rounded u64
    a = W.source_estimate([spec], 0)
    g, f = W.gradient([spec], 0, a)
    u_ex, a_ex, f_ex, g_ex = O.evaluate(G.spec.shape, G.spec.h, G.omega, m, G.spec.npml, G.v_max, G.src,
                                        G.rec_off, G.rec_idx, d, G.lam)
    assert rel(spec.u64.cpu().numpy(), u_ex) < 1e-5
    assert rel(a.cpu().numpy(), a_ex) < 1e-5
    assert rel(g[0].cpu().numpy().ravel(), g_ex) < 1e-4
    assert abs(f.item() - f_ex) <= 1e-4 * abs(f_ex)


@pytest.mark.parametrize("cfg", [18, 24])
def test_certified_pipeline_on_tma_phases_matches_oracle(W, cfg):
    """The certified configuration of the benchmark on the TMA phases (x extent 24, a multiple of 4):
    complex64 CGLS with x updated every iteration (configuration 18) or every fourth (24) inside
    FP64 refinement, the FP64 source estimate, and the gradient read off the refinement's FP64
    residual, against the oracle's exact evaluation of f4 and g4: wavefield and weights to 1e-5,
    gradient and objective to 1e-4."""
    G = case(nphys=(18, 12, 9), npml=3, nsys=3, freq=14.0)
    m, d, _ = seen(G, True)
    spec = _spec(W, G, 0)
    spec.u64 = torch.zeros(G.nsys, G.spec.n, dtype=torch.complex128, device="cuda")
    opts = W.make_opts(tol=1e-3, max_iter=200000, dtype=0, max_refine=12, refine_tol=1e-10, inner_tol=1e-3,
                       kernel=W.KERNEL_TMA(cfg))
    work = torch.empty(W.workspace_size([spec], opts), dtype=torch.uint8, device="cuda")
    it, rr, st = W.solve([spec], opts, workspace=work)
    assert st.cpu().tolist() == [W.SYS_OK] * 3
    assert 0 < float(rr.max()) <= 1e-10
    a = W.source_estimate([spec], 0, workspace=work)
    (g,), f = W.gradient_refined([spec], opts, work)
    u_ex, a_ex, f_ex, g_ex = O.evaluate(G.spec.shape, G.spec.h, G.omega, m, G.spec.npml, G.v_max, G.src,
                                        G.rec_off, G.rec_idx, d, G.lam)
    assert rel(spec.u64.cpu().numpy(), u_ex) < 1e-5
    assert rel(a.cpu().numpy(), a_ex) < 1e-5
    assert rel(g.cpu().numpy().ravel(), g_ex) < 1e-4
    assert abs(f.item() - f_ex) <= 1e-4 * abs(f_ex)


@pytest.mark.parametrize("source_free", [True, False])
def test_gradient_from_refined_residual_equals_stencil_gradient(W, source_free):
    """wri_gradient_refined reads the FP64 residual a refined solve leaves in its workspace: the same f
    and g as wri_gradient's FP64 stencil pass on the FP64 wavefield (to rounding), with two frequency
    groups in one call.  The library's record of which problem's residual a workspace holds guards the
    call."""
    G1 = case(nphys=(17, 12, 9), npml=3, nsys=3, freq=14.0)
    G2 = case(nphys=(12, 10, 8), npml=3, nsys=2, seed=8, freq=9.0)
    specs = [_spec(W, G, 0, source_free) for G in (G1, G2)]
    for sp in specs:
        sp.u64 = torch.zeros(sp.nsys, sp.n, dtype=torch.complex128, device="cuda")
    opts = W.make_opts(tol=1e-3, max_iter=200000, dtype=0, max_refine=12, refine_tol=1e-9, inner_tol=1e-3)
    work = torch.empty(W.workspace_size(specs, opts), dtype=torch.uint8, device="cuda")
    it, rr, st = W.solve(specs, opts, workspace=work)
    assert st.cpu().tolist() == [W.SYS_OK] * 5
    g_res, f_res = W.gradient_refined(specs, opts, work)
    a = W.source_estimate(specs, 0) if source_free else torch.view_as_complex(
        torch.cat([sp.alpha for sp in specs]).contiguous())
    g_st, f_st = W.gradient(specs, 0, a)
    for x, y in zip(g_res, g_st):
        assert rel(x.cpu().numpy(), y.cpu().numpy()) < 1e-9
    assert abs(f_res.item() - f_st.item()) <= 1e-10 * abs(f_st.item())
    # the residual of a fixed-budget refined solve (the benchmark's step) is also the right one
    fixed = W.make_opts(tol=0.0, max_iter=40, dtype=0, max_refine=1, refine_tol=0.0, inner_tol=1e-300)
    W.solve(specs, fixed, workspace=work)
    g_res, f_res = W.gradient_refined(specs, fixed, work)
    g_st, f_st = W.gradient(specs, 0, W.source_estimate(specs, 0) if source_free else a)
    for x, y in zip(g_res, g_st):
        assert rel(x.cpu().numpy(), y.cpu().numpy()) < 1e-9
    # an unrefined solve on the workspace drops the record, and so does a refined solve of other
    # groups: the call is refused rather than reading a residual of another problem
    W.solve(specs, W.make_opts(tol=0.0, max_iter=5, dtype=0), workspace=work)
    with pytest.raises(W.WriError) as e:
        W.gradient_refined(specs, fixed, work)
    assert e.value.code == W.EINVAL
    W.solve(specs[:1], fixed, workspace=work)
    with pytest.raises(W.WriError) as e:
        W.gradient_refined(specs, fixed, work)
    assert e.value.code == W.EINVAL


# ------------------------------------------------------------------ batching (a4)
def test_batched_equals_unbatched_and_multi_group(W):
    G1 = case(nphys=(25, 12, 10), npml=4, nsys=3, seed=5)
    G2 = case(nphys=(14, 19, 8), npml=3, nsys=2, seed=8, freq=9.0)
    opts = W.make_opts(tol=1e-6, max_iter=50000, dtype=1, zsplit=2)
    s1, s2 = _spec(W, G1, 1), _spec(W, G2, 1)
    it, rr, st = W.solve([s1, s2], opts)
    ub = []
    for G in (G1, G2):
        for s in range(G.nsys):
            one = synth.Group(G.spec, G.freq, G.v, G.src[s:s + 1], np.array([0, G.rec_off[s + 1] - G.rec_off[s]],
                              np.int32), G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]], G.lam, G.v_max, G.pml_R,
                              G.alpha[s:s + 1], G.d[G.rec_off[s]:G.rec_off[s + 1]])
            sp1 = _spec(W, one, 1)
            i1, r1, t1 = W.solve([sp1], opts)
            ub.append((sp1.u.cpu().numpy()[0], int(i1.item()), float(r1.item())))
    ub_u = [x[0] for x in ub]
    got = list(s1.u.cpu().numpy()) + list(s2.u.cpu().numpy())
    for a, b in zip(got, ub_u):
        assert np.array_equal(a, b)           # same tiles, same reduction order: bit-identical
    assert it.cpu().tolist() == [x[1] for x in ub]
    assert np.array_equal(rr.cpu().numpy(), np.array([x[2] for x in ub]))


@pytest.mark.parametrize("kernel", [0, 2 + 9])
def test_tma_batch_of_groups_equals_single_systems(W, kernel):
    """Two frequency groups on different grids (x extents multiples of 4) in one batched TMA
    solve, several orders of the work items: every system's iterate equals its own unbatched
    z-march solve (same reduction order per system, so to rounding of the FP32 stencil)."""
    G1 = case(nphys=(28, 12, 10), npml=4, nsys=3, seed=5)
    G2 = case(nphys=(16, 19, 8), npml=4, nsys=5, seed=8, freq=9.0)
    k = 20
    for order in (0, 1, 3, 6):
        s1, s2 = _spec(W, G1, 0), _spec(W, G2, 0)
        it, rr, st = W.solve([s1, s2], W.make_opts(tol=0.0, max_iter=k, dtype=0, kernel=kernel, order=order))
        assert it.cpu().tolist() == [k] * 8
        got = list(s1.u.cpu().numpy()) + list(s2.u.cpu().numpy())
        i = 0
        for G in (G1, G2):
            for s in range(G.nsys):
                one = synth.Group(G.spec, G.freq, G.v, G.src[s:s + 1], np.array([0, G.rec_off[s + 1] - G.rec_off[s]],
                                  np.int32), G.rec_idx[G.rec_off[s]:G.rec_off[s + 1]], G.lam, G.v_max, G.pml_R,
                                  G.alpha[s:s + 1], G.d[G.rec_off[s]:G.rec_off[s + 1]])
                sp1 = _spec(W, one, 0)
                W.solve([sp1], W.make_opts(tol=0.0, max_iter=k, dtype=0, kernel=W.KERNEL_MARCH))
                assert rel(got[i], sp1.u.cpu().numpy()[0]) < 1e-5, (order, i)
                i += 1


def test_autotune_choice_solves_like_default_and_is_cached(W):
    """wri_autotune picks a TMA configuration and order; solving with it gives the iterates of
    the default configuration, and a second call for the same batch shape is served from the
    cache without touching the wavefields."""
    G1 = case(nphys=(28, 12, 10), npml=4, nsys=3, seed=5)
    G2 = case(nphys=(16, 19, 8), npml=4, nsys=2, seed=8, freq=9.0)
    s1, s2 = _spec(W, G1, 0), _spec(W, G2, 0)
    base = W.make_opts(tol=0.0, max_iter=20, dtype=0)
    tuned = W.autotune([s1, s2], base, trial_iters=6)
    assert tuned.kernel in [2 + c for c in (8, 9, 12, 13, 17, 18, 22, 24)] and tuned.order in (2, 5, 6)
    s1.u.fill_(3.0)
    again = W.autotune([s1, s2], base, trial_iters=6)
    assert (again.kernel, again.order) == (tuned.kernel, tuned.order)
    assert float(s1.u.real.min()) == 3.0 == float(s1.u.real.max())
    a1, a2 = _spec(W, G1, 0), _spec(W, G2, 0)
    W.solve([a1, a2], tuned)
    b1, b2 = _spec(W, G1, 0), _spec(W, G2, 0)
    W.solve([b1, b2], base)
    assert rel(a1.u.cpu().numpy(), b1.u.cpu().numpy()) < 1e-5
    assert rel(a2.u.cpu().numpy(), b2.u.cpu().numpy()) < 1e-5


def test_autotune_disk_cache_round_trip(W, tmp_path):
    """The on-disk cache with the real library: the stored choice is the library's, and a second
    call returns it without trial solves (the wavefields stay untouched)."""
    import json
    G = case(nphys=(20, 12, 10), npml=4, nsys=2, seed=6)
    s = _spec(W, G, 0)
    base = W.make_opts(tol=0.0, max_iter=20, dtype=0)
    path = str(tmp_path / "tune.json")
    first = W.autotune([s], base, trial_iters=4, cache=path)
    with open(path) as fh:
        stored = list(json.load(fh).values())
    assert stored == [{"kernel": first.kernel, "order": first.order}]
    s.u.fill_(2.0)
    again = W.autotune([s], base, trial_iters=4, cache=path)
    assert (again.kernel, again.order) == (first.kernel, first.order)
    assert float(s.u.real.min()) == 2.0 == float(s.u.real.max())


def test_plain_path_matches_fused(W):
    G = case(nphys=(21, 13, 11), npml=4, nsys=2)
    sa, sb = _spec(W, G, 0), _spec(W, G, 0)
    ia, ra, ta = W.solve([sa], W.make_opts(tol=1e-4, max_iter=50000, dtype=0))
    ib, rb, tb = W.solve([sb], W.make_opts(tol=1e-4, max_iter=50000, dtype=0, plain=True))
    assert tb.cpu().tolist() == [W.SYS_OK] * 2
    ia, ib = ia.cpu().numpy(), ib.cpu().numpy()
    assert np.all(np.abs(ia - ib) <= np.maximum(3, 0.10 * ia))
    assert rel(sa.u.cpu().numpy(), sb.u.cpu().numpy()) < 1e-3


def test_warm_start(W):
    G = case(nphys=(15, 11, 9), npml=3, nsys=2, freq=15.0)
    s = _spec(W, G, 1)
    W.solve([s], W.make_opts(tol=1e-10, max_iter=200000, dtype=1))
    u1 = s.u.clone()
    it, rr, st = W.solve([s], W.make_opts(tol=1e-8, max_iter=200000, dtype=1, warm_start=True))
    assert it.cpu().tolist() == [0, 0] and st.cpu().tolist() == [0, 0]
    assert torch.equal(s.u, u1)
    s.u.mul_(1.01)
    it2, rr2, st2 = W.solve([s], W.make_opts(tol=1e-8, max_iter=200000, dtype=1, warm_start=True))
    assert st2.cpu().tolist() == [0, 0] and int(it2.min()) > 0
    assert float(rr2.max()) <= 1e-8
    assert rel(s.u.cpu().numpy(), u1.cpu().numpy()) < 1e-4


# ------------------------------------------------------------------ edge cases
def test_no_receivers_and_zero_data(W):
    G = case(nphys=(12, 10, 8), npml=3, nsys=2)
    G.rec_idx = G.rec_idx[G.rec_off[1]:]
    G.d = G.d[G.rec_off[1]:]
    G.rec_off = np.array([0, 0, len(G.rec_idx)], np.int32)   # system 0 has no receivers
    spec = _spec(W, G, 1)
    spec.u.fill_(7.0)
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-6, max_iter=100000, dtype=1))
    assert st.cpu().tolist() == [0, 0]
    assert int(it[0]) == 0 and float(rr[0]) == 0.0
    assert float(spec.u[0].abs().max()) == 0.0   # x0 = 0 is the solution when S^H b = 0
    assert int(it[1]) > 0
    spec.d.zero_()
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-6, max_iter=100000, dtype=1))
    assert it.cpu().tolist() == [0, 0] and float(spec.u.abs().max()) == 0.0


def test_max_iter_one_and_status(W):
    G = case(nphys=(12, 10, 8), npml=3, nsys=1)
    spec = _spec(W, G, 0)
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-12, max_iter=1, dtype=0))
    assert it.tolist() == [1] and st.tolist() == [W.SYS_MAXITER]
    with pytest.raises(W.WriError):
        W.solve([spec], W.make_opts(tol=-1.0, dtype=0))


@pytest.mark.parametrize("kernel", [0, 1])
def test_host_loop_equals_device_loop(W, kernel):
    """The host-replayed iteration graph (host_loop, kept for kernel profilers) and the device-side
    WHILE loop run the same kernels in the same order: bit-identical iterates and residuals, on a
    converged solve (tol 1e-4, so the loop's stopping decision is exercised) and a fixed budget."""
    G = case(nphys=(36, 13, 10), npml=4, nsys=3)
    for tol, k in ((1e-4, 100000), (0.0, 30)):
        out = []
        for host in (False, True):
            sp = _spec(W, G, 0)
            it, rr, st = W.solve([sp], W.make_opts(tol=tol, max_iter=k, dtype=0, kernel=kernel, host_loop=host))
            out.append((sp.u.clone(), it.clone(), rr.clone(), st.clone()))
        assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
        assert torch.equal(out[0][2], out[1][2]) and torch.equal(out[0][3], out[1][3])


@pytest.mark.parametrize("cfg", [9, 18])
def test_copy_wait_time_out_is_reported_and_the_context_recovers(W, cfg):
    """Bounded waits of the warp-specialised TMA phases.  With the test hook the copy warp of block
    0 never issues its first plane fill, so nothing ever completes that stage's barrier: the
    consumers' wait for it runs out after the 1 ms limit, the launch's error flag stops the solve
    (later launches of the solve do nothing) and wri_solve_batch returns WRI_ECUDA.  No copy is
    left in flight and no wait is unbounded, so the context stays usable: a normal solve on the
    same stream afterwards gives the reference iterates bit for bit."""
    G = case(nphys=(36, 13, 10), npml=4, nsys=3)
    k = 10
    opts = W.make_opts(tol=0.0, max_iter=k, dtype=0, kernel=W.KERNEL_TMA(cfg))
    ref = _spec(W, G, 0)
    W.solve([ref], opts)
    bad = _spec(W, G, 0)
    with pytest.raises(W.WriError) as e:
        W.solve([bad], W.make_opts(tol=0.0, max_iter=k, dtype=0, kernel=W.KERNEL_TMA(cfg), wait_limit_us=1000,
                                   test_withhold=1))
    assert e.value.code == W.ECUDA
    torch.cuda.synchronize()
    again = _spec(W, G, 0)
    it, rr, st = W.solve([again], opts)
    assert it.cpu().tolist() == [k] * 3
    assert torch.equal(again.u, ref.u)


@pytest.mark.parametrize("kernel", [0, 1])
def test_nonfinite_model_is_reported_per_group(W, kernel):
    """A NaN in one group's model: its systems end with WRI_SYS_NONFINITE, the other group's
    systems converge as usual, and the call returns (TMA phases and z-march kernels)."""
    G1 = case(nphys=(28, 12, 10), npml=4, nsys=2, seed=5)
    G2 = case(nphys=(16, 13, 9), npml=4, nsys=3, seed=8, freq=9.0)   # x extents 36 and 24: TMA-eligible
    s1, s2 = _spec(W, G1, 0), _spec(W, G2, 0)
    s2.m.view(-1)[s2.m.numel() // 2] = float("nan")
    it, rr, st = W.solve([s1, s2], W.make_opts(tol=1e-3, max_iter=100000, dtype=0, kernel=kernel))
    assert st.cpu().tolist() == [W.SYS_OK] * 2 + [W.SYS_NONFINITE] * 3
    assert float(rr[:2].max()) <= 1e-3


@pytest.mark.parametrize("tile", [1, 2, 3])
def test_tile_shapes_agree(W, tile):
    G = case(nphys=(40, 23, 9), npml=4, nsys=2)
    ref = _spec(W, G, 1)
    W.solve([ref], W.make_opts(tol=0.0, max_iter=15, dtype=1, tile=2))
    s = _spec(W, G, 1)
    W.solve([s], W.make_opts(tol=0.0, max_iter=15, dtype=1, tile=tile, zsplit=3))
    assert rel(s.u.cpu().numpy(), ref.u.cpu().numpy()) < 1e-11


# ------------------------------------------------------------------ full-size sampled checks
def test_full_size_operator_samples(W):
    """148^3 (128^3 + 10-cell layer, 8 Hz, h = 20 m): sampled rows of A and A^H
    against the oracle's sparse rows, one launch of the production tile."""
    grp = synth.workload_c4(nsrc=2, freqs=((8.0, 128),))[0]
    spec = _spec(W, grp, 0)
    x = torch.randn(1, grp.spec.n, dtype=torch.complex64, device="cuda")
    y = W.apply_A(spec, x).cpu().numpy()[0]
    yh = W.apply_A(spec, x, adjoint=True).cpu().numpy()[0]
    xs = x.cpu().numpy()[0].astype(np.complex128)
    m = grp.m.astype(np.float32).astype(np.float64)
    r = synth.rng(2)
    nodes = np.concatenate([r.integers(0, grp.spec.n, 300), [0, grp.spec.n - 1, grp.src[0]]])
    # oracle rows for the sampled nodes, from a small sub-block around each node
    A = oracle_A(grp, m)
    rows = A[nodes]
    assert rel(y[nodes], rows @ xs) < 2e-6
    assert rel(yh[nodes], rows.conj() @ xs) < 2e-6


def test_full_size_batched_iterations_consistent(W):
    """Production configuration of one group (128^3 + 10, 8 systems): after 30
    iterations the reported residual equals ||S^H (b - S u)|| / ||S^H b|| recomputed
    with the operator kernels (a property that holds at any size)."""
    grp = synth.workload_c4(nsrc=8, freqs=((8.0, 128),))[0]
    spec = _spec(W, grp, 0)
    it, rr, st = W.solve([spec], W.make_opts(tol=0.0, max_iter=30, dtype=0))
    assert it.cpu().tolist() == [30] * 8
    u = spec.u
    n = grp.spec.n
    for s in (0, 5):
        us = u[s:s + 1].to(torch.complex128)
        spec64 = _spec(W, grp, 1)
        Au = W.apply_A(spec64, us)[0]
        Au[grp.src[s]] = 0
        rec = torch.as_tensor(grp.rec_idx[grp.rec_off[s]:grp.rec_off[s + 1]].astype(np.int64)).cuda()
        d = torch.as_tensor(grp.d[grp.rec_off[s]:grp.rec_off[s + 1]].astype(np.complex64).astype(np.complex128)).cuda()
        r1 = -Au
        r2 = grp.lam * (d - us[0, rec])
        sv = W.apply_A(spec64, r1[None], adjoint=True)[0]
        sv[rec] += grp.lam * r2
        sb = torch.zeros(n, dtype=torch.complex128, device="cuda")
        sb[rec] = grp.lam ** 2 * d
        true_rr = (sv.norm() / sb.norm()).item()
        assert abs(true_rr - rr[s].item()) <= 2e-3 * true_rr, (true_rr, rr[s].item())


def test_config5_scale_refinement_residual(W):
    """256 x 256 x 160 physical nodes + 10-cell layer (276 x 276 x 180 = 13.7 M nodes), h = 8 m, salt
    body, 10 Hz, 2 systems, complex64 with FP64 refinement: after one refinement step of 60 inner
    iterations the reported FP64 residual equals ||S^H (b - S u64)|| / ||S^H b|| recomputed with the
    complex128 operator kernels (same float32 model and complex64 data), and u is u64 rounded."""
    grp = synth.workload_c5(nsrc=2)
    n = grp.spec.n
    m32 = grp.m.astype(np.float32).astype(np.float64)
    d32 = grp.d.astype(np.complex64).astype(np.complex128)
    from paper_2410_18429_gb300.problem import to_device
    spec = to_device(grp, 0, "cuda")
    spec.u64 = torch.zeros(2, n, dtype=torch.complex128, device="cuda")
    it, rr, st = W.solve([spec], W.make_opts(tol=1e-3, max_iter=60, dtype=0, max_refine=1, refine_tol=1e-12,
                                             inner_tol=1e-12))
    assert it.cpu().tolist() == [60, 60] and st.cpu().tolist() == [W.SYS_MAXITER] * 2
    assert rel(spec.u.cpu().numpy(), spec.u64.cpu().numpy()) < 1e-7
    spec64 = to_device(grp, 1, "cuda", m=m32, d=d32)
    for s in range(2):
        us = spec.u64[s:s + 1]
        Au = W.apply_A(spec64, us)[0]
        Au[grp.src[s]] = 0
        rec = torch.as_tensor(grp.rec_idx[grp.rec_off[s]:grp.rec_off[s + 1]].astype(np.int64)).cuda()
        d = torch.as_tensor(d32[grp.rec_off[s]:grp.rec_off[s + 1]]).cuda()
        r2 = grp.lam * (d - us[0, rec])
        sv = W.apply_A(spec64, (-Au)[None], adjoint=True)[0]
        sv[rec] += grp.lam * r2
        sb = torch.zeros(n, dtype=torch.complex128, device="cuda")
        sb[rec] = grp.lam ** 2 * d
        true_rr = (sv.norm() / sb.norm()).item()
        assert abs(true_rr - rr[s].item()) <= 1e-6 * true_rr, (true_rr, rr[s].item())
    del spec, spec64
    torch.cuda.empty_cache()


def test_config2_tolerance_halving_with_warm_starts(W):
    """Configuration 2's batch shape (64^3 + 10-cell layer, layered model, surface sources, 5 Hz and
    7 Hz groups in one batched complex64 solve; 2 sources per frequency) through the tolerance
    halving of Algorithm 2 (eps, eps/2, eps/4 from eps = 0.2), each step warm-started from the last:
    every system meets each tolerance, and the warm-started last step needs fewer iterations than a
    cold solve to the same tolerance.  (At 50-100 points per wavelength unpreconditioned CGLS needs
    more than 1e5 iterations even for loose tolerances on this grid: the schedule starts at 0.2 and
    the 3 Hz group, about 100 points per wavelength, is left out.)"""
    from paper_2410_18429_gb300.problem import to_device
    groups = []
    for g in synth.workload_c2()[1:]:
        groups.append(synth.Group(g.spec, g.freq, g.v, g.src[:2], g.rec_off[:3] - g.rec_off[0],
                                  g.rec_idx[g.rec_off[0]:g.rec_off[2]], g.lam, g.v_max, g.pml_R, g.alpha[:2],
                                  g.d[g.rec_off[0]:g.rec_off[2]]))
    specs = [to_device(g, 0, "cuda") for g in groups]
    nsys = sum(g.nsys for g in groups)
    tols = [0.2, 0.1, 0.05]
    iters = []
    for k, tol in enumerate(tols):
        it, rr, st = W.solve(specs, W.make_opts(tol=tol, max_iter=100000, dtype=0, warm_start=k > 0))
        assert st.cpu().tolist() == [W.SYS_OK] * nsys
        assert 0 < float(rr.min()) and float(rr.max()) <= tol
        iters.append(it.cpu().numpy())
    cold = [to_device(g, 0, "cuda") for g in groups]
    it_cold, rr_cold, st_cold = W.solve(cold, W.make_opts(tol=tols[-1], max_iter=100000, dtype=0))
    assert st_cold.cpu().tolist() == [W.SYS_OK] * nsys
    assert np.all(iters[-1] < it_cold.cpu().numpy())
