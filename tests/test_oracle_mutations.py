"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle, on the CPU, by wrapping one of the oracle's own
functions (a dropped term, a wrong sign, a wrong index, a conjugate-transposed operand, a
misplaced coefficient), and runs the pin that should catch it: the pin must fail.  (A^H u in
place of A u at the source node is no mistake: A is complex symmetric and real on every row away
from the absorbing layer, so the two agree there; the conjugate-transposed operand is planted in
the gradient's residual instead, where the layer's rows make it differ.)  Mistakes
are planted for the duration of one test only (pytest's monkeypatch), in both the ``oracle``
package namespace (calls made by the pins) and ``oracle.wri_oracle`` (calls inside the oracle).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.awri_oracle as AW
import oracle.wri_oracle as W
import test_oracle_fwi as F
import test_oracle_pins as P


def _plant(monkeypatch, module, name, make):
    orig = getattr(module, name)
    fn = make(orig)
    monkeypatch.setattr(module, name, fn)
    if module is W:
        monkeypatch.setattr(oracle, name, fn)


def _laplacian_without_h2(orig):
    def f(shape, h, omega, m, npml=0, v_max=1.0, R=1e-3):
        A = orig(shape, h, omega, m, npml, v_max, R)
        D = sp.diags(omega ** 2 * W.stretch_weight(shape, h, omega, npml, v_max, R) * np.ravel(m))
        return (D + h * h * (A - D)).tocsr()
    return f


def _mass_without_stretch_weight(orig):
    def f(shape, h, omega, m, npml=0, v_max=1.0, R=1e-3):
        A = orig(shape, h, omega, m, npml, v_max, R)
        w = W.stretch_weight(shape, h, omega, npml, v_max, R)
        return (A + sp.diags(omega ** 2 * (1.0 - w) * np.ravel(m))).tocsr()
    return f


MUTATIONS = [
    # (what is planted, module, function, wrapper, pin, pin arguments)
    ("stretch: growing waves (sign of the damping)", W, "stretch",
     lambda o: (lambda *a, **k: tuple(np.conj(s) for s in o(*a, **k))),
     P.test_stretch_zero_padding_and_profile_shape, {}),
    ("stretch: half-node factors shifted by one node", W, "stretch",
     lambda o: (lambda *a, **k: (lambda s, sh: (s, np.roll(sh, 1)))(*o(*a, **k))),
     P.test_stretch_zero_padding_and_profile_shape, {}),
    ("operator: Laplacian without 1/h^2", W, "helmholtz_matrix", _laplacian_without_h2,
     P.test_interior_is_textbook_stencil, {}),
    ("operator: omega^2 m without the stretch weight w", W, "helmholtz_matrix", _mass_without_stretch_weight,
     P.test_operator_complex_symmetric_and_stretch_weight, {}),
    ("mask Z dropped in the source-free operator", W, "augmented_operator",
     lambda o: (lambda A, Pm, src, lam, source_free=True: o(A, Pm, src, lam, False)),
     P.test_masked_problem_equals_joint_block_solve, {}),
    ("data rows weighted by lambda^2 instead of lambda", W, "augmented_operator",
     lambda o: (lambda A, Pm, src, lam, source_free=True: o(A, Pm, src, lam * lam, source_free)),
     P.test_exact_solvers_agree_with_dense_lstsq, {"source_free": True}),
    ("right-hand side: data scaled by lambda^2", W, "rhs",
     lambda o: (lambda n, src, d, lam, alpha=None, source_free=True: o(n, src, lam * np.asarray(d), lam, alpha,
                                                                       source_free)),
     P.test_exact_solvers_agree_with_dense_lstsq, {"source_free": False}),
    ("receiver-space solve: lambda where lambda^2 belongs", W, "solve_dataspace",
     lambda o: (lambda lu, n, src, rec, d, lam, alpha=None, source_free=True: o(lu, n, src, rec, d, np.sqrt(lam),
                                                                                alpha, source_free)),
     P.test_exact_solvers_agree_with_dense_lstsq, {"source_free": True}),
    ("gradient: A^H u instead of A u in the residual", W, "gradient",
     lambda o: (lambda A, u, src, alpha, omega, w: o(A.conj().T.tocsr(), u, src, alpha, omega, w)),
     P.test_gradient_matches_central_differences, {"source_free": True}),
    ("source estimate: neighbouring node", W, "source_estimate",
     lambda o: (lambda A, u, src: o(A, u, int(src) + 1)),
     P.test_masked_problem_equals_joint_block_solve, {}),
    ("objective: data term dropped", W, "objective",
     lambda o: (lambda A, Pm, u, src, d, lam, alpha: o(A, Pm, u, src, d, 0.0, alpha)),
     P.test_objective_is_compact_form, {}),
    ("objective: 1/2 on the PDE term only", W, "objective",
     lambda o: (lambda A, Pm, u, src, d, lam, alpha: o(A, Pm, u, src, d, lam * np.sqrt(2.0), alpha)),
     P.test_objective_is_compact_form, {}),
    ("gradient: sign", W, "gradient",
     lambda o: (lambda A, u, src, alpha, omega, w: -o(A, u, src, alpha, omega, w)),
     P.test_gradient_matches_central_differences, {"source_free": True}),
    ("gradient: omega instead of omega^2", W, "gradient",
     lambda o: (lambda A, u, src, alpha, omega, w: o(A, u, src, alpha, omega, w) / omega),
     P.test_gradient_matches_central_differences, {"source_free": True}),
    ("gradient: conj dropped from the stretch weight", W, "gradient",
     lambda o: (lambda A, u, src, alpha, omega, w: o(A, u, src, alpha, omega, np.conj(w))),
     P.test_gradient_matches_central_differences, {"source_free": True}),
    ("gradient: weight term a e dropped (known weight)", W, "gradient",
     lambda o: (lambda A, u, src, alpha, omega, w: o(A, u, src, 0.0, omega, w)),
     P.test_gradient_matches_central_differences, {"source_free": False}),
    ("total variation: smoothing beta dropped", W, "total_variation",
     lambda o: (lambda m, beta: o(m, 0.0)),
     P.test_total_variation_pins, {}),
    ("total variation: gradient sign", W, "total_variation",
     lambda o: (lambda m, beta: (lambda tv, g: (tv, -g))(*o(m, beta))),
     P.test_total_variation_pins, {}),
    ("l-BFGS: pairs taken newest first", AW, "two_loop",
     lambda o: (lambda g, S, Y, h0=None: o(g, S[::-1], Y[::-1], h0)),
     P.test_two_loop_recursion_equals_dense_bfgs_inverse, {}),
    ("reduced FWI: gradient sign", W, "fwi_evaluate",
     lambda o: (lambda *a, **k: (lambda u, al, f, g: (u, al, f, -g))(*o(*a, **k))),
     F.test_fwi_gradient_matches_central_differences, {"source_free": True}),
    ("reduced FWI: omega in place of omega^2", W, "fwi_evaluate",
     lambda o: (lambda *a, **k: (lambda u, al, f, g: (u, al, f, g / a[2]))(*o(*a, **k))),
     F.test_fwi_gradient_matches_central_differences, {"source_free": False}),
    ("reduced FWI: stretch weight dropped from the gradient", W, "stretch_weight",
     lambda o: (lambda *a, **k: np.ones_like(o(*a, **k))),
     F.test_fwi_gradient_matches_central_differences, {"source_free": False}),
]


@pytest.mark.filterwarnings("ignore::RuntimeWarning")    # beta = 0 divides by zero on a constant model
@pytest.mark.parametrize("what,module,name,make,pin,kwargs", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(monkeypatch, what, module, name, make, pin, kwargs):
    _plant(monkeypatch, module, name, make)
    with pytest.raises(AssertionError):
        pin(**kwargs)


def test_pins_pass_without_a_mistake():
    """The same pins, unmodified oracle: they pass (so the failures above come from the
    planted mistakes)."""
    seen = set()
    for *_, pin, kwargs in MUTATIONS:
        key = (pin.__name__, tuple(sorted(kwargs.items())))
        if key not in seen:
            seen.add(key)
            pin(**kwargs)
