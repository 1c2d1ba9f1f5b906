"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (on the CPU, through monkeypatch: a
dropped stencil term, a wrong sign, a wrong transfer weight, a swapped colour order,
a wrong residual sign, a wrong coarsest solve, a wrong relaxation scaling, a Jacobi step
without its omega, a W cycle visiting its coarse level once, ghosts
without the odd-reflection sign; for periodic grids a coarsest solution off zero mean or a
missing wrap-around; for cubic transfers bilinear or wrong taps) and runs a battery of the
pins of `test_oracle.py`, `test_oracle_periodic.py` or `test_oracle_cubic.py`
(printed stencils, the paper's symbols, printed Galerkin operators and transfers, the
two-level direct-solver theorem, the Schur-complement identity, printed rates and LFA
rates, the exact Fourier spectral radius of the Jacobi two-grid cycle, the cycle's
operator against the error-propagation recursion, agreement with a direct solve). At least one pin must fail for every mistake,
and none without one.
"""
import numpy as np
import pytest

import oracle.mg as omg
import test_oracle as pins
import test_oracle_cubic as cpins
import test_oracle_periodic as ppins

BATTERY = [
    ("fine stencil (order 4)", lambda: pins.test_fine_operator_matches_printed_stencil(4, 8)),
    ("fine stencil (order 2)", lambda: pins.test_fine_operator_matches_printed_stencil(2, 8)),
    ("paper symbol", lambda: pins.test_sine_modes_are_eigenvectors_with_paper_symbol(4, 3, 5)),
    ("printed L_G1", pins.test_first_galerkin_rbc_equals_printed_L_G1),
    ("printed L_2h_G", pins.test_first_galerkin_sc_equals_printed_L_2h_G),
    ("printed transfers", pins.test_transfers_match_printed_stencils),
    ("two-level direct solver", pins.test_two_level_rbc_galerkin_is_direct_solver),
    ("Schur complement", pins.test_red_black_reduction_schur_complement_is_twice_galerkin),
    ("three-level printed rates", pins.test_three_level_rbc_printed_rates),
    ("LFA two-level rate", lambda: pins.test_two_level_rbc_nongalerkin_rate_matches_lfa(1.0)),
    ("Jacobi two-grid RFA", lambda: pins.test_jacobi_two_grid_spectrum_equals_rfa(0.8, 1, 1)),
    ("RBC two-level RFA", lambda: pins.test_two_level_rbc_spectrum_equals_rfa(omg.NONGALERKIN, 0.9, 1, 1)),
    ("cycle operator recursion",
     lambda: pins.test_cycle_operator_equals_error_propagation_recursion(omg.REDBLACK, 2, 0.97, 1, 1, 3)),
    ("converged = direct solve", pins.test_converged_multilevel_solution_equals_direct_solve),
    ("closed-form sine solution", pins.test_converged_solution_equals_closed_form_for_sine_rhs),
]


PERIODIC_BATTERY = [
    ("printed block circulant", ppins.test_five_point_matrix_is_the_printed_block_circulant),
    ("periodic Schur complement", ppins.test_red_black_reduction_schur_complement_is_twice_galerkin),
    ("Fourier eigenvectors", lambda: ppins.test_fourier_modes_are_exact_eigenvectors(4, 3, 5)),
    ("two-level direct solver (periodic)", ppins.test_two_level_rbc_galerkin_is_direct_solver),
    ("discrete LFA rate", lambda: ppins.test_two_level_rate_equals_discrete_lfa("nongalerkin", 1.0)),
    ("zero-mean converged solution", ppins.test_converged_solution_is_the_zero_mean_solution),
    ("printed periodic rates", ppins.test_printed_three_level_and_two_level_sc_rates),
]

CUBIC_BATTERY = [
    ("printed cubic transfers", cpins.test_cubic_transfers_match_printed_stencils),
    ("printed restriction symbol", lambda: cpins.test_restriction_symbol_is_the_printed_one(2, 3)),
    ("tensor cubics reproduced", cpins.test_interpolation_reproduces_tensor_cubics_away_from_the_boundary),
    ("fourth order up to the boundary", cpins.test_interpolation_is_fourth_order_up_to_the_boundary),
    ("cubic transfers converge faster", cpins.test_fourth_order_transfers_and_coarse_operator_converge_faster),
]


def failures(battery=None):
    out = []
    for name, pin in battery or BATTERY:
        try:
            with np.errstate(all="ignore"):
                pin()
        except Exception:  # an assertion, or the mistake breaking the computation
            out.append(name)
    return out


def drop_term(monkeypatch):
    orig = omg.stencil_weights

    def bad(level, stencil, factor):
        st = dict(stencil)
        off = sorted(k for k in st if k != (0, 0))
        st.pop(off[-1])  # one neighbour forgotten
        return orig(level, st, factor)

    monkeypatch.setattr(omg, "stencil_weights", bad)


def flip_sign(monkeypatch):
    orig = omg.stencil_weights

    def bad(level, stencil, factor):
        st = dict(stencil)
        off = sorted(k for k in st if k != (0, 0))
        st[off[0]] = -st[off[0]]  # one neighbour with the wrong sign
        return orig(level, st, factor)

    monkeypatch.setattr(omg, "stencil_weights", bad)


def interpolation_weight(monkeypatch):
    orig = omg.interpolation

    def bad(fine, coarse, coarsening, order=2):
        P = orig(fine, coarse, coarsening, order).tocsr(copy=True)
        P.data = np.where(P.data < 1.0, 2.0 * P.data, P.data)  # averages summed, not averaged
        return P

    monkeypatch.setattr(omg, "interpolation", bad)


def transfer_scale(monkeypatch):
    orig = omg.interpolation
    monkeypatch.setattr(omg, "interpolation", lambda *a, **k: (2.0 * orig(*a, **k)).tocsr())


def black_first(monkeypatch):
    def bad(self, l, u, f):
        u = self.half_sweep(l, u, f, red=False)
        return self.half_sweep(l, u, f, red=True)

    monkeypatch.setattr(omg.Oracle, "smooth", bad)


def residual_sign(monkeypatch):
    def bad(self, l, u, f, red):
        mask = self.levels[l].red if red else ~self.levels[l].red
        r = self._Au(l, u) - f
        return np.where(mask, u + r * self.wd[l], u)

    monkeypatch.setattr(omg.Oracle, "half_sweep", bad)


def jacobi_scaling(monkeypatch):
    def bad(self, l, u, f, red):
        mask = self.levels[l].red if red else ~self.levels[l].red
        r = f - self._Au(l, u)
        return np.where(mask, u + r * self.wd[l] * 0.5, u)  # omega / (2 a_pp)

    monkeypatch.setattr(omg.Oracle, "half_sweep", bad)


def jacobi_without_omega(monkeypatch):
    def bad(self, l, u, f):
        if self.opt.smoother != "jacobi":
            return orig(self, l, u, f)
        r = f - self._Au(l, u)
        return u + r * self.wd[l] / self.opt.omega  # 1 / a_pp: omega forgotten

    orig = omg.Oracle.smooth
    monkeypatch.setattr(omg.Oracle, "smooth", bad)


def gamma_ignored(monkeypatch):
    monkeypatch.setattr(omg.Oracle, "gamma_at", lambda self, l: 1)  # W and Wn run as V


def coarsest_diagonal(monkeypatch):
    def bad(self, d):
        return d / np.diag(self._coarse_dense)

    monkeypatch.setattr(omg.Oracle, "coarse_solve", bad)


def restriction_transposed_weight(monkeypatch):
    orig_init = omg.Oracle.__init__

    def bad(self, *a, **k):
        orig_init(self, *a, **k)
        # R = P^T instead of 1/2 P^T (red-black) / 1/4 P^T (standard) in the cycle
        self._R = [omg.Ell(P.T.tocsr()) for P in self.P]

    monkeypatch.setattr(omg.Oracle, "__init__", bad)


def even_reflection(monkeypatch):
    orig = omg.fold

    def bad(t, n):
        tp, sign, on_boundary = orig(t, n)
        return tp, np.ones_like(sign), on_boundary  # ghosts mirrored without the sign flip

    monkeypatch.setattr(omg, "fold", bad)


def periodic_not_zero_mean(monkeypatch):
    orig = omg.Oracle.coarse_solve

    def bad(self, d):
        v = orig(self, d)
        if self.periodic:  # the singular coarse solve left with a constant in its solution
            v = v + 1.0
        return v

    monkeypatch.setattr(omg.Oracle, "coarse_solve", bad)


def periodic_wrap_dropped(monkeypatch):
    orig = omg.stencil_weights

    def bad(level, stencil, factor):
        if not level.periodic:
            return orig(level, stencil, factor)
        level.periodic = False  # wrap-around terms treated as Dirichlet ghosts
        try:
            return orig(level, stencil, factor)
        finally:
            level.periodic = True

    monkeypatch.setattr(omg, "stencil_weights", bad)


def cubic_as_bilinear(monkeypatch):
    monkeypatch.setattr(omg, "_cubic_interpolation",
                        lambda fine, coarse: omg.interpolation(fine, coarse, omg.STANDARD, 2))


def cubic_taps_swapped(monkeypatch):
    orig = omg._cubic_interpolation

    def bad(fine, coarse):
        P = orig(fine, coarse).tocsr(copy=True)
        P.data = np.where(np.abs(P.data) == 9.0 / 16, P.data * 0.5, P.data)  # 9/32 for 9/16
        return P

    monkeypatch.setattr(omg, "_cubic_interpolation", bad)


MUTATIONS = {
    "even instead of odd reflection at the boundary": even_reflection,
    "dropped stencil term": drop_term,
    "wrong sign of a stencil term": flip_sign,
    "interpolation weights summed": interpolation_weight,
    "transfers scaled by 2": transfer_scale,
    "black half-sweep first": black_first,
    "residual sign in the smoother": residual_sign,
    "relaxation scaled by 1/2": jacobi_scaling,
    "coarsest solve by the diagonal": coarsest_diagonal,
    "Jacobi step without omega": jacobi_without_omega,
    "W cycle visits the coarse level once": gamma_ignored,
    "restriction without its 1/2, 1/4 factor": restriction_transposed_weight,
}


def test_battery_passes_on_the_oracle_as_written():
    assert failures() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    caught = failures()
    assert caught, f"no pin caught: {name}"


def test_periodic_and_cubic_batteries_pass_on_the_oracle_as_written():
    assert failures(PERIODIC_BATTERY) == []
    assert failures(CUBIC_BATTERY) == []


PERIODIC_MUTATIONS = {
    "periodic coarsest solution not normalised to zero mean": periodic_not_zero_mean,
    "periodic wrap-around dropped": periodic_wrap_dropped,
    "dropped stencil term (periodic)": drop_term,
    "black half-sweep first (periodic)": black_first,
}


@pytest.mark.parametrize("name", sorted(PERIODIC_MUTATIONS))
def test_planted_periodic_mistake_is_caught(name, monkeypatch):
    PERIODIC_MUTATIONS[name](monkeypatch)
    assert failures(PERIODIC_BATTERY), f"no periodic pin caught: {name}"


CUBIC_MUTATIONS = {
    "cubic transfers built as bilinear": cubic_as_bilinear,
    "cubic tap 9/16 halved": cubic_taps_swapped,
    "even instead of odd reflection (cubic ghosts)": even_reflection,
}


@pytest.mark.parametrize("name", sorted(CUBIC_MUTATIONS))
def test_planted_cubic_mistake_is_caught(name, monkeypatch):
    CUBIC_MUTATIONS[name](monkeypatch)
    assert failures(CUBIC_BATTERY), f"no cubic pin caught: {name}"


def test_fp64_galerkin_products_fail_the_deep_level_pin(monkeypatch):
    """Planted mistake: the Galerkin recursion in plain FP64 sparse products (no exact
    recursion once the coefficients outgrow 53 bits). The deep-level pin must fail."""
    import test_oracle_deep_galerkin as deep
    monkeypatch.setattr(omg, "_fp64_product_is_exact", lambda *a: True)
    o = omg.Oracle(deep.N, 2, omg.REDBLACK, omg.GALERKIN)
    with pytest.raises(AssertionError):
        deep.test_deep_galerkin_rows_are_the_exact_product_rounded_once(o, 19)


import test_oracle_dense_coarse as dpins

DENSE_BATTERY = [
    ("exact rational solution", lambda: dpins.test_dense_solve_matches_exact_rational_solution(
        4, omg.REDBLACK, omg.GALERKIN, 8)),
    ("library Cholesky factor", lambda: dpins.test_inverse_factor_inverts_the_library_cholesky_factor(8)),
    ("single-level closed form", lambda: dpins.test_single_level_hierarchy_is_the_closed_form_solve(4)),
    ("two-level direct solver (dense)", dpins.test_two_level_direct_solver_with_dense_coarsest_level),
]


def dense_not_transposed(monkeypatch):
    """Back substitution with G instead of G^T."""
    orig = omg.Oracle.coarse_solve

    def bad_solve(self, d):
        if self._coarse_G is None:
            return orig(self, d)
        y = self._coarse_G @ d
        return self._coarse_G @ y
    monkeypatch.setattr(omg.Oracle, "coarse_solve", bad_solve)


def dense_inverse_sign(monkeypatch):
    """The inverse factor's off-diagonal entries without their minus sign."""
    orig = omg.dense_coarse_factor

    def bad(A):
        G = orig(A)
        return np.diag(np.diag(G)) - np.tril(G, -1)
    monkeypatch.setattr(omg, "dense_coarse_factor", bad)


def dense_pivot_not_inverted(monkeypatch):
    """L_ij = t / r_j written as t * L_jj (the pivot not inverted) in the factor."""
    def bad(A):
        m = A.shape[0]
        L = np.zeros((m, m))
        for j in range(m):
            s = A[j, j] - np.dot(L[j, :j], L[j, :j])
            L[j, j] = np.sqrt(s)
            L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) * L[j, j]
        return np.linalg.inv(L)
    monkeypatch.setattr(omg, "dense_coarse_factor", bad)


DENSE_MUTATIONS = {
    "dense coarsest: back substitution with G, not G^T": dense_not_transposed,
    "dense coarsest: inverse factor sign dropped": dense_inverse_sign,
    "dense coarsest: pivot not inverted": dense_pivot_not_inverted,
}


def test_dense_battery_passes_on_the_oracle_as_written():
    assert failures(DENSE_BATTERY) == []


@pytest.mark.parametrize("name", sorted(DENSE_MUTATIONS))
def test_planted_dense_coarsest_mistake_is_caught(name, monkeypatch):
    DENSE_MUTATIONS[name](monkeypatch)
    assert failures(DENSE_BATTERY), f"no dense-coarsest pin caught: {name}"
