"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (on the CPU, through monkeypatch: a
dropped stencil term, a wrong sign, a wrong transfer weight, a swapped colour order,
a wrong residual sign, a wrong coarsest solve, a wrong relaxation scaling) and runs
a battery of the pins of `test_oracle.py` (printed stencils, the paper's symbol,
printed Galerkin operators and transfers, the two-level direct-solver theorem, the
Schur-complement identity, printed rates and the LFA rate, agreement with a direct
solve). At least one pin must fail for every mistake, and none without one.
"""
import numpy as np
import pytest

import oracle.mg as omg
import test_oracle as pins

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
    ("converged = direct solve", pins.test_converged_multilevel_solution_equals_direct_solve),
    ("closed-form sine solution", pins.test_converged_solution_equals_closed_form_for_sine_rhs),
]


def failures():
    out = []
    for name, pin in BATTERY:
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


MUTATIONS = {
    "dropped stencil term": drop_term,
    "wrong sign of a stencil term": flip_sign,
    "interpolation weights summed": interpolation_weight,
    "transfers scaled by 2": transfer_scale,
    "black half-sweep first": black_first,
    "residual sign in the smoother": residual_sign,
    "relaxation scaled by 1/2": jacobi_scaling,
    "coarsest solve by the diagonal": coarsest_diagonal,
    "restriction without its 1/2, 1/4 factor": restriction_transposed_weight,
}


def test_battery_passes_on_the_oracle_as_written():
    assert failures() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    caught = failures()
    assert caught, f"no pin caught: {name}"
