"""Pins of the periodic oracle (the paper's computational setting, Sec. 2.2) against
what the paper and the mathematics fix: the printed block-circulant matrix, the
red-black reduction, exact Fourier eigenvectors, local Fourier analysis (exact on
periodic grids), the two-level direct-solver theorem, and the printed rates."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import lfa
from oracle.mg import (G1, GALERKIN, GN, NONGALERKIN, PERIODIC, REDBLACK, STANDARD, TRUE_HIGH,
                       VARIABLE, Options, Oracle)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def per(n, order=2, co=REDBLACK, op=GALERKIN, **opts):
    return Oracle(n, order, co, op, Options(**opts), boundary=PERIODIC)


def test_five_point_matrix_is_the_printed_block_circulant():
    """Sec. "Red-black reduction in two dimensions": row-wise ordering gives blocks
    T (4 on the diagonal, -1 beside it and in the corners) and -I, block-cyclic."""
    for n in (4, 8, 16):
        o = per(n)
        C = np.roll(np.eye(n), 1, axis=1) + np.roll(np.eye(n), -1, axis=1)  # cyclic neighbours
        T = 4.0 * np.eye(n) - C
        A = np.kron(np.eye(n), T) - np.kron(C, np.eye(n))
        assert np.array_equal(o.levels[0].W.toarray(), A)
        assert o.levels[0].s == float(n * n)


def test_red_black_reduction_schur_complement_is_twice_galerkin():
    """Eliminating the red unknowns of the periodic 5-point matrix (the factorisation
    A = L diag(4I, A_H) L^T of that section) leaves 2 R A P on the black points."""
    n = 16
    o = per(n)
    lev = o.levels[0]
    A = lev.A.toarray()
    red, blk = lev.red, ~lev.red
    Arr, Arb, Abr, Abb = A[np.ix_(red, red)], A[np.ix_(red, blk)], A[np.ix_(blk, red)], A[np.ix_(blk, blk)]
    assert np.array_equal(Arr, 4.0 * n * n * np.eye(red.sum()))
    S = Abb - Abr @ np.diag(1.0 / np.diag(Arr)) @ Arb
    assert np.array_equal(lev.pi[blk], o.levels[1].pi) and np.array_equal(lev.pj[blk], o.levels[1].pj)
    assert np.array_equal(S, 2.0 * o.levels[1].A.toarray())


def _symbol(order, t1, t2, h):
    if order == 2:
        return lfa.symbol_L2(t1, t2, h)
    if order == 4:
        return lfa.symbol_L4(t1, t2, h)
    axis = lambda t: 490 - 540 * math.cos(t) + 54 * math.cos(2 * t) - 4 * math.cos(3 * t)
    return (axis(t1) + axis(t2)) / (180.0 * h * h)


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("k,l", [(1, 0), (3, 5), (7, 2), (8, 8)])
def test_fourier_modes_are_exact_eigenvectors(order, k, l):
    """cos(2 pi k x) cos(2 pi l y) is an eigenvector of the periodic operator with
    eigenvalue = the symbol at theta = 2 pi (k, l) h (no boundary closure at all)."""
    n = 16
    o = per(n, order)
    v = o.to_vec(synth.rhs_periodic_mode(n, k, l))
    lam = _symbol(order, 2 * math.pi * k / n, 2 * math.pi * l / n, 1.0 / n)
    assert np.max(np.abs(o.apply(0, v) - lam * v)) <= 1e-12 * lam * np.max(np.abs(v))


@pytest.mark.parametrize("co,op,order", [(REDBLACK, GALERKIN, 2), (REDBLACK, NONGALERKIN, 4),
                                         (REDBLACK, G1, 2), (REDBLACK, GN, 2), (REDBLACK, TRUE_HIGH, 4),
                                         (STANDARD, GALERKIN, 6), (VARIABLE, GALERKIN, 4)])
def test_every_level_annihilates_constants_and_coarsens_to_one_node(co, op, order):
    """The constants span the null space of every periodic level (rows sum to 0
    exactly); the hierarchy ends in a single node whose operator row is 0."""
    o = per(32, order, co, op)
    for lev in o.levels:
        assert np.all(lev.W @ np.ones(lev.size) == 0.0)
    assert o.levels[-1].size == 1 and o.levels[-1].A.toarray()[0, 0] == 0.0
    # interpolation reproduces constants; restriction keeps zero sums at zero
    for P, R in zip(o.P, o.R):
        assert np.all(P @ np.ones(P.shape[1]) == 1.0)
        x = synth.normal(3, R.shape[1])
        x -= x.mean()
        assert abs(np.sum(R @ x)) <= 1e-13 * np.sum(np.abs(x))


def test_level_sizes():
    assert [lev.size for lev in per(16).levels] == [256, 128, 64, 32, 16, 8, 4, 2, 1]
    assert [lev.size for lev in per(16, co=STANDARD).levels] == [256, 64, 16, 4, 1]


def test_two_level_rbc_galerkin_is_direct_solver():
    """Theorem (Sec. 4.3) on the periodic grid: one cycle solves exactly."""
    n = 32
    for nu1, nu2 in ((1, 1), (0, 1)):
        o = per(n, nu1=nu1, nu2=nu2, max_levels=2)
        f = o.to_vec(synth.rhs_periodic_normal(n, 3))
        _, h = o.solve(f, max_cycles=1, fixed_cycles=True)
        assert h[1] < 1e-13


def _power_cr(o, iters=60, seed=5):
    """Asymptotic residual reduction per cycle: power iteration on the error
    (f = 0), the constant (null-space) component removed each step."""
    u = o.to_vec(synth.rhs_periodic_normal(o.n, seed))
    z = np.zeros_like(u)
    r = 0.0
    for _ in range(iters):
        d0 = np.linalg.norm(o.apply(0, u))
        u = o.cycle(u, z)
        d1 = np.linalg.norm(o.apply(0, u))
        r = d1 / d0
        u = (u - u.mean()) / d1
    return r


@pytest.mark.parametrize("coarse,omega", [("nongalerkin", 0.8), ("nongalerkin", 1.0),
                                          ("nongalerkin", 1.1), ("galerkin", 0.9)])
def test_two_level_rate_equals_discrete_lfa(coarse, omega):
    """LFA is exact on a periodic grid: the measured two-level RBC rate equals the
    largest spectral radius of the 2x2 symbols (Sec. 4.3) over the grid's frequencies."""
    n = 32
    rho = lfa.rbc_two_level_rho_periodic(n, omega, 1, 1, coarse)
    o = per(n, op=NONGALERKIN if coarse == "nongalerkin" else GALERKIN, omega=omega, max_levels=2)
    assert _power_cr(o) == pytest.approx(rho, rel=1e-2)


def test_converged_solution_is_the_zero_mean_solution():
    """Converged cycles give the minimum-norm solution up to a constant; a single
    Fourier mode is solved by f / symbol."""
    n = 32
    for order, co, op in ((2, REDBLACK, GALERKIN), (4, REDBLACK, NONGALERKIN), (4, STANDARD, GALERKIN)):
        o = per(n, order, co, op, nu1=2 if order == 4 else 1)
        f = o.to_vec(synth.rhs_periodic_normal(n, 7))
        u, _ = o.solve(f, rtol=1e-13, max_cycles=40)
        ud = o.direct(f)
        assert np.max(np.abs((u - u.mean()) - (ud - ud.mean()))) <= 1e-11 * np.max(np.abs(ud))
        k, l = 3, 5
        f = o.to_vec(synth.rhs_periodic_mode(n, k, l))
        lam = _symbol(order, 2 * math.pi * k / n, 2 * math.pi * l / n, 1.0 / n)
        u, _ = o.solve(f, rtol=1e-14, max_cycles=40)
        assert np.max(np.abs((u - u.mean()) - f / lam)) <= 1e-12 * np.max(np.abs(f / lam))


def _cr(o, seed=5, cycles=12):
    f = o.to_vec(synth.rhs_periodic_normal(o.n, seed))
    _, h = o.solve(f, max_cycles=cycles, fixed_cycles=True)
    rates = [h[i + 1] / h[i] for i in range(len(h) - 1) if h[i + 1] > 1e-12]
    return rates[-1]


def _in_band(ref, x):
    lo, hi = ref["band"]
    return lo * ref["value"] <= x <= hi * ref["value"]


def test_printed_three_level_and_two_level_sc_rates():
    g = golden("paper_rates_periodic.json")
    ref = g["rbc_3level_W11_g1_cr"]
    cr = _cr(per(ref["N"], op=ref["coarse_op"], omega=ref["omega"], gamma=2, max_levels=3))
    assert _in_band(ref, cr), cr
    ref = g["rbc_3level_V11_best_cr"]
    cr = min(_cr(per(ref["N"], op=op, omega=w, max_levels=3)) for op in ref["coarse_ops"] for w in ref["omegas"])
    assert _in_band(ref, cr), cr
    ref = g["sc_2level_V11_galerkin_cr"]
    cr = min(_cr(per(ref["N"], co=STANDARD, omega=w, max_levels=2)) for w in ref["omegas"])
    assert _in_band(ref, cr), cr


def test_printed_multilevel_ecr():
    g = golden("paper_rates_periodic.json")
    nu = 2
    ref = g["rbc_7level_V11_ecr"]
    cr = min(_cr(per(ref["N"], op=op, omega=w, max_levels=7)) for op in ref["coarse_ops"] for w in ref["omegas"])
    assert _in_band(ref, cr ** (1.0 / (2 * (nu + 2)))), cr
    ref = g["rbc_7level_W11_ecr"]
    cr_w = _cr(per(ref["N"], op=ref["coarse_op"], omega=ref["omega"], gamma=2, max_levels=7), cycles=6)
    assert _in_band(ref, cr_w ** (1.0 / (6 * (nu + 2)))), cr_w
    ref = g["sc_4level_V11_ecr"]
    cr = min(_cr(per(ref["N"], co=STANDARD, op=ref["coarse_op"], omega=w, max_levels=4)) for w in ref["omegas"])
    assert _in_band(ref, cr ** (1.0 / (4.0 / 3.0 * (nu + 2)))), cr
    ref = g["rbc_7level_Wn11_vs_W11_cr"]
    cr_wn = _cr(per(ref["N"], op=ref["coarse_op"], omega=ref["omega"], gamma=3, max_levels=7), cycles=6)
    assert _in_band(ref, cr_wn / cr_w), (cr_wn, cr_w)
    ref = g["vc_5level_W11_ecr"]
    cr = _cr(per(ref["N"], co=VARIABLE, op=ref["coarse_op"], omega=ref["omega"], gamma=2, max_levels=5), cycles=6)
    assert _in_band(ref, cr ** (1.0 / ((nu + 2) * (1 + 2 / 2 + 4 / 4 + 8 / 16)))), cr


def test_printed_three_level_ecr_and_operator_ranking():
    """App. A: three-level V[1,1] / W[1,1] ECR with Galerkin coarse operators (WU from
    the appendix formula, which counts the coarsest solve), and the ranking stated
    there: the true Galerkin operator is best for V and W, G1 and Gn close behind for W."""
    g = golden("paper_rates_periodic.json")
    for key, gamma, wu in (("rbc_3level_V11_galerkin_ecr", 1, 10.0), ("rbc_3level_W11_galerkin_ecr", 2, 16.0)):
        ref = g[key]
        cr = min(_cr(per(ref["N"], op=GALERKIN, omega=w, gamma=gamma, max_levels=3)) for w in ref["omegas"])
        assert _in_band(ref, cr ** (1.0 / wu)), (key, cr)
    for gamma in (1, 2):
        crs = {op: _cr(per(32, op=op, gamma=gamma, max_levels=3)) for op in (GALERKIN, G1, GN, NONGALERKIN)}
        assert crs[GALERKIN] == min(crs.values()), crs
        if gamma == 2:
            assert max(crs[G1], crs[GN]) < 0.1 * crs[NONGALERKIN], crs


def test_printed_fourth_order_two_level_ecr():
    """Sec. 4.4: fourth-order fine operator, red-black coarsening, second-order
    non-Galerkin coarse operator: two-level V[1,1] ECR 0.6 (WU = 2 (nu + 2))."""
    ref = golden("paper_rates_periodic.json")["rbc_2level_V11_order4_ng2_ecr"]
    cr = min(_cr(per(ref["N"], 4, op=NONGALERKIN, omega=w, max_levels=2)) for w in ref["omegas"])
    assert _in_band(ref, cr ** (1.0 / 8.0)), cr
