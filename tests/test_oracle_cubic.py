"""Pins of the oracle's cubic transfers (App. A, Eq. interp_2d4o / restr_2d4o) and
fourth-order non-Galerkin coarse operator (Eq. L_H_4n_2d) against the printed
stencils, the printed restriction symbol, polynomial exactness, the order of accuracy,
an exact rational Galerkin recursion, and the paper's remark on convergence."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle.mg import (DIRICHLET, FOURTH_ORDER, GALERKIN, NONGALERKIN, NONGALERKIN_HIGH, PERIODIC,
                       STANDARD, TRUE_HIGH, Options, Oracle)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def printed(entry):
    w = np.array(entry["weights"], dtype=float)
    r = w.shape[0] // 2
    return {(col - r, r - row): w[row, col] for row in range(w.shape[0]) for col in range(w.shape[1])
            if w[row, col] != 0}


def cubic(n, op=GALERKIN, boundary=DIRICHLET, order=4, **opts):
    return Oracle(n, order, STANDARD, op, Options(transfer_order=4, **opts), boundary=boundary)


def test_cubic_transfers_match_printed_stencils():
    g = golden("paper_stencils.json")
    o = cubic(32)
    f0, c1 = o.levels[0], o.levels[1]
    c = c1.index[8, 8]  # coarse node (8, 8) = fine node (16, 16)
    row = o.R[0].getrow(c)
    got = {(int(f0.pi[q] - 16), int(f0.pj[q] - 16)): v for q, v in zip(row.indices, row.data)}
    assert got == {k: w / 1024 for k, w in printed(g["restriction_cubic"]).items()}
    col = o.P[0].getcol(c).tocoo()
    got = {(int(f0.pi[q] - 16), int(f0.pj[q] - 16)): v for q, v in zip(col.row, col.data)}
    assert got == {k: w / 256 for k, w in printed(g["interpolation_cubic"]).items()}
    assert abs(o.P[0] - 4 * o.R[0].T).max() == 0


@pytest.mark.parametrize("k,l", [(1, 0), (2, 3), (5, 7), (8, 1)])
def test_restriction_symbol_is_the_printed_one(k, l):
    """On a periodic grid R maps the fine mode cos(t1 i) cos(t2 j) to I(t) times the
    coarse mode, I(t) = prod [1 - sin^4(t/2) (3 - 2 sin^2(t/2))] (App. A)."""
    n = 32
    o = cubic(n, boundary=PERIODIC)
    fine = o.to_vec(synth.rhs_periodic_mode(n, k, l))
    t1, t2 = 2 * math.pi * k / n, 2 * math.pi * l / n
    sym = lambda t: 1 - math.sin(t / 2) ** 4 * (3 - 2 * math.sin(t / 2) ** 2)
    coarse = o.to_vec(synth.rhs_periodic_mode(n // 2, k, l), 1)
    assert np.max(np.abs(o.restrict(0, fine) - sym(t1) * sym(t2) * coarse)) <= 1e-14


def test_interpolation_reproduces_tensor_cubics_away_from_the_boundary():
    n = 32
    o = cubic(n)
    f0, c1 = o.levels[0], o.levels[1]
    p = lambda x, y: (x ** 3 - 2 * x ** 2 + x / 3 + 0.1) * (y ** 3 + y ** 2 - y + 0.2)
    uf = p(f0.pi / n, f0.pj / n)
    uc = p(c1.pi / (n // 2), c1.pj / (n // 2))
    # every cubic tap (fine offsets up to 3) on an interior coarse node
    inside = (f0.pi >= 5) & (f0.pi <= n - 5) & (f0.pj >= 5) & (f0.pj <= n - 5)
    assert np.max(np.abs((o.prolong(0, uc) - uf)[inside])) <= 1e-14


def test_interpolation_is_fourth_order_up_to_the_boundary():
    """Odd-reflection ghosts keep the fourth order next to the boundary for data that
    vanish there (sines): the error falls 16x per halving of h; bilinear gives 4x."""
    errs = {}
    for to in (2, 4):
        e = []
        for n in (32, 64):
            o = Oracle(n, 4, STANDARD, GALERKIN, Options(transfer_order=to))
            s = lambda lev, m: np.sin(math.pi * lev.pi / m) * np.sin(2 * math.pi * lev.pj / m)
            e.append(np.max(np.abs(o.prolong(0, s(o.levels[1], n // 2)) - s(o.levels[0], n))))
        errs[to] = e[0] / e[1]
    assert 14.0 <= errs[4] <= 18.0 and 3.5 <= errs[2] <= 4.5, errs


def test_nongalerkin_high_is_the_fourth_order_stencil_with_spacing_H():
    """Eq. (L_H_4n_2d): the fine fourth-order stencil with h replaced by H = 2h."""
    n = 32
    o = Oracle(n, 4, STANDARD, NONGALERKIN_HIGH)
    lev = o.levels[1]
    row = lev.A.getrow(lev.index[8, 8])
    got = {(int(lev.pi[q] - 8), int(lev.pj[q] - 8)): v for q, v in zip(row.indices, row.data)}
    H = 2.0 / n
    assert got == {k: w / (12 * H * H) for k, w in FOURTH_ORDER.items()}


# ---- exact Galerkin recursion: independent rational convolution on the lattice ----
def _conv(a, b):
    out = {}
    for (x1, y1), w1 in a.items():
        for (x2, y2), w2 in b.items():
            out[(x1 + x2, y1 + y2)] = out.get((x1 + x2, y1 + y2), 0) + w1 * w2
    return {k: v for k, v in out.items() if v != 0}


def _galerkin_fraction(W):
    taps = {0: Fraction(1), 1: Fraction(9, 16), -1: Fraction(9, 16), 3: Fraction(-1, 16), -3: Fraction(-1, 16)}
    P = {(a, b): taps[a] * taps[b] for a in taps for b in taps}
    T = _conv(P, _conv(W, P))  # R W P with R = P^T / 4 on the infinite lattice
    return {(a // 2, b // 2): v / 4 for (a, b), v in T.items() if a % 2 == 0 and b % 2 == 0}


@pytest.mark.parametrize("op", [GALERKIN, TRUE_HIGH])
def test_galerkin_recursion_is_exact_and_rounded_once(op):
    """Level l's periodic row = the exact infinite-lattice Galerkin stencil, wrapped
    (exact sums), rounded once; the exact values outgrow 53 bits from level 4 on."""
    n = 128
    o = cubic(n, op, boundary=PERIODIC)
    if op == GALERKIN:
        W = {(0, 0): Fraction(4), (1, 0): Fraction(-1), (-1, 0): Fraction(-1), (0, 1): Fraction(-1), (0, -1): Fraction(-1)}
    else:
        W = {k: Fraction(int(v)) for k, v in FOURTH_ORDER.items()}
    inexact = 0
    for l in range(1, len(o.levels) - 1):
        W = _galerkin_fraction(W)
        lev = o.levels[l]
        m = lev.n
        row = {}
        for (a, b), v in W.items():
            row[(a % m, b % m)] = row.get((a % m, b % m), 0) + v
        inexact += any(float(v) != v for v in row.values())
        want = {k: float(v) for k, v in row.items() if v != 0}
        r = lev.W.getrow(lev.index[0, 0])
        got = {(int(lev.pi[q]), int(lev.pj[q])): x for q, x in zip(r.indices, r.data) if x != 0}
        assert got == want, l
    assert inexact >= 2  # the single rounding matters on the deep levels


def test_fourth_order_transfers_and_coarse_operator_converge_faster():
    """App. A: fourth-order transfers with fourth-order coarse operators bring the rates
    closer to the smoothing rate. Two- and three-level V(1,1), nG^(4), periodic N = 64,
    best over omega: cubic transfers beat bilinear by a clear margin."""
    def power_cr(o, iters=40, seed=5):
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
    for levels in (2, 3):
        best = {to: min(power_cr(Oracle(64, 4, STANDARD, NONGALERKIN_HIGH,
                                        Options(omega=w, transfer_order=to, max_levels=levels),
                                        boundary=PERIODIC)) for w in (1.0, 1.1, 1.2))
                for to in (2, 4)}
        assert best[4] < 0.75 * best[2], (levels, best)


@pytest.mark.parametrize("op", [GALERKIN, TRUE_HIGH, NONGALERKIN_HIGH, NONGALERKIN])
def test_cubic_hierarchies_are_spd_and_converge(op):
    o = cubic(32, op, nu1=2)
    for lev in o.levels:
        A = lev.A.toarray()
        assert np.abs(A - A.T).max() == 0
        assert np.linalg.eigvalsh(A).min() > 0
    f = o.to_vec(synth.rhs_normal(32, 3))
    u, h = o.solve(f, rtol=1e-12, max_cycles=30)
    assert h[-1] < 1e-12 and len(h) <= 14
