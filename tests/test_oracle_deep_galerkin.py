"""Pin of the oracle's deep Galerkin levels (Eq. L_G_l, Sec. 4.4), where the recursion's
dyadic coefficients need more than FP64's 53 bits (red-black coarsening: the interior
stencil from level 19, about 3 bits more per level).

Reading: the recursion L_{l+1} = R L_l P is exact and each level is rounded once to
FP64. The reference here is independent of the oracle's sparse products: the
infinite-lattice stencil recursion in exact rationals (fractions.Fraction) with the
paper's transfers (Eq. transfer_r2: interpolation 1/4 from the four neighbours, R = 1/2
P^T), folded onto the Dirichlet level by odd reflection (the reading that makes the
truncated matrices' product equal the folded infinite-lattice product), merged exactly,
then rounded once. Every row of the oracle's deep levels must equal it bit for bit."""
from fractions import Fraction

import numpy as np
import pytest

from oracle.mg import GALERKIN, REDBLACK, Oracle

N = 2048  # 21 levels; levels 19 and 20 need more than 53 bits


def taps(kind):
    """Interpolation taps ((dx, dy), weight) from a coarse node at the origin, on the fine
    level's lattice: an axis level interpolates its red nodes from the four axis
    neighbours, a rotated level its odd-i nodes from the four diagonal neighbours."""
    q = Fraction(1, 4)
    if kind == "axis":
        return [((0, 0), Fraction(1)), ((1, 0), q), ((-1, 0), q), ((0, 1), q), ((0, -1), q)]
    return [((0, 0), Fraction(1)), ((1, 1), q), ((-1, 1), q), ((1, -1), q), ((-1, -1), q)]


def galerkin(W, kind):
    """Coarse stencil R W P on the infinite lattice. Axis -> rotated: coarse nodes are the
    fine lattice's black points (offsets with a + b even, same lattice units); rotated ->
    axis: coarse nodes are the even points, coarse offset (a, b) = fine offset (2a, 2b)."""
    P = taps(kind)
    step = 1 if kind == "axis" else 2
    out = {}
    for b in range(-8, 9):
        for a in range(-8, 9):
            if kind == "axis" and (a + b) % 2:
                continue
            v = {}
            for (dx, dy), w in P:
                key = (step * a + dx, step * b + dy)
                v[key] = v.get(key, 0) + w
            g = Fraction(0)
            for (rx, ry), rw in P:
                s = sum((ww * v.get((rx + wx, ry + wy), 0) for (wx, wy), ww in W.items()), Fraction(0))
                g += Fraction(1, 2) * rw * s
            if g:
                out[(a, b)] = g
    return out


def fold_row(W, n, i, j):
    row = {}
    for (dx, dy), w in W.items():
        t = []
        for x in (i + dx, j + dy):
            m = x % (2 * n)
            t.append((m, 1) if m <= n else (2 * n - m, -1))
        (ti, si), (tj, sj) = t
        if ti in (0, n) or tj in (0, n):
            continue
        row[(ti, tj)] = row.get((ti, tj), 0) + si * sj * w
    return {k: v for k, v in row.items() if v}


@pytest.fixture(scope="module")
def oracle():
    return Oracle(N, 2, REDBLACK, GALERKIN)


def test_deep_levels_need_more_than_53_bits(oracle):
    """The premise: without the exact recursion these levels would be rounded."""
    W = {(0, 0): Fraction(4), (1, 0): Fraction(-1), (-1, 0): Fraction(-1), (0, 1): Fraction(-1),
         (0, -1): Fraction(-1)}
    for l in range(1, 19):
        W = galerkin(W, oracle.levels[l - 1].kind)
    # dyadic values: the significant bits are those of the (odd) reduced numerator
    assert max(abs(w.numerator).bit_length() for w in W.values()) <= 53
    W = galerkin(W, oracle.levels[18].kind)
    assert max(abs(w.numerator).bit_length() for w in W.values()) > 53


@pytest.mark.parametrize("level", [17, 18, 19, 20])
def test_deep_galerkin_rows_are_the_exact_product_rounded_once(oracle, level):
    W = {(0, 0): Fraction(4), (1, 0): Fraction(-1), (-1, 0): Fraction(-1), (0, 1): Fraction(-1),
         (0, -1): Fraction(-1)}
    for l in range(1, level + 1):
        W = galerkin(W, oracle.levels[l - 1].kind)
    lev = oracle.levels[level]
    M = lev.W.tocsr()
    for r in range(lev.size):
        i, j = int(lev.pi[r]), int(lev.pj[r])
        got = {(int(lev.pi[c]), int(lev.pj[c])): v for c, v in zip(M.indices[M.indptr[r]:M.indptr[r + 1]],
                                                                 M.data[M.indptr[r]:M.indptr[r + 1]]) if v != 0}
        want = {k: float(v) for k, v in fold_row(W, lev.n, i, j).items()}
        assert got == want, (level, i, j)
