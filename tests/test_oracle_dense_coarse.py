"""Pins of the oracle's exact coarsest solve for more than one unknown.

Algorithm "MG" (Sec. 2.2) solves the coarsest level exactly. With n_min > 2 (or a
truncated hierarchy) the coarsest Dirichlet system has many unknowns; the oracle factors
it once (Cholesky, inverse factor G = L^-1) and solves x = G^T (G d) in a fixed order.
Pinned here against things that do not share its arithmetic: the exact rational solution
(brute force on small systems), LAPACK's Cholesky factor, the closed-form Fourier
solution of the fine operator when the hierarchy is a single level, and the two-level
direct-solver theorem with a dense coarsest level."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import spectral
from oracle.mg import (GALERKIN, NONGALERKIN, REDBLACK, STANDARD, Options, Oracle, dense_coarse_factor,
                       dense_coarse_solve)

EPS = np.finfo(np.float64).eps


def _exact_solve(A: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Gaussian elimination in rational arithmetic (A's and d's FP64 values taken exactly)."""
    m = A.shape[0]
    M = [[Fraction(float(A[i, j])) for j in range(m)] + [Fraction(float(d[i]))] for i in range(m)]
    for c in range(m):
        p = next(r for r in range(c, m) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(c + 1, m):
            if M[r][c] != 0:
                q = M[r][c] / M[c][c]
                M[r] = [a - q * b for a, b in zip(M[r], M[c])]
    x = [Fraction(0)] * m
    for r in range(m - 1, -1, -1):
        s = M[r][m] - sum(M[r][k] * x[k] for k in range(r + 1, m))
        x[r] = s / M[r][r]
    return np.array([float(v) for v in x])


@pytest.mark.parametrize("order,co,op,n_min", [(2, STANDARD, NONGALERKIN, 4), (4, REDBLACK, GALERKIN, 4),
                                               (4, REDBLACK, GALERKIN, 8), (2, STANDARD, GALERKIN, 8)])
def test_dense_solve_matches_exact_rational_solution(order, co, op, n_min):
    o = Oracle(32, order, co, op, Options(n_min=n_min))
    A = o._coarse_dense
    m = A.shape[0]
    assert m == (n_min - 1) ** 2 and o._coarse_G is not None
    d = np.random.default_rng(n_min + order).standard_normal(m)
    x = o.coarse_solve(d)
    xe = _exact_solve(A, d)
    kappa = np.linalg.cond(A)
    # forward error of a backward-stable solve: a small multiple of m eps kappa
    assert np.max(np.abs(x - xe)) <= 4 * m * EPS * kappa * np.max(np.abs(xe)), (np.max(np.abs(x - xe)), kappa)


@pytest.mark.parametrize("n_min", [8, 16, 32])
def test_inverse_factor_inverts_the_library_cholesky_factor(n_min):
    o = Oracle(64, 4, REDBLACK, GALERKIN, Options(n_min=n_min))
    A = o._coarse_dense
    G = o._coarse_G
    m = A.shape[0]
    assert np.array_equal(np.triu(G, 1), np.zeros_like(G)) and np.all(np.diag(G) > 0)
    Lref = np.linalg.cholesky(A)
    assert np.max(np.abs(G @ Lref - np.eye(m))) <= 8 * m * EPS * np.linalg.cond(Lref)
    # and G A G^T = I
    assert np.max(np.abs(G @ A @ G.T - np.eye(m))) <= 8 * m * EPS * np.linalg.cond(A)


@pytest.mark.parametrize("order", [2, 4])
def test_single_level_hierarchy_is_the_closed_form_solve(order):
    """n_min = N: the hierarchy is level 0 alone and one cycle is the exact solve; it must
    equal the Fourier (DST-I) solution of the fine operator."""
    n = 16
    o = Oracle(n, order, REDBLACK, GALERKIN, Options(n_min=n))
    assert o.lmax == 0 and o._coarse_G is not None
    F = synth.rhs_normal(n, seed=21 + order)
    u = o.cycle(np.zeros(o.levels[0].size), o.to_vec(F))
    us = o.to_vec(spectral.solve(F, order))
    assert np.linalg.norm(u - us) <= 1e-13 * np.linalg.norm(us)


def test_two_level_direct_solver_with_dense_coarsest_level():
    """The two-level theorem (Sec. 4.3: red-black relaxation plus the Galerkin coarse
    operator on the black points, omega = 1, solves the 5-point problem in one cycle)
    holds with the dense coarsest solve as the exact coarse solve."""
    for n in (8, 32):
        o = Oracle(n, 2, REDBLACK, GALERKIN, Options(nu1=1, nu2=1, max_levels=2))
        assert o._coarse_G is not None
        f = o.to_vec(synth.rhs_normal(n, 4))
        _, h = o.solve(f, max_cycles=1, fixed_cycles=True)
        assert h[1] < 1e-13


def test_solve_order_is_the_stated_one():
    """x = G^T (G d) with the stated summation order, checked by summing in Python floats
    term by term on a small factor."""
    o = Oracle(16, 4, REDBLACK, GALERKIN, Options(n_min=4))
    G = o._coarse_G
    m = G.shape[0]
    d = np.random.default_rng(3).standard_normal(m)
    y = []
    for i in range(m):
        s = float(G[i, 0]) * float(d[0])
        for k in range(1, i + 1):
            s = s + float(G[i, k]) * float(d[k])
        y.append(s)
    x = []
    for i in range(m):
        s = float(G[i, i]) * y[i]
        for k in range(i + 1, m):
            s = s + float(G[k, i]) * y[k]
        x.append(s)
    assert np.array_equal(dense_coarse_solve(G, d), np.array(x))


def test_factor_rejects_an_indefinite_matrix():
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(AssertionError):
        dense_coarse_factor(A)
