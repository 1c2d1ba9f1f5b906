"""Pins of the oracle's Fourier-diagonalisation solver (oracle/spectral.py).

The spectral solver gives A^-1 f from the fine operator's symbol (Sec. 2.4; Eq. xi_r2,
Eq. L_hat_2d_4o) without assembling a matrix. It is pinned here to the sparse LU
(Dirichlet) or least-squares (periodic, zero-mean) solve of the oracle's own assembled
level-0 matrix, an independent route, on grids small enough for both."""
import numpy as np
import pytest

import synth
from oracle import spectral
from oracle.mg import GALERKIN, PERIODIC, REDBLACK, Oracle


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("n", [8, 32])
def test_dirichlet_spectral_solution_equals_sparse_direct_solve(order, n):
    F = synth.rhs_normal(n, seed=11 + n)
    o = Oracle(n, order, REDBLACK, GALERKIN)
    ud = o.direct(o.to_vec(F))
    us = o.to_vec(spectral.solve(F, order))
    assert np.linalg.norm(us - ud) <= 1e-13 * np.linalg.norm(ud)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_periodic_spectral_solution_equals_zero_mean_least_squares(order):
    n = 16
    F = synth.rhs_periodic_normal(n, seed=4)
    o = Oracle(n, order, REDBLACK, GALERKIN, boundary=PERIODIC)
    ud = o.direct(o.to_vec(F))
    U = spectral.solve(F, order, periodic=True)
    us = o.to_vec(U)
    assert abs(us.mean()) < 1e-13 * np.abs(us).max()
    assert np.linalg.norm(us - ud) <= 1e-12 * np.linalg.norm(ud)
    assert np.array_equal(U[n, :], U[0, :]) and np.array_equal(U[:, n], U[:, 0])


def test_domain_length_scales_the_solution_by_length_squared():
    n = 16
    F = synth.rhs_normal(n, seed=2)
    u1 = spectral.solve(F, 4)
    u3 = spectral.solve(F, 4, length=3.0)
    assert np.allclose(u3, 9.0 * u1, rtol=1e-13, atol=0)
    o = Oracle(n, 4, REDBLACK, GALERKIN, length=3.0)
    ud = o.direct(o.to_vec(F))
    assert np.linalg.norm(o.to_vec(u3) - ud) <= 1e-13 * np.linalg.norm(ud)


def test_single_mode_solution_is_the_mode_over_the_symbol():
    """f = sin(k pi x) sin(l pi y) gives u = f / symbol exactly (up to rounding)."""
    n, k, l = 64, 5, 9
    F = synth.rhs_single_mode(n, k, l)
    from oracle import lfa
    lam = lfa.symbol_L4(k * np.pi / n, l * np.pi / n, 1.0 / n)
    U = spectral.solve(F, 4)
    assert np.allclose(U, F / lam, rtol=0, atol=1e-14 * np.abs(F / lam).max())


def test_sixth_order_axis_symbol_matches_stencil_weights():
    """The sixth-order axis symbol equals the cosine series of the printed cross
    Eq. (LhOrder6): weights (-2, 27, -270, 490, -270, 27, -2) / (180 h^2) per axis."""
    t = np.linspace(0, np.pi, 17)
    w = {0: 490.0, 1: -270.0, 2: 27.0, 3: -2.0}
    direct = sum((wv if m == 0 else 2 * wv) * np.cos(m * t) for m, wv in w.items()) / 180.0
    assert np.allclose(spectral.axis_symbol(6, t, 1.0), direct, rtol=0, atol=1e-12)
