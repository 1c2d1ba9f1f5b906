"""Exact discrete solutions of the fine-level problem by Fourier diagonalisation.

TEST INFRASTRUCTURE ONLY (see the package docstring). The library never calls it.

The fine operators are constant stencils, so Fourier modes are their eigenfunctions
with the eigenvalue given by the operator's symbol (Sec. 2.4, local Fourier analysis):

* second order, Eq. (L_h_2): symbol (8 / h^2) xi, xi = (sin^2(t1/2) + sin^2(t2/2)) / 2
  (Eq. xi_r2);
* fourth order, Eq. (L_h_2d_4o): the symbol Eq. (L_hat_2d_4o),
  (8 / h^2) (xi + xi2 / 3), xi2 = (sin^4(t1/2) + sin^4(t2/2)) / 2;
* sixth order, Eq. (LhOrder6): the symbol of its weights read off the stencil,
  per axis (490 - 540 cos t + 54 cos 2t - 4 cos 3t) / (180 h^2).

Dirichlet problems (homogeneous data, interior unknowns 0 < i, j < N) close the wide
stencils by odd reflection, so the discrete sine modes sin(k pi x) sin(l pi y),
1 <= k, l <= N - 1, are exact eigenvectors of the assembled matrix with eigenvalue
symbol(k pi h, l pi h); they are orthogonal, so the type-I discrete sine transform
diagonalises the operator and A^-1 f = DST^-1 (DST(f) / symbol). Periodic problems
(unknowns 0 <= i, j < N) are diagonalised by the discrete Fourier transform with
t = 2 pi k / N; the operator annihilates constants, and the zero-mean solution is
returned (the k = l = 0 coefficient set to 0).

This is a different route to A^-1 f than the multigrid oracle and its sparse direct
solve (no assembled matrix, no elimination): the tests pin it to the sparse LU of the
oracle's own matrices on small grids. Its rounding error is about eps * sqrt(log N)
relative to ||u|| for right-hand sides with a flat spectrum, so it serves as the FP64
reference solution at sizes the sparse oracle cannot reach (8193^2).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def axis_symbol(order: int, t: np.ndarray, h: float) -> np.ndarray:
    """One axis' share of the fine operator's symbol at frequency t (the 2D symbol is
    the sum over both axes, since each stencil is a cross)."""
    s2 = np.sin(t / 2.0) ** 2
    if order == 2:  # (8/h^2) * (1/2) sin^2(t/2) per axis
        return 4.0 * s2 / (h * h)
    if order == 4:  # (8/h^2) * ((1/2) s2 + (1/6) s2^2) per axis, Eq. (L_hat_2d_4o)
        return (4.0 * s2 + (4.0 / 3.0) * s2 * s2) / (h * h)
    if order == 6:
        return (490.0 - 540.0 * np.cos(t) + 54.0 * np.cos(2 * t) - 4.0 * np.cos(3 * t)) / (180.0 * h * h)
    raise ValueError("order must be 2, 4 or 6")


def symbol_grid(n: int, order: int, periodic: bool = False, length: float = 1.0) -> np.ndarray:
    """Eigenvalues on the transform's frequency grid, indexed [l, k] (y, x)."""
    h = length / n
    if periodic:
        t = 2.0 * np.pi * np.arange(n) / n
    else:
        t = np.pi * np.arange(1, n) / n
    s = axis_symbol(order, t, h)
    return s[:, None] + s[None, :]


def solve(F: np.ndarray, order: int, periodic: bool = False, length: float = 1.0,
          workers: int | None = None) -> np.ndarray:
    """u = L_h^{-1} f on an (N+1) x (N+1) node grid (row j, column i).

    Dirichlet: the interior of F is the right-hand side; the returned grid is zero on
    the boundary. Periodic: rows and columns 0 .. N-1 are the unknowns (row/column N
    is ignored and returned as the wrap-around copy); f is projected onto zero mean
    and the zero-mean solution is returned.
    """
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0] - 1
    assert F.shape == (n + 1, n + 1)
    lam = symbol_grid(n, order, periodic, length)
    U = np.zeros_like(F)
    if periodic:
        fh = sfft.fft2(F[:n, :n], workers=workers)
        lam = lam.copy()
        lam[0, 0] = 1.0
        fh = fh / lam
        fh[0, 0] = 0.0
        U[:n, :n] = sfft.ifft2(fh, workers=workers).real
        U[n, :n] = U[0, :n]
        U[:, n] = U[:, 0]
        return U
    fh = sfft.dstn(F[1:n, 1:n], type=1, norm="ortho", workers=workers)
    fh /= lam
    U[1:n, 1:n] = sfft.idstn(fh, type=1, norm="ortho", workers=workers)
    return U
