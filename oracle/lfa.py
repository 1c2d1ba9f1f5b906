"""Local Fourier analysis symbols from the paper, for pinning the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Two-level red-black-coarsening analysis of Sec. 4.3 (Theorem "Th_rbC_LFA"):
on each two-dimensional subspace E_theta = span{phi(theta), phi(theta_bar)}
the red-black smoother, the transfers and the coarse operator act as 2x2 /
1x2 / 2x1 / 1x1 matrices written in terms of
    xi = (sin^2(theta1/2) + sin^2(theta2/2)) / 2            (Eq. xi_r2)
and the iteration matrix M = S^nu2 K S^nu1 with K = I - P L_H^{-1} R L_h.
"""
from __future__ import annotations

import numpy as np


def xi(t1, t2):
    return 0.5 * (np.sin(t1 / 2) ** 2 + np.sin(t2 / 2) ** 2)


def symbol_L2(t1, t2, h=1.0):
    """Symbol of the 5-point -Laplacian: (8/h^2) xi (Sec. 4.2)."""
    return 8.0 / h ** 2 * xi(t1, t2)


def symbol_L4(t1, t2, h=1.0):
    """Symbol of the fourth-order -Laplacian, Eq. (L_hat_2d_4o)."""
    xb = 0.5 * (np.sin(t1 / 2) ** 2 + np.sin(t2 / 2) ** 2)
    x2b = 0.5 * (np.sin(t1 / 2) ** 4 + np.sin(t2 / 2) ** 4)
    return 8.0 / h ** 2 * (xb + x2b / 3.0)


def rbc_two_level_matrix(t1, t2, omega=1.0, nu1=1, nu2=1, coarse="galerkin"):
    """2x2 symbol of the two-level RBC iteration operator on E_theta (h = 1)."""
    x = xi(t1, t2)
    D = np.diag([x, 1.0 - x])
    SR = np.eye(2) - omega * np.array([[1.0, -1.0], [-1.0, 1.0]]) @ D  # Eq. S_hat_RB_2d
    SB = np.eye(2) - omega * np.array([[1.0, 1.0], [1.0, 1.0]]) @ D
    S = SB @ SR  # Eq. S_hat_2d
    Lh = 8.0 * D
    R = np.array([[1.0 - x, x]])  # restriction symbol (1x2)
    P = R.T
    if coarse == "galerkin":  # Eq. L_G1 symbol
        LH = 8.0 * x * (1.0 - x)
    else:  # non-Galerkin 5-point on the rotated grid
        LH = 8.0 * (x - np.sin(t1 / 2) ** 2 * np.sin(t2 / 2) ** 2)
    K = np.eye(2) - P @ (R @ Lh) / LH  # Eq. K_hat_2d_rb
    return np.linalg.matrix_power(S, nu2) @ K @ np.linalg.matrix_power(S, nu1)


def rbc_two_level_rho(omega=1.0, nu1=1, nu2=1, coarse="galerkin", m=128):
    """sup over Theta_low^rb (theta != 0) of rho(M(theta)), Eq. (rho_2d_rb), on a grid."""
    ts = -np.pi + 2 * np.pi * (np.arange(m) + 0.5) / m
    best = 0.0
    for t1 in ts:
        for t2 in ts:
            if not (-np.pi <= t1 - t2 < np.pi and -np.pi <= t1 + t2 < np.pi):
                continue  # Theta_low^rb, Eq. Th_L_2d_rb
            M = rbc_two_level_matrix(t1, t2, omega, nu1, nu2, coarse)
            best = max(best, float(np.max(np.abs(np.linalg.eigvals(M)))))
    return best


def jacobi_optimal(r: float, d: int = 2):
    """omega*(r) and mu*(r) of omega-Jacobi with factor-r coarsening (Sec. 5.3)."""
    zeta = np.sin(np.pi / (2 * r)) ** 2 / d
    return 1.0 / (1.0 + zeta), (1.0 - zeta) / (1.0 + zeta)


def jacobi_smoothing_factor(omega: float, r: float = 2.0, d: int = 2, m: int = 256):
    """Brute-force sup over the high frequencies of |1 - 2 omega xi| (Sec. 5.3)."""
    ts = -np.pi + 2 * np.pi * (np.arange(m) + 0.5) / m
    T = np.meshgrid(*([ts] * d), indexing="ij")
    high = np.zeros_like(T[0], dtype=bool)
    for t in T:
        high |= np.abs(t) >= np.pi / r
    x = sum(np.sin(t / 2) ** 2 for t in T) / d
    return float(np.max(np.abs(1 - 2 * omega * x)[high]))


def rbc_two_level_rho_periodic(n: int, omega=1.0, nu1=1, nu2=1, coarse="galerkin"):
    """The same supremum over the frequencies a periodic N x N grid carries,
    theta = 2 pi k / N (k integer), theta != 0 (the constant mode is the null space
    of the periodic operator). On a periodic grid the red-black smoother, the
    transfers and the coarse operator leave every E_theta invariant, so this is
    the exact spectral radius of the two-level iteration there."""
    ks = np.arange(-n // 2, n // 2)
    best = 0.0
    for k1 in ks:
        for k2 in ks:
            if k1 == 0 and k2 == 0:
                continue
            t1, t2 = 2 * np.pi * k1 / n, 2 * np.pi * k2 / n
            if not (-np.pi <= t1 - t2 < np.pi and -np.pi <= t1 + t2 < np.pi):
                continue
            M = rbc_two_level_matrix(t1, t2, omega, nu1, nu2, coarse)
            best = max(best, float(np.max(np.abs(np.linalg.eigvals(M)))))
    return best
