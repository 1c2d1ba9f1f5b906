"""Seeded synthetic right-hand sides for 2D Poisson problems on the unit square.

This module is shared by the CUDA path's tests/bench and by the FP64 oracle's
tests. It generates inputs only and contains none of the multigrid method's
arithmetic.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value k of
stream `seed` is mix64(seed * 2^32 + k + 1) times the golden-gamma increment, so any
element can be regenerated independently of the others.

Grids have N cells per side (N a power of two) and (N+1) x (N+1) nodes, stored
row-major with x fastest: a[j, i] is the node (x_i, y_j) = (i/N, j/N). Boundary
entries of every right-hand side are zero (they are ignored by the solver).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Return `count` 64-bit outputs of SplitMix64 stream `seed`, starting at `offset`."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    base = np.uint64((int(seed) << 32) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = (base + k * _GOLDEN).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2^-53."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [-1, 1)."""
    return 2.0 * uniform01(seed, count, offset) - 1.0


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """N(0,1) doubles by the Box-Muller transform of consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]: log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def node_coords(n: int):
    x = np.arange(n + 1, dtype=np.float64) / n
    return x


def _zero_boundary(a: np.ndarray) -> np.ndarray:
    a[0, :] = 0.0
    a[-1, :] = 0.0
    a[:, 0] = 0.0
    a[:, -1] = 0.0
    return a


def rhs_manufactured_noise(n: int, seed: int = 0) -> np.ndarray:
    """f = 2 pi^2 sin(pi x) sin(pi y) + eta, eta i.i.d. U[-1, 1) on interior nodes.

    2 pi^2 sin(pi x) sin(pi y) is -Laplace of the manufactured solution
    u = sin(pi x) sin(pi y); eta is drawn in row-major order over interior nodes.
    """
    x = node_coords(n)
    s = np.sin(math.pi * x)
    f = 2.0 * math.pi ** 2 * np.outer(s, s)
    eta = uniform_pm1(seed, (n - 1) * (n - 1)).reshape(n - 1, n - 1)
    f[1:-1, 1:-1] += eta
    return _zero_boundary(f)


def sine_modes(seed: int, n_modes: int = 16, kmax: int = 64):
    """(k, l, a) for `n_modes` modes: k, l uniform integers in [1, kmax], a ~ N(0,1)."""
    z = splitmix64(seed, 2 * n_modes)
    ks = (z[0::2] % np.uint64(kmax)).astype(np.int64) + 1
    ls = (z[1::2] % np.uint64(kmax)).astype(np.int64) + 1
    amps = normal(seed + 0x5EED, n_modes)
    return [(int(k), int(l), float(a)) for k, l, a in zip(ks, ls, amps)]


def rhs_sine_modes(n: int, seed: int = 0, n_modes: int = 16, kmax: int = 64) -> np.ndarray:
    """f = sum_m a_m sin(k_m pi x) sin(l_m pi y) with the modes of `sine_modes`."""
    x = node_coords(n)
    f = np.zeros((n + 1, n + 1))
    for k, l, a in sine_modes(seed, n_modes, kmax):
        f += a * np.outer(np.sin(l * math.pi * x), np.sin(k * math.pi * x))
    return _zero_boundary(f)


def rhs_normal(n: int, seed: int = 0) -> np.ndarray:
    """f i.i.d. N(0,1) on interior nodes, row-major."""
    f = np.zeros((n + 1, n + 1))
    f[1:-1, 1:-1] = normal(seed, (n - 1) * (n - 1)).reshape(n - 1, n - 1)
    return f


def rhs_single_mode(n: int, k: int, l: int) -> np.ndarray:
    """f = sin(k pi x) sin(l pi y) (x along columns)."""
    x = node_coords(n)
    f = np.outer(np.sin(l * math.pi * x), np.sin(k * math.pi * x))
    return _zero_boundary(f)


# ---- periodic problems: unknowns are the nodes 0 <= i, j < n; row and column n of
# the (n+1) x (n+1) arrays are not unknowns and are left 0 ------------------------
def rhs_periodic_normal(n: int, seed: int = 0) -> np.ndarray:
    """f i.i.d. N(0,1) on the nodes 0 <= i, j < n (row-major), minus its mean, so that
    the singular periodic problem is solvable (f orthogonal to the constants)."""
    f = np.zeros((n + 1, n + 1))
    g = normal(seed, n * n).reshape(n, n)
    f[:n, :n] = g - g.mean()
    return f


def rhs_periodic_mode(n: int, k: int, l: int) -> np.ndarray:
    """f = cos(2 pi k x) cos(2 pi l y) on the nodes 0 <= i, j < n (x along columns);
    zero mean for (k, l) != (0, 0) modulo n."""
    x = np.arange(n, dtype=np.float64) / n
    f = np.zeros((n + 1, n + 1))
    f[:n, :n] = np.outer(np.cos(2 * math.pi * l * x), np.cos(2 * math.pi * k * x))
    return f


# ---- the same generator with torch tensors (on any device) --------------------------
# Used where a right-hand side is made on the GPU next to the solve (e.g. one per
# served request), so no host generation or host-to-device copy sits in the request
# path. SplitMix64 with 64-bit wrap-around arithmetic in signed int64 (two's
# complement gives the same bits as unsigned arithmetic; right shifts are made
# logical by masking). The uniforms are bit-identical to `uniform01`; the normals
# agree with `normal` to within the rounding of log / cos / sin on the device.
def _i64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def _lsr(z, s: int):
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(z, s), (1 << (64 - s)) - 1)


def uniform01_torch(seed: int, count: int, device="cpu", offset: int = 0):
    import torch
    k = torch.arange(offset + 1, offset + count + 1, dtype=torch.int64, device=device)
    base = _i64((int(seed) << 32) & 0xFFFFFFFFFFFFFFFF)
    z = base + k * _i64(int(_GOLDEN))
    z = torch.bitwise_xor(z, _lsr(z, 30)) * _i64(int(_M1))
    z = torch.bitwise_xor(z, _lsr(z, 27)) * _i64(int(_M2))
    z = torch.bitwise_xor(z, _lsr(z, 31))
    return _lsr(z, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def normal_torch(seed: int, count: int, device="cpu"):
    import torch
    m = (count + 1) // 2
    u = uniform01_torch(seed, 2 * m, device)
    r = torch.sqrt(-2.0 * torch.log(1.0 - u[0::2]))
    t = (2.0 * math.pi) * u[1::2]
    z = torch.stack((r * torch.cos(t), r * torch.sin(t)), dim=1).reshape(-1)
    return z[:count]


def rhs_normal_torch(n: int, seed: int = 0, device="cpu", out=None):
    """`rhs_normal` generated on `device` (into `out` if given, an (n+1) x (n+1) float64
    tensor): i.i.d. N(0,1) on interior nodes, row-major, zero boundary."""
    import torch
    if out is None:
        out = torch.zeros((n + 1, n + 1), dtype=torch.float64, device=device)
    else:
        out.zero_()
    out[1:-1, 1:-1] = normal_torch(seed, (n - 1) * (n - 1), out.device).reshape(n - 1, n - 1)
    return out
