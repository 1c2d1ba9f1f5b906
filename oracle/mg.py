"""Plain FP64 multigrid for 2D Poisson with red-black or standard coarsening.

TEST INFRASTRUCTURE ONLY (see the package docstring). Parity of the CUDA library
is measured against this module; the library never calls it.

What is computed, and where the paper defines it (Liu & Henshaw, "Multigrid with
nonstandard coarsening", arXiv:2008.03885):

* Problem: -Laplace u = f on the square [0, L]^2 (L = 1 by default), N cells per side (h = 1/N, N a power
  of two), Eq. (G_h_N). Homogeneous Dirichlet data with the interior nodes as
  unknowns (Sec. 2.1), or periodic boundaries, the setting of the paper's computed
  results (Sec. 2.2, computations), with the nodes 0 <= i, j < N as unknowns: every
  stencil and transfer wraps around modulo the level's lattice size (the block-
  circulant matrix of Sec. "Red-black reduction in two dimensions").
* Fine operators: the 5-point second-order Laplacian, Eq. (L_h_2), the wide
  9-point fourth-order one, Eq. (L_h_2d_4o), and the 13-point sixth-order one,
  Eq. (LhOrder6). Next to the boundary the wide stencils reach nodes outside; those
  ghosts are closed by odd reflection u(-x) = -u(x) (the paper analyses infinite or
  periodic grids and is silent here).
* Coarse grids: standard coarsening H = 2h (Eq. G_H_d) or red-black coarsening
  (Sec. 4.3, Eq. G_r2, Fig. "redBlackCoarseLevelGrids"): level 2m is an axis grid
  of spacing 2^m h, level 2m+1 is the set of black points (i+j even) of level 2m,
  a rotated grid of spacing 2^m sqrt(2) h. Coarsening stops at an axis grid with
  n_min cells per side.
* Transfers: red-black coarsening uses Eq. (transfer_r2) in each fine level's own
  frame: interpolation 1/4 ]. 1 .; 1 4 1; . 1 .[ and restriction R = 1/2 P^T;
  standard coarsening uses bilinear interpolation and full weighting R = 1/4 P^T,
  Eq. (transfer_2d), or (transfer_order = 4, Sec. "High-order accurate transfer
  operators") cubic interpolation Eq. (interp_2d4o) with its adjoint restriction
  Eq. (restr_2d4o), R = 1/4 P^T. The cubic stencil reaches coarse nodes beyond the
  boundary; those ghosts are odd reflections (Dirichlet) or wrap (periodic), as for
  the wide fine stencils. All are assembled here as explicit sparse matrices.
* Coarse operators (Sec. 2.3 notation, Sec. 4.4): non-Galerkin = the 5-point
  stencil on the coarse grid with spacing H (Eq. L_H_2d; for fourth order this is
  nG^(2)); "non-Galerkin high" = the fine operator's own stencil with spacing H
  (for fourth order nG^(4), Eq. L_H_4n_2d); Galerkin = the recursion L_{l+1} = R L_l P, Eq. (L_G_l), formed here by
  an explicit sparse product; for a fourth-order fine level the recursion starts
  from the second-order L_h^(2), Eq. (L_H_2G_2d), i.e. G^(2); "true high" starts it
  from the fourth-order L_h itself; G1 = the first-generation Galerkin stencil
  Eq. (L_G1) on every coarse level; Gn = Galerkin on level 1, non-Galerkin below.
* Smoother: red-black relaxation S = S^B S^R, Eq. (S_rb), red = (i+j) odd on axis
  grids; on a rotated grid the colour is the parity of k1+k2 in the rotated frame,
  which is the parity of i. Within one colour every point is updated from the
  values at the start of the half-sweep (Jacobi within a colour); for the 5-point
  stencil this is exactly red-black Gauss-Seidel (Sec. 4.2, S^GS = S^J).
  Weighted Jacobi, S = I - omega h^2/(2d) L_h (Sec. 5.3), is the other option.
* Cycle: the gamma-cycle MG(f; maxIters) of Sec. 2.2 (Algorithm "MG"): pre-smooth,
  residual, restrict, recurse (zero initial guess, Eq. L_H_approx) or solve exactly
  on the coarsest level, interpolate, correct, post-smooth. A periodic operator is
  singular (the constants are its null space); its exact coarsest solve is the
  zero-mean solution, computed with the constant mode removed explicitly. Periodic
  hierarchies coarsen down to a single node, whose operator row is zero (up to the
  rounding of deep Galerkin products) and whose zero-mean solution is 0.
* Exact coarsest solve with more than one unknown (Dirichlet, n_min > 2 or a
  truncated hierarchy; Algorithm "MG" asks only for an exact solve, so this is a
  reading): the coarsest operator A (symmetric positive definite) is factored once as
  A = L L^T by Cholesky, its inverse factor G = L^-1 is formed, and each solve is
  x = G^T (G d): two triangular products with no sequential dependence between rows.
  The operation order is fixed (see dense_coarse_factor) so that an implementation
  following it reproduces x bit for bit. One unknown keeps x = d / a_pp.

Floating-point evaluation order (so that any implementation following the same
order reproduces every iterate bit for bit): in each operator application
y_p = sum_q a_pq x_q the row's nonzeros are split into groups of equal value a_g, the
groups ordered by their first column and each group's columns in increasing order of
a row-major (j, then i) numbering of the level's unknowns; y_p = sum_g a_g (x_g1 +
x_g2 + ...), every sum left to right and every product and sum rounded separately (no
fused multiply-add). The paper writes its stencils in this factored form (a weight
times a sum of equally weighted neighbours, e.g. Eq. L_h_2d_4o), which this reading
follows; the grid transfers R and P sum their products in column order. Coefficients
are exact dyadic weights w times one scale s per level (a_pq = fl(w_pq * s)); a
relaxation is u + r * fl(omega / a_pp) with r = f - (A u); a correction is u + (P v).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

REDBLACK = "redblack"
STANDARD = "standard"
VARIABLE = "variable"  # red-black for coarse levels 1 and 2, standard below (Sec. 4.4 "VC")

NONGALERKIN = "nongalerkin"
GALERKIN = "galerkin"
G1 = "g1"
GN = "gn"
TRUE_HIGH = "galerkin_true_high"
NONGALERKIN_HIGH = "nongalerkin_high"

# Stencils in a level's own frame, as {(a, b): weight}; a along the frame's first
# axis, b along its second. Scales are applied separately.
FIVE_POINT = {(0, 0): 4.0, (-1, 0): -1.0, (1, 0): -1.0, (0, -1): -1.0, (0, 1): -1.0}  # Eq. L_h_2
FOURTH_ORDER = {  # Eq. L_h_2d_4o, times 12 h^2
    (0, 0): 60.0,
    (-1, 0): -16.0, (1, 0): -16.0, (0, -1): -16.0, (0, 1): -16.0,
    (-2, 0): 1.0, (2, 0): 1.0, (0, -2): 1.0, (0, 2): 1.0,
}
SIXTH_ORDER = {  # Eq. LhOrder6, times 180 h^2 (printed "27 -2" read as "27, -2")
    (0, 0): 980.0,
    (-1, 0): -270.0, (1, 0): -270.0, (0, -1): -270.0, (0, 1): -270.0,
    (-2, 0): 27.0, (2, 0): 27.0, (0, -2): 27.0, (0, 2): 27.0,
    (-3, 0): -2.0, (3, 0): -2.0, (0, -3): -2.0, (0, 3): -2.0,
}
FIRST_GALERKIN = {  # Eq. L_G1 / Eq. L_2h_G, times H^2
    (0, 0): 3.0,
    (-1, 0): -0.5, (1, 0): -0.5, (0, -1): -0.5, (0, 1): -0.5,
    (-1, -1): -0.25, (1, -1): -0.25, (-1, 1): -0.25, (1, 1): -0.25,
}


DIRICHLET = "dirichlet"
PERIODIC = "periodic"


def fold(t: np.ndarray, n: int):
    """Odd-periodic reflection of lattice coordinate t into [0, n].

    Returns (t', sign, on_boundary). The odd extension of a grid function that
    vanishes on x = 0 and x = n has period 2n and flips sign at each reflection.
    """
    m = np.mod(t, 2 * n)
    sign = np.where(m <= n, 1.0, -1.0)
    tp = np.where(m <= n, m, 2 * n - m)
    return tp, sign, (tp == 0) | (tp == n)


@dataclass
class Level:
    kind: str  # "axis" or "rot"
    n: int  # cells per side of the lattice the level's points live on
    h2: float  # squared grid spacing of this level (in the level's own frame)
    periodic: bool = False
    pi: np.ndarray = field(repr=False, default=None)  # unknowns' lattice i
    pj: np.ndarray = field(repr=False, default=None)  # unknowns' lattice j
    index: np.ndarray = field(repr=False, default=None)  # (n+1, n+1) -> unknown or -1
    red: np.ndarray = field(repr=False, default=None)  # colour mask over unknowns
    W: sp.csr_matrix = field(repr=False, default=None)  # dyadic weights
    s: float = 1.0  # scale: A = fl(W * s)
    A: sp.csr_matrix = field(repr=False, default=None)

    @property
    def size(self) -> int:
        return int(self.pi.size)

    def frame(self, a: int, b: int):
        """Own-frame stencil offset -> lattice offset (dx, dy).

        Rotated frame: k1 = (i - j)/2, k2 = (i + j)/2 (r = U x, Eq. G_r2), so the
        frame offset (a, b) is the lattice offset (a + b, b - a).
        """
        return (a, b) if self.kind == "axis" else (a + b, b - a)


def _make_level(kind: str, n: int, h2: float, periodic: bool = False) -> Level:
    lo, hi = (0, n) if periodic else (1, n)  # unknowns lo <= i, j < hi
    jj, ii = np.meshgrid(np.arange(lo, hi), np.arange(lo, hi), indexing="ij")
    pi, pj = ii.ravel(), jj.ravel()  # row-major: j major, i minor
    if kind == "rot":
        keep = (pi + pj) % 2 == 0
        pi, pj = pi[keep], pj[keep]
    index = -np.ones((n + 1, n + 1), dtype=np.int64)
    index[pj, pi] = np.arange(pi.size)
    red = ((pi + pj) % 2 == 1) if kind == "axis" else (pi % 2 == 1)
    return Level(kind=kind, n=n, h2=h2, periodic=periodic, pi=pi, pj=pj, index=index, red=red)


def level_shapes(n: int, coarsening: str, n_min: int = 2, max_levels: int | None = None):
    """(kind, lattice n, h^2 / h0^2) of every level, finest first."""
    shapes = [("axis", n, 1.0)]
    while True:
        kind, m, r2 = shapes[-1]
        if max_levels is not None and len(shapes) >= max_levels:
            break
        if kind == "axis" and m <= n_min:
            break
        if coarsening == REDBLACK or (coarsening == VARIABLE and len(shapes) < 3):
            shapes.append(("rot", m, 2.0 * r2) if kind == "axis" else ("axis", m // 2, 2.0 * r2))
        else:
            shapes.append(("axis", m // 2, 4.0 * r2))
    return shapes


def stencil_weights(level: Level, stencil: dict, factor: float) -> sp.csr_matrix:
    """Matrix of an own-frame stencil (times `factor`): Dirichlet with odd-reflection
    ghosts, or periodic (offsets wrap modulo the lattice size)."""
    n = level.n
    rows, cols, vals = [], [], []
    for (a, b), w in stencil.items():
        dx, dy = level.frame(a, b)
        if level.periodic:
            ti, tj = np.mod(level.pi + dx, n), np.mod(level.pj + dy, n)
            si = sj = np.ones(level.size)
            keep = np.ones(level.size, dtype=bool)
        else:
            ti, si, bi = fold(level.pi + dx, n)
            tj, sj, bj = fold(level.pj + dy, n)
            keep = ~(bi | bj)
        rows.append(np.nonzero(keep)[0])
        cols.append(level.index[tj[keep], ti[keep]])
        vals.append((si * sj)[keep] * (w * factor))
    m = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(level.size, level.size),
    ).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return m


def _cubic_interpolation(fine: Level, coarse: Level) -> sp.csr_matrix:
    """Eq. (interp_2d4o): per axis, a fine node at an even position takes its coarse
    node (weight 1); at an odd position the coarse nodes at fine offsets -3, -1, 1, 3
    with weights -1/16, 9/16, 9/16, -1/16; the 2D weights are products. Ghost coarse
    nodes: odd reflection with sign (Dirichlet; coarse boundary nodes carry nothing)
    or wrap-around (periodic)."""
    nc = coarse.n
    taps = {0: ((0, 1.0),), 1: ((-3, -1.0 / 16), (-1, 9.0 / 16), (1, 9.0 / 16), (3, -1.0 / 16))}
    rows, cols, vals = [], [], []
    for px in (0, 1):
        for py in (0, 1):
            sel = np.nonzero((fine.pi % 2 == px) & (fine.pj % 2 == py))[0]
            fi, fj = fine.pi[sel], fine.pj[sel]
            for ox, wx in taps[px]:
                for oy, wy in taps[py]:
                    ci, cj = (fi + ox) // 2, (fj + oy) // 2
                    if coarse.periodic:
                        ci, cj = np.mod(ci, nc), np.mod(cj, nc)
                        sign = np.ones(sel.size)
                        keep = np.ones(sel.size, dtype=bool)
                    else:
                        ci, si, bi = fold(ci, nc)
                        cj, sj, bj = fold(cj, nc)
                        sign, keep = si * sj, ~(bi | bj)
                    rows.append(sel[keep])
                    cols.append(coarse.index[cj[keep], ci[keep]])
                    vals.append(sign[keep] * (wx * wy))
    m = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(fine.size, coarse.size),
    ).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return m


def interpolation(fine: Level, coarse: Level, coarsening: str, order: int = 2) -> sp.csr_matrix:
    """Explicit interpolation P: coarse unknowns -> fine unknowns. Dirichlet: coarse
    boundary nodes contribute nothing; periodic: coarse positions wrap modulo the
    coarse lattice size."""
    if order == 4:
        assert coarsening == STANDARD
        return _cubic_interpolation(fine, coarse)
    rows, cols, vals = [], [], []
    fi, fj = fine.pi, fine.pj
    nf, nc = fine.n, coarse.n

    def add(mask, ci, cj, w):
        if coarse.periodic:
            ci, cj = np.mod(ci, nc), np.mod(cj, nc)
        inside = mask & (ci >= 1) & (ci <= nc - 1) & (cj >= 1) & (cj <= nc - 1)
        if coarse.periodic:
            inside = mask
        r = np.nonzero(inside)[0]
        rows.append(r)
        cols.append(coarse.index[cj[inside], ci[inside]])
        vals.append(np.full(r.size, w))

    if coarsening == REDBLACK and fine.kind == "axis":
        # coarse = black points of the same lattice; red points average 4 axis nbrs
        black = ~fine.red
        add(black, fi, fj, 1.0)
        for dx, dy in ((0, -1), (-1, 0), (1, 0), (0, 1)):
            add(fine.red, fi + dx, fj + dy, 0.25)
    elif coarsening == REDBLACK:
        # rotated fine level: coarse = points with i, j even (lattice n/2)
        black = ~fine.red
        add(black, fi // 2, fj // 2, 1.0)
        for dx, dy in ((-1, -1), (1, -1), (-1, 1), (1, 1)):
            add(fine.red, (fi + dx) // 2, (fj + dy) // 2, 0.25)
    else:
        # bilinear, Eq. transfer_2d
        assert nf == 2 * nc
        for ox, wx in ((0, 1.0), (-1, 0.5), (1, 0.5)):
            for oy, wy in ((0, 1.0), (-1, 0.5), (1, 0.5)):
                okx = (fi % 2 == 0) if ox == 0 else (fi % 2 == 1)
                oky = (fj % 2 == 0) if oy == 0 else (fj % 2 == 1)
                add(okx & oky, (fi + ox) // 2, (fj + oy) // 2, wx * wy)
    m = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(fine.size, coarse.size),
    ).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return m


# ---- exact dyadic sparse products (the Galerkin recursion) ----------------------
# Galerkin coefficients are dyadic fractions whose numerators grow every level (about
# 3 bits per red-black level, 14 per cubic level), so on deep hierarchies "R A P" has
# no unique FP64 value. The recursion is formed exactly and each level rounded once.
# A matrix is (rows, cols, numerators, e): entry = numerator / 2^e, numerators Python
# integers (numpy object arrays), so products and sums are exact at any depth.
def _dyadic_exponent(data: np.ndarray) -> int:
    """Smallest e >= 0 with every entry times 2^e an integer (every double is a dyadic
    fraction: mantissa m / 2^53 times 2^ex, so it needs 53 - ex - (trailing zero bits
    of m) fraction bits)."""
    d = data[data != 0]
    if d.size == 0:
        return 0
    m, ex = np.frexp(np.abs(d))
    M = (m * 2.0 ** 53).astype(np.int64)
    tz = np.log2((M & -M).astype(np.float64)).astype(np.int64)
    e = int(max(0, int((53 - ex - tz).max())))
    assert np.all(np.floor(d * 2.0 ** e) == d * 2.0 ** e)
    return e


def _exact_from(m: sp.csr_matrix, e: int | None = None):
    c = m.tocoo()
    if e is None:
        e = _dyadic_exponent(c.data)
    num = np.array([int(v * 2 ** e) for v in c.data], dtype=object)
    assert all(float(n) == v * 2 ** e for n, v in zip(num, c.data)), "not a multiple of 2^-e"
    return c.row.astype(np.int64), c.col.astype(np.int64), num, e


def _fp64_product_is_exact(R: sp.csr_matrix, W: sp.csr_matrix, P: sp.csr_matrix) -> bool:
    """Whether the FP64 product R W P is exact in any evaluation order: with every factor
    written as an integer matrix times 2^-e (smallest e), each product and partial sum is
    an integer times 2^-(eR + eW + eP) of magnitude at most ||N_R|| ||N_W|| ||N_P||
    (infinity norms of the integer matrices); below 2^53 all of them are representable."""
    bound = 1.0
    for m in (R, W, P):
        e = _dyadic_exponent(m.data)
        bound *= float(abs(m).sum(axis=1).max()) * 2.0 ** e if m.nnz else 0.0
    return bound < 2.0 ** 53


def _exact_mul(A, B, shape):
    """Exact sparse product A B."""
    ra, ca, na, ea = A
    rb, cb, nb, eb = B
    order = np.argsort(rb, kind="stable")
    rb, cb, nb = rb[order], cb[order], nb[order]
    ptr = np.searchsorted(rb, np.arange(shape[1] + 1))
    cnt = ptr[ca + 1] - ptr[ca]
    total = int(cnt.sum())
    first = np.repeat(ptr[ca], cnt)
    pos = first + np.arange(total) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    if total == 0:  # e.g. a periodic operator times the constant interpolation
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, dtype=object), ea + eb
    rows = np.repeat(ra, cnt)
    cols = cb[pos]
    vals = np.repeat(na, cnt) * nb[pos]
    key = rows * shape[2] + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    starts = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
    sums = np.add.reduceat(vals, starts)
    keep = np.array([v != 0 for v in sums], dtype=bool)
    k = key[starts][keep]
    return k // shape[2], k % shape[2], sums[keep], ea + eb


def _exact_normalize(E):
    """Drop factors of two common to every numerator (keeps the integers small)."""
    r, c, num, e = E
    while e > 0 and len(num) and bool(np.all(num % 2 == 0)):
        num = num // 2
        e -= 1
    return r, c, num, e


def _exact_round(E, shape) -> sp.csr_matrix:
    """Each exact entry rounded once to the nearest double (int / int division is
    correctly rounded)."""
    r, c, num, e = E
    vals = np.array([n / (1 << e) for n in num], dtype=np.float64)
    m = sp.coo_matrix((vals, (r, c)), shape=shape).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return m


DENSE_MAX_UNKNOWNS = 1024  # coarsest systems up to this size use the factored solve


def dense_coarse_factor(A: np.ndarray) -> np.ndarray:
    """Inverse Cholesky factor G = L^-1 of a symmetric positive definite A (FP64), in a
    fixed order, every product and sum rounded separately:

    Cholesky by columns j = 0, 1, ...: s = A_jj - L_j0 L_j0 - L_j1 L_j1 - ... (k
    ascending), L_jj = sqrt(s), r_j = 1 / L_jj; for i > j, t = A_ij - L_i0 L_j0 - ...
    - L_i,j-1 L_j,j-1 and L_ij = t r_j.
    Inverse factor by rows i: G_ii = r_i and, for c < i, G_ic = -((L_ic G_cc +
    L_i,c+1 G_c+1,c + ... + L_i,i-1 G_i-1,c) r_i), the sum from its first product with
    k ascending. G L = I follows from the forward substitution L G = I read row by row."""
    m = A.shape[0]
    L = np.zeros((m, m))
    r = np.zeros(m)
    for j in range(m):
        s = A[j, j]
        col = A[j + 1:, j].copy()
        for k in range(j):
            s = s - L[j, k] * L[j, k]
            col = col - L[j + 1:, k] * L[j, k]
        assert s > 0.0, "coarsest operator is not positive definite"
        L[j, j] = math.sqrt(s)
        r[j] = 1.0 / L[j, j]
        L[j + 1:, j] = col * r[j]
    G = np.zeros((m, m))
    for i in range(m):
        G[i, i] = r[i]
        acc = np.zeros(i)
        for k in range(i):
            acc[k] = L[i, k] * G[k, k]  # first product of column k's sum
            acc[:k] = acc[:k] + L[i, k] * G[k, :k]
        G[i, :i] = -(acc * r[i])
    return G


def dense_coarse_solve(G: np.ndarray, d: np.ndarray) -> np.ndarray:
    """x = G^T (G d) with G lower triangular: y_i = G_i0 d_0 + ... + G_ii d_i and
    x_i = G_ii y_i + G_i+1,i y_i+1 + ... + G_m-1,i y_m-1, each sum from its first product
    with k ascending, products and sums rounded separately."""
    m = d.size
    y = G[:, 0] * d[0]
    for k in range(1, m):
        y[k:] = y[k:] + G[k:, k] * d[k]
    x = np.zeros(m)
    for k in range(m):
        x[k] = G[k, k] * y[k]
        x[:k] = x[:k] + G[k, :k] * y[k]
    return x


class ColumnEll:
    """A CSR matrix as padded rows with sorted columns, applied in column order: the
    grid transfers, y = sum_k a_k x_k from the first product, left to right."""

    def __init__(self, m: sp.csr_matrix):
        m = m.tocsr()
        m.sort_indices()
        nrow = m.shape[0]
        counts = np.diff(m.indptr)
        width = int(counts.max()) if nrow else 0
        self.shape = m.shape
        self.cols = np.zeros((width, nrow), dtype=np.int64)
        self.vals = np.zeros((width, nrow))
        self.cols[:, :] = np.minimum(np.arange(nrow), max(m.shape[1] - 1, 0))[None, :]
        row_of = np.repeat(np.arange(nrow), counts)
        pos = np.arange(m.nnz) - np.repeat(m.indptr[:-1], counts)
        self.cols[pos, row_of] = m.indices
        self.vals[pos, row_of] = m.data
        self.width = width

    def __matmul__(self, x: np.ndarray) -> np.ndarray:
        if self.width == 0:
            return np.zeros(self.shape[0])
        y = self.vals[0] * x[self.cols[0]]
        for k in range(1, self.width):
            y = y + self.vals[k] * x[self.cols[k]]
        return y


class Ell:
    """A level operator applied row by row in the evaluation order of the header: each
    row's nonzeros are split into groups of equal value, the groups ordered by the
    column of their first nonzero and each group's nonzeros by column; the row's value
    is sum_g c_g * (x_g1 + x_g2 + ...), every sum left to right and every operation
    rounded separately (numpy FP64 ufuncs, one per operation, never fused). Stored as
    padded slots [group, position in group, row]."""

    def __init__(self, m: sp.csr_matrix):
        m = m.tocsr()
        m.sort_indices()
        nrow = m.shape[0]
        self.shape = m.shape
        counts = np.diff(m.indptr)
        W = int(counts.max()) if nrow else 0
        if m.nnz == 0:
            self.G = self.K = 0
            return
        # dense [row, column rank] copies of the rows (NaN-padded values never compare equal)
        rows = np.repeat(np.arange(nrow), counts)
        pos = np.arange(m.nnz) - np.repeat(m.indptr[:-1], counts)
        V = np.full((nrow, W), np.nan)
        C = np.zeros((nrow, W), dtype=np.int64)
        V[rows, pos] = m.data
        C[rows, pos] = m.indices
        valid = ~np.isnan(V)
        # first[r, k]: column rank of the first nonzero of row r equal in value to nonzero k.
        # Rows repeat (every interior row of a level is the same stencil), so it is worked
        # out once per distinct row: rows are bucketed by two hashes of their values' bit
        # patterns and each bucket is checked to hold one distinct row.
        Vh = np.where(valid, V, 0.0)
        bits = Vh.view(np.uint64) ^ valid.astype(np.uint64)  # exact: the values' bit patterns

        def mix(z):  # SplitMix64's finaliser: every output bit depends on every input bit
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            return z ^ (z >> np.uint64(31))

        with np.errstate(over="ignore"):
            # each word mixed together with its position, so that rearranged rows differ
            posk = np.arange(1, W + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
            m1 = mix(bits ^ posk[None, :])
            h1 = m1.sum(axis=1, dtype=np.uint64)
            h2 = mix(m1 + posk[None, :]).sum(axis=1, dtype=np.uint64)
        keys = np.stack([h1, h2, counts.astype(np.uint64)], axis=1)
        _, rep, inv = np.unique(keys, axis=0, return_index=True, return_inverse=True)
        inv = inv.reshape(-1)
        assert np.array_equal(Vh, Vh[rep][inv]) and np.array_equal(counts, counts[rep][inv]), \
            "two distinct operator rows share a bucket"
        Vu = V[rep]
        fu = np.tile(np.arange(W), (len(rep), 1))
        for j in range(W):
            for k in range(j + 1, W):
                hit = (fu[:, k] == k) & (Vu[:, k] == Vu[:, j])
                fu[hit, k] = j
        first = fu[inv]
        key = np.where(valid, first * (W + 1) + np.arange(W)[None, :], W * (W + 1) + np.arange(W)[None, :])
        order = np.argsort(key, axis=1, kind="stable")
        Vs = np.take_along_axis(V, order, axis=1)
        Cs = np.take_along_axis(C, order, axis=1)
        Fs = np.take_along_axis(first, order, axis=1)
        vs = np.take_along_axis(valid, order, axis=1)
        gstart = np.ones((nrow, W), dtype=bool)
        gstart[:, 1:] = Fs[:, 1:] != Fs[:, :-1]
        gstart &= vs
        g_in_row = np.cumsum(gstart, axis=1) - 1
        idx = np.tile(np.arange(W), (nrow, 1))
        k_in_g = idx - np.maximum.accumulate(np.where(gstart, idx, 0), axis=1)
        self.G = int(g_in_row[vs].max()) + 1
        self.K = int(k_in_g[vs].max()) + 1
        rr = np.tile(np.arange(nrow)[:, None], (1, W))
        self.cols = np.zeros((self.G, self.K, nrow), dtype=np.int64)
        self.valid = np.zeros((self.G, self.K, nrow), dtype=bool)
        self.gval = np.zeros((self.G, nrow))
        self.cols[g_in_row[vs], k_in_g[vs], rr[vs]] = Cs[vs]
        self.valid[g_in_row[vs], k_in_g[vs], rr[vs]] = True
        self.gval[g_in_row[gstart], rr[gstart]] = Vs[gstart]  # value of the group's first nonzero
        self.gvalid = self.valid[:, 0, :]
        self.full = [[bool(self.valid[g, k].all()) for k in range(self.K)] for g in range(self.G)]
        self.any = [[bool(self.valid[g, k].any()) for k in range(self.K)] for g in range(self.G)]

    def __matmul__(self, x: np.ndarray) -> np.ndarray:
        if self.G == 0:
            return np.zeros(self.shape[0])
        y = None
        for g in range(self.G):
            S = x[self.cols[g, 0]]
            for k in range(1, self.K):
                if not self.any[g][k]:
                    continue
                t = S + x[self.cols[g, k]]
                S = t if self.full[g][k] else np.where(self.valid[g, k], t, S)
            P = self.gval[g] * S
            if y is None:
                y = np.where(self.gvalid[0], P, 0.0)
            else:
                t = y + P
                y = t if self.full[g][0] else np.where(self.gvalid[g], t, y)
        return y


@dataclass
class Options:
    omega: float = 1.0
    nu1: int = 1
    nu2: int = 1
    gamma: int = 1  # 1 = V, 2 = W, 3 = "Wn" (2 on levels 0 and 1, 1 below; Sec. 4.4)
    smoother: str = "rb"  # "rb" or "jacobi"
    n_min: int | None = None  # coarsest axis lattice size: 2 (Dirichlet) / 1 (periodic) by default
    transfer_order: int = 2  # 4: cubic transfers (standard coarsening only)
    max_levels: int | None = None


class Oracle:
    """Multigrid hierarchy over explicit sparse matrices (FP64)."""

    def __init__(self, n: int, order: int = 2, coarsening: str = REDBLACK,
                 coarse_op: str = GALERKIN, options: Options | None = None,
                 boundary: str = DIRICHLET, length: float = 1.0):
        assert n >= 2 and (n & (n - 1)) == 0, "N must be a power of two"
        assert order in (2, 4, 6)
        assert boundary in (DIRICHLET, PERIODIC)
        self.n, self.order, self.coarsening, self.coarse_op = n, order, coarsening, coarse_op
        self.boundary = boundary
        self.periodic = boundary == PERIODIC
        self.opt = options or Options()
        h = length / n  # the square [0, length]^2 (the paper's unit square: length 1)
        n_min = self.opt.n_min if self.opt.n_min is not None else (1 if self.periodic else 2)
        self.levels = [_make_level(k, m, r2, self.periodic) for k, m, r2 in
                       level_shapes(n, coarsening, n_min, self.opt.max_levels)]
        self.P, self.R = [], []
        assert self.opt.transfer_order in (2, 4)
        assert self.opt.transfer_order == 2 or coarsening == STANDARD
        for l in range(len(self.levels) - 1):
            step = coarsening if coarsening != VARIABLE else (REDBLACK if l < 2 else STANDARD)
            P = interpolation(self.levels[l], self.levels[l + 1], step, self.opt.transfer_order)
            R = (P.T * (0.5 if step == REDBLACK else 0.25)).tocsr()
            R.sort_indices()
            self.P.append(P)
            self.R.append(R)

        s2 = 1.0 / (h * h)  # scale of operators derived from L_h^(2)
        s4 = 1.0 / (12.0 * h * h)  # scale of operators derived from L_h^(4)
        L0 = self.levels[0]
        if order == 2:
            L0.W, L0.s = stencil_weights(L0, FIVE_POINT, 1.0), s2
            base_W, base_s = L0.W, s2
        else:
            s6 = 1.0 / (180.0 * h * h)  # scale of the sixth-order operator
            L0.W = stencil_weights(L0, FOURTH_ORDER if order == 4 else SIXTH_ORDER, 1.0)
            L0.s = s4 if order == 4 else s6
            if coarse_op == TRUE_HIGH:
                base_W, base_s = L0.W, L0.s
            else:
                base_W, base_s = stencil_weights(L0, FIVE_POINT, 1.0), s2  # L_h^(2)
        gal_W = base_W
        # The Galerkin recursion is exact and each level is rounded once: its dyadic
        # coefficients outgrow FP64's 53 bits on deep hierarchies (about 3 bits per
        # red-black level, 14 per cubic level). While a bound proves the FP64 sparse
        # product exact it is used as is; from the first level where it does not, the
        # recursion continues in exact integer arithmetic.
        gal_E = None
        galerkin = coarse_op in (GALERKIN, TRUE_HIGH, GN)
        for l in range(1, len(self.levels)):
            lev = self.levels[l]
            if galerkin and (coarse_op != GN or l == 1):
                R, P = self.R[l - 1], self.P[l - 1]
                if gal_E is None and _fp64_product_is_exact(R, gal_W, P):
                    gal_W = (R @ gal_W @ P).tocsr()
                    gal_W.sort_indices()
                else:
                    if gal_E is None:
                        gal_E = _exact_from(gal_W)
                    nf, nc = self.levels[l - 1].size, lev.size
                    WP = _exact_mul(gal_E, _exact_from(P), (nf, nf, nc))
                    gal_E = _exact_normalize(_exact_mul(_exact_from(R), WP, (nc, nf, nc)))
                    gal_W = _exact_round(gal_E, (nc, nc))
            hh = lev.h2  # (h_l / h_0)^2
            if coarse_op in (GALERKIN, TRUE_HIGH) or (coarse_op == GN and l == 1):
                lev.W, lev.s = gal_W, base_s
            elif coarse_op == G1:
                lev.W, lev.s = stencil_weights(lev, FIRST_GALERKIN, 1.0 / hh), s2
            elif coarse_op == NONGALERKIN_HIGH:  # the fine stencil with spacing H (nG^(4) at order 4)
                fine_st = {2: FIVE_POINT, 4: FOURTH_ORDER, 6: SIXTH_ORDER}[order]
                lev.W, lev.s = stencil_weights(lev, fine_st, 1.0 / hh), L0.s
            else:  # non-Galerkin 5-point with spacing H = h_l
                lev.W, lev.s = stencil_weights(lev, FIVE_POINT, 1.0 / hh), s2
        for lev in self.levels:
            lev.A = (lev.W * lev.s).tocsr()  # elementwise fl(w * s)
            lev.A.sort_indices()
        self._A = [Ell(lev.A) for lev in self.levels]
        self._P = [ColumnEll(P) for P in self.P]
        self._R = [ColumnEll(R) for R in self.R]
        with np.errstate(divide="ignore"):  # a periodic single-node level has a_pp = 0 (never smoothed)
            self.wd = [self.opt.omega / lev.A.diagonal() for lev in self.levels]
        last = self.levels[-1]
        self._coarse_dense = last.A.toarray()
        self._coarse_G = None
        if not self.periodic and 1 < last.size <= DENSE_MAX_UNKNOWNS:
            self._coarse_G = dense_coarse_factor(self._coarse_dense)
        self._g = None  # nonzero Dirichlet data (set_boundary), level 0 only

    # ---- nonzero Dirichlet data (second order) ------------------------------
    def set_boundary(self, grid: np.ndarray) -> None:
        """Use the boundary entries of an (n+1) x (n+1) grid as Dirichlet data g (the
        paper's B u = g, Sec. 2.1), order 2 only. Level 0 then applies the 5-point stencil
        to the full grid [interior u; boundary g], summing in increasing full-grid
        (row-major) column order; the coarse levels keep solving homogeneous correction
        equations."""
        assert self.order == 2 and not self.periodic
        lev = self.levels[0]
        n = lev.n
        rows, cols, vals = [], [], []
        for (a, b), w in FIVE_POINT.items():
            rows.append(np.arange(lev.size))
            cols.append((lev.pj + b) * (n + 1) + (lev.pi + a))
            vals.append(np.full(lev.size, w))
        W = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(lev.size, (n + 1) ** 2)).tocsr()
        W.sort_indices()
        self._A0_full = Ell((W * lev.s).tocsr())
        self._interior = lev.pj * (n + 1) + lev.pi
        self._g = np.ascontiguousarray(grid, dtype=np.float64).ravel().copy()

    def _Au(self, l: int, u: np.ndarray) -> np.ndarray:
        if l == 0 and self._g is not None:
            full = self._g.copy()
            full[self._interior] = u
            return self._A0_full @ full
        return self._A[l] @ u

    # ---- grid <-> vector -------------------------------------------------
    def to_vec(self, grid: np.ndarray, level: int = 0) -> np.ndarray:
        lev = self.levels[level]
        return np.ascontiguousarray(grid[lev.pj, lev.pi], dtype=np.float64)

    def to_grid(self, v: np.ndarray, level: int = 0) -> np.ndarray:
        lev = self.levels[level]
        g = np.zeros((lev.n + 1, lev.n + 1))
        g[lev.pj, lev.pi] = v
        return g

    @property
    def lmax(self) -> int:
        return len(self.levels) - 1

    # ---- level operations ------------------------------------------------
    def apply(self, l: int, u: np.ndarray) -> np.ndarray:
        return self._Au(l, u)

    def residual(self, l: int, u: np.ndarray, f: np.ndarray) -> np.ndarray:
        return f - self._Au(l, u)

    def restrict(self, l: int, d: np.ndarray) -> np.ndarray:
        return self._R[l] @ d

    def prolong(self, l: int, v: np.ndarray) -> np.ndarray:
        return self._P[l] @ v

    def half_sweep(self, l: int, u: np.ndarray, f: np.ndarray, red: bool) -> np.ndarray:
        mask = self.levels[l].red if red else ~self.levels[l].red
        r = f - self._Au(l, u)
        return np.where(mask, u + r * self.wd[l], u)

    def smooth(self, l: int, u: np.ndarray, f: np.ndarray) -> np.ndarray:
        if self.opt.smoother == "jacobi":
            r = f - self._Au(l, u)
            return u + r * self.wd[l]
        u = self.half_sweep(l, u, f, red=True)
        return self.half_sweep(l, u, f, red=False)

    def coarse_solve(self, d: np.ndarray) -> np.ndarray:
        if self.periodic:
            # singular (constants): the zero-mean solution of A v = Q d, Q the projector
            # onto zero-mean vectors, from the nonsingular (A + 1 1^T / m) v = Q d: its
            # solution has 1^T v = 0 because 1^T A = 0. The constant mode is removed
            # explicitly, so rounding left in a deep Galerkin operator's row sums
            # cannot put a near-zero pivot on it (one node: v = 0).
            m = d.size
            return np.linalg.solve(self._coarse_dense + np.full((m, m), 1.0 / m), d - d.mean())
        if d.size == 1:
            return d / self._coarse_dense[0, 0]
        if self._coarse_G is not None:
            return dense_coarse_solve(self._coarse_G, d)
        # larger truncated hierarchies (printed-rate pins only): LAPACK's solve
        return np.linalg.solve(self._coarse_dense, d)

    def cycle_level(self, l: int, u: np.ndarray, f: np.ndarray) -> np.ndarray:
        o = self.opt
        for _ in range(o.nu1):
            u = self.smooth(l, u, f)
        d = f - self._Au(l, u)
        fc = self._R[l] @ d
        if l + 1 == self.lmax:
            uc = self.coarse_solve(fc)
        else:
            uc = np.zeros_like(fc)
            for _ in range(self.gamma_at(l)):
                uc = self.cycle_level(l + 1, uc, fc)
        u = u + self._P[l] @ uc
        for _ in range(o.nu2):
            u = self.smooth(l, u, f)
        return u

    def gamma_at(self, l: int) -> int:
        """Coarse-level cycles per visit of level l (Wn: 2 on levels 0 and 1, 1 below)."""
        if self.opt.gamma == 3:
            return 2 if l <= 1 else 1
        return self.opt.gamma

    def cycle(self, u: np.ndarray, f: np.ndarray) -> np.ndarray:
        if self.lmax == 0:
            return self.coarse_solve(f)
        return self.cycle_level(0, u, f)

    def rel_residual(self, u: np.ndarray, f: np.ndarray) -> float:
        d = f - self._Au(0, u)
        return math.sqrt(float(np.dot(d, d))) / math.sqrt(float(np.dot(f, f)))

    def solve(self, f: np.ndarray, u: np.ndarray | None = None, rtol: float = 1e-10,
              max_cycles: int = 50, fixed_cycles: bool = False):
        """Cycle until ||f - A u|| / ||f|| < rtol (or max_cycles); return (u, history)."""
        u = np.zeros_like(f) if u is None else u.copy()
        hist = [self.rel_residual(u, f)]
        for _ in range(max_cycles):
            if not fixed_cycles and hist[-1] < rtol:
                break
            u = self.cycle(u, f)
            hist.append(self.rel_residual(u, f))
        return u, hist

    def direct(self, f: np.ndarray) -> np.ndarray:
        """Direct solution of A_0 u = f (a check, not part of the cycle); periodic:
        the zero-mean (minimum-norm) solution from a dense least-squares solve."""
        if self.periodic:
            return np.linalg.lstsq(self.levels[0].A.toarray(), f, rcond=None)[0]
        import scipy.sparse.linalg as spla
        return spla.spsolve(self.levels[0].A.tocsc(), f)


def work_units(oracle: Oracle) -> float:
    """Work units of one cycle: sum over levels of (nu1 + nu2 + 1) sweeps weighted by
    the level's share of fine points, plus the transfers (Sec. 4.4 estimate form)."""
    o = oracle.opt
    n0 = oracle.levels[0].size
    wu = 0.0
    visits = 1
    for l, lev in enumerate(oracle.levels[:-1]):
        wu += visits * (o.nu1 + o.nu2 + 2) * lev.size / n0
        visits *= oracle.gamma_at(l) if l + 1 < oracle.lmax else 1
    return wu
