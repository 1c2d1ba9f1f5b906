"""Parity at the full sizes of the bench workloads, in the launch configuration the
bench times (default options, the same kernels the cycle uses).

At 4097^2 the oracle cannot build its matrices in a test's time, so single steps of the
cycle (operator, residual, one red-black sweep, restriction, interpolation) are
checked bit for bit on sampled nodes whose values are computed here one at a time from
the definition: the level's stencil weights (independent of N; read off an interior
row of a small oracle hierarchy), folded by odd reflection with the oracle's `fold`,
merged, evaluated in the library's order (groups of equal coefficient, each group's
values summed, then multiplied; transfers in column order), every operation rounded
separately. Whole solves at
4097^2 (FP64) and 8193^2 (mixed precision) are checked by an independent plain-PyTorch
FP64 residual of the returned solution.
"""
import math

import numpy as np
import pytest

import synth
from oracle.mg import FOURTH_ORDER, GALERKIN, REDBLACK, Options, Oracle, fold

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines skip the module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402

N = 4096


def interior_stencil(o, l):
    """{(dx, dy): weight} of level l's interior row (lattice offsets), from a node whose
    stencil stays clear of the small hierarchy's boundary."""
    lev = o.levels[l]
    i = j = lev.n // 2
    if lev.kind == "rot" and (i + j) % 2:
        i += 1
    row = lev.W.getrow(lev.index[j, i])
    return {(int(lev.pi[q] - i), int(lev.pj[q] - j)): float(v) for q, v in zip(row.indices, row.data)}


def node_row(st, n, i, j, scale):
    """Merged Dirichlet row of node (i, j): [(tj, ti, coefficient)] in column order."""
    acc = {}
    for (dx, dy), w in st.items():
        ti, si, bi = fold(np.array([i + dx]), n)
        tj, sj, bj = fold(np.array([j + dy]), n)
        if bi[0] or bj[0]:
            continue
        key = (int(tj[0]), int(ti[0]))
        acc[key] = acc.get(key, 0.0) + float(si[0] * sj[0]) * w
    return [(tj, ti, w * scale) for (tj, ti), w in sorted(acc.items())]


def grouped_sum(terms, val):
    """An operator row in the evaluation order: the terms (column order) split into groups
    of equal coefficient, groups ordered by their first term; sum_g c_g * (x_g1 + ...),
    every operation rounded (plain Python floats)."""
    groups = []
    for tj, ti, c in terms:
        for g in groups:
            if g[0] == c:
                g[1].append(val(ti, tj))
                break
        else:
            groups.append([c, [val(ti, tj)]])
    s = None
    for c, xs in groups:
        g = xs[0]
        for x in xs[1:]:
            g = g + x
        p = c * g
        s = p if s is None else s + p
    return s


def ordered_sum(terms, val):
    s = None
    for tj, ti, c in terms:
        p = c * val(ti, tj)
        s = p if s is None else s + p
    return s


class Grid:
    """A level's storage on the host: node (i, j) at [j, i] (axis) or [j, i >> 1] (rot)."""

    def __init__(self, arr, kind):
        self.a, self.kind = arr, kind

    def __call__(self, i, j):
        return float(self.a[j, i >> 1] if self.kind == 1 else self.a[j, i])


def random_level(h, l, seed, scale):
    info = mg.mg_get_level_info(h, l)
    a = synth.uniform_pm1(seed, info.rows * info.pitch).reshape(info.rows, info.pitch) * scale
    jj, qq = np.meshgrid(np.arange(info.rows), np.arange(info.pitch), indexing="ij")
    ii = 2 * qq + (jj & 1) if info.kind == 1 else qq
    unknown = (ii >= 1) & (ii <= info.n - 1) & (jj >= 1) & (jj <= info.n - 1) & (qq < info.cols)
    a[~unknown] = 0.0
    return torch.tensor(a, dtype=torch.float64, device="cuda"), a


def sample_nodes(n, kind, seed, count=600):
    """Random unknowns plus every near-boundary class (offsets 1..6 from each edge)."""
    z = synth.splitmix64(seed, 2 * count)
    pts = [(1 + int(z[2 * k] % np.uint64(n - 1)), 1 + int(z[2 * k + 1] % np.uint64(n - 1))) for k in range(count)]
    edge = [1, 2, 3, 4, 5, 6, n - 6, n - 5, n - 4, n - 3, n - 2, n - 1]
    mid = [n // 3, n // 2 + 1, 2 * n // 3]
    pts += [(a, b) for a in edge for b in edge + mid] + [(b, a) for a in edge for b in mid]
    if kind == 1:
        pts = [(i if (i + j) % 2 == 0 else i - 1 if i > 1 else i + 1, j) for i, j in pts]
    return sorted(set(p for p in pts if 1 <= p[0] <= n - 1 and 1 <= p[1] <= n - 1))


@pytest.fixture(scope="module")
def hier():
    h = mg.mg_setup(N, 4, "redblack", "galerkin", nu1=2, nu2=1)
    small = Oracle(64, 4, REDBLACK, GALERKIN, Options(nu1=2))
    hh = 1.0 / N
    scales = [1.0 / (12.0 * hh * hh)] + [1.0 / (hh * hh)] * (len(small.levels) - 1)
    stencils = [dict(FOURTH_ORDER)]  # axis frame: (a, b) is the lattice offset
    stencils += [interior_stencil(small, l) for l in range(1, 3)]
    yield h, stencils, scales
    h.close()


@pytest.mark.parametrize("l", [0, 1, 2])
def test_operator_residual_and_sweep_on_sampled_nodes(hier, l):
    h, stencils, scales = hier
    info = mg.mg_get_level_info(h, l)
    n, kind = info.n, info.kind
    st, sc = stencils[l], scales[l]
    du, hu = random_level(h, l, 100 + l, 3.0)
    df, hf = random_level(h, l, 200 + l, 1e3 * sc / 1e6)
    out = mg.level_array(h, l)
    mg.mg_level_apply(h, l, du, out)
    ga = Grid(out.cpu().numpy(), kind)
    mg.mg_level_residual(h, l, du, df, out)
    gr = Grid(out.cpu().numpy(), kind)
    us = du.clone()
    mg.mg_level_smooth(h, l, us, df, 1)
    gs = Grid(us.cpu().numpy(), kind)
    U, F = Grid(hu, kind), Grid(hf, kind)
    red = (lambda i, j: (i + j) % 2 == 1) if kind == 0 else (lambda i, j: i % 2 == 1)

    rows = {}

    def row(i, j):
        if (i, j) not in rows:
            rows[(i, j)] = node_row(st, n, i, j, sc)
        return rows[(i, j)]

    def relax(i, j, val):
        r = row(i, j)
        diag = [c for tj, ti, c in r if ti == i and tj == j][0]
        return val(i, j) + (F(i, j) - grouped_sum(r, val)) * (1.0 / diag)

    half = {}

    def after_red(i, j):
        if not red(i, j) or not (1 <= i <= n - 1 and 1 <= j <= n - 1):
            return U(i, j)
        if (i, j) not in half:
            half[(i, j)] = relax(i, j, U)
        return half[(i, j)]

    for i, j in sample_nodes(n, kind, 300 + l):
        s = grouped_sum(row(i, j), U)
        assert ga(i, j) == s, ("apply", l, i, j)
        assert gr(i, j) == F(i, j) - s, ("residual", l, i, j)
        want = after_red(i, j) if red(i, j) else relax(i, j, after_red)
        assert gs(i, j) == want, ("sweep", l, i, j)


@pytest.mark.parametrize("l", [0, 1])
def test_restriction_and_interpolation_on_sampled_nodes(hier, l):
    h, _, _ = hier
    fi_info, co_info = mg.mg_get_level_info(h, l), mg.mg_get_level_info(h, l + 1)
    nf, nc = fi_info.n, co_info.n
    dd, hd = random_level(h, l, 400 + l, 1.0)
    dv, hv = random_level(h, l + 1, 500 + l, 1.0)
    fc = mg.level_array(h, l + 1)
    mg.mg_level_restrict(h, l, dd, fc)
    gfc = Grid(fc.cpu().numpy(), co_info.kind)
    du, hu = random_level(h, l, 600 + l, 1.0)
    mg.mg_level_prolong_add(h, l, du, dv)
    gu = Grid(du.cpu().numpy(), fi_info.kind)
    D, V, U = Grid(hd, fi_info.kind), Grid(hv, co_info.kind), Grid(hu, fi_info.kind)
    fine_ok = lambda i, j: 1 <= i <= nf - 1 and 1 <= j <= nf - 1
    coarse_ok = lambda i, j: 1 <= i <= nc - 1 and 1 <= j <= nc - 1
    if l == 0:  # axis -> its black points (Eq. transfer_r2, axis frame)
        to_fine = lambda i, j: (i, j)
        nbrs = [(0, -1), (-1, 0), (1, 0), (0, 1)]
    else:  # rotated -> axis n/2 (Eq. transfer_r2, rotated frame)
        to_fine = lambda i, j: (2 * i, 2 * j)
        nbrs = [(-1, -1), (1, -1), (-1, 1), (1, 1)]
    for i, j in sample_nodes(nc, co_info.kind, 700 + l):
        fi, fj = to_fine(i, j)
        terms = [(fj + dy, fi + dx, 0.125) for dx, dy in nbrs if fine_ok(fi + dx, fj + dy)]
        terms.append((fj, fi, 0.5))
        assert gfc(i, j) == ordered_sum(sorted(terms), D), ("restrict", l, i, j)
    for i, j in sample_nodes(nf, fi_info.kind, 800 + l):
        if l == 0:
            black = (i + j) % 2 == 0
            src = [(i, j)] if black else [(i + dx, j + dy) for dx, dy in nbrs]
        else:
            black = i % 2 == 0
            src = [(i // 2, j // 2)] if black else [((i + dx) // 2, (j + dy) // 2) for dx, dy in nbrs]
        w = 1.0 if black else 0.25
        terms = sorted((cj, ci, w) for ci, cj in src if coarse_ok(ci, cj))
        e = ordered_sum(terms, V) if terms else 0.0
        assert gu(i, j) == U(i, j) + e, ("prolong", l, i, j)


def torch_residual(u, f, order):
    """Relative residual ||f - L u|| / ||f|| over interior nodes, plain PyTorch FP64,
    odd-reflection ghosts for the fourth-order stencil (independent of the library)."""
    n = u.shape[0] - 1
    h2 = 1.0 / (n * n)
    g = torch.nn.functional.pad(u[None, None], (2, 2, 2, 2))[0, 0]
    g[:, 1], g[:, -2] = -g[:, 3], -g[:, -4]  # u(-h) = -u(h) about the boundary lines
    g[1, :], g[-2, :] = -g[3, :], -g[-4, :]
    c = g[2:-2, 2:-2]
    if order == 2:
        lu = (4 * c - g[1:-3, 2:-2] - g[3:-1, 2:-2] - g[2:-2, 1:-3] - g[2:-2, 3:-1]) / h2
    else:
        lu = (60 * c - 16 * (g[1:-3, 2:-2] + g[3:-1, 2:-2] + g[2:-2, 1:-3] + g[2:-2, 3:-1])
              + g[:-4, 2:-2] + g[4:, 2:-2] + g[2:-2, :-4] + g[2:-2, 4:]) / (12 * h2)
    r = (f - lu)[1:-1, 1:-1]
    return float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(f[1:-1, 1:-1]))


def test_bench_workload_fp64_solve_reaches_tolerance():
    """4097^2, order 4, red-black coarsening, Galerkin G^(2), V(2,1), FP64, to 1e-10."""
    f = torch.tensor(synth.rhs_sine_modes(N, 0), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(N, 4, "redblack", "galerkin", nu1=2, nu2=1)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=30)
    finally:
        h.close()
    assert k <= 8 and hist[-1] < 1e-10
    assert all(hist[m + 1] < hist[m] for m in range(k))
    rr = torch_residual(u, f, 4)
    # both evaluate the same residual up to rounding order (~1e-13 of ||f|| here)
    assert abs(rr - hist[-1]) <= 0.2 * hist[-1] + 1e-13, (rr, hist[-1])


@pytest.mark.parametrize("order", [2, 4])
def test_mixed_precision_8193_reaches_tolerance(order):
    """8193^2, N(0,1) right-hand side, FP32 inner cycles inside FP64 refinement."""
    n = 8192
    f = torch.tensor(synth.rhs_normal(n, 17), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, order, "redblack", "galerkin", nu1=2 if order == 4 else 1, nu2=1,
                    precision=mg.MG_PREC_MIXED_FP32, fma_contract=1)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=40)
    finally:
        h.close()
    assert hist[-1] < 1e-10 and k <= 10
    rr = torch_residual(u, f, order)
    assert rr < 1.5e-10, rr
    del f, u
    torch.cuda.empty_cache()
    assert math.isfinite(rr)


def test_batched_workload_512_problems_reach_tolerance():
    """512 problems, sides 2^k + 1 with k uniform in {7..11}, order 2 or 4 (50/50),
    N(0,1) right-hand sides, mixed precision, one level-synchronous batched solve to 1e-8;
    every problem's reported residual and, for a sample, an independent FP64 residual."""
    count = 512
    z = synth.uniform01(91, 2 * count)
    specs = [(2 ** (7 + int(z[2 * i] * 5)), 2 if z[2 * i + 1] < 0.5 else 4) for i in range(count)]
    hs, us, fs = [], [], []
    try:
        for p, (n, order) in enumerate(specs):
            hs.append(mg.mg_setup(n, order, "redblack", "galerkin", nu1=2, nu2=1,  # one schedule per batch
                                  precision=mg.MG_PREC_MIXED_FP32, fma_contract=1))
            fs.append(torch.tensor(synth.rhs_normal(n, 1000 + p), dtype=torch.float64, device="cuda"))
            us.append(torch.zeros_like(fs[-1]))
        cycles, rr = mg.mg_solve_batched(hs, us, fs, rtol=1e-8, max_cycles=40)
        assert max(rr) < 1e-8 and max(cycles) <= 12
        for p in range(0, count, 64):
            assert torch_residual(us[p], fs[p], specs[p][1]) < 1.5e-8, p
    finally:
        for h in hs:
            h.close()
