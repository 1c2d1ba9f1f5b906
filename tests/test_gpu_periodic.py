"""Periodic boundaries (the paper's computational setting, Sec. 2.2): the CUDA path
through the C ABI against the periodic FP64 oracle. Same contract as the Dirichlet
parity tests: single steps and iterates bit for bit (FP64, fma_contract = 0),
residual histories to 1e-12 relative."""
import numpy as np
import pytest

import synth
from oracle.mg import (G1, GALERKIN, GN, NONGALERKIN, PERIODIC, REDBLACK, STANDARD, TRUE_HIGH, VARIABLE,
                       Options, Oracle)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines skip the module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402

HIST_RTOL = 1e-12
ORACLE_OPTS = ("omega", "nu1", "nu2", "gamma", "smoother")

CONFIGS = [(2, REDBLACK, GALERKIN), (2, REDBLACK, NONGALERKIN), (2, REDBLACK, G1), (2, REDBLACK, GN),
           (4, REDBLACK, GALERKIN), (4, REDBLACK, NONGALERKIN), (4, REDBLACK, TRUE_HIGH),
           (6, REDBLACK, GALERKIN), (2, STANDARD, GALERKIN), (4, STANDARD, NONGALERKIN),
           (4, STANDARD, TRUE_HIGH), (2, VARIABLE, GALERKIN), (4, VARIABLE, GN)]


def oracle(n, order, co, op, **opts):
    return Oracle(n, order, co, op, Options(**{k: v for k, v in opts.items() if k in ORACLE_OPTS}),
                  boundary=PERIODIC)


def setup(n, order, co, op, **opts):
    o = dict(opts)
    if o.get("smoother") == "jacobi":
        o["smoother"] = mg.MG_SMOOTH_JACOBI
    return mg.mg_setup(n, order, co, op, boundary="periodic", **o)


def to_dev(h, level, vec):
    i, j, row, col = mg.level_nodes(h, level)
    a = mg.level_array(h, level)
    a[torch.as_tensor(row), torch.as_tensor(col)] = torch.as_tensor(vec, dtype=torch.float64).cuda()
    return a


def from_dev(h, level, a):
    i, j, row, col = mg.level_nodes(h, level)
    return a.cpu().numpy()[row, col]


@pytest.mark.parametrize("order,co,op", CONFIGS)
def test_level_steps_bitwise(order, co, op):
    n = 64
    o = oracle(n, order, co, op)
    h = setup(n, order, co, op)
    try:
        assert mg.mg_num_levels(h) == len(o.levels)
        for l, lev in enumerate(o.levels):
            i, j, _, _ = mg.level_nodes(h, l)
            assert np.array_equal(i, lev.pi) and np.array_equal(j, lev.pj)
            assert mg.mg_get_level_info(h, l).unknowns == lev.size
            u = synth.uniform_pm1(1000 + l, lev.size) * 3.0
            f = synth.uniform_pm1(2000 + l, lev.size) * 1e3
            du, df = to_dev(h, l, u), to_dev(h, l, f)
            out = mg.level_array(h, l)
            mg.mg_level_apply(h, l, du, out)
            assert np.array_equal(from_dev(h, l, out), o.apply(l, u)), ("apply", l)
            mg.mg_level_residual(h, l, du, df, out)
            assert np.array_equal(from_dev(h, l, out), o.residual(l, u, f)), ("residual", l)
            if l + 1 < len(o.levels):  # the single-node level is only ever solved, not smoothed
                us = du.clone()
                mg.mg_level_smooth(h, l, us, df, 2)
                assert np.array_equal(from_dev(h, l, us), o.smooth(l, o.smooth(l, u, f), f)), ("smooth", l)
                fc = mg.level_array(h, l + 1)
                mg.mg_level_restrict(h, l, df, fc)
                assert np.array_equal(from_dev(h, l + 1, fc), o.restrict(l, f)), ("restrict", l)
                v = synth.uniform_pm1(3000 + l, o.levels[l + 1].size)
                dv = to_dev(h, l + 1, v)
                uu = du.clone()
                mg.mg_level_prolong_add(h, l, uu, dv)
                assert np.array_equal(from_dev(h, l, uu), u + o.prolong(l, v)), ("prolong", l)
        torch.cuda.synchronize()
    finally:
        h.close()


def run_pair(n, order, co, op, F, cycles, **opts):
    o = oracle(n, order, co, op, **opts)
    uo, ho = o.solve(o.to_vec(F), max_cycles=cycles, fixed_cycles=True)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = setup(n, order, co, op, **opts)
    try:
        k, hg = mg.mg_solve(h, u, f, rtol=0.0, max_cycles=cycles, raise_not_converged=False)
    finally:
        h.close()
    assert k == cycles
    return np.array(hg), np.array(ho), o.to_vec(u.cpu().numpy()), uo


@pytest.mark.parametrize("order,co,op", CONFIGS)
def test_cycle_histories_and_iterates_match_oracle(order, co, op):
    n = 128
    F = synth.rhs_periodic_normal(n, seed=4)
    nu1 = 2 if order > 2 else 1
    hg, ho, ug, uo = run_pair(n, order, co, op, F, 10, nu1=nu1)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("opts", [dict(gamma=2), dict(gamma=3), dict(omega=1.1, nu1=2, nu2=1),
                                  dict(smoother="jacobi", omega=0.8, nu1=2, nu2=2),
                                  dict(tail_unknowns=-1), dict(tail_unknowns=4096, tail_ctas=4)])
def test_cycle_variants_match_oracle(opts):
    n = 64
    F = synth.rhs_periodic_normal(n, seed=5)
    hg, ho, ug, uo = run_pair(n, 2, REDBLACK, GALERKIN, F, 8, **opts)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("n", [4, 8, 16])
@pytest.mark.parametrize("co", [REDBLACK, STANDARD])
def test_small_grids_match_oracle(n, co):
    F = synth.rhs_periodic_normal(n, seed=6)
    hg, ho, ug, uo = run_pair(n, 4, co, GALERKIN, F, 6, nu1=2)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


def test_row_and_column_n_are_neither_read_nor_written():
    n = 64
    F = synth.rhs_periodic_normal(n, seed=8)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    f[n, :] = float("nan")
    f[:, n] = float("nan")
    u = torch.zeros_like(f)
    u[n, :] = 7.0
    u[:, n] = 7.0
    h = setup(n, 2, REDBLACK, GALERKIN)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=30)
    finally:
        h.close()
    assert hist[-1] < 1e-10
    un = u.cpu().numpy()
    assert np.all(un[n, :] == 7.0) and np.all(un[:, n] == 7.0)
    o = oracle(n, 2, REDBLACK, GALERKIN)
    uo, _ = o.solve(o.to_vec(F), rtol=1e-10, max_cycles=30)
    assert np.array_equal(o.to_vec(un), uo)


def test_fourier_mode_is_solved_by_f_over_symbol():
    """A zero-mean single mode cos(2 pi k x) cos(2 pi l y): the converged GPU solution,
    minus its mean, is f / symbol (closed form, no oracle involved)."""
    n, k, l = 256, 3, 11
    F = synth.rhs_periodic_mode(n, k, l)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = setup(n, 2, REDBLACK, GALERKIN)
    try:
        mg.mg_solve(h, u, f, rtol=1e-13, max_cycles=40)
    finally:
        h.close()
    t1, t2 = 2 * np.pi * k / n, 2 * np.pi * l / n
    lam = (4 - 2 * np.cos(t1) - 2 * np.cos(t2)) * n * n
    ug = u.cpu().numpy()[:n, :n]
    assert np.max(np.abs((ug - ug.mean()) - F[:n, :n] / lam)) <= 1e-11 * np.max(np.abs(F / lam))


@pytest.mark.parametrize("order,co,op", [(2, REDBLACK, GALERKIN), (4, REDBLACK, GALERKIN), (4, STANDARD, NONGALERKIN)])
def test_mixed_precision_reaches_1e10(order, co, op):
    n = 256
    F = synth.rhs_periodic_normal(n, seed=9)
    nu1 = 2 if order == 4 else 1
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = setup(n, order, co, op, nu1=nu1, precision=mg.MG_PREC_MIXED_FP32)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=40)
    finally:
        h.close()
    assert hist[-1] < 1e-10
    o = oracle(n, order, co, op, nu1=nu1)
    fv, ug = o.to_vec(F), o.to_vec(u.cpu().numpy())
    assert o.rel_residual(ug, fv) < 1.5e-10
    uo, _ = o.solve(fv, rtol=1e-13, max_cycles=60)
    d = (ug - ug.mean()) - (uo - uo.mean())
    assert np.linalg.norm(d) / np.linalg.norm(uo - uo.mean()) <= 1e-8


def test_fma_contract_converges_to_the_oracle_solution():
    n = 128
    F = synth.rhs_periodic_normal(n, seed=10)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = setup(n, 4, REDBLACK, GALERKIN, nu1=2, fma_contract=1)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=40)
    finally:
        h.close()
    o = oracle(n, 4, REDBLACK, GALERKIN, nu1=2)
    fv, ug = o.to_vec(F), o.to_vec(u.cpu().numpy())
    assert o.rel_residual(ug, fv) < 1.5e-10
    uo, _ = o.solve(fv, rtol=1e-13, max_cycles=60)
    d = (ug - ug.mean()) - (uo - uo.mean())
    assert np.linalg.norm(d) / np.linalg.norm(uo - uo.mean()) <= 1e-8


def test_batch_and_tile_kernel_reject_periodic():
    h = setup(32, 2, REDBLACK, GALERKIN)
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_batch_create([h])
        assert e.value.status == mg.MG_ERR_UNSUPPORTED
    finally:
        h.close()
    with pytest.raises(mg.MGError) as e:
        setup(32, 2, REDBLACK, GALERKIN, sweep_kernel=2)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED
