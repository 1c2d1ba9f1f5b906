"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 with fma_contract = 0 follows the same evaluation order as the oracle, so
single steps and whole iterates are compared bit for bit; residual norms differ
only by the order of the final sum of squares, and per-cycle relative residual
histories must agree to 1e-12 relative.
"""
import numpy as np
import pytest

import synth
from oracle.mg import (G1, GALERKIN, GN, NONGALERKIN, REDBLACK, STANDARD, TRUE_HIGH, VARIABLE,
                       Options, Oracle)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines skip the module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402

HIST_RTOL = 1e-12

ALL_CONFIGS = [(order, co, op) for order in (2, 4) for co in (REDBLACK, STANDARD)
               for op in (NONGALERKIN, GALERKIN, G1, GN, TRUE_HIGH)]


def to_dev(h, level, vec):
    i, j, row, col = mg.level_nodes(h, level)
    a = mg.level_array(h, level)
    a[torch.as_tensor(row), torch.as_tensor(col)] = torch.as_tensor(vec, dtype=torch.float64).cuda()
    return a


def from_dev(h, level, a):
    i, j, row, col = mg.level_nodes(h, level)
    return a.cpu().numpy()[row, col]


def check_order_matches(h, o):
    for l in range(mg.mg_num_levels(h)):
        i, j, _, _ = mg.level_nodes(h, l)
        assert np.array_equal(i, o.levels[l].pi) and np.array_equal(j, o.levels[l].pj)


def rng_vec(seed, n):
    return synth.uniform_pm1(seed, n)


@pytest.mark.parametrize("order,co,op", ALL_CONFIGS)
@pytest.mark.parametrize("n", [64, 128])
def test_level_steps_bitwise(order, co, op, n):
    if n == 128 and op in (G1, GN):
        pytest.skip("covered at n=64")
    o = Oracle(n, order, co, op)
    h = mg.mg_setup(n, order, co, op)
    try:
        assert mg.mg_num_levels(h) == len(o.levels)
        check_order_matches(h, o)
        for l, lev in enumerate(o.levels):
            m = lev.size
            u = rng_vec(1000 + l, m) * 3.0
            f = rng_vec(2000 + l, m) * 1e3
            du, df = to_dev(h, l, u), to_dev(h, l, f)
            out = mg.level_array(h, l)
            mg.mg_level_apply(h, l, du, out)
            assert np.array_equal(from_dev(h, l, out), o.apply(l, u)), ("apply", l)
            mg.mg_level_residual(h, l, du, df, out)
            assert np.array_equal(from_dev(h, l, out), o.residual(l, u, f)), ("residual", l)
            us = du.clone()
            mg.mg_level_smooth(h, l, us, df, 2)
            ref = o.smooth(l, o.smooth(l, u, f), f)
            assert np.array_equal(from_dev(h, l, us), ref), ("smooth", l)
            if l + 1 < len(o.levels):
                fc = mg.level_array(h, l + 1)
                mg.mg_level_restrict(h, l, df, fc)
                assert np.array_equal(from_dev(h, l + 1, fc), o.restrict(l, f)), ("restrict", l)
                v = rng_vec(3000 + l, o.levels[l + 1].size)
                dv = to_dev(h, l + 1, v)
                uu = du.clone()
                mg.mg_level_prolong_add(h, l, uu, dv)
                assert np.array_equal(from_dev(h, l, uu), u + o.prolong(l, v)), ("prolong", l)
        torch.cuda.synchronize()
    finally:
        h.close()


def run_pair(n, order, co, op, F, cycles, **opts):
    o = Oracle(n, order, co, op, Options(**{k: v for k, v in opts.items() if k in ("omega", "nu1", "nu2", "gamma", "smoother")}))
    uo, ho = o.solve(o.to_vec(F), max_cycles=cycles, fixed_cycles=True)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    mgopts = dict(opts)
    if mgopts.get("smoother") == "jacobi":
        mgopts["smoother"] = mg.MG_SMOOTH_JACOBI
    h = mg.mg_setup(n, order, co, op, **mgopts)
    try:
        k, hg = mg.mg_solve(h, u, f, rtol=0.0, max_cycles=cycles, raise_not_converged=False)
    finally:
        h.close()
    assert k == cycles
    ug = u.cpu().numpy()[o.levels[0].pj, o.levels[0].pi]
    return np.array(hg), np.array(ho), ug, uo


def test_config_a_history_matches_oracle():
    """65x65, order 2, RBC, Galerkin, V(1,1), omega = 1, 15 cycles."""
    n = 64
    F = synth.rhs_manufactured_noise(n, seed=0)
    hg, ho, ug, uo = run_pair(n, 2, REDBLACK, GALERKIN, F, 15)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)
    assert ho[-1] < 1e-12


@pytest.mark.parametrize("order,co,op", ALL_CONFIGS)
def test_cycle_histories_match_oracle(order, co, op):
    n = 128
    F = synth.rhs_sine_modes(n, seed=1, n_modes=16, kmax=64) + 0.1 * synth.rhs_normal(n, seed=2)
    nu1 = 2 if order == 4 else 1
    omega = 1.1 if (order == 4 and co == STANDARD) else 1.0
    hg, ho, ug, uo = run_pair(n, order, co, op, F, 10, nu1=nu1, omega=omega)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("opts", [dict(gamma=2), dict(gamma=3), dict(nu1=0, nu2=2), dict(omega=0.9, nu1=3, nu2=2),
                                  dict(smoother="jacobi", omega=0.8, nu1=2, nu2=2)])
def test_cycle_variants_match_oracle(opts):
    n = 64
    F = synth.rhs_normal(n, seed=4)
    co = STANDARD if opts.get("smoother") == "jacobi" else REDBLACK
    hg, ho, ug, uo = run_pair(n, 2, co, GALERKIN, F, 8, **opts)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_small_grids_match_oracle(n):
    for order, co, op in ((2, REDBLACK, GALERKIN), (4, REDBLACK, TRUE_HIGH), (4, STANDARD, G1)):
        F = synth.rhs_normal(n, seed=n)
        hg, ho, ug, uo = run_pair(n, order, co, op, F, 5)
        assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
        assert np.array_equal(ug, uo)


def test_solve_reaches_tolerance_and_reports_history():
    n = 256
    F = synth.rhs_sine_modes(n, seed=0)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, 4, "redblack", "galerkin", nu1=2, nu2=1)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=40)
    finally:
        h.close()
    assert hist[-1] < 1e-10 and all(hist[i + 1] < hist[i] for i in range(k))


def test_boundary_of_u_is_reset_and_f_boundary_ignored():
    n = 32
    F = synth.rhs_normal(n, seed=9)
    F2 = F.copy()
    F2[0, :] = 5.0
    F2[:, -1] = -7.0
    outs = []
    for FF, u0 in ((F, 0.0), (F2, 3.0)):
        f = torch.tensor(FF, dtype=torch.float64, device="cuda")
        u = torch.full_like(f, u0)
        u[1:-1, 1:-1] = 0.0
        h = mg.mg_setup(n, 2)
        try:
            mg.mg_solve(h, u, f, rtol=0.0, max_cycles=3, raise_not_converged=False)
        finally:
            h.close()
        outs.append(u.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.all(outs[1][0, :] == 0) and np.all(outs[1][:, -1] == 0)


def test_zero_rhs_and_nonfinite_rhs_are_reported():
    n = 16
    h = mg.mg_setup(n, 2)
    try:
        f = torch.zeros((n + 1, n + 1), dtype=torch.float64, device="cuda")
        u = torch.zeros_like(f)
        with pytest.raises(mg.MGError) as e:
            mg.mg_solve(h, u, f)
        assert e.value.status == mg.MG_ERR_INVALID
        f[3, 4] = float("nan")
        with pytest.raises(mg.MGError) as e:
            mg.mg_solve(h, u, f)
        assert e.value.status == mg.MG_ERR_NONFINITE
    finally:
        h.close()


@pytest.mark.parametrize("order,co,op", [(2, REDBLACK, GALERKIN), (4, REDBLACK, GALERKIN), (4, STANDARD, NONGALERKIN)])
def test_fma_contract_mode_converges_to_the_oracle_solution(order, co, op):
    """fma_contract = 1 changes rounding only: the per-cycle histories agree with the
    oracle to 1e-12 relative while the residual is far above roundoff (first two
    cycles), and the converged solution matches the oracle's within cond(L) * rtol."""
    n = 128
    F = synth.rhs_normal(n, seed=21)
    nu1 = 2 if order == 4 else 1
    o = Oracle(n, order, co, op, Options(nu1=nu1))
    f = o.to_vec(F)
    uo, ho = o.solve(f, rtol=1e-13, max_cycles=60)
    ft = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(ft)
    h = mg.mg_setup(n, order, co, op, nu1=nu1, fma_contract=1)
    try:
        k, hg = mg.mg_solve(h, u, ft, rtol=1e-10, max_cycles=40)
    finally:
        h.close()
    assert hg[-1] < 1e-10
    rel = [abs(a - b) / b for a, b in zip(hg[:3], ho[:3])]
    kappa = 8.0 * n * n / (2 * np.pi ** 2)
    # FMA rounding differs by O(eps * cond) relative to ||f|| in each residual
    assert max(rel[1:]) <= kappa * 1e-14 / min(ho[1:3])
    ug = o.to_vec(u.cpu().numpy())
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) <= kappa * 1e-10


@pytest.mark.parametrize("order,co,op", [(2, REDBLACK, GALERKIN), (4, REDBLACK, GALERKIN), (4, REDBLACK, TRUE_HIGH),
                                         (4, STANDARD, NONGALERKIN), (2, STANDARD, G1)])
@pytest.mark.parametrize("nu1,nu2", [(2, 1), (1, 1)])
def test_tile_sweep_kernel_is_bitwise_identical(order, co, op, nu1, nu2):
    """The shared-memory tile kernel (one launch per red-black sweep, out of place)
    reproduces the oracle bit for bit, including odd sweep counts (parity flip)."""
    n = 256
    F = synth.rhs_normal(n, seed=31)
    hg, ho, ug, uo = run_pair(n, order, co, op, F, 6, nu1=nu1, nu2=nu2, sweep_kernel=2)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("order,co,op", [(4, REDBLACK, GALERKIN), (4, REDBLACK, TRUE_HIGH), (2, STANDARD, GN)])
def test_tile_sweep_single_steps_bitwise(order, co, op):
    n = 128
    o = Oracle(n, order, co, op)
    h = mg.mg_setup(n, order, co, op, sweep_kernel=2)
    try:
        for l, lev in enumerate(o.levels):
            u = rng_vec(5000 + l, lev.size)
            f = rng_vec(6000 + l, lev.size) * 100.0
            du, df = to_dev(h, l, u), to_dev(h, l, f)
            mg.mg_level_smooth(h, l, du, df, 3)
            ref = o.smooth(l, o.smooth(l, o.smooth(l, u, f), f), f)
            assert np.array_equal(from_dev(h, l, du), ref), l
    finally:
        h.close()


@pytest.mark.parametrize("tail", [-1, 64, 100000])
def test_tail_cluster_threshold_does_not_change_bits(tail):
    n = 128
    F = synth.rhs_normal(n, seed=41)
    hg, ho, ug, uo = run_pair(n, 4, REDBLACK, GALERKIN, F, 5, nu1=2, tail_unknowns=tail)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("order,op", [(2, GALERKIN), (4, GALERKIN), (4, NONGALERKIN), (2, G1), (4, TRUE_HIGH)])
def test_variable_coarsening_bitwise(order, op):
    n = 128
    F = synth.rhs_normal(n, seed=51)
    hg, ho, ug, uo = run_pair(n, order, VARIABLE, op, F, 6, nu1=2 if order == 4 else 1)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)
    o = Oracle(n, order, VARIABLE, op)
    h = mg.mg_setup(n, order, VARIABLE, op)
    try:
        check_order_matches(h, o)
        for l, lev in enumerate(o.levels[:-1]):
            v = rng_vec(7000 + l, o.levels[l + 1].size)
            d = rng_vec(8000 + l, lev.size)
            fc = mg.level_array(h, l + 1)
            mg.mg_level_restrict(h, l, to_dev(h, l, d), fc)
            assert np.array_equal(from_dev(h, l + 1, fc), o.restrict(l, d)), l
    finally:
        h.close()


@pytest.mark.parametrize("co,op", [(REDBLACK, GALERKIN), (REDBLACK, NONGALERKIN), (REDBLACK, TRUE_HIGH),
                                   (STANDARD, GALERKIN), (VARIABLE, GN)])
def test_sixth_order_bitwise(co, op):
    n = 128
    F = synth.rhs_normal(n, seed=61)
    hg, ho, ug, uo = run_pair(n, 6, co, op, F, 6, nu1=2)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("precision", [mg.MG_PREC_FP64, mg.MG_PREC_MIXED_FP32])
def test_host_buffer_solve_equals_device_solve(precision):
    """mg_solve_host (u, f in host memory, pageable numpy or pinned torch) gives the
    device solve's iterate bit for bit and the same history, on repeated calls."""
    n = 128
    F = synth.rhs_sine_modes(n, seed=4, n_modes=8, kmax=32)
    h = mg.mg_setup(n, 4, REDBLACK, GALERKIN, nu1=2, precision=precision)
    try:
        f = torch.tensor(F, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(f)
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=30)
        for rep in range(2):
            uh = np.zeros((n + 1, n + 1))
            kh, hh = mg.mg_solve_host(h, uh, np.ascontiguousarray(F), rtol=1e-10, max_cycles=30)
            assert kh == k and hh == hist
            assert np.array_equal(uh, u.cpu().numpy())
        up = torch.zeros((n + 1, n + 1), dtype=torch.float64).pin_memory()
        mg.mg_solve_host(h, up, torch.tensor(F).pin_memory(), rtol=1e-10, max_cycles=30)
        assert torch.equal(up, u.cpu())
    finally:
        h.close()


@pytest.mark.parametrize("length", [2.5, 0.25])
def test_domain_length_matches_oracle(length):
    n = 64
    F = synth.rhs_normal(n, seed=31)
    o = Oracle(n, 4, REDBLACK, GALERKIN, Options(nu1=2), length=length)
    uo, ho = o.solve(o.to_vec(F), max_cycles=8, fixed_cycles=True)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, 4, REDBLACK, GALERKIN, nu1=2, length=length)
    try:
        k, hg = mg.mg_solve(h, u, f, rtol=0.0, max_cycles=8, raise_not_converged=False)
    finally:
        h.close()
    assert np.max(np.abs(np.array(hg) - np.array(ho)) / np.array(ho)) <= HIST_RTOL
    assert np.array_equal(o.to_vec(u.cpu().numpy()), uo)


def test_torch_caching_allocator_holds_the_hierarchy():
    """allocator="torch": every handle buffer comes from torch's caching allocator
    (visible in torch.cuda.memory_allocated, returned on close) and the iterates are
    those of the cudaMalloc path bit for bit."""
    n = 256
    F = synth.rhs_normal(n, seed=5)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    outs = []
    for allocator in (None, "torch"):
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        h = mg.mg_setup(n, 4, REDBLACK, GALERKIN, nu1=2, allocator=allocator,
                        precision=mg.MG_PREC_MIXED_FP32)
        held = torch.cuda.memory_allocated() - before
        u = torch.zeros_like(f)
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=30)
        h.close()
        torch.cuda.synchronize()
        outs.append((u.cpu().numpy(), hist))
        if allocator == "torch":
            assert held >= mg.mg_workspace_bytes(n, 4, REDBLACK, GALERKIN, precision=mg.MG_PREC_MIXED_FP32)
            assert torch.cuda.memory_allocated() == before
        else:
            assert held == 0
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


@pytest.mark.parametrize("co,op", [(REDBLACK, GALERKIN), (STANDARD, NONGALERKIN)])
def test_nonzero_dirichlet_data_matches_oracle(co, op):
    """dirichlet_data = 1 (second order): the boundary entries of u hold g and stay;
    iterates and histories bitwise those of the oracle with the same data."""
    n = 128
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)
    G = np.sin(3 * X) * np.cosh(2 * Y) + X * Y  # boundary data
    F = synth.rhs_normal(n, seed=12)
    o = Oracle(n, 2, co, op)
    o.set_boundary(G)
    uo, ho = o.solve(o.to_vec(F), max_cycles=8, fixed_cycles=True)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.tensor(G, dtype=torch.float64, device="cuda")
    u[1:-1, 1:-1] = 0.0
    h = mg.mg_setup(n, 2, co, op, dirichlet_data=1)
    try:
        k, hg = mg.mg_solve(h, u, f, rtol=0.0, max_cycles=8, raise_not_converged=False)
    finally:
        h.close()
    ug = u.cpu().numpy()
    assert np.max(np.abs(np.array(hg) - np.array(ho)) / np.array(ho)) <= HIST_RTOL
    assert np.array_equal(o.to_vec(ug), uo)
    edge = np.ones((n + 1, n + 1), dtype=bool)
    edge[1:-1, 1:-1] = False
    assert np.array_equal(ug[edge], G[edge])


def test_dirichlet_data_quadratic_is_exact_in_mixed_precision():
    n = 512
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)
    U = X ** 2 - 2 * Y ** 2 + 3 * X * Y
    f = torch.full((n + 1, n + 1), 2.0, dtype=torch.float64, device="cuda")
    u = torch.tensor(U, dtype=torch.float64, device="cuda")
    u[1:-1, 1:-1] = 0.0
    h = mg.mg_setup(n, 2, REDBLACK, GALERKIN, dirichlet_data=1, precision=mg.MG_PREC_MIXED_FP32)
    try:
        # the rounding floor of the residual is ~1e-10 here (terms ~1e6 against f = 2)
        k, hist = mg.mg_solve(h, u, f, rtol=1e-9, max_cycles=30)
    finally:
        h.close()
    assert np.max(np.abs(u.cpu().numpy() - U)) <= 1e-8


def test_dirichlet_data_rejected_for_wide_stencils():
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, 4, REDBLACK, GALERKIN, dirichlet_data=1)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED


@pytest.mark.parametrize("opts", [dict(order=4, co=REDBLACK, op=GALERKIN, nu1=2),
                                  dict(order=2, co=REDBLACK, op=GALERKIN, nu1=1),
                                  dict(order=4, co=STANDARD, op=NONGALERKIN, nu1=1, nu2=2),
                                  dict(order=4, co=REDBLACK, op=GALERKIN, nu1=2, boundary="periodic"),
                                  dict(order=2, co=REDBLACK, op=GALERKIN, nu1=1, dirichlet_data=1)])
def test_solve_with_norm_fused_half_sweep_equals_single_cycles(opts):
    """mg_solve lets each residual-norm kernel also do the next cycle's first (red)
    half-sweep and starts the cycle with black; mg_cycle runs whole cycles. K cycles of
    either must give the same iterate bit for bit and the same relative residuals."""
    opts = dict(opts)
    order, co, op = opts.pop("order"), opts.pop("co"), opts.pop("op")
    n, K = 128, 4
    F = synth.rhs_normal(n, seed=23)
    if opts.get("boundary") == "periodic":
        F = F - F[:n, :n].mean()
        F[n, :] = 0.0
        F[:, n] = 0.0
    h = mg.mg_setup(n, order, co, op, **opts)
    try:
        f = torch.tensor(F, dtype=torch.float64, device="cuda")
        u0 = torch.zeros_like(f)
        if opts.get("dirichlet_data"):
            x = torch.linspace(0, 1, n + 1, dtype=torch.float64, device="cuda")
            g = (x[None, :] ** 2 + 2 * x[:, None]).contiguous()
            u0[0, :], u0[n, :], u0[:, 0], u0[:, n] = g[0, :], g[n, :], g[:, 0], g[:, n]
        us = u0.clone()
        k, hist = mg.mg_solve(h, us, f, rtol=0.0, max_cycles=K, raise_not_converged=False)
        assert k == K
        uc = u0.clone()
        rr = [mg.mg_cycle(h, uc, f) for _ in range(K)]
        assert torch.equal(us, uc)
        assert np.allclose(hist[1:], rr, rtol=1e-13, atol=0.0)
    finally:
        h.close()
