"""Cubic transfers (App. A, Eq. interp_2d4o / restr_2d4o) and the fourth-order
non-Galerkin coarse operator nG^(4) (Eq. L_H_4n_2d) on the GPU against the oracle:
single steps and iterates bit for bit (FP64, fma_contract = 0), histories to 1e-12,
for Dirichlet and periodic boundaries, including the Galerkin recursion that is exact
only up to the third coarse level (both sides round the exact product once)."""
import numpy as np
import pytest

import synth
from oracle.mg import (DIRICHLET, GALERKIN, GN, NONGALERKIN, NONGALERKIN_HIGH, PERIODIC, STANDARD, TRUE_HIGH,
                       Options, Oracle)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines skip the module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402

HIST_RTOL = 1e-12
CONFIGS = [(4, NONGALERKIN_HIGH, 4), (4, TRUE_HIGH, 4), (4, GALERKIN, 4), (2, GALERKIN, 4), (6, NONGALERKIN_HIGH, 4),
           (4, GN, 4), (4, NONGALERKIN, 4), (4, NONGALERKIN_HIGH, 2), (6, TRUE_HIGH, 4)]


def rhs(n, bnd, seed):
    return synth.rhs_periodic_normal(n, seed) if bnd == PERIODIC else synth.rhs_normal(n, seed)


def pair(n, order, op, to, bnd, **opts):
    o = Oracle(n, order, STANDARD, op, Options(transfer_order=to, **{k: v for k, v in opts.items()
                                                                     if k in ("omega", "nu1", "nu2", "gamma")}),
               boundary=bnd)
    h = mg.mg_setup(n, order, "standard", op, transfer_order=to, boundary=bnd, **opts)
    return o, h


def to_dev(h, level, vec):
    i, j, row, col = mg.level_nodes(h, level)
    a = mg.level_array(h, level)
    a[torch.as_tensor(row), torch.as_tensor(col)] = torch.as_tensor(vec, dtype=torch.float64).cuda()
    return a


def from_dev(h, level, a):
    i, j, row, col = mg.level_nodes(h, level)
    return a.cpu().numpy()[row, col]


@pytest.mark.parametrize("bnd", [DIRICHLET, PERIODIC])
@pytest.mark.parametrize("order,op,to", CONFIGS)
def test_level_steps_bitwise(order, op, to, bnd):
    n = 64
    o, h = pair(n, order, op, to, bnd)
    try:
        assert mg.mg_num_levels(h) == len(o.levels)
        for l, lev in enumerate(o.levels):
            u = synth.uniform_pm1(1000 + l, lev.size) * 3.0
            f = synth.uniform_pm1(2000 + l, lev.size) * 1e3
            du, df = to_dev(h, l, u), to_dev(h, l, f)
            out = mg.level_array(h, l)
            mg.mg_level_apply(h, l, du, out)
            assert np.array_equal(from_dev(h, l, out), o.apply(l, u)), ("apply", l)
            if l + 1 < len(o.levels):
                us = du.clone()
                mg.mg_level_smooth(h, l, us, df, 2)
                assert np.array_equal(from_dev(h, l, us), o.smooth(l, o.smooth(l, u, f), f)), ("smooth", l)
                fc = mg.level_array(h, l + 1)
                mg.mg_level_restrict(h, l, df, fc)
                assert np.array_equal(from_dev(h, l + 1, fc), o.restrict(l, f)), ("restrict", l)
                v = synth.uniform_pm1(3000 + l, o.levels[l + 1].size)
                uu = du.clone()
                mg.mg_level_prolong_add(h, l, uu, to_dev(h, l + 1, v))
                assert np.array_equal(from_dev(h, l, uu), u + o.prolong(l, v)), ("prolong", l)
        torch.cuda.synchronize()
    finally:
        h.close()


def run(n, order, op, to, bnd, cycles, **opts):
    o, h = pair(n, order, op, to, bnd, **opts)
    F = rhs(n, bnd, 4)
    uo, ho = o.solve(o.to_vec(F), max_cycles=cycles, fixed_cycles=True)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    try:
        k, hg = mg.mg_solve(h, u, f, rtol=0.0, max_cycles=cycles, raise_not_converged=False)
    finally:
        h.close()
    return np.array(hg), np.array(ho), o.to_vec(u.cpu().numpy()), uo


@pytest.mark.parametrize("bnd", [DIRICHLET, PERIODIC])
@pytest.mark.parametrize("order,op,to", CONFIGS)
def test_cycle_histories_and_iterates_match_oracle(order, op, to, bnd):
    hg, ho, ug, uo = run(128, order, op, to, bnd, 8, nu1=2)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("op", [TRUE_HIGH, GALERKIN])
def test_deep_galerkin_levels_round_the_exact_product_once(op):
    """N = 256: seven coarse levels, four of them past FP64's exact range."""
    hg, ho, ug, uo = run(256, 4, op, 4, DIRICHLET, 6, nu1=2)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("opts", [dict(gamma=2), dict(tail_unknowns=-1), dict(tail_unknowns=4096, tail_ctas=4)])
def test_variants_match_oracle(opts):
    hg, ho, ug, uo = run(64, 4, TRUE_HIGH, 4, DIRICHLET, 6, nu1=2, **opts)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("bnd", [DIRICHLET, PERIODIC])
def test_mixed_precision_reaches_1e10(bnd):
    n = 256
    F = rhs(n, bnd, 9)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, 4, "standard", "nongalerkin_high", transfer_order=4, boundary=bnd, nu1=2,
                    precision=mg.MG_PREC_MIXED_FP32)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=40)
    finally:
        h.close()
    assert hist[-1] < 1e-10
    o = Oracle(n, 4, STANDARD, NONGALERKIN_HIGH, Options(nu1=2, transfer_order=4), boundary=bnd)
    assert o.rel_residual(o.to_vec(u.cpu().numpy()), o.to_vec(F)) < 1.5e-10


def test_batch_rejects_cubic_transfers():
    h = mg.mg_setup(32, 4, "standard", "galerkin", transfer_order=4)
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_batch_create([h])
        assert e.value.status == mg.MG_ERR_UNSUPPORTED
    finally:
        h.close()
