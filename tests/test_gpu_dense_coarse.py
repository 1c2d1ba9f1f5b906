"""The exact coarsest solve with several unknowns (n_min > 2, truncated hierarchies)
against the FP64 oracle: whole iterates bit for bit and per-cycle histories to 1e-12,
through every place the solve runs (the shared-memory tail, the cluster tail, a
standalone kernel, the batched schedule), and the mixed-precision path to the oracle's
converged solution."""
import numpy as np
import pytest

import synth
from oracle.mg import GALERKIN, NONGALERKIN, REDBLACK, STANDARD, TRUE_HIGH, VARIABLE, Options, Oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines skip the module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402

HIST_RTOL = 1e-12
ORACLE_KEYS = ("omega", "nu1", "nu2", "gamma", "n_min", "max_levels")


def run_pair(n, order, co, op, F, cycles, **opts):
    o = Oracle(n, order, co, op, Options(**{k: v for k, v in opts.items() if k in ORACLE_KEYS}))
    uo, ho = o.solve(o.to_vec(F), max_cycles=cycles, fixed_cycles=True)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, order, co, op, **opts)
    try:
        assert mg.mg_num_levels(h) == len(o.levels)
        k, hg = mg.mg_solve(h, u, f, rtol=0.0, max_cycles=cycles, raise_not_converged=False)
    finally:
        h.close()
    assert k == cycles
    ug = u.cpu().numpy()[o.levels[0].pj, o.levels[0].pi]
    return np.array(hg), np.array(ho), ug, uo


CASES = [  # (n, order, coarsening, coarse_op, n_min, extra options)
    (64, 2, REDBLACK, GALERKIN, 4, {}),
    (64, 4, REDBLACK, GALERKIN, 8, dict(nu1=2)),
    (128, 2, STANDARD, NONGALERKIN, 16, {}),
    (128, 4, REDBLACK, TRUE_HIGH, 16, dict(nu1=2)),
    (64, 2, VARIABLE, GALERKIN, 8, dict(gamma=2)),
    (256, 4, STANDARD, GALERKIN, 32, dict(nu1=2, omega=1.1)),
]


@pytest.mark.parametrize("tail", [0, -1, 300])  # shared-memory tail, no tail, cluster tail
@pytest.mark.parametrize("n,order,co,op,n_min,extra", CASES)
def test_dense_coarsest_cycles_bitwise(n, order, co, op, n_min, extra, tail):
    F = synth.rhs_normal(n, seed=n + n_min)
    hg, ho, ug, uo = run_pair(n, order, co, op, F, 6, n_min=n_min, tail_unknowns=tail, **extra)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)


@pytest.mark.parametrize("n,co,max_levels", [(8, REDBLACK, 2), (32, REDBLACK, 2), (64, REDBLACK, 5),
                                             (64, STANDARD, 3)])
def test_truncated_hierarchies_bitwise(n, co, max_levels):
    """max_levels: the coarsest level may be rotated (red-black level 1 at max_levels = 2,
    the two-level direct solver of Sec. 4.3 with omega = 1: one cycle is exact)."""
    F = synth.rhs_normal(n, seed=3 * n + max_levels)
    hg, ho, ug, uo = run_pair(n, 2, co, GALERKIN, F, 4, max_levels=max_levels)
    assert np.max(np.abs(hg - ho) / ho) <= HIST_RTOL
    assert np.array_equal(ug, uo)
    if co == REDBLACK and max_levels == 2:
        assert hg[1] < 1e-13


def test_coarsest_too_large_is_rejected():
    with pytest.raises(mg.MGError) as e:  # rotated level 1 of N = 128: 8065 unknowns
        mg.mg_setup(128, 2, "redblack", "galerkin", max_levels=2)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED


@pytest.mark.parametrize("order", [2, 4])
def test_mixed_precision_with_dense_coarsest_reaches_the_oracle_solution(order):
    n = 256
    F = synth.rhs_normal(n, seed=40 + order)
    o = Oracle(n, order, REDBLACK, GALERKIN, Options(nu1=2, n_min=16))
    uo, _ = o.solve(o.to_vec(F), rtol=1e-12, max_cycles=40)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, order, "redblack", "galerkin", nu1=2, n_min=16, precision=mg.MG_PREC_MIXED_FP32,
                    fma_contract=1)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=1e-11, max_cycles=40)
    finally:
        h.close()
    assert hist[-1] < 1e-11 and k < 15
    ug = u.cpu().numpy()[o.levels[0].pj, o.levels[0].pi]
    assert np.linalg.norm(ug - uo) <= 1e-9 * np.linalg.norm(uo)


def test_fma_handle_with_dense_coarsest_tracks_the_oracle():
    n = 128
    F = synth.rhs_normal(n, seed=77)
    o = Oracle(n, 2, REDBLACK, GALERKIN, Options(n_min=16))
    _, ho = o.solve(o.to_vec(F), max_cycles=6, fixed_cycles=True)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, 2, "redblack", "galerkin", n_min=16, fma_contract=1)
    try:
        _, hg = mg.mg_solve(h, u, f, rtol=0.0, max_cycles=6, raise_not_converged=False)
    finally:
        h.close()
    # fused products change the last bits of every iterate: histories agree to 1e-6
    # relative until they reach the rounding floor (~1e-15 of ||f|| at this size)
    hg, ho = np.array(hg), np.array(ho)
    assert np.all(np.abs(hg - ho) <= 1e-6 * ho + 1e-15), (hg, ho)


BATCH = [(64, 2, "redblack", "galerkin"), (128, 4, "redblack", "galerkin"), (32, 2, "standard", "galerkin"),
         (256, 4, "redblack", "nongalerkin"), (16, 2, "redblack", "galerkin")]


@pytest.mark.parametrize("opts", [dict(), dict(precision=mg.MG_PREC_MIXED_FP32, fma_contract=1)])
def test_batch_with_dense_coarsest_matches_individual_solves_bitwise(opts):
    """Problems of different sizes stopping at n_min = 8 (dense solves of 49 unknowns
    at different depths); the batch's per-problem results are bitwise those of mg_solve
    alone."""
    def make():
        hs, us, fs = [], [], []
        for k, (n, order, co, op) in enumerate(BATCH):
            hs.append(mg.mg_setup(n, order, co, op, nu1=2, nu2=1, n_min=8, **opts))
            fs.append(torch.tensor(synth.rhs_normal(n, seed=500 + k), dtype=torch.float64, device="cuda"))
            us.append(torch.zeros_like(fs[-1]))
        return hs, us, fs

    hs, us, fs = make()
    ref = []
    for h, u, f in zip(hs, us, fs):
        k, hist = mg.mg_solve(h, u, f, rtol=1e-10, max_cycles=40)
        ref.append((k, hist[-1], u.cpu().numpy()))
        u.zero_()
    b = mg.mg_batch_create(hs)
    try:
        cyc, rr = mg.mg_batch_solve(b, us, fs, rtol=1e-10, max_cycles=40)
        torch.cuda.synchronize()
        for p, (k, r, u_ref) in enumerate(ref):
            assert cyc[p] == k, (p, cyc[p], k)
            assert abs(rr[p] - r) <= 1e-12 * r
            assert np.array_equal(us[p].cpu().numpy(), u_ref), p
    finally:
        b.close()
        for h in hs:
            h.close()
