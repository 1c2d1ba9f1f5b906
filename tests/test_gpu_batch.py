"""Batched (level-synchronous) solves against the same problems solved one by one,
and against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle.mg import Options, Oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402

PROBLEMS = [  # (n, order, coarsening, coarse_op)
    (16, 2, "redblack", "galerkin"), (64, 4, "redblack", "galerkin"), (32, 2, "standard", "galerkin"),
    (128, 4, "redblack", "nongalerkin"), (64, 2, "redblack", "g1"), (128, 2, "redblack", "galerkin"),
    (32, 4, "standard", "nongalerkin"), (256, 4, "redblack", "galerkin"), (8, 2, "redblack", "gn"),
    (64, 4, "redblack", "galerkin_true_high"),
]


def make(problems, **opts):
    hs, us, fs = [], [], []
    for k, (n, order, co, op) in enumerate(problems):
        hs.append(mg.mg_setup(n, order, co, op, nu1=2, nu2=1, **opts))
        F = synth.rhs_normal(n, seed=100 + k)
        fs.append(torch.tensor(F, dtype=torch.float64, device="cuda"))
        us.append(torch.zeros_like(fs[-1]))
    return hs, us, fs


def solo(problems, rtol, **opts):
    hs, us, fs = make(problems, **opts)
    out = []
    for h, u, f in zip(hs, us, fs):
        k, hist = mg.mg_solve(h, u, f, rtol=rtol, max_cycles=40)
        out.append((k, hist[-1], u.cpu().numpy()))
        h.close()
    return out


@pytest.mark.parametrize("opts", [dict(), dict(precision=mg.MG_PREC_MIXED_FP32, fma_contract=1)])
def test_batch_matches_individual_solves_bitwise(opts):
    rtol = 1e-10
    ref = solo(PROBLEMS, rtol, **opts)
    hs, us, fs = make(PROBLEMS, **opts)
    b = mg.mg_batch_create(hs)
    try:
        for rep in range(2):  # the batch is reusable
            for u in us:
                u.zero_()
            cyc, rr = mg.mg_batch_solve(b, us, fs, rtol=rtol, max_cycles=40)
            torch.cuda.synchronize()
            for p, (k, r, u_ref) in enumerate(ref):
                assert cyc[p] == k, (p, cyc[p], k)
                assert abs(rr[p] - r) <= 1e-12 * r
                assert np.array_equal(us[p].cpu().numpy(), u_ref), p
    finally:
        b.close()
        for h in hs:
            h.close()


def test_batch_uneven_sizes_reach_tolerance_and_oracle_agrees():
    rng = np.random.default_rng(7)
    problems = []
    for k in range(24):
        n = int(2 ** rng.integers(5, 10))  # 32 .. 512
        problems.append((n, int(rng.choice([2, 4])), "redblack", "galerkin"))
    hs, us, fs = make(problems, precision=mg.MG_PREC_MIXED_FP32, fma_contract=1)
    try:
        cyc, rr = mg.mg_solve_batched(hs, us, fs, rtol=1e-8, max_cycles=40)
        assert max(rr) < 1e-8
        for p in (0, 5, 11):
            n, order, co, op = problems[p]
            o = Oracle(n, order, co, op, Options(nu1=2, nu2=1))
            f = o.to_vec(fs[p].cpu().numpy())
            assert o.rel_residual(o.to_vec(us[p].cpu().numpy()), f) < 1.5e-8
    finally:
        for h in hs:
            h.close()


def test_batch_rejects_mismatched_schedules():
    h1 = mg.mg_setup(32, 2, nu1=1)
    h2 = mg.mg_setup(32, 2, nu1=2)
    h3 = mg.mg_setup(32, 2, gamma=2)
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_batch_create([h1, h2])
        assert e.value.status == mg.MG_ERR_INVALID
        with pytest.raises(mg.MGError) as e:
            mg.mg_batch_create([h3])
        assert e.value.status == mg.MG_ERR_UNSUPPORTED
    finally:
        for h in (h1, h2, h3):
            h.close()


def test_batch_launch_count_is_per_level_not_per_problem():
    problems = [(64, 2, "redblack", "galerkin")] * 16
    hs, us, fs = make(problems)
    b = mg.mg_batch_create(hs)
    try:
        before = mg.mg_batch_get_launches(b)
        cyc, rr = mg.mg_batch_solve(b, us, fs, rtol=1e-10, max_cycles=40)
        launched = mg.mg_batch_get_launches(b) - before
        per_cycle_one = 120  # ~10 kernels per level of one 65^2 problem (11 levels)
        assert launched < (max(cyc) + 2) * per_cycle_one + 16 + 8
    finally:
        b.close()
        for h in hs:
            h.close()


@pytest.mark.parametrize("solo_min_n,workers", [(64, 3), (8, 2), (128, 1)])
@pytest.mark.parametrize("opts", [dict(), dict(precision=mg.MG_PREC_MIXED_FP32, fma_contract=1)])
def test_hybrid_batch_matches_individual_solves_bitwise(opts, solo_min_n, workers):
    """The hybrid schedule: problems with N >= solo_min_n solved alone on worker streams
    (all of them at 8), the rest level-synchronously, concurrently; every result is
    bitwise that of mg_solve alone, reported in the caller's problem order."""
    rtol = 1e-10
    ref = solo(PROBLEMS, rtol, **opts)
    hs, us, fs = make(PROBLEMS, **opts)
    b = mg.mg_batch_create(hs, solo_min_n=solo_min_n, workers=workers)
    try:
        for rep in range(2):
            for u in us:
                u.zero_()
            before = mg.mg_batch_get_launches(b)
            cyc, rr = mg.mg_batch_solve(b, us, fs, rtol=rtol, max_cycles=40)
            torch.cuda.synchronize()
            assert mg.mg_batch_get_launches(b) - before >= sum(cyc)
            for p, (k, r, u_ref) in enumerate(ref):
                assert cyc[p] == k, (p, cyc[p], k)
                assert abs(rr[p] - r) <= 1e-12 * r
                assert np.array_equal(us[p].cpu().numpy(), u_ref), p
    finally:
        b.close()
        for h in hs:
            h.close()


def test_hybrid_batch_on_a_side_stream_and_not_converged_status():
    """The caller's stream waits for the worker streams; a missed tolerance in either
    part comes back as MG_ERR_NOT_CONVERGED with every problem's count and residual."""
    problems = [(128, 2, "redblack", "galerkin"), (32, 4, "redblack", "galerkin"), (256, 4, "redblack", "galerkin")]
    hs, us, fs = make(problems)
    b = mg.mg_batch_create(hs, solo_min_n=128, workers=2)
    side = torch.cuda.Stream()
    try:
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            cyc, rr = mg.mg_batch_solve(b, us, fs, rtol=1e-14, max_cycles=2, stream=side,
                                        raise_not_converged=False)
            norms = [torch.linalg.vector_norm(u).item() for u in us]  # ordered after the solve on `side`
        assert cyc == [2, 2, 2] and all(1e-14 < r < 1 for r in rr) and all(x > 0 for x in norms)
        for u in us:
            u.zero_()
        with pytest.raises(mg.MGError) as e:
            mg.mg_batch_solve(b, us, fs, rtol=1e-14, max_cycles=2)
        assert e.value.status == mg.MG_ERR_NOT_CONVERGED
    finally:
        b.close()
        for h in hs:
            h.close()


def test_batch_rejects_a_repeated_handle_and_bad_options():
    h1 = mg.mg_setup(32, 2)
    h2 = mg.mg_setup(32, 2)
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_batch_create([h1, h2, h1])
        assert e.value.status == mg.MG_ERR_INVALID
        for kw in (dict(solo_min_n=-1), dict(workers=-2), dict(workers=65)):
            with pytest.raises(mg.MGError) as e:
                mg.mg_batch_create([h1, h2], **kw)
            assert e.value.status == mg.MG_ERR_INVALID
    finally:
        h1.close()
        h2.close()
