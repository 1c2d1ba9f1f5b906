"""Serving with continuous batching: every result equals the same request solved
alone, every result is checked against the FP64 oracle, and the budget is respected."""
import numpy as np
import pytest

from oracle import spectral
from oracle.mg import REDBLACK, Options, Oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402
from paper_2008_03885_gb300 import serve  # noqa: E402


def alone(r, **opts):
    f = torch.tensor(r.f, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(r.n, r.order, "redblack", r.coarse_op, **opts)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=r.rtol, max_cycles=60)
    finally:
        h.close()
    return u.cpu().numpy(), k


@pytest.mark.parametrize("opts", [dict(nu1=2, nu2=1),
                                  dict(nu1=2, nu2=1, precision=mg.MG_PREC_MIXED_FP32, fma_contract=1)])
def test_results_identical_alone_and_in_the_mix(opts):
    reqs = serve.poisson_stream(seed=5, count=40, rate=2000.0, k_lo=4, k_hi=8, rtol=1e-8)
    srv = serve.Server(slots=6, budget_bytes=8e9, **opts)
    try:
        results, stats = srv.run(reqs, realtime=True)
    finally:
        srv.close()
    assert stats["requests"] == 40 and stats["p99_ms"] >= stats["p50_ms"] > 0
    for r in reqs:
        res = results[r.rid]
        assert res.rel_res < 1e-8
        u, k = alone(r, **opts)
        assert res.cycles == k
        assert np.array_equal(res.u, u), r.rid


class OracleCache:
    """One oracle hierarchy per problem shape (the served requests repeat shapes)."""

    def __init__(self, **opts):
        self.opts, self.cache = opts, {}

    def __call__(self, r):
        key = (r.n, r.order, r.coarse_op)
        if key not in self.cache:
            self.cache[key] = Oracle(r.n, r.order, REDBLACK, r.coarse_op, Options(**self.opts))
        return self.cache[key]


@pytest.mark.parametrize("mixed", [False, True])
def test_served_results_against_the_oracle(mixed):
    """Every served solution meets the tolerance by the oracle's own FP64 residual and is
    close to the exact discrete solution (oracle/spectral.py). FP64 with the exact
    evaluation order: every served solution equals the oracle's iterate after the same
    number of cycles bit for bit (Algorithm "MG", Sec. 2.2, stopped by its while-test)."""
    opts = dict(nu1=2, nu2=1)
    if mixed:
        opts.update(precision=mg.MG_PREC_MIXED_FP32, fma_contract=1)
    reqs = serve.poisson_stream(seed=21, count=32, rate=3000.0, k_lo=4, k_hi=8, rtol=1e-8)
    srv = serve.Server(slots=5, budget_bytes=8e9, **opts)
    try:
        results, stats = srv.run(reqs, realtime=True)
    finally:
        srv.close()
    oracles = OracleCache(nu1=2, nu2=1)
    for r in reqs:
        res = results[r.rid]
        o = oracles(r)
        ug = o.to_vec(res.u)
        fv = o.to_vec(r.f)
        rr = o.rel_residual(ug, fv)
        assert rr < 1.5e-8, (r.rid, rr)
        assert abs(rr - res.rel_res) <= 1e-6 * rr, (r.rid, rr, res.rel_res)
        U = o.to_vec(spectral.solve(r.f, r.order))
        assert np.linalg.norm(ug - U) <= 1e-6 * np.linalg.norm(U), r.rid
        if not mixed:
            uo, ho = o.solve(fv, rtol=r.rtol, max_cycles=60)
            assert res.cycles == len(ho) - 1, r.rid
            assert np.array_equal(ug, uo), r.rid


def test_small_budget_evicts_and_stays_correct():
    reqs = serve.poisson_stream(seed=9, count=24, rate=5000.0, k_lo=5, k_hi=8, rtol=1e-8)
    big = max(mg.mg_workspace_bytes(r.n, r.order, "redblack", r.coarse_op, nu1=2, nu2=1) + 2 * (r.n + 1) ** 2 * 8
              for r in reqs)
    srv = serve.Server(slots=3, budget_bytes=1.6 * big, nu1=2, nu2=1)
    try:
        results, stats = srv.run(reqs, realtime=False)
    finally:
        srv.close()
    assert stats["hierarchies_evicted"] > 0
    assert stats["hbm_peak_gb"] * 1e9 <= 1.6 * big + 1
    for r in reqs[:6]:
        u, _ = alone(r, nu1=2, nu2=1)
        assert np.array_equal(results[r.rid].u, u)
