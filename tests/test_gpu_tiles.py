"""The TMA-staged tile kernels of the FP32 inner cycle (sweep_kernel = 0, the default)
give the same bits as the per-step half-sweep, residual and restriction kernels
(sweep_kernel = 1): whole mixed-precision solves are compared bit for bit (iterates and
residual histories) over both orders, red-black and standard coarsening, Galerkin and
non-Galerkin coarse operators, nu1, nu2 in {1, 2}, one and two inner cycles, and both
rounding modes; sizes from 257^2 (the smallest level the tile kernels take, with ragged
last tiles in both directions) upward. Red-black Galerkin hierarchies also run the
rotated tile kernels on level 1 (the first Galerkin 9-point stencil)."""
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402


def solve(n, order, co, op, F, steps, **opts):
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, order, co, op, precision=mg.MG_PREC_MIXED_FP32, **opts)
    try:
        mg.mg_reset_counters(h)
        k, hist = mg.mg_solve(h, u, f, rtol=0.0, max_cycles=steps, raise_not_converged=False)
        launches, _ = mg.mg_get_counters(h)
    finally:
        h.close()
    torch.cuda.synchronize()
    return u, hist, launches


CASES = [
    # (n, order, coarsening, coarse op, nu1, nu2, inner cycles, fma)
    (256, 4, "redblack", "galerkin", 2, 1, 1, 1),
    (256, 2, "redblack", "galerkin", 2, 2, 1, 0),
    (512, 2, "redblack", "galerkin", 1, 1, 1, 1),
    (512, 4, "redblack", "nongalerkin", 2, 1, 1, 1),
    (512, 2, "redblack", "nongalerkin", 2, 2, 1, 0),
    (512, 4, "redblack", "galerkin", 1, 2, 2, 1),
    (512, 4, "standard", "nongalerkin", 2, 1, 1, 1),
    (512, 2, "standard", "galerkin", 1, 1, 2, 0),
    (1024, 4, "redblack", "galerkin", 2, 1, 1, 0),
    (4096, 4, "redblack", "galerkin", 2, 1, 1, 1),
]


@pytest.mark.parametrize("n,order,co,op,nu1,nu2,inner,fma", CASES)
def test_tile_kernels_give_the_same_bits(n, order, co, op, nu1, nu2, inner, fma):
    F = synth.rhs_normal(n, seed=n + order)
    opts = dict(nu1=nu1, nu2=nu2, inner_cycles=inner, fma_contract=fma,
                omega=1.1 if (co == "standard" and order == 4) else 1.0)
    steps = 4
    ut, ht, lt = solve(n, order, co, op, F, steps, sweep_kernel=0, **opts)
    uh, hh, lh = solve(n, order, co, op, F, steps, sweep_kernel=1, **opts)
    assert ht == hh
    assert torch.equal(ut, uh), int((ut != uh).sum())
    assert lt < lh  # the tile path makes fewer launches
