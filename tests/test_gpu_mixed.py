"""Mixed-precision solves (FP64 residual and update, FP32 inner cycles) against the
FP64 oracle: the oracle recomputes the final residual of the GPU iterate, and the
GPU solution is compared with the oracle's converged FP64 solution."""
import math

import numpy as np
import pytest

import synth
from oracle.mg import GALERKIN, NONGALERKIN, REDBLACK, STANDARD, Options, Oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402


def mixed_solve(n, order, co, op, F, rtol=1e-10, **opts):
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, order, co, op, precision=mg.MG_PREC_MIXED_FP32, **opts)
    try:
        k, hist = mg.mg_solve(h, u, f, rtol=rtol, max_cycles=40)
    finally:
        h.close()
    return u.cpu().numpy(), k, hist


@pytest.mark.parametrize("order,co,op", [(2, REDBLACK, GALERKIN), (4, REDBLACK, GALERKIN),
                                         (4, REDBLACK, NONGALERKIN), (4, STANDARD, GALERKIN),
                                         (2, STANDARD, NONGALERKIN)])
@pytest.mark.parametrize("n", [128, 512])
def test_mixed_reaches_1e10_and_matches_fp64_oracle(order, co, op, n):
    F = synth.rhs_normal(n, seed=11)
    nu1 = 2 if order == 4 else 1
    omega = 1.1 if (order == 4 and co == STANDARD) else 1.0
    u, k, hist = mixed_solve(n, order, co, op, F, nu1=nu1, omega=omega)
    assert hist[-1] < 1e-10
    o = Oracle(n, order, co, op, Options(nu1=nu1, omega=omega))
    f = o.to_vec(F)
    ug = o.to_vec(u)
    # the oracle's own FP64 residual of the GPU iterate
    assert o.rel_residual(ug, f) < 1.5e-10
    uo, ho = o.solve(f, rtol=1e-13, max_cycles=60)
    err = np.linalg.norm(ug - uo) / np.linalg.norm(uo)
    # ||u - u*|| / ||u*|| <= cond(L) ||r|| / ||f||, cond(L) < 8 N^2 / (2 pi^2)
    kappa = 8.0 * n * n / (2 * math.pi ** 2)
    assert err <= kappa * 1e-10
    assert err <= 1e-8


def test_mixed_history_is_monotone_and_fast():
    n = 1024
    F = synth.rhs_sine_modes(n, seed=0)
    u, k, hist = mixed_solve(n, 4, REDBLACK, GALERKIN, F, nu1=2)
    assert hist[-1] < 1e-10
    assert k <= 8
    assert all(hist[i + 1] < hist[i] for i in range(k))


@pytest.mark.parametrize("bf16_levels", [1, 2])
def test_bf16_storage_trial_still_reaches_1e10(bf16_levels):
    """Values stored on the finest FP32 inner levels rounded to bfloat16: the FP64
    refinement still reaches 1e-10 (more steps), checked by the oracle's residual."""
    n = 256
    F = synth.rhs_normal(n, seed=13)
    u, k, hist = mixed_solve(n, 4, REDBLACK, GALERKIN, F, nu1=2, bf16_levels=bf16_levels)
    assert hist[-1] < 1e-10
    o = Oracle(n, 4, REDBLACK, GALERKIN, Options(nu1=2))
    assert o.rel_residual(o.to_vec(u), o.to_vec(F)) < 1.5e-10
    _, k0, _ = mixed_solve(n, 4, REDBLACK, GALERKIN, F, nu1=2)
    assert k >= k0


def test_bf16_trial_is_rejected_outside_mixed_precision():
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, 2, bf16_levels=1)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED
