"""The allocation-free relative-residual entry point, checked against mg_cycle and the oracle.

mg_rel_residual_static is for callers that must not allocate device memory at the
point where they need a residual norm: a loop that cannot afford cudaMalloc's implicit
device synchronisation, or a host that fixes the library's memory at set-up (a budget
or an arena it manages itself). Its partial sums live in a fixed device array inside
the library instead of the handle's workspace. Each case calls it twice in a row (the
array keeps the previous call's partials) and compares it with the norm mg_cycle
returns from the handle's workspace and with the FP64 oracle's residual norm. This
file is collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle.mg import GALERKIN, PERIODIC, REDBLACK, STANDARD, Options, Oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402

HIST_RTOL = 1e-12  # the per-cycle residual tolerance of the parity tests
FMA_RTOL = 1e-9    # handles that let products fuse: the residual's rounding differs from the oracle's


def _fn():
    fn = mg._lib.mg_rel_residual_static
    fn.argtypes = [ctypes.c_void_p] * 5
    fn.restype = ctypes.c_int
    return fn


def static_rel_residual(h, u, f):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = _fn()(h.ptr, u.data_ptr(), f.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == mg.MG_OK, st
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("n,order,coarsening", [(64, 2, "redblack"), (512, 4, "standard"), (4096, 4, "redblack")])
def test_static_scratch_residual_matches_cycle_residual(n, order, coarsening):
    F = synth.rhs_sine_modes(n, seed=3) if n >= 512 else synth.rhs_normal(n, seed=3)
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = mg.mg_setup(n, order, coarsening, "galerkin", nu1=2 if order == 4 else 1)
    try:
        for _ in range(2):  # two calls in a row: the array keeps the previous call's partials
            rr = mg.mg_cycle(h, u, f)  # relative residual from the handle's workspace
            rs = static_rel_residual(h, u, f)
            assert abs(rs - rr) <= HIST_RTOL * rr, (rs, rr)
    finally:
        h.close()


def _oracle_case(kind):
    """(handle options, oracle, F, initial u grid, tolerance) of one handle kind."""
    n = 64
    if kind == "periodic":
        F = synth.rhs_periodic_normal(n, seed=8)
        o = Oracle(n, 4, REDBLACK, GALERKIN, Options(nu1=2), boundary=PERIODIC)
        return dict(order=4, co=REDBLACK, nu1=2, boundary="periodic"), o, F, np.zeros_like(F), HIST_RTOL
    if kind == "dirichlet_data":
        x = np.arange(n + 1) / n
        X, Y = np.meshgrid(x, x)
        G = np.cos(2 * X) * np.sinh(Y) + X
        G[1:-1, 1:-1] = 0.0
        F = synth.rhs_normal(n, seed=9)
        o = Oracle(n, 2, STANDARD, GALERKIN)
        o.set_boundary(G)
        return dict(order=2, co=STANDARD, nu1=1, dirichlet_data=1), o, F, G, HIST_RTOL
    if kind == "mixed":
        F = synth.rhs_normal(n, seed=10)
        o = Oracle(n, 4, REDBLACK, GALERKIN, Options(nu1=2))
        return (dict(order=4, co=REDBLACK, nu1=2, precision=mg.MG_PREC_MIXED_FP32, fma_contract=1), o, F,
                np.zeros_like(F), FMA_RTOL)
    assert kind == "fma"
    F = synth.rhs_normal(n, seed=11)
    o = Oracle(n, 2, REDBLACK, GALERKIN)
    return dict(order=2, co=REDBLACK, nu1=1, fma_contract=1), o, F, np.zeros_like(F), FMA_RTOL


@pytest.mark.parametrize("kind", ["periodic", "dirichlet_data", "mixed", "fma"])
def test_static_scratch_residual_matches_oracle(kind):
    """Other handle kinds: periodic boundaries, nonzero Dirichlet data (the boundary of u
    is read as stored), a mixed-precision handle (its FP64 finest level, products fused)
    and an FMA handle; the norm is the oracle's relative residual of the same iterate."""
    opts, o, F, U0, tol = _oracle_case(kind)
    order, co = opts.pop("order"), opts.pop("co")
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.tensor(U0, dtype=torch.float64, device="cuda")
    h = mg.mg_setup(64, order, co, "galerkin", **opts)
    try:
        for _ in range(2):
            mg.mg_cycle(h, u, f)
            rs = static_rel_residual(h, u, f)
            ug = u.cpu().numpy()
            ro = o.rel_residual(o.to_vec(ug), o.to_vec(F))
            assert abs(rs - ro) <= tol * ro, (kind, rs, ro)
    finally:
        h.close()


def test_static_scratch_residual_rejects_null_arguments():
    n = 32
    f = torch.tensor(synth.rhs_normal(n, seed=1), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    h = mg.mg_setup(n, 2, "redblack", "galerkin")
    fn = _fn()
    s = torch.cuda.current_stream().cuda_stream
    try:
        assert fn(None, u.data_ptr(), f.data_ptr(), out.data_ptr(), s) == mg.MG_ERR_INVALID
        assert fn(h.ptr, None, f.data_ptr(), out.data_ptr(), s) == mg.MG_ERR_INVALID
        assert fn(h.ptr, u.data_ptr(), None, out.data_ptr(), s) == mg.MG_ERR_INVALID
        assert fn(h.ptr, u.data_ptr(), f.data_ptr(), None, s) == mg.MG_ERR_INVALID
        # a valid call after the rejected ones still answers
        rr = mg.mg_cycle(h, u, f)
        assert abs(static_rel_residual(h, u, f) - rr) <= HIST_RTOL * rr
    finally:
        h.close()
