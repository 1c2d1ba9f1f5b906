"""The allocation-free relative-residual entry point, checked against mg_cycle.

mg_rel_residual_static serves callers that may not allocate device memory when
they need a residual norm (for example while a stream is being captured into a
CUDA graph, or in a loop that must not pay cudaMalloc's implicit device
synchronisation). Its partial sums live in a fixed device array inside the
library instead of the handle's workspace. This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2008_03885_gb300 as mg  # noqa: E402

HIST_RTOL = 1e-12  # the per-cycle residual tolerance of the parity tests


def static_rel_residual(h, u, f):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    lib = mg._lib
    lib.mg_rel_residual_static.argtypes = [ctypes.c_void_p] * 5
    lib.mg_rel_residual_static.restype = ctypes.c_int
    st = lib.mg_rel_residual_static(h.ptr, u.data_ptr(), f.data_ptr(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
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
