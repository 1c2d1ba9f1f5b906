"""Python binding of libnsmg.so, the GB300 multigrid library (nonstandard coarsening).

Argument marshalling only: every step of the multigrid cycle runs in the CUDA
kernels of the library. Device arrays are torch CUDA tensors (FP64, contiguous);
streams are torch CUDA streams. The functions keep the C ABI's names
(include/nsmg.h) and raise `MGError` on a non-zero status.

There is no CPU fallback: importing this package loads the compiled library
and fails loudly if it has not been built (`python -c "import __graft_entry__ as
g; g.build()"`).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnsmg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libnsmg.so is not built ({LIB_PATH} missing); run the package build first")

_lib = ctypes.CDLL(LIB_PATH)

# ---- enums (mirror include/nsmg.h) ------------------------------------------
MG_OK, MG_ERR_INVALID, MG_ERR_UNSUPPORTED, MG_ERR_OOM, MG_ERR_BUDGET, MG_ERR_CUDA, \
    MG_ERR_NONFINITE, MG_ERR_NOT_CONVERGED, MG_ERR_TIMEOUT = range(9)
MG_COARSEN_STANDARD, MG_COARSEN_REDBLACK, MG_COARSEN_VARIABLE = 0, 1, 2
(MG_OP_NONGALERKIN, MG_OP_GALERKIN, MG_OP_GALERKIN_G1, MG_OP_GALERKIN_GN, MG_OP_GALERKIN_TRUE_HIGH,
 MG_OP_NONGALERKIN_HIGH) = range(6)
MG_SMOOTH_REDBLACK, MG_SMOOTH_JACOBI = 0, 1
MG_PREC_FP64, MG_PREC_MIXED_FP32 = 0, 1
MG_BOUNDARY_DIRICHLET, MG_BOUNDARY_PERIODIC = 0, 1

COARSENING = {"standard": MG_COARSEN_STANDARD, "redblack": MG_COARSEN_REDBLACK, "variable": MG_COARSEN_VARIABLE}
COARSE_OP = {"nongalerkin": MG_OP_NONGALERKIN, "galerkin": MG_OP_GALERKIN, "g1": MG_OP_GALERKIN_G1,
             "gn": MG_OP_GALERKIN_GN, "galerkin_true_high": MG_OP_GALERKIN_TRUE_HIGH,
             "nongalerkin_high": MG_OP_NONGALERKIN_HIGH}


class mg_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("length", ctypes.c_double)]


class mg_options(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32),
                ("gamma", ctypes.c_int32), ("smoother", ctypes.c_int32), ("n_min", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("fma_contract", ctypes.c_int32), ("inner_cycles", ctypes.c_int32),
                ("tail_unknowns", ctypes.c_int32), ("tail_ctas", ctypes.c_int32),
                ("sweep_kernel", ctypes.c_int32), ("bf16_levels", ctypes.c_int32),
                ("boundary", ctypes.c_int32), ("transfer_order", ctypes.c_int32),
                ("dirichlet_data", ctypes.c_int32),
                ("dev_alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)),
                ("dev_free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)),
                ("alloc_ctx", ctypes.c_void_p)]


class mg_level_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("cols", ctypes.c_int32), ("pitch", ctypes.c_int32), ("unknowns", ctypes.c_int32),
                ("nterms", ctypes.c_int32), ("periodic", ctypes.c_int32)]


_vp, _dp, _ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)

_lib.mg_default_options.argtypes = [ctypes.POINTER(mg_options)]
_lib.mg_default_options.restype = None
_lib.mg_setup.argtypes = [ctypes.POINTER(mg_grid), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.POINTER(mg_options), ctypes.POINTER(_vp)]
_lib.mg_cycle.argtypes = [_vp, _vp, _vp, _dp, _vp]
_lib.mg_solve.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _ip, _dp, _vp]
_lib.mg_solve_host.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _ip, _dp, _vp]
_lib.mg_destroy.argtypes = [_vp]
_lib.mg_status_string.argtypes = [ctypes.c_int]
_lib.mg_status_string.restype = ctypes.c_char_p
_lib.mg_workspace_bytes.argtypes = [ctypes.POINTER(mg_grid), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(mg_options)]
_lib.mg_workspace_bytes.restype = ctypes.c_size_t
_lib.mg_num_levels.argtypes = [_vp]
_lib.mg_get_level_info.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(mg_level_info)]
_lib.mg_level_apply.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
_lib.mg_level_residual.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.mg_level_smooth.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp]
_lib.mg_level_restrict.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
_lib.mg_level_prolong_add.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
_lib.mg_get_counters.argtypes = [_vp, _vp]
_lib.mg_reset_counters.argtypes = [_vp]
_lib.mg_set_timing.argtypes = [_vp, ctypes.c_int]
_lib.mg_get_timing.argtypes = [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int64)]
for _name in ("mg_get_counters", "mg_reset_counters", "mg_set_timing", "mg_get_timing", "mg_setup", "mg_cycle", "mg_solve", "mg_destroy", "mg_get_level_info", "mg_level_apply",
              "mg_level_residual", "mg_level_smooth", "mg_level_restrict", "mg_level_prolong_add"):
    getattr(_lib, _name).restype = ctypes.c_int
_lib.mg_num_levels.restype = ctypes.c_int


MG_KERNEL_SMOOTH, MG_KERNEL_RESIDUAL, MG_KERNEL_RESTRICT, MG_KERNEL_PROLONG, MG_KERNEL_NORM = range(5)


class mg_counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("cycles", ctypes.c_int64)]


class MGError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib.mg_status_string(status).decode()} (status {status})")


def _check(status: int, what: str):
    if status != MG_OK:
        raise MGError(status, what)


def _ptr(t) -> int:
    """Device pointer of a torch CUDA tensor (contiguous); ints pass through."""
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


BOUNDARY = {"dirichlet": MG_BOUNDARY_DIRICHLET, "periodic": MG_BOUNDARY_PERIODIC}


def mg_default_options(**overrides) -> mg_options:
    o = mg_options()
    _lib.mg_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "boundary":
            v = BOUNDARY.get(v, v)
        setattr(o, k, v)
    return o


def mg_workspace_bytes(n: int, order: int = 2, coarsening="redblack", coarse_op="galerkin", length: float = 1.0,
                       **opts) -> int:
    g = mg_grid(n, length)
    o = mg_default_options(**opts)
    return int(_lib.mg_workspace_bytes(ctypes.byref(g), order, COARSENING.get(coarsening, coarsening),
                                       COARSE_OP.get(coarse_op, coarse_op), ctypes.byref(o)))


class Handle:
    """Owns an mg_handle; freed by close() or garbage collection."""

    def __init__(self, ptr: int):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            _lib.mg_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _torch_allocator():
    """(dev_alloc, dev_free) callbacks drawing the handle's buffers from torch's CUDA
    caching allocator on the current device."""
    import torch
    dev = torch.cuda.current_device()
    alloc_t = mg_options._fields_[-3][1]
    free_t = mg_options._fields_[-2][1]

    def alloc(size, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), dev)
        except Exception:  # out of memory: the library reports MG_ERR_OOM
            return None

    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return alloc_t(alloc), free_t(free)


def mg_setup(n: int, order: int = 2, coarsening="redblack", coarse_op="galerkin", length: float = 1.0,
             allocator=None, **opts) -> Handle:
    """Build a hierarchy for the square [0, length]^2 with n cells per side.
    allocator=None: cudaMalloc; "torch": torch's CUDA caching allocator."""
    g = mg_grid(n, length)
    o = mg_default_options(**opts)
    keep = None
    if allocator == "torch":
        keep = _torch_allocator()
        o.dev_alloc, o.dev_free = keep
    elif allocator is not None:
        raise ValueError("allocator must be None or 'torch'")
    out = _vp()
    _check(_lib.mg_setup(ctypes.byref(g), order, COARSENING.get(coarsening, coarsening),
                         COARSE_OP.get(coarse_op, coarse_op), ctypes.byref(o), ctypes.byref(out)), "mg_setup")
    h = Handle(out.value)
    h._callbacks = keep  # the callbacks must outlive the handle
    return h


def mg_destroy(h: Handle):
    h.close()


def mg_cycle(h: Handle, u, f, stream=None) -> float:
    rr = ctypes.c_double()
    _check(_lib.mg_cycle(h.ptr, _ptr(u), _ptr(f), ctypes.byref(rr), _stream(stream)), "mg_cycle")
    return rr.value


def mg_solve(h: Handle, u, f, rtol: float = 1e-10, max_cycles: int = 50, stream=None,
             raise_not_converged: bool = True):
    """Returns (cycles, history list of relative residuals)."""
    hist = (ctypes.c_double * (max_cycles + 1))()
    cyc = ctypes.c_int()
    st = _lib.mg_solve(h.ptr, _ptr(u), _ptr(f), rtol, max_cycles, ctypes.byref(cyc), hist, _stream(stream))
    if st != MG_OK and not (st == MG_ERR_NOT_CONVERGED and not raise_not_converged):
        raise MGError(st, "mg_solve")
    return cyc.value, [hist[k] for k in range(cyc.value + 1)]


def _host_ptr(a, writable: bool) -> int:
    """Address of a C-contiguous float64 host array: numpy, or a CPU torch tensor."""
    if hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise ValueError("expected a contiguous float64 CPU tensor")
        return a.data_ptr()
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous float64 numpy array")
    if writable and not a.flags["WRITEABLE"]:
        raise ValueError("u must be writable")
    return a.ctypes.data


def mg_solve_host(h: Handle, u, f, rtol: float = 1e-10, max_cycles: int = 50, stream=None,
                  raise_not_converged: bool = True):
    """mg_solve on host arrays ((N+1) x (N+1) float64; pinned memory copies fastest):
    u is overwritten with the new iterate. Returns (cycles, history)."""
    hist = (ctypes.c_double * (max_cycles + 1))()
    cyc = ctypes.c_int()
    st = _lib.mg_solve_host(h.ptr, _host_ptr(u, True), _host_ptr(f, False), rtol, max_cycles,
                            ctypes.byref(cyc), hist, _stream(stream))
    if st != MG_OK and not (st == MG_ERR_NOT_CONVERGED and not raise_not_converged):
        raise MGError(st, "mg_solve_host")
    return cyc.value, [hist[k] for k in range(cyc.value + 1)]


def mg_num_levels(h: Handle) -> int:
    return _lib.mg_num_levels(h.ptr)


def mg_get_level_info(h: Handle, level: int) -> mg_level_info:
    info = mg_level_info()
    _check(_lib.mg_get_level_info(h.ptr, level, ctypes.byref(info)), "mg_get_level_info")
    return info


def mg_level_apply(h: Handle, level: int, u, out, stream=None):
    _check(_lib.mg_level_apply(h.ptr, level, _ptr(u), _ptr(out), _stream(stream)), "mg_level_apply")


def mg_level_residual(h: Handle, level: int, u, f, d, stream=None):
    _check(_lib.mg_level_residual(h.ptr, level, _ptr(u), _ptr(f), _ptr(d), _stream(stream)), "mg_level_residual")


def mg_level_smooth(h: Handle, level: int, u, f, sweeps: int = 1, stream=None):
    _check(_lib.mg_level_smooth(h.ptr, level, _ptr(u), _ptr(f), sweeps, _stream(stream)), "mg_level_smooth")


def mg_level_restrict(h: Handle, level: int, d_fine, f_coarse, stream=None):
    _check(_lib.mg_level_restrict(h.ptr, level, _ptr(d_fine), _ptr(f_coarse), _stream(stream)), "mg_level_restrict")


def mg_level_prolong_add(h: Handle, level: int, u_fine, v_coarse, stream=None):
    _check(_lib.mg_level_prolong_add(h.ptr, level, _ptr(u_fine), _ptr(v_coarse), _stream(stream)),
           "mg_level_prolong_add")


def level_array(h: Handle, level: int, device="cuda"):
    """A zeroed FP64 torch tensor in the storage layout of `level` (rows x pitch)."""
    import torch
    info = mg_get_level_info(h, level)
    return torch.zeros((info.rows, info.pitch), dtype=torch.float64, device=device)


def level_nodes(h: Handle, level: int):
    """(i, j, row, col) numpy index arrays of the level's unknowns (interior nodes, or
    nodes 0 <= i, j < n of a periodic level) in row-major (j, then i) order, with their
    storage row/column."""
    import numpy as np
    info = mg_get_level_info(h, level)
    n = info.n
    lo = 0 if info.periodic else 1
    jj, ii = np.meshgrid(np.arange(lo, n), np.arange(lo, n), indexing="ij")
    i, j = ii.ravel(), jj.ravel()
    if info.kind == 1:
        keep = (i + j) % 2 == 0
        i, j = i[keep], j[keep]
        col = i >> 1
    else:
        col = i
    return i, j, j, col


def mg_get_counters(h: Handle):
    """(kernel launches, cycles) since the last reset."""
    c = mg_counters()
    _check(_lib.mg_get_counters(h.ptr, ctypes.byref(c)), "mg_get_counters")
    return c.launches, c.cycles


def mg_reset_counters(h: Handle):
    _check(_lib.mg_reset_counters(h.ptr), "mg_reset_counters")


def mg_set_timing(h: Handle, enable=True):
    """True / 1: finest-level kernels; 2: every level (class k of level l is k + 5 l)."""
    _check(_lib.mg_set_timing(h.ptr, int(enable)), "mg_set_timing")


def mg_get_timing(h: Handle, kernel_class: int):
    """(total device ms, launches) of a finest-level kernel class since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(_lib.mg_get_timing(h.ptr, kernel_class, ctypes.byref(ms), ctypes.byref(n)), "mg_get_timing")
    return ms.value, n.value


_lib.mg_rel_residual_static.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.mg_rel_residual_static.restype = ctypes.c_int


def mg_rel_residual_static(h: Handle, u, f, rel_res_dev, stream=None):
    """Relative residual of the finest level into the device scalar `rel_res_dev`,
    without any device allocation (partial sums in the library's fixed device array)."""
    _check(_lib.mg_rel_residual_static(h.ptr, _ptr(u), _ptr(f), _ptr(rel_res_dev), _stream(stream)),
           "mg_rel_residual_static")


# ---- batched solves ---------------------------------------------------------
_lib.mg_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp)]


class mg_batch_options(ctypes.Structure):
    _fields_ = [("solo_min_n", ctypes.c_int), ("workers", ctypes.c_int)]


_lib.mg_batch_create_ex.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(mg_batch_options),
                                    ctypes.POINTER(_vp)]
_lib.mg_batch_solve.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_double, ctypes.c_int,
                                _ip, _dp, _vp]
_lib.mg_batch_destroy.argtypes = [_vp]
_lib.mg_batch_get_launches.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
_lib.mg_solve_batched.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int,
                                  ctypes.c_double, ctypes.c_int, _ip, _dp, _vp]
for _name in ("mg_batch_create", "mg_batch_create_ex", "mg_batch_solve", "mg_batch_destroy", "mg_batch_get_launches", "mg_solve_batched"):
    getattr(_lib, _name).restype = ctypes.c_int


class Batch:
    """Owns an mg_batch over a list of Handles (which must outlive it)."""

    def __init__(self, handles, solo_min_n: int = 0, workers: int = 0):
        self.handles = list(handles)
        arr = (_vp * len(self.handles))(*[h.ptr for h in self.handles])
        out = _vp()
        o = mg_batch_options(solo_min_n, workers)
        _check(_lib.mg_batch_create_ex(arr, len(self.handles), ctypes.byref(o), ctypes.byref(out)),
               "mg_batch_create_ex")
        self.ptr = out.value

    def close(self):
        if self.ptr:
            _lib.mg_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_batch_create(handles, solo_min_n: int = 0, workers: int = 0) -> Batch:
    """solo_min_n / workers: the hybrid schedule's options (0: the library defaults,
    solo_min_n above 16384: level-synchronous only)."""
    return Batch(handles, solo_min_n, workers)


def mg_batch_solve(b: Batch, us, fs, rtol: float = 1e-8, max_cycles: int = 50, stream=None,
                   raise_not_converged: bool = True):
    """Returns (cycles list, final relative residual list)."""
    n = len(b.handles)
    ua = (_vp * n)(*[_ptr(x) for x in us])
    fa = (_vp * n)(*[_ptr(x) for x in fs])
    cyc = (ctypes.c_int * n)()
    rr = (ctypes.c_double * n)()
    st = _lib.mg_batch_solve(b.ptr, ua, fa, rtol, max_cycles, cyc, rr, _stream(stream))
    if st != MG_OK and not (st == MG_ERR_NOT_CONVERGED and not raise_not_converged):
        raise MGError(st, "mg_batch_solve")
    return list(cyc), list(rr)


def mg_batch_destroy(b: Batch):
    b.close()


def mg_batch_get_launches(b: Batch) -> int:
    v = ctypes.c_int64()
    _check(_lib.mg_batch_get_launches(b.ptr, ctypes.byref(v)), "mg_batch_get_launches")
    return v.value


def mg_solve_batched(handles, us, fs, rtol: float = 1e-8, max_cycles: int = 50, stream=None):
    n = len(handles)
    ha = (_vp * n)(*[h.ptr for h in handles])
    ua = (_vp * n)(*[_ptr(x) for x in us])
    fa = (_vp * n)(*[_ptr(x) for x in fs])
    cyc = (ctypes.c_int * n)()
    rr = (ctypes.c_double * n)()
    _check(_lib.mg_solve_batched(ha, ua, fa, n, rtol, max_cycles, cyc, rr, _stream(stream)), "mg_solve_batched")
    return list(cyc), list(rr)
