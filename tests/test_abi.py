"""CPU checks of the C ABI: the library builds, loads without a GPU and exports
every function include/nsmg.h declares; host-side argument validation."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nsmg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mg_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    b = __graft_entry__._load_builder()
    if not os.path.exists(b.LIB):
        b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mg_setup", "mg_cycle", "mg_solve", "mg_destroy", "mg_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults(lib):
    import paper_2008_03885_gb300 as mg
    for s in range(9):
        assert mg._lib.mg_status_string(s)
    o = mg.mg_default_options()
    assert o.omega == 1.0 and o.nu1 == 1 and o.nu2 == 1 and o.gamma == 1 and o.n_min == 2
    assert o.boundary == mg.MG_BOUNDARY_DIRICHLET and o.transfer_order == 2


def test_workspace_bytes_validates_without_gpu(lib):
    import paper_2008_03885_gb300 as mg
    assert mg.mg_workspace_bytes(64) > 0
    assert mg.mg_workspace_bytes(63) == 0  # not a power of two
    assert mg.mg_workspace_bytes(64, order=3) == 0 and mg.mg_workspace_bytes(64, order=6) > 0
    assert mg.mg_workspace_bytes(2) == 0
    # periodic hierarchies coarsen to one node: more (tiny) levels, about the same bytes
    bp, bd = mg.mg_workspace_bytes(64, boundary="periodic"), mg.mg_workspace_bytes(64)
    assert bd < bp < 1.2 * bd
    # FP64 red-black V: roughly 2 arrays on level 0 plus 4 per coarse level
    b = mg.mg_workspace_bytes(1024)
    assert 2 * 1025 * 1025 * 8 <= b <= 12 * 1025 * 1025 * 8
    # n_min = 16: fewer levels, plus the dense coarsest factor (2 x 225^2 doubles)
    b16 = mg.mg_workspace_bytes(1024, n_min=16)
    assert b16 - b >= 2 * 225 * 225 * 8 - 4 * 17 * 17 * 8 * 8


def test_setup_rejects_bad_arguments_before_touching_the_gpu(lib):
    import paper_2008_03885_gb300 as mg
    for kwargs in (dict(n=48), dict(n=64, order=8), dict(n=64, order=3)):
        with pytest.raises(mg.MGError) as e:
            mg.mg_setup(kwargs.pop("n"), **kwargs)
        assert e.value.status == mg.MG_ERR_INVALID
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, omega=2.5)
    assert e.value.status == mg.MG_ERR_INVALID
    # n_min: a power of two from 2 to N / 2; above 2 (several coarsest unknowns, the
    # dense solve) Dirichlet only; at least two levels
    for kwargs, status in ((dict(n_min=3), mg.MG_ERR_INVALID), (dict(n_min=0), mg.MG_ERR_INVALID),
                           (dict(n_min=64), mg.MG_ERR_UNSUPPORTED), (dict(max_levels=-1), mg.MG_ERR_INVALID),
                           (dict(max_levels=1), mg.MG_ERR_UNSUPPORTED),
                           (dict(n_min=8, boundary="periodic"), mg.MG_ERR_UNSUPPORTED),
                           (dict(max_levels=3, boundary="periodic"), mg.MG_ERR_UNSUPPORTED)):
        with pytest.raises(mg.MGError) as e:
            mg.mg_setup(64, **kwargs)
        assert e.value.status == status, kwargs
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, length=-1.0)
    assert e.value.status == mg.MG_ERR_INVALID
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, length=float("inf"))
    assert e.value.status == mg.MG_ERR_INVALID
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, boundary=2)
    assert e.value.status == mg.MG_ERR_INVALID
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, boundary="periodic", sweep_kernel=2)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, 4, "standard", transfer_order=3)
    assert e.value.status == mg.MG_ERR_INVALID
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, 4, "redblack", transfer_order=4)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED
    with pytest.raises(mg.MGError) as e:
        mg.mg_setup(64, 4, "standard", 6)
    assert e.value.status == mg.MG_ERR_INVALID


def test_batch_arguments_are_checked_before_the_gpu(lib):
    """The batch entry points validate their arguments on the host: an empty list, a
    NULL handle and out-of-range options are MG_ERR_INVALID without a device; the
    options struct is two C ints."""
    import paper_2008_03885_gb300 as mg
    assert ctypes.sizeof(mg.mg_batch_options) == 2 * ctypes.sizeof(ctypes.c_int)
    with pytest.raises(mg.MGError) as e:
        mg.mg_batch_create([])
    assert e.value.status == mg.MG_ERR_INVALID
    none = (ctypes.c_void_p * 1)(None)
    out = ctypes.c_void_p()
    for solo_min_n, workers in ((0, 0), (-1, 0), (0, -1), (0, 65)):
        o = mg.mg_batch_options(solo_min_n, workers)
        assert lib.mg_batch_create_ex(none, 1, ctypes.byref(o), ctypes.byref(out)) == mg.MG_ERR_INVALID
        assert out.value is None
    assert lib.mg_batch_destroy(None) == mg.MG_OK
