"""The C-ABI library loads without a GPU and exports every function include/vd.h declares.

No compute call is made here (no GPU on this machine); the GPU tests exercise them.
"""

import ctypes
import os

import pytest

import paper_2403_06654_gb300 as vd


def _lib_or_skip():
    if not os.path.exists(vd.LIB_PATH):
        pytest.skip("libvd.so not built (run __graft_entry__.build())")
    return vd.lib()


def test_header_declares_the_boundary():
    names = vd.header_functions()
    for required in ("vd_grid_create", "vd_grid_destroy", "vd_density_set", "vd_density_bytes",
                     "vd_workspace_bytes", "vd_apply_op", "vd_apply_precond", "vd_solve", "vd_last_error",
                     "vd_divergence", "vd_gradient"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = _lib_or_skip()
    for name in vd.header_functions():
        assert hasattr(L, name), name


def test_binding_wraps_every_declared_function():
    missing = [n for n in vd.header_functions() if n not in vd._SIGS]
    assert not missing, missing


def test_host_side_argument_checks_without_gpu():
    L = _lib_or_skip()
    h = ctypes.c_void_p()
    nn = (ctypes.c_int * 3)(6, 1, 1)
    ll = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    # invalid sizes are rejected before any device call
    for bad in ((0, nn), (4, nn)):
        assert L.vd_grid_create(bad[0], bad[1], ll, ctypes.byref(h)) == vd.VD_ERR_INVALID_ARG
    odd = (ctypes.c_int * 3)(7, 1, 1)
    assert L.vd_grid_create(1, odd, ll, ctypes.byref(h)) == vd.VD_ERR_INVALID_ARG
    seven = (ctypes.c_int * 3)(14, 1, 1)   # 14 = 2 * 7: not a 2-3-5 size
    assert L.vd_grid_create(1, seven, ll, ctypes.byref(h)) == vd.VD_ERR_INVALID_ARG
    assert b"2, 3 and 5" in L.vd_last_error()
    assert L.vd_solve(None, 0, 0, None, None, None, None, None, None, 0, None) == vd.VD_ERR_INVALID_ARG
    assert L.vd_version().startswith(b"vdspectral")


def test_profiler_modes_checked_on_the_host():
    """Profile mode 0 off, 1 every launch, 2 spans; anything else is refused before any
    device call, and reading an unknown class is refused too."""
    L = _lib_or_skip()
    for bad in (-1, 3, 7):
        assert L.vd_profile_enable(bad) == vd.VD_ERR_INVALID_ARG
    assert b"profile mode" in L.vd_last_error()
    assert L.vd_profile_enable(0) == vd.VD_OK
    n = ctypes.c_longlong()
    ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    for bad in (-1, 10):
        assert L.vd_profile_read(bad, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by),
                                 ctypes.byref(fl)) == vd.VD_ERR_INVALID_ARG
    assert vd.PROFILE_SPAN_INNER_F32 == 9 and 9 not in vd.PROFILE_CLASSES


def test_pointer_marshalling_rejects_noncontiguous():
    """Every pointer of the C interface addresses a dense row-major array: strided tensors are refused."""
    import torch
    t = torch.zeros((4, 6), dtype=torch.float64).t()
    with pytest.raises(vd.VDError) as e:
        vd._ptr(t)
    assert e.value.status == vd.VD_ERR_INVALID_ARG
    c = t.contiguous()
    assert vd._ptr(c).value == c.data_ptr()


def test_make_request_checks_tensors():
    import torch
    n, L = (8, 6), (1.0, 1.0)
    good = torch.zeros((6, 8), dtype=torch.float64)
    # host tensors are refused (the server reads device memory)
    with pytest.raises(vd.VDError):
        vd.make_request(0, n, L, good, good, good)
    # wrong shape or dtype is refused before any device check matters
    with pytest.raises(vd.VDError):
        vd.make_request(0, n, L, good.t(), good, good)
    with pytest.raises(vd.VDError):
        vd.make_request(0, n, L, good.float(), good, good)


def test_batch_size_query_host_only():
    """vd_batch_bytes is a host computation: positive for supported grids, 0 for a length with
    a prime factor above 5 or an empty batch."""
    import math
    shapes = [(64, 48), (24, 20, 16)]
    arr = (vd.vd_batch_item * 2)()
    for i, n in enumerate(shapes):
        nd = len(n)
        arr[i].ndim = nd
        arr[i].n = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - nd)))
        arr[i].L = (ctypes.c_double * 3)(*([2 * math.pi] * 3))
        arr[i].rho = arr[i].b_vel = arr[i].x_vel = arr[i].b_pres = arr[i].x_pres = 1
    p = vd.vd_batch_params(vd.VD_SOLVER_GMRES, vd.VD_SOLVER_CG, 1e-10, 400, 20)
    both = vd.lib().vd_batch_bytes(arr, 2, ctypes.byref(p))
    one = vd.lib().vd_batch_bytes(arr, 1, ctypes.byref(p))
    assert both > one > 0
    arr[1].n = (ctypes.c_int * 3)(24, 20, 28)
    assert vd.lib().vd_batch_bytes(arr, 2, ctypes.byref(p)) == 0
    assert vd.lib().vd_batch_bytes(arr, 0, ctypes.byref(p)) == 0
