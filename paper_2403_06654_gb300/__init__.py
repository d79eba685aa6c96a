"""GB300 (sm_103a) variable-density spectral elliptic solver: Python binding of libvd.so.

The binding only marshals arguments: every step of an operator apply or a solve runs in
the CUDA kernels of ``libvd.so`` (declared in ``include/vd.h``).  PyTorch supplies device
memory (tensors passed as raw pointers) and the current CUDA stream.

Module-level functions carry the C names (``vd_grid_create``, ``vd_density_set``,
``vd_apply_op``, ``vd_apply_precond``, ``vd_solve``, ...).  ``Grid`` is a convenience
wrapper that allocates the workspaces with torch and calls them.

If the shared library is missing, every call raises ``VDError``: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libvd.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "vd.h")

VD_OK, VD_ERR_INVALID_ARG, VD_ERR_OOM, VD_ERR_CUDA = 0, 1, 2, 3
VD_ERR_NOT_CONVERGED, VD_ERR_BREAKDOWN, VD_ERR_DIVERGED, VD_ERR_NONFINITE, VD_ERR_NO_DENSITY = 4, 5, 6, 7, 8
VD_ERR_RHS_NOT_IN_RANGE, VD_ERR_TIMEOUT = 9, 10
STATUS_NAMES = {0: "converged", 1: "invalid_arg", 2: "oom", 3: "cuda", 4: "max_iter", 5: "breakdown",
                6: "diverged", 7: "nonfinite", 8: "no_density", 9: "rhs_not_in_range", 10: "timeout"}
STATUS_CODES = {v: k for k, v in STATUS_NAMES.items()}
VD_OP_PRESSURE, VD_OP_VELOCITY, VD_OP_KRHO = 0, 1, 2
VD_SOLVER_CG, VD_SOLVER_GMRES, VD_SOLVER_RMR = 0, 1, 2
VD_PREC_FP64, VD_PREC_MIXED, VD_PREC_MIXED_DD = 0, 1, 2
OPS = {"pressure": VD_OP_PRESSURE, "velocity": VD_OP_VELOCITY, "krho": VD_OP_KRHO}
SOLVERS = {"cg": VD_SOLVER_CG, "gmres": VD_SOLVER_GMRES, "rmr": VD_SOLVER_RMR}
PRECISIONS = {"fp64": VD_PREC_FP64, "mixed": VD_PREC_MIXED, "mixed_dd": VD_PREC_MIXED_DD}


class VDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class vd_op_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("inv_sc", ctypes.c_double)]


class vd_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_it", ctypes.c_int), ("restart", ctypes.c_int),
                ("use_x0", ctypes.c_int), ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("coef_pair", ctypes.c_int), ("range_tol", ctypes.c_double)]


class vd_flow_params(ctypes.Structure):
    _fields_ = [("Re", ctypes.c_double), ("Sc", ctypes.c_double), ("Fr", ctypes.c_double),
                ("gravity_axis", ctypes.c_int), ("vel_solver", ctypes.c_int), ("pres_solver", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_it", ctypes.c_int), ("restart", ctypes.c_int),
                ("precision", ctypes.c_int)]


class vd_step_info(ctypes.Structure):
    _fields_ = [("vel_iters", ctypes.c_int), ("pres_iters", ctypes.c_int), ("vel_status", ctypes.c_int),
                ("pres_status", ctypes.c_int), ("vel_relres", ctypes.c_double), ("pres_relres", ctypes.c_double)]


class vd_server_params(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int), ("hbm_budget", ctypes.c_size_t)]


class vd_request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_ulonglong), ("ndim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("L", ctypes.c_double * 3), ("rho", ctypes.c_void_p), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("solver", ctypes.c_int), ("tol", ctypes.c_double), ("max_it", ctypes.c_int),
                ("restart", ctypes.c_int), ("precision", ctypes.c_int)]


class vd_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_ulonglong), ("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("relres_true", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("x", ctypes.c_void_p)]


class vd_batch_item(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3),
                ("rho", ctypes.c_void_p), ("b_vel", ctypes.c_void_p), ("x_vel", ctypes.c_void_p),
                ("a", ctypes.c_double), ("inv_sc", ctypes.c_double),
                ("b_pres", ctypes.c_void_p), ("x_pres", ctypes.c_void_p)]


class vd_batch_params(ctypes.Structure):
    _fields_ = [("vel_solver", ctypes.c_int), ("pres_solver", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_it", ctypes.c_int), ("restart", ctypes.c_int), ("precision", ctypes.c_int)]


class vd_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("status", ctypes.c_int),
                ("relres", ctypes.c_double), ("relres_true", ctypes.c_double),
                ("hist", ctypes.POINTER(ctypes.c_double)), ("hist_cap", ctypes.c_int), ("hist_len", ctypes.c_int),
                ("rhs_removed", ctypes.c_double), ("coef_pair", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_SZ = ctypes.c_size_t
_I = ctypes.c_int

_SIGS = {
    "vd_last_error": (ctypes.c_char_p, []),
    "vd_version": (ctypes.c_char_p, []),
    "vd_grid_create": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_P)]),
    "vd_grid_destroy": (_I, [_P]),
    "vd_grid_points": (_SZ, [_P]),
    "vd_grid_modes": (_SZ, [_P]),
    "vd_density_bytes": (_SZ, [_P, _I]),
    "vd_density_set": (_I, [_P, _I, _P, _P, _SZ, _P]),
    "vd_workspace_bytes": (_SZ, [_P, _I, _I, ctypes.POINTER(vd_solve_params)]),
    "vd_apply_op": (_I, [_P, _I, ctypes.POINTER(vd_op_params), _P, _P, _P, _SZ, _P]),
    "vd_apply_precond": (_I, [_P, _I, ctypes.POINTER(vd_op_params), _P, _P, _P, _SZ, _P]),
    "vd_solve": (_I, [_P, _I, _I, ctypes.POINTER(vd_op_params), ctypes.POINTER(vd_solve_params), _P, _P,
                      ctypes.POINTER(vd_solve_info), _P, _SZ, _P]),
    "vd_transform_ws_bytes": (_SZ, [_P, _I]),
    "vd_fft_r2c": (_I, [_P, _I, _P, _P, _P, _SZ, _P]),
    "vd_fft_c2r": (_I, [_P, _I, _P, _P, _P, _SZ, _P]),
    "vd_divergence": (_I, [_P, _P, _P, _P, _SZ, _P]),
    "vd_gradient": (_I, [_P, _P, _P, _P, _SZ, _P]),
    "vd_autotune_bytes": (_SZ, [_P]),
    "vd_autotune": (_I, [_P, _I, _P, _SZ, _P]),
    "vd_autotune_table": (_I, [ctypes.POINTER(_I), _I]),
    "vd_autotune_set": (_I, [_I, _I, _I, _I, _I, _I]),
    "vd_batch_bytes": (_SZ, [ctypes.POINTER(vd_batch_item), _I, ctypes.POINTER(vd_batch_params)]),
    "vd_batch_create": (_I, [ctypes.POINTER(vd_batch_item), _I, ctypes.POINTER(vd_batch_params), _P, _SZ, _P,
                             ctypes.POINTER(_P)]),
    "vd_batch_run": (_I, [_P, _P]),
    "vd_batch_info": (_I, [_P, _I, ctypes.POINTER(vd_solve_info), ctypes.POINTER(vd_solve_info)]),
    "vd_batch_graph_nodes": (_SZ, [_P]),
    "vd_batch_destroy": (_I, [_P]),
    "vd_apply_pressure_noalloc": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double), _P, _P, _P, _P]),
    "vd_flow_bytes": (_SZ, [_P, ctypes.POINTER(vd_flow_params)]),
    "vd_flow_create": (_I, [_P, ctypes.POINTER(vd_flow_params), _P, _SZ, ctypes.POINTER(_P)]),
    "vd_flow_destroy": (_I, [_P]),
    "vd_flow_set_state": (_I, [_P, _P, _P, _P]),
    "vd_flow_get_state": (_I, [_P, _P, _P, _P, _P, _P]),
    "vd_flow_set_sources": (_I, [_P, _P, _P, _P]),
    "vd_flow_step": (_I, [_P, ctypes.c_double, ctypes.POINTER(vd_step_info), _P]),
    "vd_flow_snapshot_bytes": (_SZ, [_P]),
    "vd_flow_save": (_I, [_P, _P, _SZ, _P]),
    "vd_flow_load": (_I, [_P, _P, _SZ, _P]),
    "vd_server_create": (_I, [ctypes.POINTER(vd_server_params), ctypes.POINTER(_P)]),
    "vd_server_request_bytes": (_SZ, [ctypes.POINTER(vd_request)]),
    "vd_server_submit": (_I, [_P, ctypes.POINTER(vd_request), _SZ]),
    "vd_server_cancel": (_I, [_P, ctypes.c_ulonglong]),
    "vd_server_poll": (_I, [_P, ctypes.POINTER(vd_completion), _I]),
    "vd_server_fetch": (_I, [_P, ctypes.c_ulonglong, _P, _P]),
    "vd_server_release": (_I, [_P, ctypes.c_ulonglong]),
    "vd_server_drain": (_I, [_P]),
    "vd_server_stats": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "vd_server_destroy": (_I, [_P]),
    "vd_launch_count": (ctypes.c_longlong, []),
    "vd_alu_rate": (_I, [_I, ctypes.POINTER(ctypes.c_double), _P]),
    "vd_profile_enable": (_I, [_I]),
    "vd_profile_reset": (_I, []),
    "vd_profile_read": (_I, [_I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
}


def lib():
    """Load libvd.so (raises VDError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise VDError(VD_ERR_CUDA, f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def header_functions(path: str = HEADER) -> list:
    """Names of the functions declared in include/vd.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vd_[a-z0-9_]+)\s*\(", txt)))


def _check(st):
    if st != VD_OK:
        raise VDError(st, lib().vd_last_error().decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    # every pointer of the C interface addresses a dense row-major array
    if not t.is_contiguous():
        raise VDError(VD_ERR_INVALID_ARG, "tensor passed to the C interface must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------------------------------
# thin wrappers with the C names
# ------------------------------------------------------------------------------------------

def vd_grid_create(n, L):
    nd = len(n)
    nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - nd)))
    ll = (ctypes.c_double * 3)(*(list(L) + [1.0] * (3 - nd)))
    h = ctypes.c_void_p()
    _check(lib().vd_grid_create(nd, nn, ll, ctypes.byref(h)))
    return h


def vd_grid_destroy(h):
    _check(lib().vd_grid_destroy(h))


def vd_density_bytes(h, op):
    return int(lib().vd_density_bytes(h, op))


def vd_workspace_bytes(h, op, solver, params: vd_solve_params | None):
    return int(lib().vd_workspace_bytes(h, op, solver, ctypes.byref(params) if params is not None else None))


def vd_density_set(h, op, rho, ws, stream=None):
    _check(lib().vd_density_set(h, op, _ptr(rho), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def vd_apply_op(h, op, params, x, out, ws, stream=None):
    _check(lib().vd_apply_op(h, op, ctypes.byref(params) if params is not None else None, _ptr(x), _ptr(out),
                             _ptr(ws), ws.numel(), _stream(stream)))


def vd_apply_precond(h, op, params, x, out, ws, stream=None):
    _check(lib().vd_apply_precond(h, op, ctypes.byref(params) if params is not None else None, _ptr(x), _ptr(out),
                                  _ptr(ws), ws.numel(), _stream(stream)))


def vd_solve(h, op, solver, op_params, params, b, x, info, ws, stream=None):
    """Returns the raw status (not raised: non-convergence is a result, not an error)."""
    st = lib().vd_solve(h, op, solver, ctypes.byref(op_params) if op_params is not None else None,
                        ctypes.byref(params), _ptr(b), _ptr(x), ctypes.byref(info), _ptr(ws), ws.numel(),
                        _stream(stream))
    if st in (VD_ERR_INVALID_ARG, VD_ERR_OOM, VD_ERR_CUDA, VD_ERR_NO_DENSITY, VD_ERR_RHS_NOT_IN_RANGE, VD_ERR_TIMEOUT):
        _check(st)
    return st


def vd_transform_ws_bytes(h, prec):
    return int(lib().vd_transform_ws_bytes(h, prec))


def vd_fft_r2c(h, prec, x, out, ws, stream=None):
    _check(lib().vd_fft_r2c(h, prec, _ptr(x), _ptr(out), _ptr(ws), ws.numel() * ws.element_size(),
                            _stream(stream)))


def vd_fft_c2r(h, prec, x, out, ws, stream=None):
    _check(lib().vd_fft_c2r(h, prec, _ptr(x), _ptr(out), _ptr(ws), ws.numel() * ws.element_size(),
                            _stream(stream)))


def vd_alu_rate(kind, stream=None):
    """Measured flop/s of the GPU: kind 0 FP64 FMA, 1 FP32 FMA, 2 float-pair multiply-add."""
    v = ctypes.c_double()
    _check(lib().vd_alu_rate(kind, ctypes.byref(v), _stream(stream)))
    return v.value


def vd_divergence(h, u, out, ws, stream=None):
    _check(lib().vd_divergence(h, _ptr(u), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))


def vd_gradient(h, phi, out, ws, stream=None):
    _check(lib().vd_gradient(h, _ptr(phi), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))


def vd_apply_pressure_noalloc(n, L, rho, x, out, stream=None):
    """Pressure apply through the entry point that allocates no device memory: for callers
    that cannot allocate (a host framework's pool owns the device, fixed-footprint plugins,
    loops that must not synchronise through an allocation).  Only marshalling here."""
    nd = len(n)
    nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - nd)))
    ll = (ctypes.c_double * 3)(*(list(L) + [1.0] * (3 - nd)))
    _check(lib().vd_apply_pressure_noalloc(nd, nn, ll, _ptr(rho), _ptr(x), _ptr(out), _stream(stream)))


def vd_flow_bytes(h, params):
    return int(lib().vd_flow_bytes(h, ctypes.byref(params)))


def vd_flow_create(h, params, mem):
    f = ctypes.c_void_p()
    _check(lib().vd_flow_create(h, ctypes.byref(params), _ptr(mem), mem.numel(), ctypes.byref(f)))
    return f


def vd_flow_destroy(f):
    _check(lib().vd_flow_destroy(f))


def vd_flow_set_state(f, rho, u, stream=None):
    _check(lib().vd_flow_set_state(f, _ptr(rho), _ptr(u), _stream(stream)))


def vd_flow_get_state(f, rho=None, u=None, gradp=None, phi=None, stream=None):
    p = lambda t: _ptr(t) if t is not None else None  # noqa: E731
    _check(lib().vd_flow_get_state(f, p(rho), p(u), p(gradp), p(phi), _stream(stream)))


def vd_flow_set_sources(f, mass_source=None, force=None, stream=None):
    p = lambda t: _ptr(t) if t is not None else None  # noqa: E731
    _check(lib().vd_flow_set_sources(f, p(mass_source), p(force), _stream(stream)))


def vd_flow_step(f, dt, info, stream=None):
    """Returns the raw status (an unconverged solve is a result, not an error)."""
    st = lib().vd_flow_step(f, ctypes.c_double(dt), ctypes.byref(info), _stream(stream))
    if st in (VD_ERR_INVALID_ARG, VD_ERR_OOM, VD_ERR_CUDA, VD_ERR_NO_DENSITY):
        _check(st)
    return st


def vd_server_create(max_inflight=4, hbm_budget=0):
    h = ctypes.c_void_p()
    _check(lib().vd_server_create(ctypes.byref(vd_server_params(max_inflight, hbm_budget)), ctypes.byref(h)))
    return h


def vd_server_request_bytes(req):
    return int(lib().vd_server_request_bytes(ctypes.byref(req)))


def vd_server_submit(h, req, nbytes):
    _check(lib().vd_server_submit(h, ctypes.byref(req), nbytes))


def vd_server_cancel(h, rid):
    _check(lib().vd_server_cancel(h, rid))


def vd_server_poll(h, max_n=256):
    buf = (vd_completion * max_n)()
    k = lib().vd_server_poll(h, buf, max_n)
    return [buf[i] for i in range(k)]


def vd_server_fetch(h, rid, dst, stream=None):
    """Copy the server-owned solution of request rid into dst (device tensor) and free it."""
    _check(lib().vd_server_fetch(h, rid, _ptr(dst), _stream(stream)))


def vd_server_release(h, rid):
    _check(lib().vd_server_release(h, rid))


def vd_server_drain(h):
    _check(lib().vd_server_drain(h))


def vd_server_stats(h):
    a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    d, e = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().vd_server_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                                 ctypes.byref(e)))
    return {"submitted": a.value, "completed": b.value, "inflight": c.value, "reserved": d.value, "budget": e.value}


def vd_server_destroy(h):
    _check(lib().vd_server_destroy(h))


def make_request(rid, n, L, rho, b, x=None, solver="cg", tol=1e-10, max_it=500, restart=30, precision="mixed_dd"):
    """Build a vd_request from device tensors (marshalling only); x None: server-owned solution."""
    nd = len(n)
    r = vd_request()
    r.id = rid
    r.ndim = nd
    r.n = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - nd)))
    r.L = (ctypes.c_double * 3)(*(list(L) + [1.0] * (3 - nd)))
    import torch
    for name, t in (("rho", rho), ("b", b), ("x", x)):
        if t is None and name == "x":
            continue
        if t.dtype != torch.float64 or not t.is_cuda or tuple(t.shape) != tuple(reversed(n)):
            raise VDError(VD_ERR_INVALID_ARG, f"{name} must be a float64 CUDA tensor of shape {tuple(reversed(n))}")
    r.rho, r.b = _ptr(rho).value, _ptr(b).value
    r.x = _ptr(x).value if x is not None else None
    r.solver = SOLVERS[solver]
    r.tol = tol
    r.max_it = max_it
    r.restart = restart
    r.precision = PRECISIONS[precision]
    return r


def vd_launch_count():
    return int(lib().vd_launch_count())


def vd_profile_enable(on):
    """0 off, 1 (or True) every launch bracketed by events, 2 span mode (whole inner solves)."""
    _check(lib().vd_profile_enable(int(on)))


def vd_profile_reset():
    _check(lib().vd_profile_reset())


PROFILE_CLASSES = {0: "axis_f64", 1: "axis_f32", 2: "xpass_f64", 3: "xpass_f32", 5: "axis_dd", 6: "xpass_dd",
                   7: "vec_f32", 8: "vec_f64"}
PROFILE_SPAN_INNER_F32 = 9   # span mode: whole inner float solves


def vd_profile_read(cls):
    n = ctypes.c_longlong()
    ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().vd_profile_read(cls, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl)))
    return {"launches": n.value, "ms": ms.value, "alg_bytes": by.value, "alg_flops": fl.value}


# ------------------------------------------------------------------------------------------
# convenience object
# ------------------------------------------------------------------------------------------

class Grid:
    """A periodic grid with its density; fields are float64 CUDA tensors shaped (n2, n1, n0)
    (trailing axes dropped for 2D/1D), vector fields (ndim, ...)."""

    def __init__(self, n, L, device="cuda"):
        import torch
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.ndim = len(self.n)
        self.shape = tuple(reversed(self.n))
        self.device = torch.device(device)
        self.h = vd_grid_create(self.n, self.L)
        self._dens = None
        self._ws = {}
        self._op_set = None

    def close(self):
        if self.h:
            vd_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def modes(self):
        return int(lib().vd_grid_modes(self.h))

    def _field(self, t, ncomp=0, name="field"):
        """float64 contiguous device copy of t, checked against the grid shape; ncomp = 0 for
        a scalar field, else the number of components of a vector field (ncomp, *shape)."""
        import torch
        t = t.to(device=self.device, dtype=torch.float64).contiguous()
        want = ((ncomp,) if ncomp > 0 else ()) + self.shape
        if tuple(t.shape) != want:
            raise VDError(VD_ERR_INVALID_ARG, f"{name} has shape {tuple(t.shape)}, expected {want}")
        return t

    def _ncomp(self, op):
        return self.ndim if OPS[op] == VD_OP_VELOCITY else 0

    def _workspace(self, nbytes):
        import torch
        key = "ws"
        t = self._ws.get(key)
        if t is None or t.numel() < nbytes:
            t = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
            self._ws[key] = t
        return t

    def set_density(self, rho, op="pressure", stream=None):
        import torch
        opc = OPS[op]
        rho = self._field(rho, 0, "rho")
        nb = vd_density_bytes(self.h, opc)
        self._dens = torch.empty(nb, dtype=torch.uint8, device=self.device)
        vd_density_set(self.h, opc, rho, self._dens, stream)
        self._op_set = op

    def apply(self, op, x, a=0.0, inv_sc=1.0, stream=None):
        import torch
        opc = OPS[op]
        x = self._field(x, self._ncomp(op), "x")
        out = torch.empty_like(x)
        p = vd_solve_params(tol=0.0, max_it=1, restart=1, use_x0=0, precision=0, inner_tol=0.0, check_every=1)
        ws = self._workspace(vd_workspace_bytes(self.h, opc, VD_SOLVER_RMR, p))
        vd_apply_op(self.h, opc, vd_op_params(a, inv_sc) if opc == VD_OP_VELOCITY else None, x, out, ws, stream)
        return out

    def precond(self, op, x, a=0.0, stream=None):
        import torch
        opc = OPS[op]
        x = self._field(x, self._ncomp(op), "x")
        out = torch.empty_like(x)
        p = vd_solve_params(tol=0.0, max_it=1, restart=1, use_x0=0, precision=0, inner_tol=0.0, check_every=1)
        ws = self._workspace(vd_workspace_bytes(self.h, opc, VD_SOLVER_RMR, p))
        vd_apply_precond(self.h, opc, vd_op_params(a, 1.0) if opc == VD_OP_VELOCITY else None, x, out, ws, stream)
        return out

    def solve_params(self, tol=1e-10, max_it=500, restart=30, use_x0=False, precision="fp64", inner_tol=0.0,
                     check_every=1, coef_pair=0, range_tol=0.0):
        return vd_solve_params(tol=tol, max_it=max_it, restart=restart, use_x0=int(bool(use_x0)),
                               precision=PRECISIONS[precision], inner_tol=inner_tol, check_every=check_every,
                               coef_pair=int(coef_pair), range_tol=float(range_tol))

    def workspace_bytes(self, op, solver, **kw):
        return vd_workspace_bytes(self.h, OPS[op], SOLVERS[solver], self.solve_params(**kw))

    def solve(self, op, solver, b, x0=None, a=0.0, inv_sc=1.0, stream=None, hist_cap=0, out=None, **kw):
        """Solve A x = b; returns (x, info dict)."""
        import torch
        opc, sc = OPS[op], SOLVERS[solver]
        b = self._field(b, self._ncomp(op), "b")
        if out is None:
            out = torch.zeros_like(b)
        if x0 is not None:
            out.copy_(x0)
            kw["use_x0"] = True
        p = self.solve_params(**kw)
        ws = self._workspace(vd_workspace_bytes(self.h, opc, sc, p))
        info = vd_solve_info()
        hist = None
        if hist_cap > 0:
            hist = (ctypes.c_double * hist_cap)()
            info.hist = hist
            info.hist_cap = hist_cap
        st = vd_solve(self.h, opc, sc, vd_op_params(a, inv_sc) if opc == VD_OP_VELOCITY else None, p, b, out, info,
                      ws, stream)
        res = {"status": STATUS_NAMES.get(st, st), "iters": info.iters, "outer_iters": info.outer_iters,
               "relres": info.relres, "relres_true": info.relres_true, "rhs_removed": info.rhs_removed,
               "coef_pair": bool(info.coef_pair)}
        if hist is not None:
            res["hist"] = [hist[i] for i in range(info.hist_len)]
        return out, res

    def fft_r2c(self, x, precision="fp64", out=None, stream=None):
        """Half spectrum (complex tensor, shape (n2, n1, n0/2+1) with trailing axes dropped)
        of the real field x: unnormalised forward DFT; float32 fields with precision="mixed"."""
        import torch
        prec = PRECISIONS[precision]
        rdt, cdt = (torch.float32, torch.complex64) if prec == VD_PREC_MIXED else (torch.float64, torch.complex128)
        if x.dtype != rdt or not x.is_cuda or tuple(x.shape) != self.shape:
            raise VDError(VD_ERR_INVALID_ARG, f"x must be a {rdt} CUDA tensor of shape {self.shape}")
        hshape = self.shape[:-1] + (self.n[0] // 2 + 1,)
        if out is None:
            out = torch.empty(hshape, dtype=cdt, device=self.device)
        ws = self._workspace(vd_transform_ws_bytes(self.h, prec))
        vd_fft_r2c(self.h, prec, x, out, ws, stream)
        return out

    def fft_c2r(self, xh, precision="fp64", out=None, stream=None):
        """Real field of the half spectrum xh (inverse DFT divided by N)."""
        import torch
        prec = PRECISIONS[precision]
        rdt, cdt = (torch.float32, torch.complex64) if prec == VD_PREC_MIXED else (torch.float64, torch.complex128)
        hshape = self.shape[:-1] + (self.n[0] // 2 + 1,)
        if xh.dtype != cdt or not xh.is_cuda or tuple(xh.shape) != hshape:
            raise VDError(VD_ERR_INVALID_ARG, f"xh must be a {cdt} CUDA tensor of shape {hshape}")
        if out is None:
            out = torch.empty(self.shape, dtype=rdt, device=self.device)
        ws = self._workspace(vd_transform_ws_bytes(self.h, prec))
        vd_fft_c2r(self.h, prec, xh, out, ws, stream)
        return out

    def divergence(self, u, stream=None):
        import torch
        u = self._field(u, self.ndim, "u")
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        ws = self._workspace(16 * self.modes * 3 + 256)
        vd_divergence(self.h, u, out, ws, stream)
        return out

    def gradient(self, phi, stream=None):
        import torch
        phi = self._field(phi, 0, "phi")
        out = torch.empty((self.ndim,) + self.shape, dtype=torch.float64, device=self.device)
        ws = self._workspace(16 * self.modes * 3 + 256)
        vd_gradient(self.h, phi, out, ws, stream)
        return out


class Flow:
    """Semi-implicit variable-density flow on a Grid (state on the device)."""

    def __init__(self, grid: Grid, Re, Sc=1.0, Fr=1.0, gravity_axis=-1, vel_solver="rmr", pres_solver="gmres",
                 tol=1e-10, max_it=200, restart=30, precision="fp64"):
        import torch
        self.grid = grid
        self.params = vd_flow_params(Re=Re, Sc=Sc, Fr=Fr, gravity_axis=gravity_axis,
                                     vel_solver=SOLVERS[vel_solver], pres_solver=SOLVERS[pres_solver], tol=tol,
                                     max_it=max_it, restart=restart, precision=PRECISIONS[precision])
        nb = vd_flow_bytes(grid.h, self.params)
        if nb == 0:
            raise VDError(VD_ERR_INVALID_ARG, lib().vd_last_error().decode())
        self.mem = torch.empty(nb, dtype=torch.uint8, device=grid.device)
        self.h = vd_flow_create(grid.h, self.params, self.mem)

    def close(self):
        if self.h:
            vd_flow_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, rho, u, stream=None):
        g = self.grid
        vd_flow_set_state(self.h, g._field(rho, 0, "rho"), g._field(u, g.ndim, "u"), stream)

    def set_sources(self, mass_source=None, force=None, stream=None):
        """Mass source (scalar field) and body force (ndim fields) at the next step's mid-time;
        None removes a term."""
        g = self.grid
        ms = g._field(mass_source, 0, "mass_source") if mass_source is not None else None
        fo = g._field(force, g.ndim, "force") if force is not None else None
        vd_flow_set_sources(self.h, ms, fo, stream)
        self._sources = (ms, fo)   # keep the tensors alive until the copies have run

    def state(self, stream=None):
        import torch
        g = self.grid
        rho = torch.empty(g.shape, dtype=torch.float64, device=g.device)
        u = torch.empty((g.ndim,) + g.shape, dtype=torch.float64, device=g.device)
        gp = torch.empty_like(u)
        phi = torch.empty_like(rho)
        vd_flow_get_state(self.h, rho, u, gp, phi, stream)
        return rho, u, gp, phi

    def save(self, stream=None):
        """Snapshot of the complete step state in host memory (bytes)."""
        nb = int(lib().vd_flow_snapshot_bytes(self.h))
        buf = (ctypes.c_char * nb)()
        _check(lib().vd_flow_save(self.h, buf, nb, _stream(stream)))
        return bytes(buf)

    def load(self, snap, stream=None):
        """Restore a snapshot taken by save() on a grid of the same sizes."""
        buf = ctypes.create_string_buffer(snap, len(snap))
        _check(lib().vd_flow_load(self.h, buf, len(snap), _stream(stream)))

    def step(self, dt, stream=None):
        info = vd_step_info()
        st = vd_flow_step(self.h, dt, info, stream)
        return {"status": STATUS_NAMES.get(st, st), "vel_iters": info.vel_iters, "pres_iters": info.pres_iters,
                "vel_status": STATUS_NAMES.get(info.vel_status, info.vel_status),
                "pres_status": STATUS_NAMES.get(info.pres_status, info.pres_status),
                "vel_relres": info.vel_relres, "pres_relres": info.pres_relres}


class Batch:
    """Many uneven solves recorded into one CUDA graph (marshalling over vd_batch_*).

    items: list of dicts with keys n, L, rho and optionally b_vel/x_vel (with a, inv_sc)
    and b_pres/x_pres (device float64 tensors).  run() is a single graph launch."""

    def __init__(self, items, vel_solver="gmres", pres_solver="cg", tol=1e-10, max_it=500, restart=30,
                 precision="fp64", device=None, stream=None):
        import torch
        self._keep = []
        arr = (vd_batch_item * len(items))()
        for i, it in enumerate(items):
            n = tuple(it["n"])
            nd = len(n)
            arr[i].ndim = nd
            arr[i].n = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - nd)))
            arr[i].L = (ctypes.c_double * 3)(*(list(it["L"]) + [1.0] * (3 - nd)))
            for key in ("rho", "b_vel", "x_vel", "b_pres", "x_pres"):
                t = it.get(key)
                if t is not None:
                    want = ((nd,) if key.endswith("_vel") else ()) + tuple(reversed(n))
                    if t.dtype != torch.float64 or not t.is_cuda or tuple(t.shape) != want:
                        raise VDError(VD_ERR_INVALID_ARG, f"item {i}: {key} must be float64 CUDA of shape {want}")
                    setattr(arr[i], key, _ptr(t).value)
                    self._keep.append(t)
            arr[i].a = float(it.get("a", 0.0))
            arr[i].inv_sc = float(it.get("inv_sc", 1.0))
        self.params = vd_batch_params(SOLVERS[vel_solver], SOLVERS[pres_solver], tol, max_it, restart,
                                      PRECISIONS[precision])
        self.items = arr
        self.count = len(items)
        nb = int(lib().vd_batch_bytes(arr, len(items), ctypes.byref(self.params)))
        if nb == 0:
            raise VDError(VD_ERR_INVALID_ARG, "unsupported batch")
        self.mem = torch.empty(nb, dtype=torch.uint8, device=device or "cuda")
        self.h = ctypes.c_void_p()
        _check(lib().vd_batch_create(arr, len(items), ctypes.byref(self.params), _ptr(self.mem), nb,
                                     _stream(stream), ctypes.byref(self.h)))

    def run(self, stream=None):
        _check(lib().vd_batch_run(self.h, _stream(stream)))

    def info(self, i):
        v, p = vd_solve_info(), vd_solve_info()
        _check(lib().vd_batch_info(self.h, i, ctypes.byref(v), ctypes.byref(p)))
        conv = lambda x: {"status": STATUS_NAMES.get(x.status, x.status), "iters": x.iters,  # noqa: E731
                          "outer_iters": x.outer_iters, "relres": x.relres, "relres_true": x.relres_true}
        return conv(v), conv(p)

    def graph_nodes(self):
        return int(lib().vd_batch_graph_nodes(self.h))

    def close(self):
        if self.h:
            lib().vd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vd_autotune(grid, precisions=("fp64", "mixed", "mixed_dd"), stream=None):
    """Tune the transform launch shapes for this grid (Grid object) and the arithmetic types the
    precision modes use: fp64 -> double, mixed -> float, mixed_dd -> float + float-pair."""
    import torch
    bits = 0
    for p in precisions:
        bits |= {"fp64": 1, "mixed": 2, "mixed_dd": 6}[p]
    nb = int(lib().vd_autotune_bytes(grid.h))
    scratch = torch.empty(nb, dtype=torch.uint8, device=grid.device)
    _check(lib().vd_autotune(grid.h, bits, _ptr(scratch), nb, _stream(stream)))


def vd_autotune_table():
    """List of (kind, type, length, axis, dir, choice) entries of the launch-shape table."""
    n = lib().vd_autotune_table(None, 0)
    buf = (ctypes.c_int * (6 * max(n, 1)))()
    n = lib().vd_autotune_table(buf, n)
    return [tuple(buf[6 * i:6 * i + 6]) for i in range(n)]


def vd_autotune_set(kind, type_, n, axis, dir_, choice):
    _check(lib().vd_autotune_set(kind, type_, n, axis, dir_, choice))
