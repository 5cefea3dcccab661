"""ctypes binding of libgfc (include/gfc.h): argument marshalling only.

Every evaluation runs in the library's CUDA kernels. PyTorch provides device
memory and streams. If the shared library cannot be built or loaded, every
call raises; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

from . import build as _build

GFC_OK, GFC_EINVAL, GFC_ENOMEM, GFC_EBUDGET, GFC_ECUDA = 0, -1, -2, -3, -4
GFC_ETIMEOUT, GFC_ECANCELED, GFC_EBUSY, GFC_ENOTFOUND = -5, -6, -7, -8
GFC_PROP_SCALAR, GFC_PROP_CPAIR, GFC_PROP_DRESSED = 0, 1, 2
GFC_FP64, GFC_MIXED, GFC_F32X2 = 0, 1, 2
_PRECISION = {"fp64": GFC_FP64, "mixed": GFC_MIXED, "f32x2": GFC_F32X2}
ANGULAR_RULES = {"gl": 0, "tanh-sinh": 1, "chebyshev1": 2, "chebyshev2": 3, "exact": 4}
RADIAL_RULES = {"mapped": 0, "clustered": 1}


class GfcError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class _Prop(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("m2", ctypes.c_double),
                ("mk2_re", ctypes.c_double), ("mk2_im", ctypes.c_double),
                ("mq2_re", ctypes.c_double), ("mq2_im", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("mu2", ctypes.c_double),
                ("n_radial", ctypes.c_int), ("n_angular", ctypes.c_int),
                ("radial_scale", ctypes.c_double), ("detour_radius", ctypes.c_double),
                ("precision", ctypes.c_int), ("cut_band", ctypes.c_double),
                ("pinch_angle", ctypes.c_double), ("mixed_rtol", ctypes.c_double),
                ("mixed_fallback", ctypes.c_int), ("angular_rule", ctypes.c_int),
                ("radial_rule", ctypes.c_int)]


class _Grid(ctypes.Structure):
    _fields_ = [("re0", ctypes.c_double), ("re1", ctypes.c_double),
                ("im0", ctypes.c_double), ("im1", ctypes.c_double),
                ("m", ctypes.c_int), ("n", ctypes.c_int)]


class _EvalStats(ctypes.Structure):
    _fields_ = [("points", ctypes.c_int64), ("points_fp64", ctypes.c_int64),
                ("node_evals", ctypes.c_int64), ("kernel_launches", ctypes.c_int),
                ("pairs_evaluated", ctypes.c_int64), ("node_evals_fallback", ctypes.c_int64),
                ("pairs_fallback", ctypes.c_int64), ("pairs_full_table", ctypes.c_int64),
                ("pairs_full_table_fallback", ctypes.c_int64), ("points_partial", ctypes.c_int64),
                ("node_evals_list64", ctypes.c_int64), ("pairs_list64", ctypes.c_int64),
                ("pairs_full_table_list64", ctypes.c_int64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("canceled", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("points_per_s", ctypes.c_double), ("points_done", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_budget", ctypes.c_size_t),
                ("launches", ctypes.c_int64), ("queued", ctypes.c_int), ("active", ctypes.c_int)]


class _PipePeaks(ctypes.Structure):
    _fields_ = [("dfma_per_s", ctypes.c_double), ("dmul_per_s", ctypes.c_double),
                ("dadd_per_s", ctypes.c_double), ("ffma_per_s", ctypes.c_double),
                ("rcp32_per_s", ctypes.c_double), ("sm_count", ctypes.c_int),
                ("dfma_mhz", ctypes.c_double), ("ffma_mhz", ctypes.c_double),
                ("fp64_mix_per_s", ctypes.c_double)]


class _RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("state", ctypes.c_int),
                ("points", ctypes.c_int64), ("points_routed", ctypes.c_int64),
                ("queue_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("launches", ctypes.c_int64), ("bytes", ctypes.c_size_t)]


# every symbol of include/gfc.h with (argtypes, restype)
_P = ctypes.c_void_p
_SIGS = {
    "gfc_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "gfc_last_error": ([], ctypes.c_char_p),
    "gfc_version": ([ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "gfc_params_default": ([ctypes.POINTER(_Params)], ctypes.c_int),
    "gfc_eval_points": ([ctypes.POINTER(_Prop), ctypes.POINTER(_Params), _P, ctypes.c_int64, _P,
                         _P], ctypes.c_int),
    "gfc_eval_points_cond": ([ctypes.POINTER(_Prop), ctypes.POINTER(_Params), _P, ctypes.c_int64,
                              _P, _P, _P], ctypes.c_int),
    "gfc_eval_grid": ([ctypes.POINTER(_Prop), ctypes.POINTER(_Params), ctypes.POINTER(_Grid), _P,
                       _P], ctypes.c_int),
    "gfc_eval_points_noalloc": ([ctypes.POINTER(_Prop), ctypes.POINTER(_Params), _P,
                                 ctypes.c_int64, _P, _P], ctypes.c_int),
    "gfc_grid_points": ([ctypes.POINTER(_Grid), _P, _P], ctypes.c_int),
    "gfc_eval_points_host": ([ctypes.POINTER(_Prop), ctypes.POINTER(_Params), _P, ctypes.c_int64,
                              _P, _P], ctypes.c_int),
    "gfc_last_stats": ([ctypes.POINTER(_EvalStats)], ctypes.c_int),
    "gfc_release": ([], ctypes.c_int),
    "gfc_server_create": ([ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_P)],
                          ctypes.c_int),
    "gfc_server_submit": ([_P, ctypes.POINTER(_Prop), ctypes.POINTER(_Params),
                           ctypes.POINTER(_Grid), _P, ctypes.POINTER(ctypes.c_uint64)],
                          ctypes.c_int),
    "gfc_server_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "gfc_server_wait": ([_P, ctypes.c_uint64, ctypes.c_int], ctypes.c_int),
    "gfc_server_cancel": ([_P, ctypes.c_uint64], ctypes.c_int),
    "gfc_server_stats": ([_P, ctypes.POINTER(_ServerStats)], ctypes.c_int),
    "gfc_server_request_info": ([_P, ctypes.c_uint64, ctypes.POINTER(_RequestInfo)], ctypes.c_int),
    "gfc_server_destroy": ([_P], ctypes.c_int),
    "gfc_server_load": ([_P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gfc_router_create": ([ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_size_t, ctypes.c_int,
                           ctypes.POINTER(_P)], ctypes.c_int),
    "gfc_router_submit": ([_P, ctypes.POINTER(_Prop), ctypes.POINTER(_Params),
                           ctypes.POINTER(_Grid), _P, ctypes.POINTER(ctypes.c_uint64)],
                          ctypes.c_int),
    "gfc_router_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "gfc_router_wait": ([_P, ctypes.c_uint64, ctypes.c_int], ctypes.c_int),
    "gfc_router_cancel": ([_P, ctypes.c_uint64], ctypes.c_int),
    "gfc_router_server": ([_P, ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
    "gfc_router_server_of": ([_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "gfc_router_destroy": ([_P], ctypes.c_int),
    "gfc_angular_map": ([ctypes.POINTER(_Prop), ctypes.POINTER(_Params), ctypes.c_double,
                         ctypes.c_double, _P, ctypes.c_int64, _P, _P], ctypes.c_int),
    "gfc_region_map": ([ctypes.POINTER(_Prop), _P, ctypes.c_int64, _P, _P], ctypes.c_int),
    "gfc_test_fail_allocations": ([ctypes.c_int], ctypes.c_int),
    "gfc_test_fail_launches": ([ctypes.c_int], ctypes.c_int),
    "gfc_measure_pipe_peaks": ([ctypes.POINTER(_PipePeaks), ctypes.c_double, _P], ctypes.c_int),
    "gfc_test_full_angular_rule": ([ctypes.c_int], ctypes.c_int),
    "gfc_test_angular_rules": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int), _P, ctypes.c_int, _P, _P,
                                ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads libgfc.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            lib = ctypes.CDLL(path)
            for name, (argt, rest) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = argt
                fn.restype = rest
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != GFC_OK:
        lib = load_library()
        detail = lib.gfc_last_error().decode() or lib.gfc_strerror(status).decode()
        raise GfcError(status, where, detail)


# --------------------------------------------------------------------------
# argument types
# --------------------------------------------------------------------------

def make_prop(spec) -> _Prop:
    """``spec``: {'kind': 'scalar', 'm2': ...} | {'kind': 'cpair', 'mk2': c, 'mq2': c}
    | {'kind': 'dressed', 'a': .., 'b': .., 'c': ..}"""
    if isinstance(spec, _Prop):
        return spec
    p = _Prop()
    k = spec["kind"]
    if k == "scalar":
        p.kind, p.m2 = GFC_PROP_SCALAR, float(spec["m2"])
    elif k == "cpair":
        mk2, mq2 = complex(spec["mk2"]), complex(spec["mq2"])
        p.kind = GFC_PROP_CPAIR
        p.mk2_re, p.mk2_im, p.mq2_re, p.mq2_im = mk2.real, mk2.imag, mq2.real, mq2.imag
    elif k == "dressed":
        p.kind = GFC_PROP_DRESSED
        p.a, p.b, p.c = float(spec["a"]), float(spec["b"]), float(spec["c"])
    else:
        raise ValueError(f"unknown propagator kind {k!r}")
    return p


def make_params(spec=None, **kw) -> _Params:
    """Defaults of gfc_params_default, overridden by ``spec``/keywords;
    ``precision`` and ``mixed_fallback`` may be 'fp64', 'mixed' or 'f32x2',
    ``angular_rule`` 'gl', 'tanh-sinh', 'chebyshev1', 'chebyshev2' or 'exact',
    ``radial_rule`` 'mapped' or 'clustered'."""
    if isinstance(spec, _Params) and not kw:
        return spec
    lib = load_library()
    q = _Params()
    _check(lib.gfc_params_default(ctypes.byref(q)), "gfc_params_default")
    d = dict(spec or {})
    d.update(kw)
    for k, v in d.items():
        if k in ("precision", "mixed_fallback"):
            v = _PRECISION.get(v, v)
        if k == "angular_rule":
            v = ANGULAR_RULES.get(v, v)
        if k == "radial_rule":
            v = RADIAL_RULES.get(v, v)
        if not hasattr(q, k):
            raise ValueError(f"unknown parameter {k!r}")
        setattr(q, k, type(getattr(q, k))(v))
    return q


def make_grid(re0, re1, im0, im1, m, n) -> _Grid:
    return _Grid(float(re0), float(re1), float(im0), float(im1), int(m), int(n))


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------
# one-shot evaluation
# --------------------------------------------------------------------------

def eval_points(prop, params, x, out=None, stream=None):
    """G at the complex128 CUDA tensor ``x`` (any shape); returns a complex128
    tensor of the same shape, enqueued on ``stream`` (default: current)."""
    import torch
    lib = load_library()
    if x.dtype != torch.complex128 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous complex128 CUDA tensor")
    G = out if out is not None else torch.empty_like(x)
    _check(lib.gfc_eval_points(ctypes.byref(make_prop(prop)), ctypes.byref(make_params(params)),
                               ctypes.c_void_p(x.data_ptr()), x.numel(),
                               ctypes.c_void_p(G.data_ptr()), _stream_ptr(stream)),
           "gfc_eval_points")
    return G


def eval_points_cond(prop, params, x, out=None, cond=None, stream=None):
    """As eval_points, also returning the per-point magnitude scale
    K_D sum_k M_k (float64 CUDA tensor) of gfc_eval_points_cond."""
    import torch
    lib = load_library()
    if x.dtype != torch.complex128 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous complex128 CUDA tensor")
    G = out if out is not None else torch.empty_like(x)
    c = cond if cond is not None else torch.empty(x.shape, dtype=torch.float64, device=x.device)
    _check(lib.gfc_eval_points_cond(ctypes.byref(make_prop(prop)),
                                    ctypes.byref(make_params(params)),
                                    ctypes.c_void_p(x.data_ptr()), x.numel(),
                                    ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                    _stream_ptr(stream)),
           "gfc_eval_points_cond")
    return G, c


def eval_grid(prop, params, grid, out=None, stream=None, device=None):
    """G on the cell-centred grid as an (m, n) complex128 CUDA tensor."""
    import torch
    lib = load_library()
    g = grid if isinstance(grid, _Grid) else make_grid(*grid)
    G = out if out is not None else torch.empty((g.m, g.n), dtype=torch.complex128,
                                                device=device or "cuda")
    _check(lib.gfc_eval_grid(ctypes.byref(make_prop(prop)), ctypes.byref(make_params(params)),
                             ctypes.byref(g), ctypes.c_void_p(G.data_ptr()), _stream_ptr(stream)),
           "gfc_eval_grid")
    return G


def grid_points(grid, stream=None, device=None):
    """Kernel 1 alone: the (m, n) grid of x as a complex128 CUDA tensor."""
    import torch
    lib = load_library()
    g = grid if isinstance(grid, _Grid) else make_grid(*grid)
    x = torch.empty((g.m, g.n), dtype=torch.complex128, device=device or "cuda")
    _check(lib.gfc_grid_points(ctypes.byref(g), ctypes.c_void_p(x.data_ptr()), _stream_ptr(stream)),
           "gfc_grid_points")
    return x


def eval_points_host(prop, params, x_host, G_host=None, stream=None):
    """End-to-end call on host arrays (numpy complex128 or pinned CPU tensors):
    copy in, evaluate, copy out, wait."""
    import numpy as np
    lib = load_library()
    if isinstance(x_host, np.ndarray):
        x_host = np.ascontiguousarray(x_host, dtype=np.complex128)
        G = G_host if G_host is not None else np.empty_like(x_host)
        xp, gp, n = x_host.ctypes.data, G.ctypes.data, x_host.size
    else:
        G = G_host if G_host is not None else x_host.new_empty(x_host.shape)
        xp, gp, n = x_host.data_ptr(), G.data_ptr(), x_host.numel()
    _check(lib.gfc_eval_points_host(ctypes.byref(make_prop(prop)),
                                    ctypes.byref(make_params(params)), ctypes.c_void_p(xp), n,
                                    ctypes.c_void_p(gp), _stream_ptr(stream)),
           "gfc_eval_points_host")
    return G


@dataclass
class EvalStats:
    points: int
    points_fp64: int
    node_evals: int
    kernel_launches: int
    pairs_evaluated: int
    node_evals_fallback: int = 0
    pairs_fallback: int = 0
    pairs_full_table: int = 0
    pairs_full_table_fallback: int = 0
    points_partial: int = 0
    node_evals_list64: int = 0
    pairs_list64: int = 0
    pairs_full_table_list64: int = 0


def last_stats() -> EvalStats:
    lib = load_library()
    s = _EvalStats()
    _check(lib.gfc_last_stats(ctypes.byref(s)), "gfc_last_stats")
    return EvalStats(*(getattr(s, k) for k, _ in _EvalStats._fields_))


def version():
    lib = load_library()
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib.gfc_version(ctypes.byref(a), ctypes.byref(b)), "gfc_version")
    return a.value, b.value


def release():
    _check(load_library().gfc_release(), "gfc_release")


def measure_pipe_peaks(seconds: float = 0.2, stream=None) -> dict:
    """Measured throughput of the FP64 FMA, FP32 FMA and binary32 reciprocal
    pipes of the current device (gfc_measure_pipe_peaks), thread ops/s."""
    p = _PipePeaks()
    _check(load_library().gfc_measure_pipe_peaks(ctypes.byref(p), float(seconds), _stream_ptr(stream)),
           "gfc_measure_pipe_peaks")
    return {"dfma_per_s": p.dfma_per_s, "dmul_per_s": p.dmul_per_s, "dadd_per_s": p.dadd_per_s,
            "ffma_per_s": p.ffma_per_s, "rcp32_per_s": p.rcp32_per_s, "sm_count": p.sm_count,
            "dfma_mhz": p.dfma_mhz, "ffma_mhz": p.ffma_mhz, "fp64_mix_per_s": p.fp64_mix_per_s}


# --------------------------------------------------------------------------
# serving
# --------------------------------------------------------------------------

@dataclass
class ServerStats:
    submitted: int
    completed: int
    rejected: int
    canceled: int
    p50_ms: float
    p99_ms: float
    points_per_s: float
    points_done: int
    bytes_in_use: int
    bytes_budget: int
    launches: int
    queued: int
    active: int


class Server:
    """Continuous-batching server on one device (gfc_server_*)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 40 << 30, max_slots: int = 64):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.gfc_server_create(device, hbm_budget_bytes, max_slots, ctypes.byref(h)),
               "gfc_server_create")
        self._h = h
        self._keep = {}   # ticket -> host buffer kept alive until completion

    def submit(self, prop, params, grid, out=None):
        """Queues a grid request; returns (ticket, output array). ``out`` may be
        a numpy array (host output, the default) or a complex128 CUDA tensor on
        the server's device (written in place by the kernels)."""
        import numpy as np
        g = grid if isinstance(grid, _Grid) else make_grid(*grid)
        G = out if out is not None else np.empty((g.m, g.n), dtype=np.complex128)
        ptr = G.ctypes.data if isinstance(G, np.ndarray) else G.data_ptr()
        t = ctypes.c_uint64()
        _check(self._lib.gfc_server_submit(self._h, ctypes.byref(make_prop(prop)),
                                           ctypes.byref(make_params(params)), ctypes.byref(g),
                                           ctypes.c_void_p(ptr), ctypes.byref(t)),
               "gfc_server_submit")
        self._keep[t.value] = G
        return t.value, G

    def poll(self, ticket):
        done, st = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.gfc_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(st)),
               "gfc_server_poll")
        return bool(done.value), st.value

    def wait(self, ticket, timeout_ms: int = -1) -> int:
        """Returns the request's status (GFC_ETIMEOUT if still running)."""
        return self._lib.gfc_server_wait(self._h, ticket, int(timeout_ms))

    def cancel(self, ticket) -> int:
        return self._lib.gfc_server_cancel(self._h, ticket)

    def stats(self) -> ServerStats:
        s = _ServerStats()
        _check(self._lib.gfc_server_stats(self._h, ctypes.byref(s)), "gfc_server_stats")
        return ServerStats(s.submitted, s.completed, s.rejected, s.canceled, s.p50_ms, s.p99_ms,
                           s.points_per_s, s.points_done, s.bytes_in_use, s.bytes_budget,
                           s.launches, s.queued, s.active)

    def request_info(self, ticket) -> dict:
        """One request's record (gfc_server_request_info) as a dict."""
        r = _RequestInfo()
        _check(self._lib.gfc_server_request_info(self._h, ticket, ctypes.byref(r)),
               "gfc_server_request_info")
        return {k: getattr(r, k) for k, _ in _RequestInfo._fields_}

    def load(self) -> float:
        """Estimated work not yet launched (gfc_server_load)."""
        w = ctypes.c_double()
        _check(self._lib.gfc_server_load(self._h, ctypes.byref(w)), "gfc_server_load")
        return w.value

    def close(self):
        if self._h:
            _check(self._lib.gfc_server_destroy(self._h), "gfc_server_destroy")
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _RouterServer(Server):
    """A server owned by a router (destroyed with it)."""

    def __init__(self, lib, handle):
        self._lib = lib
        self._h = handle
        self._keep = {}

    def close(self):
        self._h = None


class Router:
    """One server per listed device, each request to the least-loaded one
    (gfc_router_*)."""

    def __init__(self, devices, hbm_budget_bytes: int = 40 << 30, max_slots: int = 64):
        self._lib = load_library()
        devs = (ctypes.c_int * len(devices))(*devices)
        h = ctypes.c_void_p()
        _check(self._lib.gfc_router_create(devs, len(devices), hbm_budget_bytes, max_slots,
                                           ctypes.byref(h)), "gfc_router_create")
        self._h = h
        self._keep = {}
        self.servers = []
        for i in range(len(devices)):
            sh = ctypes.c_void_p()
            _check(self._lib.gfc_router_server(self._h, i, ctypes.byref(sh)), "gfc_router_server")
            self.servers.append(_RouterServer(self._lib, sh))

    def submit(self, prop, params, grid, out=None):
        """As Server.submit, on the least-loaded server; returns (ticket, output)."""
        import numpy as np
        g = grid if isinstance(grid, _Grid) else make_grid(*grid)
        G = out if out is not None else np.empty((g.m, g.n), dtype=np.complex128)
        ptr = G.ctypes.data if isinstance(G, np.ndarray) else G.data_ptr()
        t = ctypes.c_uint64()
        _check(self._lib.gfc_router_submit(self._h, ctypes.byref(make_prop(prop)),
                                           ctypes.byref(make_params(params)), ctypes.byref(g),
                                           ctypes.c_void_p(ptr), ctypes.byref(t)),
               "gfc_router_submit")
        self._keep[t.value] = G
        return t.value, G

    def wait(self, ticket, timeout_ms: int = -1) -> int:
        return self._lib.gfc_router_wait(self._h, ticket, int(timeout_ms))

    def poll(self, ticket):
        done, st = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.gfc_router_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(st)),
               "gfc_router_poll")
        return bool(done.value), st.value

    def cancel(self, ticket) -> int:
        return self._lib.gfc_router_cancel(self._h, ticket)

    def server_of(self, ticket):
        """(server index, server ticket) of a router ticket."""
        i, t = ctypes.c_int(), ctypes.c_uint64()
        _check(self._lib.gfc_router_server_of(self._h, ticket, ctypes.byref(i), ctypes.byref(t)),
               "gfc_router_server_of")
        return i.value, t.value

    def close(self):
        if self._h:
            _check(self._lib.gfc_router_destroy(self._h), "gfc_router_destroy")
            self._h = None
            self._keep.clear()
            self.servers = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def angular_map(prop, params, x, y, out=None, stream=None):
    """B(x, y) of gfc_angular_map at one complex x for the complex128 CUDA
    tensor y (Sect. 5, Fig. 1)."""
    import torch
    lib = load_library()
    y = y.contiguous()
    B = out if out is not None else torch.empty_like(y)
    _check(lib.gfc_angular_map(ctypes.byref(make_prop(prop)), ctypes.byref(make_params(params)),
                               float(complex(x).real), float(complex(x).imag),
                               ctypes.c_void_p(y.data_ptr()), y.numel(),
                               ctypes.c_void_p(B.data_ptr()), _stream_ptr(stream)),
           "gfc_angular_map")
    return B


def region_map(prop, x, out=None, stream=None):
    """int32 CUDA tensor: 1 where x lies in region 1 of Fig. 2 (gfc_region_map)."""
    import torch
    lib = load_library()
    x = x.contiguous()
    F = out if out is not None else torch.empty(x.shape, dtype=torch.int32, device=x.device)
    _check(lib.gfc_region_map(ctypes.byref(make_prop(prop)), ctypes.c_void_p(x.data_ptr()),
                              x.numel(), ctypes.c_void_p(F.data_ptr()), _stream_ptr(stream)),
           "gfc_region_map")
    return F


def test_fail_allocations(n: int):
    """Test hook: the next ``n`` device allocations of the library fail
    (gfc_test_fail_allocations); 0 clears it."""
    _check(load_library().gfc_test_fail_allocations(int(n)), "gfc_test_fail_allocations")


def test_fail_launches(n: int):
    """Test hook: the next ``n`` evaluation-kernel launches of the library
    report an error without launching (gfc_test_fail_launches); 0 clears it."""
    _check(load_library().gfc_test_fail_launches(int(n)), "gfc_test_fail_launches")


def test_full_angular_rule(on: bool):
    """Test switch: the full angular table instead of the compressed rules for
    every later evaluation (gfc_test_full_angular_rule)."""
    _check(load_library().gfc_test_full_angular_rule(1 if on else 0), "gfc_test_full_angular_rule")


def angular_rules(n_angular: int, dim: int = 4, angular_rule="gl"):
    """Test hook (host only): the angular pair table and the compressed rules
    the kernels use (gfc_test_angular_rules). Returns (pairs, rules, rho_min):
    pairs an (np, 3) array of (t, e, g), rules a list of (n, 3) arrays of
    (tau, gamma, gamma tau), rho_min the Bernstein-parameter threshold of each
    rule (binary64 and double-float)."""
    import numpy as np
    lib = load_library()
    rule = ANGULAR_RULES[angular_rule] if isinstance(angular_rule, str) else int(angular_rule)
    pairs = np.zeros(3 * 512, dtype=np.float64)
    rules = np.zeros(3 * 4096, dtype=np.float64)
    rule_n = np.zeros(32, dtype=np.int32)
    rho_min = np.zeros(32, dtype=np.float32)
    npair, nrule = ctypes.c_int(), ctypes.c_int()
    _check(lib.gfc_test_angular_rules(int(n_angular), int(dim), rule,
                                      ctypes.c_void_p(pairs.ctypes.data), 512, ctypes.byref(npair),
                                      ctypes.c_void_p(rules.ctypes.data), 4096,
                                      ctypes.c_void_p(rule_n.ctypes.data),
                                      ctypes.c_void_p(rho_min.ctypes.data), ctypes.byref(nrule)),
           "gfc_test_angular_rules")
    out, off = [], 0
    for r in range(nrule.value):
        n = int(rule_n[r])
        out.append(rules[3 * off:3 * (off + n)].reshape(n, 3).copy())
        off += n
    return (pairs[:3 * npair.value].reshape(-1, 3).copy(), out,
            rho_min[:nrule.value].astype(np.float64))
