"""ORACLE — test infrastructure only.

ctypes wrapper around ``gfc_oracle.c``: a plain FP64 CPU evaluation of the
Taylor-subtracted two-point integral (Steps 1-5 of Sect. 2, eqs. 11-15 and 20;
contours of Sect. 5.3). Only the tests, the smoke check (``smoke()``) and the
benchmark's CPU-baseline and reference legs may import this package. It imports nothing from
the product package and the product package imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "gfc_oracle.c")
_lock = threading.Lock()
_lib = None

PROP_SCALAR, PROP_CPAIR, PROP_DRESSED = 0, 1, 2


class _Prop(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("m2", ctypes.c_double),
                ("mk2_re", ctypes.c_double), ("mk2_im", ctypes.c_double),
                ("mq2_re", ctypes.c_double), ("mq2_im", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("mu2", ctypes.c_double),
                ("n_radial", ctypes.c_int), ("n_angular", ctypes.c_int),
                ("radial_scale", ctypes.c_double), ("detour_radius", ctypes.c_double),
                ("angular_rule", ctypes.c_int), ("radial_rule", ctypes.c_int)]

# angular rules (Sect. 4)
ANGULAR_RULES = {"gl": 0, "tanh-sinh": 1, "chebyshev1": 2, "chebyshev2": 3, "exact": 4}
# radial rules of the rays from q = 0
RADIAL_RULES = {"mapped": 0, "clustered": 1}


def _compile(out: str, defines=()) -> None:
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *defines, "-o", tmp,
                           _SRC, "-lm", "-lpthread"])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gfc_oracle.h"))):
        _compile(_SO)
    return _SO


def _bind(path: str):
    lib = ctypes.CDLL(path)
    lib.orc_eval_points.argtypes = [ctypes.POINTER(_Prop), ctypes.POINTER(_Params),
                                    ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int]
    lib.orc_eval_points.restype = ctypes.c_int
    lib.orc_grid_points.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_int,
                                                            ctypes.c_void_p]
    lib.orc_grid_points.restype = ctypes.c_int
    lib.orc_gauss_legendre.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_angular_rule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p]
    lib.orc_gauss_legendre.restype = ctypes.c_int
    lib.orc_angular_map.argtypes = [ctypes.POINTER(_Prop), ctypes.POINTER(_Params),
                                    ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                    ctypes.c_long, ctypes.c_void_p]
    lib.orc_region_map.argtypes = [ctypes.POINTER(_Prop), ctypes.c_void_p, ctypes.c_long,
                                   ctypes.c_void_p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


class Oracle:
    """The oracle's entry points bound to one compiled library."""

    def __init__(self, lib):
        self._lib = lib

    def eval_points(self, prop, params, x, nthreads=None, with_kappa=False):
        return _eval_points(self._lib, prop, params, x, nthreads, with_kappa)

    def grid_points(self, re0, re1, im0, im1, m, n):
        return _grid_points(self._lib, re0, re1, im0, im1, m, n)


def mutant(n: int, workdir: str) -> Oracle:
    """The oracle with planted mistake number ``n`` compiled in (tests only)."""
    out = os.path.join(workdir, f"liboracle_mutant{n}.so")
    _compile(out, [f"-DORC_MUTANT={int(n)}"])
    return Oracle(_bind(out))


def _prop(spec: dict) -> _Prop:
    k = spec["kind"]
    p = _Prop()
    if k == "scalar":
        p.kind, p.m2 = PROP_SCALAR, float(spec["m2"])
    elif k == "cpair":
        mk2, mq2 = complex(spec["mk2"]), complex(spec["mq2"])
        p.kind = PROP_CPAIR
        p.mk2_re, p.mk2_im, p.mq2_re, p.mq2_im = mk2.real, mk2.imag, mq2.real, mq2.imag
    elif k == "dressed":
        p.kind, p.a, p.b, p.c = PROP_DRESSED, float(spec["a"]), float(spec["b"]), float(spec["c"])
    else:
        raise ValueError(f"unknown propagator kind {k!r}")
    return p


def _params(par: dict) -> _Params:
    q = _Params()
    q.dim = int(par.get("dim", 4))
    q.mu2 = float(par.get("mu2", 0.0))
    q.n_radial = int(par["n_radial"])
    q.n_angular = int(par["n_angular"])
    q.radial_scale = float(par.get("radial_scale", 1.0))
    q.detour_radius = float(par.get("detour_radius", 0.1))
    r = par.get("angular_rule", 0)
    q.angular_rule = ANGULAR_RULES[r] if isinstance(r, str) else int(r)
    r = par.get("radial_rule", 0)
    q.radial_rule = RADIAL_RULES[r] if isinstance(r, str) else int(r)
    return q


def eval_points(prop: dict, params: dict, x, nthreads: int | None = None,
                with_kappa: bool = False):
    """G(x) = G0(x) - G0(mu2) at complex points x (physical normalisation
    int d^Dq/(2 pi)^D). Returns complex128 array (and per-point condition
    number kappa = sum|terms|/|sum| when ``with_kappa``)."""
    return _eval_points(_load(), prop, params, x, nthreads, with_kappa)


def _eval_points(lib, prop, params, x, nthreads, with_kappa):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128).ravel())
    G = np.empty_like(x)
    kap = np.empty(x.size, dtype=np.float64) if with_kappa else None
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    st = lib.orc_eval_points(ctypes.byref(_prop(prop)), ctypes.byref(_params(params)),
                             x.ctypes.data, x.size, G.ctypes.data,
                             kap.ctypes.data if kap is not None else None, int(nthreads))
    if st != 0:
        raise ValueError(f"oracle rejected the input (status {st})")
    return (G, kap) if with_kappa else G


def grid_points(re0, re1, im0, im1, m, n):
    """Kernel 1 of Sect. 4: cell-centred M x N grid, G[i*n + j] layout."""
    return _grid_points(_load(), re0, re1, im0, im1, m, n)


def _grid_points(lib, re0, re1, im0, im1, m, n):
    x = np.empty(m * n, dtype=np.complex128)
    st = lib.orc_grid_points(re0, re1, im0, im1, m, n, x.ctypes.data)
    if st != 0:
        raise ValueError("bad grid")
    return x


def angular_rule(rule, n: int, dim: int):
    """Nodes z_j = cos psi_j and weights of an angular rule (Sect. 4) for
    int_0^pi f(cos psi) sin^(D-2) psi dpsi."""
    lib = _load()
    z = np.empty(n)
    w = np.empty(n)
    r = ANGULAR_RULES[rule] if isinstance(rule, str) else int(rule)
    if lib.orc_angular_rule(r, n, dim, z.ctypes.data, w.ctypes.data) != 0:
        raise ValueError("bad angular rule, order or dimension")
    return z, w


def angular_map(prop: dict, params: dict, x: complex, y):
    """B(x, y) = int_0^pi sin^(D-2) psi [P2(s) - P2(y)] dpsi of the (p-k) leg
    as given, at complex y (Sect. 5, Fig. 1)."""
    lib = _load()
    y = np.ascontiguousarray(np.asarray(y, dtype=np.complex128).ravel())
    B = np.empty_like(y)
    rc = lib.orc_angular_map(ctypes.byref(_prop(prop)), ctypes.byref(_params(params)),
                             float(np.real(x)), float(np.imag(x)), y.ctypes.data, y.size,
                             B.ctypes.data)
    if rc != 0:
        raise ValueError(f"orc_angular_map failed ({rc})")
    return B


def region_map(prop: dict, x):
    """1 where the real-axis y contour is free of the angular integral's cut
    (region 1 of Fig. 2), else 0."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128).ravel())
    out = np.empty(x.size, dtype=np.int32)
    if lib.orc_region_map(ctypes.byref(_prop(prop)), x.ctypes.data, x.size, out.ctypes.data) != 0:
        raise ValueError("orc_region_map failed")
    return out


def gauss_legendre(n: int):
    lib = _load()
    x = np.empty(n)
    w = np.empty(n)
    if lib.orc_gauss_legendre(n, x.ctypes.data, w.ctypes.data) != 0:
        raise ValueError("bad order")
    return x, w
