"""The C-ABI library loads without a GPU and exports every function that
include/gfc.h declares; calls that fail argument checks do so on the host,
before any CUDA work, with the documented status codes."""
import ctypes
import os
import re

import pytest

import paper_1205_0752_gb300 as gfc
from paper_1205_0752_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gfc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gfc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_function_is_exported():
    lib = gfc.load_library()
    names = declared_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows the signature of each
    assert sorted(binding._SIGS) == names


def test_version_and_strings():
    assert gfc.version() == (1, 6)
    lib = gfc.load_library()
    assert lib.gfc_strerror(0) == b"ok"
    assert lib.gfc_strerror(-3) == b"request exceeds the memory budget"


def test_defaults():
    p = gfc.make_params()
    assert (p.dim, p.mu2, p.n_radial, p.n_angular) == (4, 1.0, 2048, 256)
    assert (p.radial_scale, p.detour_radius, p.precision) == (1.0, 0.1, 0)
    assert (p.cut_band, p.pinch_angle, p.mixed_rtol, p.mixed_fallback) == (0.05, 0.0, 1e-6, 2)
    assert p.angular_rule == 0


@pytest.mark.parametrize("bad", [dict(dim=2), dict(n_radial=6), dict(n_radial=20000),
                                 dict(n_angular=1), dict(n_angular=1024), dict(mu2=-1.0),
                                 dict(angular_rule="tanh-sinh", n_angular=64),
                                 dict(angular_rule=5),
                                 dict(radial_scale=-1.0), dict(precision=7),
                                 dict(mixed_rtol=-1.0), dict(mixed_fallback="mixed")])
def test_bad_params_rejected_on_the_host(bad):
    lib = gfc.load_library()
    p = gfc.make_params(**bad)
    prop = gfc.make_prop({"kind": "scalar", "m2": 1.0})
    rc = lib.gfc_eval_points(ctypes.byref(prop), ctypes.byref(p), None, 0, None, None)
    assert rc == -1
    assert lib.gfc_last_error() != b""


def test_bad_grid_and_pointers_rejected_on_the_host():
    lib = gfc.load_library()
    p = gfc.make_params()
    prop = gfc.make_prop({"kind": "scalar", "m2": 1.0})
    g = gfc.make_grid(-2.0, 1.0, -1.5, 1.5, 4, 3)     # middle row on the negative axis
    assert lib.gfc_eval_grid(ctypes.byref(prop), ctypes.byref(p), ctypes.byref(g),
                             ctypes.c_void_p(16), None) == -1
    g = gfc.make_grid(1.0, -1.0, -1.0, 1.0, 4, 4)     # empty rectangle
    assert lib.gfc_grid_points(ctypes.byref(g), ctypes.c_void_p(16), None) == -1
    g = gfc.make_grid(-1.0, 1.0, -1.0, 1.0, 4, 4)
    assert lib.gfc_eval_grid(ctypes.byref(prop), ctypes.byref(p), ctypes.byref(g),
                             ctypes.c_void_p(8), None) == -1   # misaligned
    assert lib.gfc_eval_points(ctypes.byref(prop), ctypes.byref(p), None, 5, None, None) == -1


@pytest.mark.parametrize("prop", [{"kind": "scalar", "m2": 0.0},
                                  {"kind": "cpair", "mk2": 0.5j, "mq2": 0.4j},
                                  {"kind": "cpair", "mk2": 0.05j, "mq2": -0.05j},
                                  {"kind": "dressed", "a": 1.0, "b": 3.0, "c": 2.0}])
def test_bad_propagators_rejected_on_the_host(prop):
    lib = gfc.load_library()
    p = gfc.make_params()
    g = gfc.make_grid(-1.0, 1.0, -1.0, 1.0, 4, 4)
    rc = lib.gfc_eval_grid(ctypes.byref(gfc.make_prop(prop)), ctypes.byref(p), ctypes.byref(g),
                           ctypes.c_void_p(16), None)
    assert rc == -1


def test_server_arguments_checked_on_the_host():
    lib = gfc.load_library()
    h = ctypes.c_void_p()
    assert lib.gfc_server_create(0, 1 << 30, 0, ctypes.byref(h)) == -1
    assert lib.gfc_server_create(0, 1 << 10, 4, ctypes.byref(h)) == -1
    assert lib.gfc_server_destroy(None) == -1


def test_router_rejects_bad_arguments_on_the_host():
    lib = gfc.load_library()
    h = ctypes.c_void_p()
    devs = (ctypes.c_int * 1)(0)
    assert lib.gfc_router_create(devs, 0, 1 << 30, 8, ctypes.byref(h)) == -1
    assert lib.gfc_router_create(devs, 257, 1 << 30, 8, ctypes.byref(h)) == -1
    assert lib.gfc_router_create(None, 1, 1 << 30, 8, ctypes.byref(h)) == -1
    assert lib.gfc_router_destroy(None) == -1
