"""gfc_eval_points_noalloc: the FP64 evaluation for callers that cannot
allocate device memory (its tables and scratch sit in a fixed device array
inside the library). Called through the C ABI, two calls in a row, each
checked against gfc_eval_points within the FP64 tolerance of the other
tests. Kept in a file of its own, collected last."""
import ctypes

import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_0752_gb300 as gfc  # noqa: E402

RTOL = 1e-10


def _rel(a, b):
    tau = 1e-3 * np.max(np.abs(b))
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), tau))


def _noalloc(prop, par, xt):
    lib = gfc.load_library()
    G = torch.empty_like(xt)
    rc = lib.gfc_eval_points_noalloc(ctypes.byref(gfc.make_prop(prop)),
                                     ctypes.byref(gfc.make_params(par)),
                                     ctypes.c_void_p(xt.data_ptr()), xt.numel(),
                                     ctypes.c_void_p(G.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.gfc_last_error()
    torch.cuda.synchronize()
    return G.cpu().numpy()


def test_two_calls_match_the_allocating_entry_point():
    g = si.SplitMix64(21)
    xs = np.array([complex(-8 + 12 * g.uniform(), -4 + 8 * g.uniform()) for _ in range(300)])
    xt = torch.tensor(xs, dtype=torch.complex128, device="cuda")
    a, b, c = si.dressed_draws(3, 1)[0]
    calls = [({"kind": "scalar", "m2": 1.0}, dict(dim=4, mu2=1.0, n_radial=512, n_angular=128)),
             ({"kind": "dressed", "a": a, "b": b, "c": c},
              dict(dim=3, mu2=1.0, n_radial=256, n_angular=64))]
    for prop, par in calls:
        ref = gfc.eval_points(prop, dict(par, precision="fp64"), xt)
        torch.cuda.synchronize()
        got = _noalloc(prop, dict(par, precision="fp64"), xt)
        assert _rel(got, ref.cpu().numpy()) <= RTOL


def test_makes_no_device_allocation():
    """With the library's allocation hook armed (its next device allocation
    would fail) the call still succeeds, and the device's free memory is the
    same before and after a warmed-up call."""
    from paper_1205_0752_gb300 import binding
    g = si.SplitMix64(22)
    xs = np.array([complex(-8 + 12 * g.uniform(), -4 + 8 * g.uniform()) for _ in range(64)])
    xt = torch.tensor(xs, dtype=torch.complex128, device="cuda")
    prop, par = {"kind": "scalar", "m2": 1.0}, dict(dim=4, mu2=1.0, n_radial=256, n_angular=64)
    ref = gfc.eval_points(prop, dict(par, precision="fp64"), xt).cpu().numpy()
    lib = gfc.load_library()
    G = torch.empty_like(xt)
    args = (ctypes.byref(gfc.make_prop(prop)), ctypes.byref(gfc.make_params(par)),
            ctypes.c_void_p(xt.data_ptr()), xt.numel(), ctypes.c_void_p(G.data_ptr()))
    binding.test_fail_allocations(1)
    try:
        for _ in range(2):
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            assert lib.gfc_eval_points_noalloc(*args, None) == 0, lib.gfc_last_error()
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
    finally:
        binding.test_fail_allocations(0)
    # the second call ran with every kernel loaded: nothing was allocated
    assert free1 == free0
    assert _rel(G.cpu().numpy(), ref) <= RTOL


def test_rejects_sizes_beyond_its_limits():
    lib = gfc.load_library()
    xt = torch.tensor([1 + 1j], dtype=torch.complex128, device="cuda")
    G = torch.empty_like(xt)
    for par in (dict(n_radial=8192), dict(precision="mixed")):
        rc = lib.gfc_eval_points_noalloc(ctypes.byref(gfc.make_prop({"kind": "scalar", "m2": 1.0})),
                                         ctypes.byref(gfc.make_params(par)),
                                         ctypes.c_void_p(xt.data_ptr()), 1,
                                         ctypes.c_void_p(G.data_ptr()), None)
        assert rc == -1 and lib.gfc_last_error()
