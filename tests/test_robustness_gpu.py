"""Failure paths without faulting the GPU, reproducibility, and the smallest
orders.

Allocation failures are injected on the host (gfc_test_fail_allocations):
the call reports GFC_ECUDA, leaves no half-built state behind, and the next
call succeeds. Results are bitwise reproducible: every point's sums run in a
fixed order (lanes over fixed node indices, a fixed warp reduction tree),
whichever warp takes the point and in whatever order points are listed.
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_0752_gb300 as gfc  # noqa: E402
from paper_1205_0752_gb300 import binding  # noqa: E402

SCALAR = {"kind": "scalar", "m2": 1.0}
GFC_ECUDA = -4
X = np.array([2 + 1j, -2 + 0.5j, -6 - 1j, 0.3 - 2j, -0.5 + 0.05j])


def _oracle(par, x=X):
    keep = ("dim", "mu2", "n_radial", "n_angular", "angular_rule", "radial_rule")
    return oracle.eval_points(SCALAR, {k: par[k] for k in keep if k in par}, x)


def test_injected_allocation_failure_is_reported_and_recovers():
    # an order no other test uses, so the call must build (allocate) new tables
    par = dict(dim=4, mu2=1.0, n_radial=1996, n_angular=46, precision="fp64")
    xt = torch.tensor(X, device="cuda")
    binding.test_fail_allocations(1)
    try:
        with pytest.raises(gfc.GfcError) as e:
            gfc.eval_points(SCALAR, par, xt)
        assert e.value.status == GFC_ECUDA
        assert b"cudaMalloc" in gfc.load_library().gfc_last_error()
    finally:
        binding.test_fail_allocations(0)
    G = gfc.eval_points(SCALAR, par, xt)
    torch.cuda.synchronize()
    ref = _oracle(par)
    assert np.max(np.abs(G.cpu().numpy() - ref) / np.abs(ref)) < 1e-10


def test_injected_allocation_failure_in_the_server():
    rect = si.grid_rect("small")
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=64, precision="mixed")
    with gfc.Server(0, hbm_budget_bytes=64 << 20, max_slots=4) as srv:
        binding.test_fail_allocations(1)
        try:
            t, _ = srv.submit(SCALAR, par, (*rect, 16, 16))
            assert srv.wait(t, 60000) == GFC_ECUDA
        finally:
            binding.test_fail_allocations(0)
        t, G = srv.submit(SCALAR, par, (*rect, 16, 16))
        assert srv.wait(t, 60000) == 0
    alone = gfc.eval_grid(SCALAR, par, (*rect, 16, 16))
    torch.cuda.synchronize()
    assert np.max(np.abs(G - alone.cpu().numpy()) / np.abs(alone.cpu().numpy())) < 1e-6


def test_hook_rejects_negative_counts():
    with pytest.raises(gfc.GfcError):
        binding.test_fail_allocations(-1)
    with pytest.raises(gfc.GfcError):
        binding.test_fail_launches(-1)


def test_injected_launch_failure_one_shot():
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=64, precision="fp64")
    xt = torch.tensor(X, device="cuda")
    binding.test_fail_launches(1)
    try:
        with pytest.raises(gfc.GfcError) as e:
            gfc.eval_points(SCALAR, par, xt)
        assert e.value.status == GFC_ECUDA
    finally:
        binding.test_fail_launches(0)
    G = gfc.eval_points(SCALAR, par, xt)
    torch.cuda.synchronize()
    ref = _oracle(par)
    assert np.max(np.abs(G.cpu().numpy() - ref) / np.abs(ref)) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_injected_launch_failure_in_the_server_is_not_a_result(precision):
    """A batched launch that fails finishes every request it carried with
    GFC_ECUDA, and the host array is not written; later requests succeed."""
    rect = si.grid_rect("small")
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=64, precision=precision)
    with gfc.Server(0, hbm_budget_bytes=64 << 20, max_slots=4) as srv:
        sentinel = np.full((16, 16), 7.0 + 7.0j)
        binding.test_fail_launches(1)
        try:
            t, G = srv.submit(SCALAR, par, (*rect, 16, 16), out=sentinel)
            assert srv.wait(t, 60000) == GFC_ECUDA
            assert b"launch" in gfc.load_library().gfc_last_error()
            assert srv.request_info(t)["status"] == GFC_ECUDA
            assert np.all(G == 7.0 + 7.0j)
        finally:
            binding.test_fail_launches(0)
        t, G = srv.submit(SCALAR, par, (*rect, 16, 16))
        assert srv.wait(t, 60000) == 0
        assert srv.stats().completed == 1
    alone = gfc.eval_grid(SCALAR, par, (*rect, 16, 16)).cpu().numpy()
    tol = 1e-6 if precision == "mixed" else 1e-10
    assert np.max(np.abs(G - alone) / np.abs(alone)) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
def test_results_are_bitwise_reproducible(precision):
    rect = si.grid_rect("production")
    par = dict(dim=4, mu2=1.0, n_radial=512, n_angular=64, precision=precision)
    a = gfc.eval_grid(SCALAR, par, (*rect, 96, 80)).cpu().numpy()
    b = gfc.eval_grid(SCALAR, par, (*rect, 96, 80)).cpu().numpy()
    assert np.array_equal(a, b)
    # the same points listed in another order give the same values
    x = oracle.grid_points(*rect, 96, 80)
    perm = np.random.default_rng(3).permutation(x.size)
    G = gfc.eval_points(SCALAR, par, torch.tensor(x[perm], device="cuda")).cpu().numpy()
    # (mixed: routing depends only on the point, so the permuted call routes alike)
    assert np.array_equal(G, a.ravel()[perm])


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
def test_smallest_orders(precision):
    """n_radial = 4, n_angular = 2 (one pair): coarse, but the same finite
    sums as the oracle's, on a 1 x 1 grid and on points of every kind."""
    par = dict(dim=4, mu2=1.0, n_radial=4, n_angular=2, precision=precision)
    tol = 1e-6 if precision == "mixed" else 1e-10
    G = gfc.eval_points(SCALAR, par, torch.tensor(X, device="cuda")).cpu().numpy()
    ref = _oracle(par)
    assert np.max(np.abs(G - ref) / np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))) < tol
    G1 = gfc.eval_grid(SCALAR, par, (-3.0, 1.0, -1.0, 2.0, 1, 1)).cpu().numpy().ravel()
    ref1 = _oracle(par, oracle.grid_points(-3.0, 1.0, -1.0, 2.0, 1, 1))
    assert abs(G1[0] - ref1[0]) <= tol * abs(ref1[0])
