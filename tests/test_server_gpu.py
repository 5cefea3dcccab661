"""Serving runtime (continuous batching) through the C ABI.

Each result computed in a mix of concurrently admitted requests equals the
same request evaluated alone (one-shot call), within the stated tolerances;
admission honours the memory budget; cancel, wait timeouts and stats work.
"""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_0752_gb300 as gfc  # noqa: E402

RTOL = {"fp64": 1e-10, "mixed": 1e-6, "f32x2": 1e-10}
RECT = si.grid_rect("small")


def _mix():
    a, b, c = si.dressed_draws(3, 1)[0]
    dressed = {"kind": "dressed", "a": a, "b": b, "c": c}
    return [
        ({"kind": "scalar", "m2": 1.0}, dict(dim=4, n_radial=256, n_angular=64, precision="fp64"), 64),
        ({"kind": "scalar", "m2": 0.25}, dict(dim=3, n_radial=512, n_angular=128, precision="mixed"), 48),
        (dressed, dict(dim=4, n_radial=256, n_angular=64, precision="fp64"), 40),
        (dressed, dict(dim=3, n_radial=256, n_angular=128, precision="mixed"), 32),
        ({"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j}, dict(dim=4, mu2=0.0, n_radial=256, n_angular=64,
                                                             precision="fp64"), 56),
        ({"kind": "scalar", "m2": 4.0}, dict(dim=4, n_radial=512, n_angular=256, precision="mixed"), 64),
        ({"kind": "scalar", "m2": 1.0}, dict(dim=4, n_radial=256, n_angular=10, precision="fp64"), 34),
        # other rules: same n_angular and dim as the first request, so only the
        # rules keep them out of its launches
        ({"kind": "scalar", "m2": 1.0}, dict(dim=4, n_radial=256, n_angular=64, precision="fp64",
                                             angular_rule="chebyshev2"), 40),
        ({"kind": "scalar", "m2": 1.0}, dict(dim=4, n_radial=256, n_angular=49, precision="f32x2",
                                             angular_rule="tanh-sinh"), 36),
        ({"kind": "scalar", "m2": 1.0}, dict(dim=4, n_radial=512, n_angular=64, precision="fp64",
                                             angular_rule="exact", radial_rule="clustered"), 44),
        (dressed, dict(dim=3, n_radial=512, n_angular=64, precision="mixed",
                       angular_rule="exact", radial_rule="clustered"), 30),
    ]


def _alone(prop, par, side):
    G = gfc.eval_grid(prop, par, (*RECT, side, side))
    torch.cuda.synchronize()
    return G.cpu().numpy()


def _rel(a, b):
    tau = 1e-3 * np.max(np.abs(b))
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), tau))


def test_mix_equals_alone():
    mix = _mix()
    alone = [_alone(p, q, s) for p, q, s in mix]
    # small budget and few slots: later requests wait for admission while
    # earlier ones run, so the mix overlaps admission, launches and copies
    with gfc.Server(0, hbm_budget_bytes=8 << 20, max_slots=3) as srv:
        tickets = [srv.submit(p, q, (*RECT, s, s)) for p, q, s in mix]
        for (t, _), (p, q, s) in zip(tickets, mix):
            assert srv.wait(t, 120000) == 0, gfc.load_library().gfc_last_error()
        st = srv.stats()
        assert st.completed == len(mix) and st.launches >= 2
        assert st.p99_ms >= st.p50_ms > 0
        for (t, _), (p, q, s) in zip(tickets, mix):
            info = srv.request_info(t)
            assert info["status"] == 0 and info["state"] == 2 and info["points"] == s * s
            assert 0.0 <= info["queue_ms"] <= info["total_ms"] and info["launches"] >= 1
            assert info["bytes"] >= 16 * s * s
            if q["precision"] == "mixed":
                assert 0 <= info["points_routed"] <= s * s
            else:
                assert info["points_routed"] == -1
    for (t, G), ref, (p, q, s) in zip(tickets, alone, mix):
        assert _rel(G, ref) <= RTOL[q["precision"]], (p, q, s, _rel(G, ref))


def test_each_request_alone_in_the_server():
    mix = _mix()[:3]
    with gfc.Server(0, hbm_budget_bytes=1 << 30, max_slots=8) as srv:
        for p, q, s in mix:
            t, G = srv.submit(p, q, (*RECT, s, s))
            assert srv.wait(t, 120000) == 0
            assert _rel(G, _alone(p, q, s)) <= RTOL[q["precision"]]


def test_budget_rejects_oversized_request():
    with gfc.Server(0, hbm_budget_bytes=2 << 20, max_slots=2) as srv:
        with pytest.raises(gfc.GfcError) as ei:
            srv.submit({"kind": "scalar", "m2": 1.0}, dict(precision="fp64"), (*RECT, 512, 512))
        assert ei.value.status == -3
        assert srv.stats().rejected == 1


def test_cancel_queued_and_wait_timeout():
    big = dict(dim=4, n_radial=2048, n_angular=256, precision="fp64")
    with gfc.Server(0, hbm_budget_bytes=1 << 30, max_slots=1) as srv:
        t1, _ = srv.submit({"kind": "scalar", "m2": 1.0}, big, (*RECT, 128, 128))
        t2, G2 = srv.submit({"kind": "scalar", "m2": 1.0}, big, (*RECT, 64, 64))
        G2[:] = 7.0
        assert srv.cancel(t2) == 0
        assert srv.wait(t2, 1000) == -6
        assert srv.wait(t1, 1) == -5          # still running after 1 ms
        assert srv.wait(t1, 300000) == 0
        assert np.all(G2 == 7.0)              # a cancelled request writes nothing
        st = srv.stats()
        assert st.completed == 1 and st.canceled == 1


def test_bad_requests_rejected():
    with gfc.Server(0, hbm_budget_bytes=1 << 30, max_slots=2) as srv:
        with pytest.raises(gfc.GfcError):
            srv.submit({"kind": "scalar", "m2": 1.0}, dict(n_angular=1), (*RECT, 8, 8))
        with pytest.raises(gfc.GfcError):
            srv.submit({"kind": "scalar", "m2": 1.0}, {}, (-2.0, 1.0, -1.5, 1.5, 4, 3))


def test_cancel_active_request_between_launches():
    """A request already on the device stops being scheduled: the launch in
    flight completes (launches are bounded by the server's work budget, so no
    kernel polls a flag), no further launch is made for it, its host array is
    not written, and the server goes on serving."""
    import time
    big = dict(dim=4, n_radial=2048, n_angular=256, precision="fp64")
    with gfc.Server(0, hbm_budget_bytes=1 << 30, max_slots=2) as srv:
        # 2048 x 2048 points, several launches' worth of work
        t, G = srv.submit({"kind": "scalar", "m2": 1.0}, big, (*RECT, 2048, 2048))
        G[:] = 7.0
        deadline = time.monotonic() + 60.0
        while srv.request_info(t)["state"] == 0 and time.monotonic() < deadline:
            time.sleep(0.002)
        assert srv.request_info(t)["state"] == 1      # on the device, not finished
        assert srv.cancel(t) == 0
        assert srv.wait(t, 120000) == -6
        info = srv.request_info(t)
        assert info["state"] == 2 and info["status"] == -6
        assert np.all(G == 7.0)
        # the server still serves
        t2, G2 = srv.submit({"kind": "scalar", "m2": 1.0}, dict(big, n_radial=256, n_angular=64),
                            (*RECT, 16, 16))
        assert srv.wait(t2, 60000) == 0
        assert _rel(G2, _alone({"kind": "scalar", "m2": 1.0}, dict(big, n_radial=256, n_angular=64), 16)) <= 1e-10
        assert srv.stats().canceled == 1


def test_device_output_equals_host_output():
    """G may be device memory of the server's device: the kernels write it in
    place (no output buffer counted against the budget) and the result equals
    the host-output request's and the one-shot call's."""
    mix = _mix()[:4]
    with gfc.Server(0, hbm_budget_bytes=8 << 20, max_slots=3) as srv:
        host = [srv.submit(p, q, (*RECT, s, s)) for p, q, s in mix]
        dev = [srv.submit(p, q, (*RECT, s, s),
                          out=torch.empty((s, s), dtype=torch.complex128, device="cuda"))
               for p, q, s in mix]
        for (t, _), (td, _) in zip(host, dev):
            assert srv.wait(t, 120000) == 0
            assert srv.wait(td, 120000) == 0
        for (td, _), (p, q, s) in zip(dev, mix):
            info = srv.request_info(td)
            assert info["bytes"] == (8 * s * s if q["precision"] == "mixed" else 0)
    for (_, Gh), (_, Gd), (p, q, s) in zip(host, dev, mix):
        gd = Gd.cpu().numpy()
        assert np.array_equal(gd, Gh)
        assert _rel(gd, _alone(p, q, s)) <= RTOL[q["precision"]]
