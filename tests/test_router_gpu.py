"""Requests over several servers (gfc_router_*): each request goes whole to
the server with the least estimated work outstanding, and comes back equal
to the one-shot evaluation of the same grid. The servers here share device
0 (the routing logic does not depend on how many devices there are)."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_0752_gb300 as gfc  # noqa: E402


def _rel(a, b):
    tau = 1e-3 * np.max(np.abs(b))
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), tau))


def test_requests_spread_over_servers_and_match_one_shot():
    a, b, c = si.dressed_draws(3, 1)[0]
    props = [{"kind": "scalar", "m2": 1.0}, {"kind": "dressed", "a": a, "b": b, "c": c},
             {"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j}]
    rect = si.grid_rect("small")
    reqs = []
    for i in range(12):
        prop = props[i % 3]
        cpair = prop["kind"] == "cpair"
        par = dict(dim=4 if (i % 2 or cpair) else 3, mu2=0.0 if cpair else 1.0,
                   n_radial=256, n_angular=64, precision="fp64")
        side = (16, 32, 48)[i % 3]
        reqs.append((prop, par, (*rect, side, side)))
    with gfc.Router([0, 0], hbm_budget_bytes=4 << 30, max_slots=16) as r:
        sub = [(r.submit(p, q, g), p, q, g) for p, q, g in reqs]
        for (t, _), _, _, _ in sub:
            assert r.wait(t) == 0
        assert {r.server_of(t)[0] for (t, _), _, _, _ in sub} == {0, 1}
        assert sum(s.stats().completed for s in r.servers) == len(reqs)
        assert all(s.load() == 0.0 for s in r.servers)
        for (t, G), p, q, g in sub:
            ref = gfc.eval_grid(p, q, g).cpu().numpy()
            assert _rel(G, ref) <= 1e-12
