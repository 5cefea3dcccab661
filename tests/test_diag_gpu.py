"""Step 3 diagnostics on the GPU against the oracle (Sect. 5, Figs. 1-2):
the angular integral B(x, y) over a grid of complex y, and the region-1 map
over a grid of complex x."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_0752_gb300 as gfc  # noqa: E402

PROPS = {"scalar": {"kind": "scalar", "m2": 1.0},
         "paper": {"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j},
         "dressed": {"kind": "dressed", "a": 1.0, "b": 0.5, "c": 2.0}}


def _q_poles(prop):
    """Poles s = -M2 of the (p-k) leg as given."""
    if prop["kind"] == "scalar":
        return [prop["m2"]]
    if prop["kind"] == "cpair":
        return [complex(prop["mq2"])]
    b, c = prop["b"], prop["c"]
    yp = complex(-0.5 * b, 0.5 * np.sqrt(4 * c - b * b))
    return [-yp, -np.conj(yp)]


def _cut_distance(prop, x, y):
    """Distance of each y to the branch cut of eq. 25 (sampled)."""
    th = np.linspace(0.0, np.pi, 20001)
    pts = []
    for M in _q_poles(prop):
        r = np.sqrt(-x * np.sin(th) ** 2 - M + 0j)
        for sg in (1, -1):
            pts.append((np.sqrt(x + 0j) * np.cos(th) + sg * r) ** 2)
    pts = np.concatenate(pts)
    return np.array([np.min(np.abs(pts - v)) for v in y])


@pytest.mark.parametrize("dim", [3, 4])
@pytest.mark.parametrize("rule,n", [("gl", 64), ("tanh-sinh", 49), ("exact", 2)])
@pytest.mark.parametrize("name", ["scalar", "paper", "dressed"])
def test_angular_map_matches_oracle(name, rule, n, dim):
    prop = PROPS[name]
    x = -2.0 + 1.0j
    g = np.linspace(-6.0, 6.0, 41)[:-1] + 0.15
    y = (g[:, None] + 1j * g[None, :]).ravel()
    par = dict(dim=dim, mu2=1.0, n_radial=4, n_angular=n, angular_rule=rule)
    B = gfc.angular_map(prop, par, x, torch.tensor(y, device="cuda"))
    torch.cuda.synchronize()
    B = B.cpu().numpy()
    ref = oracle.angular_map(prop, par, x, y)
    keep = _cut_distance(prop, x, y) > 1e-2
    tau = 1e-3 * np.max(np.abs(ref[keep]))
    err = np.abs(B - ref) / np.maximum(np.abs(ref), tau)
    assert keep.mean() > 0.8
    assert np.max(err[keep]) < 1e-10, (name, rule, dim, np.max(err[keep]))


@pytest.mark.parametrize("name", ["scalar", "paper", "dressed"])
def test_region_map_matches_oracle(name):
    prop = PROPS[name]
    rect = si.grid_rect("production")
    x = oracle.grid_points(*rect, 96, 80)
    F = gfc.region_map(prop, torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    F = F.cpu().numpy()
    ref = oracle.region_map(prop, x)
    # compare where the oracle's answer is the same a small step away in
    # every direction (points on the boundary may go either way)
    d = 0.03
    stable = np.ones(x.size, dtype=bool)
    for dx in (d, -d, 1j * d, -1j * d):
        stable &= oracle.region_map(prop, x + dx) == ref
    assert stable.mean() > 0.9
    assert np.array_equal(F[stable], ref[stable])
    assert 0.0 < ref.mean() < 1.0


def test_region_map_parabola_for_real_mass():
    """Region 1 for the real-mass bubble is Im^2 x < 4 m^2 (Re x + m^2)."""
    m2 = 0.25
    x = oracle.grid_points(-10.0, 5.0, -5.0, 5.0, 150, 100)
    F = gfc.region_map({"kind": "scalar", "m2": m2}, torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    par = (x.imag ** 2 < 4 * m2 * (x.real + m2)).astype(np.int32)
    far = np.abs(x.imag ** 2 - 4 * m2 * (x.real + m2)) > 0.02
    assert np.array_equal(F.cpu().numpy()[far], par[far])


def test_diagnostics_reject_bad_arguments():
    with pytest.raises(gfc.GfcError):
        gfc.angular_map({"kind": "dressed", "a": 1, "b": 3, "c": 2}, {}, 1.0,
                        torch.zeros(4, dtype=torch.complex128, device="cuda"))
    with pytest.raises(gfc.GfcError):
        gfc.region_map({"kind": "cpair", "mk2": 1j, "mq2": 1j},
                       torch.zeros(4, dtype=torch.complex128, device="cuda"))
