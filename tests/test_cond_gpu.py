"""The per-point rounding-error scale of gfc_eval_points_cond.

E = K_D (sqrt(sum_k (M_k kappa_k)^2) + sum_k M_k) over a point's contour
nodes (M_k the magnitude of node k's contribution, kappa_k its relative
condition number) is the scale that a point's rounding error is a small
multiple of, in the unit roundoff of the arithmetic that produced the value:
checked against the oracle for binary64, and against the binary64 result for
the points GFC_MIXED keeps in binary32 (the bound its routing relies on). E is
0 where nothing is summed (the cut side of the real axis, x = mu2) and where
the value came from double-float, which computes no scale. Relative to |G| it
is larger next to the negative real axis, where the angular integrand nearly
pinches, than away from it (not monotonically so: the discrete rule's nodes
meet the pinch at particular distances).
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

SCALAR = {"kind": "scalar", "m2": 1.0}
U64, U32 = 2.0 ** -53, 2.0 ** -24
PAR = dict(dim=4, mu2=1.0, n_radial=512, n_angular=64)
# regular points, one far from the axis, three next to the negative real
# axis, then the cut side and x = mu2
NEAR = [2 + 1j, -2 + 0.1j, -2 + 0.02j, -2 + 0.004j]
SPECIAL = [-3 + 0j, 1 + 0j]


def _points(n=192, seed=11):
    # seeded sample of the production 1024 x 1024 grid's cell centres
    x = oracle.grid_points(*si.grid_rect("production"), 1024, 1024)
    x = x[si.sample_indices(seed, x.size, n)]
    return np.concatenate([x, NEAR, SPECIAL])


def _cond(prop, par, x):
    G, c = gfc.eval_points_cond(prop, par, torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    return G.cpu().numpy(), c.cpu().numpy()


def test_fp64_scale_bounds_the_error_against_the_oracle():
    x = _points()
    G, c = _cond(SCALAR, dict(PAR, precision="fp64"), x)
    reg = slice(0, x.size - len(SPECIAL))
    # nothing summed on the cut side and at the subtraction point
    assert np.all(c[reg.stop:] == 0.0)
    assert np.isnan(G[-2]) and G[-1] == 0.0
    assert np.all(np.isfinite(c[reg]) & (c[reg] > 0.0))
    ref = oracle.eval_points(SCALAR, PAR, x[reg])
    err = np.abs(G[reg] - ref)
    ratio = err / (U64 * c[reg])
    k = int(np.argmax(ratio))
    assert ratio[k] <= 8.0, f"error {err[k]:.3e} = {ratio[k]:.1f} u E at x = {x[k]}"
    # the scale relative to |G| next to the negative real axis, against x = 2 + i
    n0 = reg.stop - len(NEAR)
    rel = c[n0:reg.stop] / np.abs(G[n0:reg.stop])
    assert 1.0 <= rel[0] < 30.0 and np.all(rel[1:] > 10.0 * rel[0]), rel


def test_mixed_kept_points_within_the_binary32_scale():
    x = _points(256, seed=12)
    G, c = _cond(SCALAR, dict(PAR, precision="mixed"), x)
    routed = gfc.last_stats().points_fp64
    Gf, cf = _cond(SCALAR, dict(PAR, precision="fp64"), x)
    reg = np.arange(x.size - len(SPECIAL))
    # double-float computes no scale: the routed points (band included) report 0
    assert np.count_nonzero(c[reg] == 0.0) == routed
    kept = reg[c[reg] > 0.0]
    assert kept.size > 0
    err = np.abs(G[kept] - Gf[kept])
    # the routing keeps a point when 2 u32 E <= 1e-6 |G|; the binary32 error
    # is a small multiple of u32 E (median 0.25-0.45, at most 3.5 over the
    # production grids when the factor 2 was calibrated)
    ratio = err / (U32 * c[kept])
    k = int(np.argmax(ratio))
    assert ratio[k] <= 4.0, f"error {err[k]:.3e} = {ratio[k]:.2f} u32 E at x = {x[kept[k]]}"
    assert np.median(ratio) <= 1.0
    assert np.all(2.0 * U32 * c[kept] <= 1e-6 * np.abs(G[kept]) * (1 + 1e-12))


def test_mixed_fp64_fallback_equals_the_fp64_call_bitwise():
    x = _points(128, seed=13)
    G, c = _cond(SCALAR, dict(PAR, precision="mixed", mixed_fallback="fp64"), x)
    routed = gfc.last_stats().points_fp64
    Gf, cf = _cond(SCALAR, dict(PAR, precision="fp64"), x)
    # routed points: the binary64 kernel on the list computes exactly what it
    # computes on all points, scale included
    same = (G == Gf) & (c == cf)
    assert routed > 0
    assert np.count_nonzero(same[: x.size - len(SPECIAL)]) >= routed


def test_double_float_writes_zero_scale():
    x = _points(64, seed=14)
    G, c = _cond(SCALAR, dict(PAR, precision="f32x2"), x)
    assert np.all(c == 0.0)
    assert np.all(np.isfinite(G[: x.size - 2]))
