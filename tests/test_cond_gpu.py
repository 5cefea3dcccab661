"""The per-point rounding-error scale of gfc_eval_points_cond.

E = K_D (sqrt(sum_k (M_k kappa_k)^2) + sum_k M_k) over a point's contour
nodes (M_k the magnitude of node k's contribution, kappa_k its relative
condition number) is the scale that a point's rounding error is a small
multiple of, in the unit roundoff of the arithmetic that produced the value:
checked against the oracle for binary64, and against the binary64 result for
the parts GFC_MIXED keeps in binary32 (the bound its routing relies on). E is
0 where nothing is summed (the cut side of the real axis, x = mu2), where the
value came from double-float, which computes no scale, and where GFC_MIXED
keeps nothing in binary32. Relative to |G| it
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
    """Under GFC_MIXED the scale is that of what a point keeps in binary32:
    the whole point, or the kept node groups of a partially routed point
    (its other groups are evaluated again in the fallback arithmetic and
    added), 0 where nothing is kept (next to a pinch); the cut band is
    evaluated whole in binary64 and reports the binary64 scale."""
    x = _points(256, seed=12)
    G, c = _cond(SCALAR, dict(PAR, precision="mixed"), x)
    st = gfc.last_stats()
    Gf, cf = _cond(SCALAR, dict(PAR, precision="fp64"), x)
    reg = np.arange(x.size - len(SPECIAL))
    xr = x[reg]
    d = np.where(xr.real <= -4.0, np.abs(xr.imag), np.abs(xr + 4.0))
    band = d < 0.05
    assert np.count_nonzero(band) == st.points_fp64
    assert np.array_equal(c[reg][band], cf[reg][band])        # binary64 there
    kept = reg[~band & (c[reg] > 0.0)]
    assert kept.size > 0 and st.points_partial > 0
    err = np.abs(G[kept] - Gf[kept])
    # the routing keeps a part when 2 u32 E <= 1e-6 |G| (a quarter of that for
    # a partially routed point's kept groups); the binary32 error is a small
    # multiple of u32 E (median 0.25-0.45, at most 3.5 over the production
    # grids when the factor 2 was calibrated)
    ratio = err / (U32 * c[kept])
    k = int(np.argmax(ratio))
    assert ratio[k] <= 4.0, f"error {err[k]:.3e} = {ratio[k]:.2f} u32 E at x = {x[kept[k]]}"
    assert np.median(ratio) <= 1.0
    assert np.all(2.0 * U32 * c[kept] <= 1e-6 * np.abs(G[kept]) * (1 + 1e-3))
    tau = 1e-3 * np.max(np.abs(Gf[reg]))
    assert np.all(np.abs(G[reg] - Gf[reg]) <= 1e-6 * np.maximum(np.abs(Gf[reg]), tau))


def test_mixed_fp64_fallback_equals_the_fp64_call_bitwise():
    # the sample plus points of the cut band (within 0.05 of x <= -4)
    band = np.array([-4.5 + 0.01j, -6 - 0.03j, -9 + 0.02j, -3.98 + 0.02j])
    x = np.concatenate([band, _points(128, seed=13)])
    G, c = _cond(SCALAR, dict(PAR, precision="mixed", mixed_fallback="fp64"), x)
    routed = gfc.last_stats().points_fp64
    Gf, cf = _cond(SCALAR, dict(PAR, precision="fp64"), x)
    # the band goes whole to the binary64 kernel, which computes exactly what
    # it computes on all points, scale included
    assert routed >= band.size
    assert np.array_equal(G[: band.size], Gf[: band.size])
    assert np.array_equal(c[: band.size], cf[: band.size])
    # points next to a pinch go whole to the fallback kernel, here binary64:
    # the same sums (their scale is 0, nothing being kept in binary32)
    pinch = np.flatnonzero(c[band.size:] == 0.0)[: -len(SPECIAL)] + band.size
    assert np.all(np.abs(G[pinch] - Gf[pinch]) <= 1e-13 * np.abs(Gf[pinch]))


def test_double_float_writes_zero_scale():
    x = _points(64, seed=14)
    G, c = _cond(SCALAR, dict(PAR, precision="f32x2"), x)
    assert np.all(c == 0.0)
    assert np.all(np.isfinite(G[: x.size - 2]))
