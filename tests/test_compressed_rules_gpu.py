"""The compressed angular rules reproduce the full 2048 x 256 quadrature on the
whole production grid.

Per radial node the kernels sum the angular integral over the smallest Gauss
rule of the pair table's own discrete measure that is exact to rounding for
that node (the selection runs in binary32 and is made uniform over a warp).
Here every point of the 1024 x 1024 production grid, for each mass, is
evaluated twice through the C ABI: with the compressed rules (the benchmark's
launch) and with the full angular table (gfc_test_full_angular_rule). The two
must agree to rounding level at every point: relative to max(|G|, tau) within
1e-12, and in absolute terms within a small multiple of the unit roundoff
times the point's rounding-error scale E (gfc_eval_points_cond), which is
what rounding-level agreement means where the sum cancels.

The error-scale call evaluates the scalar bubble's nodes by the general node
code, the plain call by the code in the frame of the ray; both are checked
against each other at rounding level too.
"""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_0752_gb300 as gfc  # noqa: E402
from paper_1205_0752_gb300 import binding  # noqa: E402

U64 = 2.0 ** -53


@pytest.mark.parametrize("m2", [0.25, 1.0, 4.0])
def test_compressed_equals_full_rule_on_the_production_grid(m2):
    prop = {"kind": "scalar", "m2": m2}
    par = dict(dim=4, mu2=1.0, n_radial=2048, n_angular=256, precision="fp64")
    x = gfc.grid_points((*si.grid_rect("production"), 1024, 1024)).reshape(-1)
    Gg, E = gfc.eval_points_cond(prop, par, x)
    Gc = gfc.eval_points(prop, par, x)
    st = gfc.last_stats()
    assert 0 < st.pairs_evaluated < st.node_evals // 2      # the compressed rules were used
    binding.test_full_angular_rule(True)
    try:
        Gf = gfc.eval_points(prop, par, x)
        stf = gfc.last_stats()
    finally:
        binding.test_full_angular_rule(False)
    assert stf.pairs_evaluated == stf.node_evals // 2        # every pair of the full table
    torch.cuda.synchronize()
    gc, gf, gg, e = Gc.cpu().numpy(), Gf.cpu().numpy(), Gg.cpu().numpy(), E.cpu().numpy()
    d = np.abs(gc - gf)
    tau = 1e-3 * np.max(np.abs(gf))
    rel = d / np.maximum(np.abs(gf), tau)
    scaled = d / (U64 * e)
    k = int(np.argmax(rel))
    print(f"m2={m2}: max rel {rel.max():.2e} (median {np.median(rel):.1e}) at x={x.cpu().numpy()[k]}, "
          f"max |dG|/(u E) {scaled.max():.2f}")
    assert np.all(np.isfinite(gc)) and np.all(np.isfinite(gf))
    assert rel.max() <= 1e-12, (rel.max(), x.cpu().numpy()[k])
    assert scaled.max() <= 64.0
    # the general node code (compressed rules) against the frame of the ray
    dg = np.abs(gg - gc)
    relg = dg / np.maximum(np.abs(gf), tau)
    print(f"m2={m2}: general vs ray-frame node code: max rel {relg.max():.2e}, "
          f"max |dG|/(u E) {(dg / (U64 * e)).max():.2f}")
    assert np.all(np.isfinite(gg))
    assert relg.max() <= 1e-11
    assert (dg / (U64 * e)).max() <= 64.0
