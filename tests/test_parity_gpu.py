"""Parity of the CUDA path (through the C ABI) with the oracle.

Element by element on seeded inputs at sizes the oracle finishes in seconds
(several tiles of 32-lane node slices, ragged tails), and at the full
production size on seeded samples. Tolerances (relative, with a floor tau =
1e-3 max|G| that guards the zero at x = mu2): 1e-10 for FP64, 1e-6 for MIXED.
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

RTOL = {"fp64": 1e-10, "mixed": 1e-6, "f32x2": 1e-10}


def rel_err(G, ref, floor_frac=1e-3):
    G = np.asarray(G).ravel()
    ref = np.asarray(ref).ravel()
    tau = floor_frac * np.max(np.abs(ref))
    return np.abs(G - ref) / np.maximum(np.abs(ref), tau)


def assert_parity(G, ref, rtol, x=None, what=""):
    e = rel_err(G, ref)
    k = int(np.argmax(e))
    where = f" at x={np.asarray(x).ravel()[k]}" if x is not None else ""
    assert e[k] <= rtol, f"{what}: max rel err {e[k]:.3e}{where} (G={np.ravel(G)[k]}, ref={np.ravel(ref)[k]})"


def oracle_params(p):
    return {k: p[k] for k in ("dim", "mu2", "n_radial", "n_angular", "radial_scale",
                              "detour_radius", "angular_rule", "radial_rule") if k in p}


def run_grid(prop, params, rect, m, n):
    G = gfc.eval_grid(prop, params, (*rect, m, n))
    torch.cuda.synchronize()
    return G.cpu().numpy()


SCALAR = {"kind": "scalar", "m2": 1.0}
PAPER = {"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j}


def test_grid_points_bit_exact():
    for rect, m, n in ((si.grid_rect("small"), 64, 64), (si.grid_rect("paper"), 128, 128),
                       ((-10.0, 5.0, -5.0, 5.0), 37, 53)):
        x = gfc.grid_points((*rect, m, n))
        torch.cuda.synchronize()
        xo = oracle.grid_points(*rect, m, n)
        assert np.array_equal(x.cpu().numpy().ravel(), xo)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
def test_bubble_64x64_grid(precision):
    """The 64 x 64 bubble grid (m = 1, D = 4, mu2 = 1, 256 x 64 nodes)."""
    rect = si.grid_rect("small")
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=64, precision=precision)
    G = run_grid(SCALAR, par, rect, 64, 64)
    x = oracle.grid_points(*rect, 64, 64)
    ref = oracle.eval_points(SCALAR, oracle_params(par), x)
    assert_parity(G, ref, RTOL[precision], x, f"bubble 64x64 {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
def test_paper_worked_example_grid(precision):
    """Sect. 5: 128 x 128 over [-5,5]^2, masses -+ i/2, x = 0 subtraction,
    64 nodes per sub-contour and 64 angular nodes."""
    rect = si.grid_rect("paper")
    par = dict(dim=4, mu2=0.0, n_radial=256, n_angular=64, precision=precision)
    G = run_grid(PAPER, par, rect, 128, 128)
    x = oracle.grid_points(*rect, 128, 128)
    ref = oracle.eval_points(PAPER, oracle_params(par), x)
    assert_parity(G, ref, RTOL[precision], x, f"paper example {precision}")


@pytest.mark.parametrize("dim", [3, 4])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
def test_dressed_grid(dim, precision):
    """Dressed propagator, a seeded (a, b, c) draw, ragged 48 x 40 grid."""
    a, b, c = si.dressed_draws(3, 1)[0]
    prop = {"kind": "dressed", "a": a, "b": b, "c": c}
    rect = si.grid_rect("small")
    par = dict(dim=dim, mu2=1.0, n_radial=512, n_angular=64, precision=precision)
    G = run_grid(prop, par, rect, 48, 40)
    x = oracle.grid_points(*rect, 48, 40)
    ref = oracle.eval_points(prop, oracle_params(par), x)
    assert_parity(G, ref, RTOL[precision], x, f"dressed D={dim} {precision}")


@pytest.mark.parametrize("n_angular", [2, 10, 64, 128, 256, 300])
def test_angular_orders_and_generic_path(n_angular):
    """Specialised (64, 128, 256) and generic angular orders, FP64."""
    xs = np.array([2 + 1j, -3 + 1j, -1 - 3j, 0.5 + 0.01j, -7 + 3.5j])
    par = dict(dim=4, mu2=1.0, n_radial=64, n_angular=n_angular, precision="fp64")
    G = gfc.eval_points(SCALAR, par, torch.tensor(xs, device="cuda"))
    torch.cuda.synchronize()
    ref = oracle.eval_points(SCALAR, oracle_params(par), xs)
    assert_parity(G.cpu().numpy(), ref, 1e-10, xs, f"n_angular={n_angular}")


@pytest.mark.parametrize("npts", [0, 1, 31, 33, 1000])
def test_ragged_point_counts(npts):
    g = si.SplitMix64(11)
    xs = np.array([complex(-8 + 12 * g.uniform(), -4 + 8 * g.uniform()) for _ in range(npts)])
    par = dict(dim=4, mu2=1.0, n_radial=128, n_angular=64, precision="fp64")
    xt = torch.tensor(xs, dtype=torch.complex128, device="cuda")
    G = gfc.eval_points(SCALAR, par, xt)
    torch.cuda.synchronize()
    if npts:
        ref = oracle.eval_points(SCALAR, oracle_params(par), xs)
        assert_parity(G.cpu().numpy(), ref, 1e-10, xs, f"npts={npts}")


def test_edge_points():
    """x = mu2 gives 0, the positive real axis is real, the negative real axis
    (cut side, undefined) gives NaN, the smallest contour (n_radial = 4)."""
    par = dict(dim=4, mu2=1.0, n_radial=4, n_angular=2, precision="fp64")
    xs = np.array([1.0 + 0j, 3.0 + 0j, -2.0 + 0j, 1e-9 + 1e-9j, 50.0 - 40.0j])
    G = gfc.eval_points(SCALAR, par, torch.tensor(xs, device="cuda")).cpu().numpy()
    assert G[0] == 0
    assert G[1].imag == 0 or abs(G[1].imag) < 1e-18
    assert np.isnan(G[2].real) and np.isnan(G[2].imag)
    ref = oracle.eval_points(SCALAR, oracle_params(par), xs[[0, 1, 3, 4]])
    assert_parity(G[[0, 1, 3, 4]], ref, 1e-10, xs[[0, 1, 3, 4]], "edge points")


def test_rejects_bad_arguments():
    x = torch.tensor([1 + 1j], dtype=torch.complex128, device="cuda")
    for bad in (dict(dim=5), dict(n_angular=1), dict(angular_rule="tanh-sinh", n_angular=8),
                dict(n_radial=6), dict(radial_scale=0.0)):
        with pytest.raises(gfc.GfcError):
            gfc.eval_points(SCALAR, dict(bad), x)
    with pytest.raises(gfc.GfcError):
        gfc.eval_points({"kind": "dressed", "a": 1, "b": 3, "c": 2}, {}, x)
    with pytest.raises(gfc.GfcError):   # the grid row Im x = 0 with Re x < 0
        gfc.eval_grid(SCALAR, {}, (-2.0, 1.0, -1.5, 1.5, 4, 3))


def test_host_path_matches_device_path():
    xs = oracle.grid_points(*si.grid_rect("small"), 16, 16)
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=64, precision="fp64")
    Gd = gfc.eval_points(SCALAR, par, torch.tensor(xs, device="cuda")).cpu().numpy()
    Gh = gfc.eval_points_host(SCALAR, par, xs)
    assert np.array_equal(Gd, Gh)


def test_row_shards_equal_unsharded():
    """Weak-scaling layout: disjoint row shards of a grid, evaluated as
    separate requests, reproduce the whole grid bit for bit."""
    rect = si.grid_rect("production")
    m, n = 64, 48
    par = dict(dim=4, mu2=1.0, n_radial=128, n_angular=64, precision="fp64")
    whole = run_grid(SCALAR, par, rect, m, n)
    x = oracle.grid_points(*rect, m, n).reshape(m, n)
    parts = []
    for r0, r1 in ((0, 20), (20, 41), (41, 64)):
        xs = torch.tensor(x[r0:r1].ravel(), device="cuda")
        parts.append(gfc.eval_points(SCALAR, par, xs).cpu().numpy().reshape(r1 - r0, n))
    assert np.array_equal(np.concatenate(parts), whole)


def test_interleaved_row_shards_match_the_whole_grid():
    """The benchmark's weak-scaling layout: rank r of N evaluates the rows
    i = r (mod N) of an (N side) x side grid over the production rectangle
    as a side x side grid of its own (bench.shard_rect). Each shard equals
    those rows of the whole grid; the coordinates agree to rounding (the
    shard's origin is computed apart), so the values agree to 1e-12."""
    import bench
    side, N = 16, 3
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=64, precision="fp64")
    whole = run_grid(SCALAR, par, si.grid_rect("production"), N * side, side)
    tau = 1e-3 * np.max(np.abs(whole))
    for r in range(N):
        part = run_grid(SCALAR, par, bench.shard_rect(r, N, side), side, side)
        ref = whole[r::N]
        assert np.max(np.abs(part - ref) / np.maximum(np.abs(ref), tau)) <= 1e-12, r


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
@pytest.mark.parametrize("m2", [0.25, 1.0, 4.0])
def test_production_grid_sampled(precision, m2):
    """1024 x 1024 over [-10,5] x [-5,5], 2048 x 256 nodes (the launch the
    benchmark times), checked on a seeded sample of 96 points."""
    prop = {"kind": "scalar", "m2": m2}
    rect = si.grid_rect("production")
    par = dict(dim=4, mu2=1.0, n_radial=2048, n_angular=256, precision=precision)
    G = run_grid(prop, par, rect, 1024, 1024).ravel()
    idx = si.sample_indices(2024, 1024 * 1024, 96)
    x = oracle.grid_points(*rect, 1024, 1024)[idx]
    ref = oracle.eval_points(prop, oracle_params(par), x)
    assert_parity(G[idx], ref, RTOL[precision], x, f"production m2={m2} {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
@pytest.mark.parametrize("dim", [3, 4])
def test_dressed_full_size_sampled(precision, dim):
    """The dressed workload at full size: 512 x 512 over [-8,4] x [-4,4],
    1024 x 128 nodes, two seeded (a, b, c) draws, 48 sampled points each."""
    rect = si.grid_rect("small")
    par = dict(dim=dim, mu2=1.0, n_radial=1024, n_angular=128, precision=precision)
    for k, (a, b, c) in enumerate(si.dressed_draws(3, 2)):
        prop = {"kind": "dressed", "a": a, "b": b, "c": c}
        G = run_grid(prop, par, rect, 512, 512).ravel()
        idx = si.sample_indices(300 + k, 512 * 512, 48)
        x = oracle.grid_points(*rect, 512, 512)[idx]
        ref = oracle.eval_points(prop, oracle_params(par), x)
        assert_parity(G[idx], ref, RTOL[precision], x, f"dressed 512^2 D={dim} draw {k} {precision}")


@pytest.mark.parametrize("fallback", ["f32x2", "fp64"])
@pytest.mark.parametrize("kind", ["bubble", "paper"])
def test_mixed_fallback_arithmetics(kind, fallback):
    """Mixed precision whose routed points go to the double-float kernel (the
    default) or to the binary64 kernel."""
    if kind == "bubble":
        prop, rect, m, n, mu2 = SCALAR, si.grid_rect("small"), 64, 64, 1.0
    else:
        prop, rect, m, n, mu2 = PAPER, si.grid_rect("paper"), 128, 128, 0.0
    par = dict(dim=4, mu2=mu2, n_radial=256, n_angular=64, precision="mixed",
               mixed_fallback=fallback)
    G = run_grid(prop, par, rect, m, n)
    x = oracle.grid_points(*rect, m, n)
    ref = oracle.eval_points(prop, oracle_params(par), x)
    assert_parity(G, ref, RTOL["mixed"], x, f"mixed/{fallback} {kind}")


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
@pytest.mark.parametrize("rule,n", [("tanh-sinh", 49), ("tanh-sinh", 65), ("chebyshev1", 64),
                                    ("chebyshev2", 64), ("chebyshev1", 63), ("gl", 63)])
def test_angular_rules(rule, n, precision):
    """The paper's angular rules (Sect. 4: tanh-sinh in z, Gauss-Chebyshev of
    both kinds) and odd orders, whose centre node pairs with itself; n = 63
    and 64 run the unrolled 32-pair kernels, 49 and 65 the generic loop."""
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=n, angular_rule=rule, precision=precision)
    rect = si.grid_rect("small")
    G = run_grid(SCALAR, par, rect, 48, 40)
    x = oracle.grid_points(*rect, 48, 40)
    ref = oracle.eval_points(SCALAR, oracle_params(par), x)
    assert_parity(G, ref, RTOL[precision], x, f"{rule} n={n} {precision}")


@pytest.mark.parametrize("dim", [3, 4])
def test_paper_rule_on_the_dressed_propagator(dim):
    """The paper's 49-node tanh-sinh rule with detours and two-term passes."""
    a, b, c = si.dressed_draws(3, 1)[0]
    prop = {"kind": "dressed", "a": a, "b": b, "c": c}
    par = dict(dim=dim, mu2=1.0, n_radial=512, n_angular=49, angular_rule="tanh-sinh")
    rect = si.grid_rect("small")
    G = run_grid(prop, par, rect, 32, 24)
    x = oracle.grid_points(*rect, 32, 24)
    ref = oracle.eval_points(prop, oracle_params(par), x)
    assert_parity(G, ref, RTOL["fp64"], x, f"dressed tanh-sinh D={dim}")


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
@pytest.mark.parametrize("case", ["bubble", "paper", "dressed3", "dressed4"])
def test_exact_angular(case, precision):
    """The psi integral in closed form (the kernel's own derivation, from the
    paired sum's v and w) against the oracle's (from int sin^(D-2)/(A - B cos
    psi)) on rays, detours and two-term dressed passes."""
    if case == "bubble":
        prop, rect, m, n, dim, mu2, nr = SCALAR, si.grid_rect("small"), 48, 40, 4, 1.0, 256
    elif case == "paper":
        prop, rect, m, n, dim, mu2, nr = PAPER, si.grid_rect("paper"), 64, 64, 4, 0.0, 256
    else:
        a, b, c = si.dressed_draws(3, 1)[0]
        prop = {"kind": "dressed", "a": a, "b": b, "c": c}
        rect, m, n, dim, mu2, nr = si.grid_rect("small"), 32, 24, int(case[-1]), 1.0, 512
    par = dict(dim=dim, mu2=mu2, n_radial=nr, n_angular=2, angular_rule="exact",
               precision=precision)
    G = run_grid(prop, par, rect, m, n)
    x = oracle.grid_points(*rect, m, n)
    ref = oracle.eval_points(prop, oracle_params(par), x)
    assert_parity(G, ref, RTOL[precision], x, f"exact angular {case} {precision}")


def test_exact_angular_production_sampled():
    """Production bubble grid (1024 x 1024, 8192 radial nodes) with the
    closed-form psi integral, on seeded samples the oracle computes one by one."""
    rect = si.grid_rect("production")
    par = dict(dim=4, mu2=1.0, n_radial=8192, n_angular=2, angular_rule="exact")
    G = run_grid(SCALAR, par, rect, 1024, 1024).ravel()
    idx = si.sample_indices(21, 1 << 20, 512)
    x = oracle.grid_points(*rect, 1024, 1024)[idx]
    ref = oracle.eval_points(SCALAR, oracle_params(par), x)
    assert_parity(G[idx], ref, RTOL["fp64"], x, "exact angular production")


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
@pytest.mark.parametrize("angular", ["exact", "gl"])
@pytest.mark.parametrize("case", ["bubble", "paper", "dressed3", "dressed4"])
def test_clustered_radial_rule(case, angular, precision):
    """The sinh-clustered radial rule (variant kernels) against the oracle's,
    with the closed-form angle and with the Gauss-Legendre rule."""
    if case == "bubble":
        prop, rect, m, n, dim, mu2 = SCALAR, si.grid_rect("small"), 48, 40, 4, 1.0
    elif case == "paper":
        prop, rect, m, n, dim, mu2 = PAPER, si.grid_rect("paper"), 48, 40, 4, 0.0
    else:
        a, b, c = si.dressed_draws(3, 1)[0]
        prop = {"kind": "dressed", "a": a, "b": b, "c": c}
        rect, m, n, dim, mu2 = si.grid_rect("small"), 32, 24, int(case[-1]), 1.0
    par = dict(dim=dim, mu2=mu2, n_radial=512, n_angular=2 if angular == "exact" else 64,
               angular_rule=angular, radial_rule="clustered", precision=precision)
    G = run_grid(prop, par, rect, m, n)
    x = oracle.grid_points(*rect, m, n)
    ref = oracle.eval_points(prop, oracle_params(par), x)
    # double-float carries ~48 bits; the clustered nodes come within d of a
    # pole, where a node's relative condition |y|/|y + M2| reaches ~1/d, so
    # its bound is 2^-48/d: 5e-10 here (d >= ~1e-4 on these grids)
    rtol = 5e-10 if precision == "f32x2" else RTOL[precision]
    assert_parity(G, ref, rtol, x, f"clustered {case} {angular} {precision}")


def test_clustered_near_axis_band():
    """Points within 0.05 of the negative real axis (beyond and below the
    threshold -4 m^2), 8192 radial nodes, closed-form angle: the case the
    clustered rule exists for."""
    re = np.linspace(-9.9, -0.1, 50)
    x = np.concatenate([re + 0.01j, re - 0.03j, re + 0.049j])
    par = dict(dim=4, mu2=1.0, n_radial=8192, n_angular=2, angular_rule="exact",
               radial_rule="clustered")
    G = gfc.eval_points(SCALAR, par, torch.tensor(x, device="cuda"))
    torch.cuda.synchronize()
    ref = oracle.eval_points(SCALAR, oracle_params(par), x)
    assert_parity(G.cpu().numpy(), ref, RTOL["fp64"], x, "clustered near-axis band")


_MAX_X = np.array([2 + 1j, -2 + 0.3j, -8 - 2j, 0.5 - 4j, -0.2 + 0.01j, 3.9 + 0.2j, -6 + 0.2j,
                   1e-3 + 1e-3j])
_MAX_REF = {}


@pytest.mark.parametrize("precision", ["fp64", "mixed", "f32x2"])
@pytest.mark.parametrize("name", ["scalar", "paper"])
def test_maximum_orders(name, precision):
    """The largest orders the library accepts: 16384 radial x 512 angular
    nodes (256 pairs: generic pair loop, the largest compressed rules), on
    points of every contour kind of the bubble and the paper's pair."""
    prop, mu2 = (SCALAR, 1.0) if name == "scalar" else (PAPER, 0.0)
    par = dict(dim=4, mu2=mu2, n_radial=16384, n_angular=512, precision=precision)
    G = gfc.eval_points(prop, par, torch.tensor(_MAX_X, device="cuda"))
    torch.cuda.synchronize()
    if name not in _MAX_REF:
        _MAX_REF[name] = oracle.eval_points(prop, oracle_params(par), _MAX_X)
    assert_parity(G.cpu().numpy(), _MAX_REF[name], RTOL[precision], _MAX_X,
                  f"max orders {name} {precision}")
