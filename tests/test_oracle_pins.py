"""Pins of the oracle against what the paper and the mathematics fix.

The oracle (oracle/) is a plain FP64 evaluation of the paper's quadrature.
These tests check it against values that do not come from it: the paper's
closed form eq. 18 (golden file), textbook bubble closed forms, exact analytic
continuations of the Feynman-parameter form, invariants (Schwarz reflection,
G(mu2) = 0, reality on the spacelike axis, the threshold at -4 m^2), cut-off
independence (Sect. 2, Step 2) and a library Gauss-Legendre rule. A last test
compiles the oracle with planted mistakes and shows that each one fails a pin.
"""
import json
import os

import numpy as np
import pytest

import oracle
from closed_forms import G_exact, dressed_poles

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
PI = np.pi

with open(os.path.join(GOLD, "paper_example.json")) as f:
    PAPER = json.load(f)
PAPER_PROP = {"kind": "cpair", "mk2": complex(*PAPER["mk2"]), "mq2": complex(*PAPER["mq2"])}


def _eq18_golden():
    rows = np.loadtxt(os.path.join(GOLD, "eq18_values.txt"))
    x = rows[:, 2] + 1j * rows[:, 3]
    g = rows[:, 4] + 1j * rows[:, 5]
    return rows[:, :2].astype(int), x, g


def _dist_to_cut(x, threshold):
    """distance from x to the half-line (-inf, threshold] of the real axis"""
    x = np.asarray(x)
    return np.where(x.real <= threshold, np.abs(x.imag), np.abs(x - threshold))


# bulk points of the 64 x 64 bubble rectangle [-8,4] x [-4,4], all quadrants,
# at least 0.5 away from the real axis where Re x < 0
BULK = np.array([2 + 1j, 1 - 3j, -1 + 1j, -1 + 3j, -3 + 1j, -3 + 3j, -3 - 3j, -0.5 + 4j,
                 0.3 + 0.2j, -6 - 2j, -7.5 + 3.5j, 3.9 - 3.9j, -5 + 0.7j, 0.1 - 0.05j])


def test_gauss_legendre_matches_library_rule():
    for n in (1, 2, 3, 7, 64, 256, 2048):
        x, w = oracle.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.max(np.abs(x - xr)) < 1e-14
        # numpy's own end weights lose accuracy as n grows (~1e-11 at 256,
        # ~1e-7 at 2048), so compare with it only up to n = 256
        if n <= 256:
            assert np.max(np.abs(w - wr) / wr) < 5e-11
        # exact for polynomials of degree < 2n: sum w x^k = 2/(k+1), k even
        for k in range(0, min(2 * n, 40), 2):
            assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) < 1e-13


def test_grid_is_the_papers_cell_centred_grid():
    ij, xg, _ = _eq18_golden()
    g = PAPER["grid"]
    X = oracle.grid_points(g["re0"], g["re1"], g["im0"], g["im1"], g["m"], g["n"])
    assert X.shape == (g["m"] * g["n"],)
    assert np.array_equal(X[ij[:, 0] * g["n"] + ij[:, 1]], xg)
    # no grid point on the real axis
    assert np.min(np.abs(X.imag)) > 0


def test_paper_worked_example_matches_eq18():
    """Sect. 5: the detoured contours and the leg relabelling reproduce eq. 18."""
    _, x, g18 = _eq18_golden()
    par = dict(dim=4, mu2=0.0, n_radial=1024, n_angular=128)
    G = oracle.eval_points(PAPER_PROP, par, x)
    err = np.abs(16 * PI ** 2 * G - g18) / np.abs(g18)
    d = _dist_to_cut(x, PAPER["threshold"])
    bulk = d > 0.2
    assert bulk.sum() >= 15
    assert np.max(err[bulk]) < 1e-11, err[bulk]
    # next to the cut the quadrature converges slowly, but it converges
    assert np.max(err[~bulk]) < 2e-2


def test_paper_example_at_the_papers_node_counts():
    """ngl = 64 per sub-contour suffices in well-behaved areas (Sect. 4):
    n_radial = 4 * 64 gives 64 nodes on each detour piece."""
    _, x, g18 = _eq18_golden()
    par = dict(dim=4, mu2=0.0, n_radial=4 * PAPER["ngl"], n_angular=64)
    G = oracle.eval_points(PAPER_PROP, par, x)
    err = np.abs(16 * PI ** 2 * G - g18) / np.abs(g18)
    bulk = _dist_to_cut(x, PAPER["threshold"]) > 1.0
    assert np.max(err[bulk]) < 1e-4


@pytest.mark.parametrize("dim", [4, 3])
@pytest.mark.parametrize("m2", [0.25, 1.0, 4.0])
def test_scalar_bubble_closed_form(dim, m2):
    prop = {"kind": "scalar", "m2": m2}
    par = dict(dim=dim, mu2=1.0, n_radial=2048, n_angular=256)
    # 0.2 rad or more away from the negative real axis, where the angular
    # integrand nearly pinches and the quadrature converges slowly
    xs = BULK[np.pi - np.abs(np.angle(BULK)) > 0.2]
    G = oracle.eval_points(prop, par, xs)
    ref = np.array([G_exact(prop, x, dim, 1.0) for x in xs])
    err = np.abs(G - ref) / np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
    assert np.max(err) < 1e-10, err


@pytest.mark.parametrize("dim", [4, 3])
@pytest.mark.parametrize("abc", [(1.0, 0.5, 2.0), (1.3, 0.0, 2.5), (0.7, 0.9, 1.2)])
def test_dressed_closed_form(dim, abc):
    a, b, c = abc
    prop = {"kind": "dressed", "a": a, "b": b, "c": c}
    (yp, _), _ = dressed_poles(a, b, c)
    # stay 10 degrees away from the rays arg x = +-arg y+, where the k-leg pole
    # grazes the radial path and the quadrature converges slowly
    keep = np.abs(np.abs(np.angle(BULK)) - np.angle(yp)) > np.radians(10)
    xs = BULK[keep]
    par = dict(dim=dim, mu2=1.0, n_radial=2048, n_angular=256)
    G = oracle.eval_points(prop, par, xs)
    ref = np.array([G_exact(prop, x, dim, 1.0) for x in xs])
    err = np.abs(G - ref) / np.abs(ref)
    assert np.max(err) < 1e-10, err


@pytest.mark.parametrize("prop", [
    {"kind": "scalar", "m2": 1.0},
    PAPER_PROP,
    {"kind": "dressed", "a": 1.0, "b": 0.5, "c": 2.0},
])
@pytest.mark.parametrize("dim", [3, 4])
def test_schwarz_reflection(prop, dim):
    """G(conj x) = conj G(x); for the conjugate-pair legs the two half-planes
    use different leg assignments and detours, so this is not automatic."""
    xs = np.array([2 + 1j, -1 + 1j, -3 + 3j, -0.5 + 4j, -6 + 2j, 0.3 + 0.1j])
    par = dict(dim=dim, mu2=1.0, n_radial=512, n_angular=64)
    G = oracle.eval_points(prop, par, np.concatenate([xs, np.conj(xs)]))
    n = xs.size
    assert np.max(np.abs(G[n:] - np.conj(G[:n])) / np.abs(G[:n])) < 1e-13


def test_subtraction_point_and_spacelike_axis():
    prop = {"kind": "scalar", "m2": 1.0}
    par = dict(dim=4, mu2=1.0, n_radial=512, n_angular=64)
    G = oracle.eval_points(prop, par, np.array([1.0 + 0j, 0.5, 3.0, 7.0]))
    assert G[0] == 0
    # real on the spacelike axis x > 0
    assert np.max(np.abs(G.imag)) < 1e-17
    assert np.all(np.abs(G[1:].real) > 1e-5)
    # the paper example is real on (-1, inf) too, in particular at x > 0
    G2 = oracle.eval_points(PAPER_PROP, dict(dim=4, mu2=0.0, n_radial=512, n_angular=64),
                            np.array([0.5 + 0j, 2.0, 4.0]))
    assert np.max(np.abs(G2.imag)) < 1e-17


def test_branch_cut_opens_at_threshold():
    """16 pi^2 Im G(x + i0) = -pi sqrt(1 + 4 m^2/x) below x = -4 m^2 and 0
    above it (D = 4, real mass); checked 0.05 off the axis, where the
    quadrature with 4096 x 2048 nodes has converged, so the limits hold up to
    O(0.05)."""
    prop = {"kind": "scalar", "m2": 1.0}
    par = dict(dim=4, mu2=1.0, n_radial=4096, n_angular=2048)
    d = 0.05
    xs = np.array([-2.0, -3.0, -5.0, -6.0]) + 1j * d
    G = 16 * PI ** 2 * oracle.eval_points(prop, par, np.concatenate([xs, np.conj(xs)]))
    above, below = G[:4], G[4:]
    assert np.max(np.abs(above[:2].imag)) < 0.05
    lim = -PI * np.sqrt(1 + 4 / xs[2:].real)
    assert np.max(np.abs(above[2:].imag - lim)) < 0.05
    assert np.max(np.abs(below[2:].imag + lim)) < 0.05


def test_cutoff_independence():
    """The subtracted integral does not depend on where the radial path is cut
    (Sect. 2, Step 2): changing the scale L of |q| = L t/(1-t) changes nothing."""
    prop = {"kind": "dressed", "a": 0.7, "b": 0.9, "c": 1.2}
    xs = np.array([2 + 1j, -3 + 1j, -2 - 1j])
    res = []
    for L in (0.5, 1.0, 2.0):
        res.append(oracle.eval_points(prop, dict(dim=4, mu2=1.0, n_radial=1024, n_angular=128,
                                                 radial_scale=L), xs))
    assert np.max(np.abs(res[0] - res[1]) / np.abs(res[1])) < 1e-11
    assert np.max(np.abs(res[2] - res[1]) / np.abs(res[1])) < 1e-11


def test_convergence_under_refinement():
    prop = {"kind": "scalar", "m2": 1.0}
    x = np.array([-2 + 0.5j])
    ref = G_exact(prop, x[0], 4, 1.0)
    errs = [abs(oracle.eval_points(prop, dict(dim=4, mu2=1.0, n_radial=nr, n_angular=na), x)[0]
                - ref) for nr, na in ((128, 32), (512, 128), (2048, 256))]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5 * abs(ref)


@pytest.mark.parametrize("dim", [3, 4])
@pytest.mark.parametrize("rule,n", [("gl", 64), ("tanh-sinh", 49), ("tanh-sinh", 97),
                                    ("chebyshev1", 64), ("chebyshev2", 64)])
def test_angular_rule_moments(rule, n, dim):
    """Sect. 4's angular rules against the moments int_0^pi cos^(2k) psi
    sin^(D-2) psi dpsi = Gamma(k + 1/2) Gamma((D-1)/2) / Gamma(k + D/2):
    Gauss rules are exact to their degree, tanh-sinh converges doubly
    exponentially, the Chebyshev rules are Gaussian for the weight of one
    dimension only (2nd kind: D = 4) and converge algebraically for D = 3."""
    from math import gamma
    z, w = oracle.angular_rule(rule, n, dim)
    assert np.all(np.abs(z) < 1.0) and np.all(w > 0.0)
    assert np.max(np.abs(np.sort(z) + np.sort(z)[::-1])) < 1e-15       # symmetric in z
    exact = np.array([gamma(k + 0.5) * gamma((dim - 1) / 2) / gamma(k + dim / 2) for k in range(12)])
    got = np.array([np.sum(w * z ** (2 * k)) for k in range(12)])
    err = np.abs(got - exact) / exact
    if rule == "gl" or (rule.startswith("chebyshev") and dim == 4):
        assert err.max() < 1e-13
    elif rule == "tanh-sinh":
        assert err[:4].max() < (1e-13 if n > 64 else 1e-11) and err.max() < 1e-8
    else:
        z4, w4 = oracle.angular_rule(rule, 4 * n, dim)
        err4 = abs(np.sum(w4) - exact[0]) / exact[0]
        assert 1e-6 < err[0] < 1e-2 and err4 < err[0] / 8          # O(n^-2)


@pytest.mark.parametrize("rule,n,tol", [("gl", 64, 1e-12), ("tanh-sinh", 97, 1e-11),
                                        ("chebyshev1", 64, 1e-12), ("chebyshev2", 64, 1e-12)])
def test_angular_rules_reach_the_closed_form(rule, n, tol):
    """Every angular rule reproduces the D = 4 bubble's closed form away from
    the negative real axis; the paper's 49-node tanh-sinh rule is exact there
    only where the integrand is benign and improves with the order."""
    prop = {"kind": "scalar", "m2": 1.0}
    xs = np.array([2 + 1j, -2 + 3j, 0.5 - 2j])
    ref = np.array([G_exact(prop, x, 4, 1.0) for x in xs])
    G = oracle.eval_points(prop, dict(dim=4, mu2=1.0, n_radial=1024, n_angular=n,
                                      angular_rule=rule), xs)
    assert np.max(np.abs(G - ref) / np.abs(ref)) < tol
    G49 = oracle.eval_points(prop, dict(dim=4, mu2=1.0, n_radial=1024, n_angular=49,
                                        angular_rule="tanh-sinh"), xs)
    e49 = np.abs(G49 - ref) / np.abs(ref)
    assert e49[0] < 1e-13 and e49[1] > np.max(np.abs(G - ref)[1] / np.abs(ref[1]))


@pytest.mark.parametrize("dim", [3, 4])
@pytest.mark.parametrize("prop", [{"kind": "scalar", "m2": 1.0},
                                  {"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j},
                                  {"kind": "dressed", "a": 1.0, "b": 0.5, "c": 2.0}])
def test_exact_angular_is_the_limit_of_the_rules(prop, dim):
    """The closed-form psi integral (written from int sin^(D-2)/(A - B cos psi))
    is the n -> infinity limit of the Gauss-Legendre rule, on rays and detours."""
    xs = np.array([2 + 1j, -2 + 3j, 0.5 - 2j, -1 - 1.5j, 3 + 0.2j])
    mu2 = 0.0 if prop["kind"] == "cpair" else 1.0
    base = dict(dim=dim, mu2=mu2, n_radial=512)
    Ge = oracle.eval_points(prop, dict(base, n_angular=2, angular_rule="exact"), xs)
    Gq = oracle.eval_points(prop, dict(base, n_angular=1024), xs)
    assert np.max(np.abs(Ge - Gq) / np.abs(Gq)) < 1e-11


@pytest.mark.parametrize("dim", [3, 4])
def test_exact_angular_closes_the_near_axis_gap(dim):
    """Next to the negative real axis the angular rule's error dominates (the
    integrand nearly pinches); with the psi integral in closed form the radial
    rule alone decides, and refining it reaches the closed form."""
    prop = {"kind": "scalar", "m2": 1.0}
    xs = np.array([-2 + 0.0625j, -6 + 0.0625j])
    ref = np.array([G_exact(prop, x, dim, 1.0) for x in xs])
    gl = oracle.eval_points(prop, dict(dim=dim, mu2=1.0, n_radial=8192, n_angular=256), xs)
    ex = oracle.eval_points(prop, dict(dim=dim, mu2=1.0, n_radial=8192, n_angular=2,
                                       angular_rule="exact"), xs)
    e_gl = np.abs(gl - ref) / np.abs(ref)
    e_ex = np.abs(ex - ref) / np.abs(ref)
    assert np.all(e_gl > 1e-3) and np.all(e_ex < 1e-8)


def test_exact_angular_dressed_closed_form():
    """The dressed propagator with the closed-form psi integral against its
    partial-fraction closed forms (D = 4 and 3, b = 0 and b > 0)."""
    for dim in (3, 4):
        for abc in ((1.0, 0.0, 2.0), (1.0, 0.5, 2.0)):
            prop = {"kind": "dressed", "a": abc[0], "b": abc[1], "c": abc[2]}
            xs = np.array([1.5 + 1j, -1 + 2j, 0.5 - 3j])
            ref = np.array([G_exact(prop, x, dim, 1.0) for x in xs])
            G = oracle.eval_points(prop, dict(dim=dim, mu2=1.0, n_radial=2048, n_angular=2,
                                              angular_rule="exact"), xs)
            assert np.max(np.abs(G - ref) / np.abs(ref)) < 1e-9, (dim, abc)


@pytest.mark.parametrize("m2", [0.25, 1.0])
def test_region_map_is_the_parabola(m2):
    """Region 1 of Fig. 2 for a real mass: the real-axis y contour is free of
    the angular integral's cut exactly inside Im^2 x < 4 m^2 (Re x + m^2), the
    parabola of the figure (found here from the pole condition w = 4 x y/
    (x + y + m^2)^2 >= 1 real on y > 0)."""
    re = np.linspace(-9.9, 4.9, 75)
    im = np.linspace(-4.9, 4.9, 61)
    x = (re[:, None] + 1j * im[None, :]).ravel()
    got = oracle.region_map({"kind": "scalar", "m2": m2}, x)
    par = (x.imag ** 2 < 4 * m2 * (x.real + m2)).astype(np.int32)
    far = np.abs(x.imag ** 2 - 4 * m2 * (x.real + m2)) > 0.02
    assert np.array_equal(got[far], par[far])
    assert 0.1 < got.mean() < 0.9


@pytest.mark.parametrize("dim", [3, 4])
@pytest.mark.parametrize("prop", [{"kind": "scalar", "m2": 1.0},
                                  {"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j},
                                  {"kind": "dressed", "a": 1.0, "b": 0.5, "c": 2.0}])
def test_angular_map_rule_converges_to_closed_form(prop, dim):
    """B(x, y) by the plain sum over a 1024-node rule against the closed form
    at y away from the cut (Fig. 1's integral B)."""
    x = 1.5 + 0.5j
    y = np.array([0.3 + 0.1j, 2.0 - 1.0j, 5.0 + 3.0j, 0.05 + 0.02j, 10.0 - 0.5j])
    q = oracle.angular_map(prop, dict(dim=dim, n_radial=4, n_angular=1024), x, y)
    e = oracle.angular_map(prop, dict(dim=dim, n_radial=4, n_angular=2, angular_rule="exact"),
                           x, y)
    assert np.max(np.abs(q - e) / np.abs(e)) < 1e-11


def test_angular_map_jumps_across_the_cut():
    """Across the branch cut of eq. 25 B is discontinuous; along it and away
    from it B is continuous (the paper's example, Fig. 1)."""
    prop = {"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j}
    par = dict(dim=4, n_radial=4, n_angular=2, angular_rule="exact")
    x = -2.0 + 1.0j
    th = 1.1
    k = np.sqrt(x) * np.cos(th) + np.sqrt(-x * np.sin(th) ** 2 + 0.5j)   # eq. 24, s = -Mq2
    yc = k ** 2                                                           # eq. 25
    dk = np.sqrt(x) * np.cos(th + 1e-4) + np.sqrt(-x * np.sin(th + 1e-4) ** 2 + 0.5j)
    tang = dk ** 2 - yc
    nrm = 1j * tang / abs(tang)
    eps = 1e-7
    across = oracle.angular_map(prop, par, x, [yc + eps * nrm, yc - eps * nrm])
    along = oracle.angular_map(prop, par, x, [yc + eps * nrm, yc + eps * nrm + 1e-6 * tang / abs(tang)])
    assert abs(across[0] - across[1]) > 1e-2 * abs(across[0])
    assert abs(along[0] - along[1]) < 1e-4 * abs(along[0])


@pytest.mark.parametrize("dim", [3, 4])
def test_clustered_radial_rule_beyond_threshold(dim):
    """Beyond threshold next to the negative real axis the ray passes within
    ~|Im x|/|x| of the pole y = -m^2; with the angle in closed form the
    sinh-clustered radial rule resolves it at 2048 nodes where the mapped
    rule is off by O(1) or more, and leaves benign points as accurate."""
    prop = {"kind": "scalar", "m2": 1.0}
    near = np.array([-4.5 + 0.01j, -6 + 0.0625j, -9 + 0.3j, -3.9 + 0.01j])
    benign = np.array([2 + 1j, -8 + 2j, -1 - 1j])
    base = dict(dim=dim, mu2=1.0, n_radial=2048, n_angular=2, angular_rule="exact")
    for xs, bound in ((near, 1e-4), (benign, 1e-12)):
        ref = np.array([G_exact(prop, x, dim, 1.0) for x in xs])
        cl = oracle.eval_points(prop, dict(base, radial_rule="clustered"), xs)
        assert np.max(np.abs(cl - ref) / np.abs(ref)) < bound
    mp = oracle.eval_points(prop, base, near[:1])
    assert abs(mp[0] - G_exact(prop, near[0], dim, 1.0)) > 1.0 * abs(G_exact(prop, near[0], dim, 1.0))


def test_clustered_radial_rule_dressed_and_pair():
    """The clustered rule with the dressed propagator and the paper's complex
    pair: still the closed forms at points of every kind of contour."""
    for prop, mu2 in (({"kind": "dressed", "a": 1.0, "b": 0.5, "c": 2.0}, 1.0),
                      ({"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j}, 0.0)):
        xs = np.array([1.5 + 1j, -1 + 2j, 0.5 - 3j, -3 + 0.2j, -2 - 0.1j])
        ref = np.array([G_exact(prop, x, 4, mu2) for x in xs])
        G = oracle.eval_points(prop, dict(dim=4, mu2=mu2, n_radial=2048, n_angular=2,
                                          angular_rule="exact", radial_rule="clustered"), xs)
        assert np.max(np.abs(G - ref) / np.abs(ref)) < 1e-8, prop


def test_condition_number_reported():
    """kappa = sum|terms|/|sum| grows as x approaches the negative real axis,
    where the angular integrand nearly pinches."""
    prop = {"kind": "scalar", "m2": 1.0}
    xs = np.array([2 + 1j, -2 + 0.1j, -2 + 0.02j])
    G, kap = oracle.eval_points(prop, dict(dim=4, mu2=1.0, n_radial=2048, n_angular=256),
                                xs, with_kappa=True)
    assert 1.0 <= kap[0] < 10 < kap[1] < kap[2]


@pytest.mark.parametrize("bad", [
    dict(dim=5), dict(n_angular=1), dict(n_radial=250), dict(radial_scale=0.0),
    dict(angular_rule="tanh-sinh"), dict(angular_rule=7),
])
def test_rejects_bad_parameters(bad):
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=64)
    par.update(bad)
    with pytest.raises(ValueError):
        oracle.eval_points({"kind": "scalar", "m2": 1.0}, par, np.array([1 + 1j]))


def test_rejects_bad_inputs():
    par = dict(dim=4, mu2=1.0, n_radial=256, n_angular=64)
    with pytest.raises(ValueError):   # on the cut side of the real axis
        oracle.eval_points({"kind": "scalar", "m2": 1.0}, par, np.array([-2 + 0j]))
    with pytest.raises(ValueError):   # b^2 >= 4c: no conjugate poles
        oracle.eval_points({"kind": "dressed", "a": 1, "b": 3, "c": 2}, par, np.array([1 + 1j]))
    with pytest.raises(ValueError):   # legs not a conjugate pair
        oracle.eval_points({"kind": "cpair", "mk2": 0.5j, "mq2": 0.4j}, par, np.array([1 + 1j]))


# --- planted mistakes -------------------------------------------------------

def _paper_err(orc):
    _, x, g18 = _eq18_golden()
    keep = _dist_to_cut(x, PAPER["threshold"]) > 0.2
    G = orc.eval_points(PAPER_PROP, dict(dim=4, mu2=0.0, n_radial=512, n_angular=64), x[keep])
    return np.max(np.abs(16 * PI ** 2 * G - g18[keep]) / np.abs(g18[keep]))


def _closed_err(orc, prop, dim):
    (yp, _), _ = dressed_poles(1.0, 0.5, 2.0)
    keep = (np.abs(np.abs(np.angle(BULK)) - np.angle(yp)) > np.radians(10)) & \
        (np.pi - np.abs(np.angle(BULK)) > 0.2)
    xs = BULK[keep]
    G = orc.eval_points(prop, dict(dim=dim, mu2=1.0, n_radial=1024, n_angular=128), xs)
    ref = np.array([G_exact(prop, x, dim, 1.0) for x in xs])
    return np.max(np.abs(G - ref) / np.abs(ref))


def _grid_err(orc):
    ij, xg, _ = _eq18_golden()
    g = PAPER["grid"]
    X = orc.grid_points(g["re0"], g["re1"], g["im0"], g["im1"], g["m"], g["n"])
    return np.max(np.abs(X[ij[:, 0] * g["n"] + ij[:, 1]] - xg))


DRESSED = {"kind": "dressed", "a": 1.0, "b": 0.5, "c": 2.0}
SCALAR = {"kind": "scalar", "m2": 1.0}
MUTANT_PINS = {
    1: lambda o: _paper_err(o),
    2: lambda o: _paper_err(o),
    3: lambda o: _closed_err(o, DRESSED, 3),
    4: lambda o: _closed_err(o, SCALAR, 4),
    5: lambda o: _closed_err(o, SCALAR, 3),
    6: lambda o: _closed_err(o, SCALAR, 4),
    7: lambda o: _closed_err(o, DRESSED, 4),
    8: lambda o: _grid_err(o),
    9: lambda o: _paper_err(o),
    10: lambda o: _closed_err(o, DRESSED, 4),
}


@pytest.mark.parametrize("n", sorted(MUTANT_PINS))
def test_planted_mistake_fails_a_pin(n, tmp_path):
    pin = MUTANT_PINS[n]
    # the oracle as written passes the pin at this resolution ...
    good = pin(oracle.Oracle(oracle._load()))
    assert good < 1e-4
    # ... and the oracle with mistake n compiled in fails it
    bad = pin(oracle.mutant(n, str(tmp_path)))
    assert not (bad < 1e-2), f"mutant {n} passed its pin (err {bad})"
