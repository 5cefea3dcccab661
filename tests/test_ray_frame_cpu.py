"""The ray-frame form of a contour node (the binary64 and double-float
kernels' node_rot) equals the general node form term by term.

Both are written out here in numpy complex128 from their definitions: the
general form builds y = r e2, a = x + y + M2, u = y/a, w = 4xy/a^2, the lead
(delta y - Omega (x + M2))/a - Omega1 w and the node factor
Jt P1(y)/(y + M2) / a; the ray-frame form uses only r and the per-pass
constants xi = (x + M2)/e2, eta = M2/e2, chi = 4x/e2 (g = 1/(r + xi),
h = 1/(r + eta), u = r g, w = chi u g, lead = (delta r - Omega xi) g -
Omega1 w, factor m (eD/e2^3) H h g). Three kinds of term: both legs on one
pole (H = h), the whole dressed propagator (H = R+ h+ + R- h-) and a k-leg
with a pole of its own (H = 1/(r + M2k/e2))."""
import numpy as np

RNG = np.random.default_rng(1205)


def general(x, r, e2, eD, m, m2, p1, Om, Om1, delta):
    y = r * e2
    a = x + y + m2
    u = y / a
    w = 4 * x * y / a ** 2
    lead = (delta * y - Om * (x + m2)) / a - Om1 * w
    f = (m * eD) * p1(y) / (y + m2) / a
    return u, w, lead, f


def ray_frame(x, r, e2, eD, m, m2, H, Om, Om1, delta):
    xi, eta, chi = (x + m2) / e2, m2 / e2, 4 * x / e2
    g, h = 1 / (r + xi), 1 / (r + eta)
    u = r * g
    w = chi * u * g
    lead = (delta * r - Om * xi) * g - Om1 * w
    f = m * (eD / e2 ** 3) * H(r, e2, h) * h * g
    return u, w, lead, f


def _case():
    x = complex(RNG.uniform(-10, 5), RNG.uniform(-5, 5))
    phi = np.angle(x)
    e2 = np.exp(1j * phi)
    dim = int(RNG.integers(3, 5))
    eD = e2 ** 2 if dim == 4 else e2 * np.exp(0.5j * phi)
    r = float(np.exp(RNG.uniform(-8, 12)))
    m = float(np.exp(RNG.uniform(-5, 5)))
    Om, Om1 = RNG.uniform(0.5, 2), RNG.uniform(0.1, 1)
    return x, r, e2, eD, m, Om, Om1, 4 * Om1 - Om


def _close(a, b):
    for p, q in zip(a, b):
        assert abs(p - q) <= 1e-12 * max(abs(q), 1e-300), (p, q)


def test_shared_pole():
    for _ in range(2000):
        x, r, e2, eD, m, Om, Om1, delta = _case()
        m2 = complex(RNG.uniform(0.1, 4), RNG.uniform(-2, 2) * RNG.integers(0, 2))
        G = general(x, r, e2, eD, m, m2, lambda y: 1 / (y + m2), Om, Om1, delta)
        R = ray_frame(x, r, e2, eD, m, m2, lambda r_, e, h: h, Om, Om1, delta)
        _close(R, G)


def test_whole_dressed_propagator():
    for _ in range(2000):
        x, r, e2, eD, m, Om, Om1, delta = _case()
        a, b, c = RNG.uniform(0.5, 2), RNG.uniform(0, 1), RNG.uniform(1, 4)
        yp = complex(-b / 2, np.sqrt(4 * c - b * b) / 2)
        ym = yp.conjugate()
        Rp = (yp + a) / (yp - ym)
        Rm = Rp.conjugate()
        D = lambda y: Rp / (y - yp) + Rm / (y - ym)
        s0 = complex(RNG.uniform(-3, 3), RNG.uniform(-3, 3))
        assert abs(D(s0) - (s0 + a) / (s0 * s0 + b * s0 + c)) <= 1e-12 * abs(D(s0))
        for m2, other in ((-yp, -ym), (-ym, -yp)):
            G = general(x, r, e2, eD, m, m2, D, Om, Om1, delta)
            hp = lambda r_, e, h: 1 / (r_ - yp / e)
            hm = lambda r_, e, h: 1 / (r_ - ym / e)
            R = ray_frame(x, r, e2, eD, m, m2,
                          lambda r_, e, h: Rp * hp(r_, e, h) + Rm * hm(r_, e, h), Om, Om1, delta)
            _close(R, G)


def test_distinct_k_leg_pole():
    for _ in range(2000):
        x, r, e2, eD, m, Om, Om1, delta = _case()
        yk = complex(RNG.uniform(-1, 1), RNG.uniform(0.1, 1))
        m2k, m2q = -yk, -yk.conjugate()
        G = general(x, r, e2, eD, m, m2q, lambda y: 1 / (y + m2k), Om, Om1, delta)
        R = ray_frame(x, r, e2, eD, m, m2q, lambda r_, e, h: 1 / (r_ + m2k / e), Om, Om1, delta)
        _close(R, G)
