"""Closed forms and exact analytic continuations that pin the oracle.

None of this imports the oracle or the product library. Everything here is a
textbook or paper formula evaluated independently of the 2-D quadrature:

* eq. 18 of the paper (its 4-D worked example, masses -+ i/2 on the two legs,
  subtracted at x = 0), evaluated with mpmath at 30 digits;
* the one-loop bubble with masses M1^2, M2^2 in D = 4 through its Feynman
  parameter form  16 pi^2 T(x) = -int_0^1 log(1 + a(1-a) x / D0(a)) da,
  D0(a) = a M2^2 + (1-a) M1^2, integrated in closed form over the roots of the
  quadratic and continued analytically along the arc |x| e^{i s arg x},
  s: 0 -> 1, from the positive real axis (where the straight Feynman integral
  is the momentum integral itself);
* the D = 3 bubble  T(x) = [h(x/(M1+M2)^2) - 1] / (4 pi (M1+M2)),
  h(u) = arctan(sqrt u)/sqrt u, principal roots M_i = sqrt(M_i^2).
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

mp.mp.dps = 30
PI = np.pi


def eq18(x: complex) -> complex:
    """Rescaled exact solution of the worked example, eq. 18 (= 16 pi^2 G)."""
    x = mp.mpc(x)
    if abs(x) < mp.mpf("1e-6"):
        # series of eq. 18 about 0: -pi x/4 + x^2/3 - pi x^3/16 + ...
        return complex(-mp.pi * x / 4 + x ** 2 / 3 - mp.pi * x ** 3 / 16)
    return complex(1 - mp.pi / (2 * x) + mp.sqrt(1 - x * x) / x * mp.acos(x))


def _gl(n, a, b):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * t + 0.5 * (b + a), 0.5 * (b - a) * w


_A = [_gl(800, 0.0, 0.5), _gl(800, 0.5, 1.0)]


def _feyn_straight(x: complex, M1: complex, M2: complex) -> complex:
    """int_0^1 log(1 + a(1-a)x/D0) da on the straight path, principal log."""
    s = 0.0
    for a, w in _A:
        s += np.sum(w * np.log(1 + a * (1 - a) * x / (a * M2 + (1 - a) * M1)))
    return complex(s)


def _near(prev: complex, new: complex) -> complex:
    return new + 2j * PI * np.round((prev - new).imag / (2 * PI))


def _I(L1, L0, r):
    """int_0^1 log(a - r) da given log(1-r) = L1 and log(-r) = L0."""
    return (1 - r) * L1 + r * L0 - 1


def bubble4(x: complex, M1: complex, M2: complex, steps: int = 4000) -> complex:
    """16 pi^2 * T(x), x = 0 subtracted, D = 4, analytic continuation from the
    positive real axis along the arc of radius |x|."""
    x = complex(x)
    M1, M2 = complex(M1), complex(M2)
    if x == 0:
        return 0j
    x0, ph = abs(x), np.angle(x)
    if abs(M1.real) < 1e-15 and abs(M2.real) < 1e-15 and abs(M1 + M2) < 1e-15 * abs(M1):
        # masses +- i kappa: D0(a) vanishes at a = 1/2 and the Feynman form does
        # not apply; the paper's eq. 17 gives the answer for kappa = 1/2 and
        # T(x; lambda M^2) = T(x/lambda; M^2) rescales it.
        return eq18(x / (2 * abs(M1.imag)))
    if abs(M1 - M2) < 1e-14 * max(1.0, abs(M1)):
        # equal masses: the analytic function is regular along the arc unless
        # the arc meets -4 M^2; integrate d/dx along the arc instead
        return _bubble4_equal_arc(x, M1, steps)
    r0 = M1 / (M1 - M2)
    xs = x0 * np.exp(1j * ph * np.linspace(0.0, 1.0, steps + 1))
    # roots of g(a) = -x a^2 + (x + M2 - M1) a + M1, followed continuously
    bq = xs + M2 - M1
    disc = np.sqrt(bq * bq + 4 * xs * M1)
    ra = (bq + disc) / (2 * xs)
    rb = (bq - disc) / (2 * xs)
    r1 = np.empty_like(ra)
    r2 = np.empty_like(rb)
    r1[0], r2[0] = ra[0], rb[0]
    for k in range(1, steps + 1):
        if abs(ra[k] - r1[k - 1]) + abs(rb[k] - r2[k - 1]) <= abs(rb[k] - r1[k - 1]) + abs(ra[k] - r2[k - 1]):
            r1[k], r2[k] = ra[k], rb[k]
        else:
            r1[k], r2[k] = rb[k], ra[k]

    def clog(z):
        return np.log(np.abs(z)) + 1j * np.unwrap(np.angle(z))

    c0 = _I(np.log(1 - r0), np.log(-r0), r0)
    Lx = clog(-xs / (M2 - M1))
    tot = Lx + _I(clog(1 - r1), clog(-r1), r1) + _I(clog(1 - r2), clog(-r2), r2) - c0
    ref = _feyn_straight(x0, M1, M2)
    off = 2j * PI * np.round((ref - tot[0]).imag / (2 * PI))
    assert abs(tot[0] + off - ref) < 1e-8 * max(1.0, abs(ref)), "start-point calibration failed"
    return complex(-(tot[-1] + off))


def _bubble4_equal_arc(x, M, steps):
    # 16 pi^2 T = 2 - beta log((beta+1)/(beta-1)), beta = sqrt(1 + 4 M/x); the
    # principal branches give the function cut along x in -4M [1, inf).
    beta = np.sqrt(1 + 4 * M / x)
    return complex(2 - beta * np.log((beta + 1) / (beta - 1)))


def _h(u: complex) -> complex:
    u = mp.mpc(u)
    if abs(u) < mp.mpf("1e-8"):
        return complex(1 - u / 3 + u * u / 5)
    su = mp.sqrt(u)
    return complex(mp.atan(su) / su)


def bubble3(x: complex, M1sq: complex, M2sq: complex) -> complex:
    """T(x) in D = 3 (physical normalisation d^3q/(2pi)^3), x = 0 subtracted."""
    S = complex(mp.sqrt(mp.mpc(M1sq)) + mp.sqrt(mp.mpc(M2sq)))
    return (_h(complex(x) / (S * S)) - 1.0) / (4 * PI * S)


def dressed_poles(a: float, b: float, c: float):
    yp = 0.5 * (-b + 1j * np.sqrt(4 * c - b * b))
    ym = np.conj(yp)
    Rp = (yp + a) / (yp - ym)
    Rm = (ym + a) / (ym - yp)
    return (yp, ym), (Rp, Rm)


def G_exact(prop: dict, x: complex, dim: int, mu2: float) -> complex:
    """G(x) = T(x) - T(mu2), physical normalisation int d^Dq/(2 pi)^D."""

    def T(xx):
        kind = prop["kind"]
        if kind == "scalar":
            m2 = float(prop["m2"])
            terms = [(1.0, m2, m2)]
        elif kind == "cpair":
            terms = [(1.0, complex(prop["mk2"]), complex(prop["mq2"]))]
        elif kind == "dressed":
            (yp, ym), (Rp, Rm) = dressed_poles(prop["a"], prop["b"], prop["c"])
            terms = [(Rp * Rp, -yp, -yp), (Rm * Rm, -ym, -ym), (2 * Rp * Rm, -yp, -ym)]
        else:
            raise ValueError(kind)
        s = 0j
        for coef, M1, M2 in terms:
            if dim == 4:
                s += coef * bubble4(xx, M1, M2) / (16 * PI * PI)
            else:
                s += coef * bubble3(xx, M1, M2)
        return s

    return T(complex(x)) - (T(complex(mu2)) if mu2 != 0 else 0.0)
