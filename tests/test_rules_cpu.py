"""The angular tables and compressed rules built by the library's host code
(gfc_test_angular_rules), pinned without a GPU.

Per radial node the kernels replace the full sums A = sum_j e_j/|1 - w t_j|^2
and B = sum_j g_j/|1 - w t_j|^2 over the pair table by a Gauss rule of the
discrete measure sum_j e_j delta(t - t_j): the smallest one whose threshold
rho_min the node's Bernstein-ellipse parameter rho of the poles t = 1/w,
1/conj(w) meets. Pinned here: the pair table's moments against the closed form
of int_0^pi cos^(2k) psi sin^(D-2) psi dpsi (each +-psi pair is weighted once,
so the table carries half of it); each rule's exactness for t^m, m < 2n; and
the property the kernels rely on, that A and B from the selected rule agree
with the full sums to rounding for seeded w of every Bernstein parameter.
"""
import math

import numpy as np
import pytest

from paper_1205_0752_gb300 import binding


def _moment(k, dim):
    """int_0^pi cos^(2k) psi sin^(D-2) psi dpsi"""
    return math.gamma(k + 0.5) * math.gamma((dim - 1) / 2) / math.gamma(k + dim / 2)


def _rho(w):
    """Bernstein-ellipse parameter of the pole t = 1/w for [0, 1]"""
    s0 = 2.0 / w - 1.0
    z = s0 + np.sqrt(s0 - 1.0 + 0j) * np.sqrt(s0 + 1.0 + 0j)
    m = np.abs(z)
    return np.where(m >= 1.0, m, 1.0 / m)


@pytest.mark.parametrize("n_angular,dim,rule,tol", [(256, 4, "gl", 1e-13), (128, 3, "gl", 1e-13),
                                                    (64, 4, "chebyshev2", 1e-13), (65, 4, "gl", 1e-13)])
def test_pair_table_moments(n_angular, dim, rule, tol):
    pairs, _, _ = binding.angular_rules(n_angular, dim, rule)
    t, e = pairs[:, 0], pairs[:, 1]
    assert pairs.shape[0] == (n_angular + 1) // 2
    assert np.all((t >= 0) & (t < 1)) and np.all(e >= 0)
    assert np.allclose(pairs[:, 2], e * t, rtol=1e-15, atol=0)
    for k in range(0, 12):
        # sum_j e_j t_j^k = sum_j w_j t_j^(k+2) = half the (k+2)-th moment
        got = np.sum(e * t ** k)
        want = 0.5 * _moment(k + 2, dim)
        assert abs(got - want) <= tol * want, (k, got, want)


@pytest.mark.parametrize("n_angular", [10, 64, 256, 300])
def test_each_rule_is_exact_for_polynomials(n_angular):
    pairs, rules, rho_min = binding.angular_rules(n_angular, 4)
    t, e = pairs[:, 0], pairs[:, 1]
    assert len(rules) == len(rho_min) >= 1
    assert np.all(np.diff(rho_min) < 0)          # larger rules reach closer poles
    for rl in rules:
        n = rl.shape[0]
        tau, gam = rl[:, 0], rl[:, 1]
        assert n < t.size and np.all(gam > 0) and np.all((tau >= 0) & (tau <= 1))
        assert np.allclose(rl[:, 2], gam * tau, rtol=1e-15, atol=0)
        for m in range(2 * n):
            full = np.sum(e * t ** m)
            assert abs(np.sum(gam * tau ** m) - full) <= 1e-11 * full, (n, m)


@pytest.mark.parametrize("n_angular,dim", [(256, 4), (64, 4), (128, 3), (300, 4)])
def test_selected_rule_reproduces_the_full_sums(n_angular, dim):
    pairs, rules, rho_min = binding.angular_rules(n_angular, dim)
    t, e, g = pairs[:, 0], pairs[:, 1], pairs[:, 2]
    rng = np.random.default_rng(n_angular + dim)
    w = rng.uniform(0.0, 3.0, 4000) * np.exp(1j * rng.uniform(-np.pi, np.pi, 4000))
    rho = _rho(w)
    used = 0
    worst = 0.0
    for wk, rk in zip(w, rho):
        sel = [r for r in range(len(rules)) if rk >= rho_min[r]]
        if not sel:
            continue                  # the full table: the same sum
        rl = rules[sel[0]]
        used += 1
        qf = np.abs(1.0 - wk * t) ** 2
        qr = np.abs(1.0 - wk * rl[:, 0]) ** 2
        A, B = np.sum(e / qf), np.sum(g / qf)
        Ar, Br = np.sum(rl[:, 1] / qr), np.sum(rl[:, 2] / qr)
        worst = max(worst, abs(Ar - A) / A, abs(Br - B) / B)
    assert used > 1000
    assert worst <= 1e-13, worst
