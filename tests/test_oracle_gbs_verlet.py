"""Pins for the oracle's Gragg-Bulirsch-Stoer extrapolator and Stormer-Verlet
scheme (paper Sec. 3.2), against what the mathematics fixes:

* GBS: with k columns the extrapolated value has order 2k, so it integrates
  y' = t^m exactly for m <= 2k - 1 and not for m = 2k; its local error and its
  error estimate shrink as H^(2k+1) and H^(2k-1); one column is the explicit
  midpoint rule;
* Verlet: on a separable Hamiltonian it is the textbook velocity Verlet; on a
  non-separable one it is time-reversible, symplectic (unit Jacobian), of order
  two against a closed-form solution, and its energy error stays bounded;
* whole rays: crossing radii against Mino-time quadrature, and the paper's
  accuracy ranking of the five schemes on its escaping Schwarzschild ray
  (Sec. 4.1, Fig. 1).
"""
import json
import math
import os

import numpy as np
import pytest

import kerr_exact as KE
from paper_2609_08989_gb300 import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ---------------------------------------------------------------- GBS ----

@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_gbs_polynomial_exactness(orc, k):
    t0, H = 0.3, 0.7
    for m in range(0, 2 * k + 1):
        yn, _, _ = orc.gbs_step(lambda y, m=m: [1.0, y[0] ** m], [t0, 0.0], H, k)
        exact = ((t0 + H) ** (m + 1) - t0 ** (m + 1)) / (m + 1)
        assert yn[0] == pytest.approx(t0 + H, abs=1e-15)
        if m <= 2 * k - 1:
            assert abs(yn[1] - exact) < 1e-14, (k, m)
        else:
            assert abs(yn[1] - exact) > 1e-8, (k, m)


def test_gbs_one_column_is_explicit_midpoint(orc):
    f = lambda y: [y[1], -math.sin(y[0]) + 0.1 * y[0] * y[1]]
    y0, H = np.array([0.4, -0.3]), 0.25
    yn, _, err = orc.gbs_step(f, y0, H, 1)
    k1 = np.array(f(y0))
    mid = np.array(f(y0 + 0.5 * H * k1))
    assert np.allclose(yn, y0 + H * mid, rtol=0, atol=1e-16)
    assert np.all(err == 0)


@pytest.mark.parametrize("k,hs", [(2, (0.4, 0.2, 0.1)), (3, (0.8, 0.4, 0.2))])
def test_gbs_local_orders(orc, k, hs):
    lam = -0.7 + 0.9j

    def f(y):
        z = complex(y[0], y[1]) * lam
        return [z.real, z.imag]

    errs, ests = [], []
    for H in hs:
        yn, _, e = orc.gbs_step(f, np.array([1.0, 0.0]), H, k)
        errs.append(abs(complex(*yn) - np.exp(lam * H)))
        ests.append(abs(complex(*e)))
    for i in range(2):
        p = np.log2(errs[i] / errs[i + 1])
        q = np.log2(ests[i] / ests[i + 1])
        assert 2 * k + 0.6 < p < 2 * k + 1.4, (k, p)
        assert 2 * k - 1.4 < q < 2 * k - 0.6, (k, q)


def test_gbs_fnew_is_rhs_at_solution(orc):
    f = lambda y: [y[1], -y[0] ** 3]
    yn, fn, _ = orc.gbs_step(f, np.array([0.5, 0.1]), 0.3, 6)
    assert np.allclose(fn, f(yn), rtol=0, atol=1e-16)


# ------------------------------------------------------------- Verlet ----

def test_verlet_separable_is_velocity_verlet(orc):
    # H = p^2/2 - cos q: (dH/dp, -dH/dq) = (p, -sin q)
    f = lambda y: [y[1], -math.sin(y[0])]
    h = 0.1
    y = np.array([1.1, 0.2])
    for _ in range(50):
        q, p = y
        ph = p - 0.5 * h * math.sin(q)
        q1 = q + h * ph
        p1 = ph - 0.5 * h * math.sin(q1)
        y, _ = orc.verlet_step(f, y, h)
        assert abs(y[0] - q1) < 1e-14 and abs(y[1] - p1) < 1e-14


def _nonsep(y):
    # H = (1 + q^2) p^2 / 2 + q^2 / 2 + q^4 / 4
    q, p = y
    return [(1 + q * q) * p, -(q * p * p + q + q ** 3)]


def _nonsep_H(y):
    q, p = y
    return 0.5 * (1 + q * q) * p * p + 0.5 * q * q + 0.25 * q ** 4


def test_verlet_time_reversible(orc):
    y0 = np.array([0.7, -0.4])
    y1, _ = orc.verlet_step(_nonsep, y0, 0.15)
    y2, _ = orc.verlet_step(_nonsep, y1, -0.15)
    assert np.max(np.abs(y2 - y0)) < 1e-14


def test_verlet_symplectic(orc):
    y0, h, d = np.array([0.7, -0.4]), 0.15, 1e-6
    J = np.zeros((2, 2))
    for j in range(2):
        e = np.zeros(2)
        e[j] = d
        J[:, j] = (orc.verlet_step(_nonsep, y0 + e, h)[0] - orc.verlet_step(_nonsep, y0 - e, h)[0]) / (2 * d)
    assert abs(np.linalg.det(J) - 1.0) < 1e-8
    # a non-symplectic second-order method (explicit midpoint) is visibly off
    mid, _, _ = orc.gbs_step(_nonsep, y0, h, 1)
    Jm = np.zeros((2, 2))
    for j in range(2):
        e = np.zeros(2)
        e[j] = d
        Jm[:, j] = (orc.gbs_step(_nonsep, y0 + e, h, 1)[0] - orc.gbs_step(_nonsep, y0 - e, h, 1)[0]) / (2 * d)
    assert abs(np.linalg.det(Jm) - 1.0) > 1e-5


def test_verlet_second_order_closed_form(orc):
    # H = (q p)^2 / 2: q p = c is conserved, so dq/dt = q^2 p = c q and q(t) = q0 exp(c t)
    f = lambda y: [y[0] * y[0] * y[1], -y[0] * y[1] * y[1]]
    q0, p0, T = 1.0, 0.8, 2.0
    c = q0 * p0
    errs = []
    for n in (50, 100, 200):
        y = np.array([q0, p0])
        for _ in range(n):
            y, _ = orc.verlet_step(f, y, T / n)
        errs.append(abs(y[0] - q0 * math.exp(c * T)))
    for i in range(2):
        assert 1.8 < np.log2(errs[i] / errs[i + 1]) < 2.2


def test_verlet_energy_bounded(orc):
    y = np.array([1.2, 0.3])
    H0 = _nonsep_H(y)
    dev = []
    for _ in range(4000):
        y, _ = orc.verlet_step(_nonsep, y, 0.1)
        dev.append(abs(_nonsep_H(y) - H0))
    dev = np.array(dev)
    assert dev.max() < 0.02 * H0                            # O(h^2) and small
    assert dev[2000:].max() < 1.5 * dev[:2000].max()      # no secular growth


# --------------------------------------------------------- whole rays ----

def _consts(y, inc, a):
    p = -y[4:]
    E, L = -p[0], p[3]
    Q = p[2] ** 2 + math.cos(inc) ** 2 * (-a * a * E * E + L * L / math.sin(inc) ** 2)
    return L / E, Q / E ** 2, p[2]


def _worst_vs_mino(orc, sc):
    r_stop = orc.rplus(1.0, sc.a) * (1 + sc.horizon_eps)
    rng = np.random.default_rng(21)
    pts = list(rng.uniform(-20, 20, (10, 2))) + [(4.0, 2.0), (-6.1, 0.3), (2.5, -5.5)]
    worst, n = 0.0, 0
    for al, be in pts:
        y0 = orc.initial_state(sc, al, be)
        xi, eta, pth = _consts(y0, sc.theta_obs, sc.a)
        ray = orc.trace_ray(sc, al, be, cap=2)
        ex = KE.exact_crossings(sc.a, xi, eta, sc.r_obs, sc.theta_obs, -np.sign(pth), 3, r_stop)
        assert abs(len(ex) - ray["n_cross"]) <= 1
        for k in range(min(len(ex), ray["n_cross"], 3)):
            worst = max(worst, abs(ray["r_cross"][k] - ex[k]) / ex[k])
            n += 1
    assert n >= 13
    return worst


def _open(rtol, **kw):
    return scenes.kerr_disk(64).replace(rtol=rtol, atol=rtol, r_in=1e-6, r_out=1e12, max_crossings=3, **kw)


@pytest.mark.parametrize("rtol,tol", [(1e-12, 5e-11), (1e-10, 5e-9)])
def test_gbs_crossings_vs_mino_time(orc, rtol, tol):
    assert _worst_vs_mino(orc, _open(rtol, method=scenes.GBS)) < tol


def test_verlet_crossings_vs_mino_time_second_order(orc):
    e2 = _worst_vs_mino(orc, _open(1e-12, method=scenes.VERLET, h0=0.02))
    e1 = _worst_vs_mino(orc, _open(1e-12, method=scenes.VERLET, h0=0.01))
    assert e2 < 2e-4
    assert 3.5 < e2 / e1 < 4.5


def test_paper_accuracy_ranking_escape_ray(orc):
    """Sec. 4.1, Fig. 1: on the escaping b = 6 ray at tolerances 1e-10 the
    extrapolator keeps |H| lowest, the three pairs stay near or below 1e-9, and
    fixed-step Verlet drifts most (its step is not given; 0.01 M here)."""
    g = GOLD["escape_ray"]
    D, b = g["D"], g["b"]
    hm = {}
    for m in (scenes.DOPRI5, scenes.CASH_KARP, scenes.FEHLBERG, scenes.GBS, scenes.VERLET):
        sc = scenes.Scene(a=0.0, r_obs=D, theta_obs=math.pi / 2, rtol=g["rtol"], atol=g["atol"], method=m,
                          h0=0.01 if m == scenes.VERLET else 0.0)
        ray = orc.trace_ray(sc, b * math.sqrt(1 - 2.0 / D), 0.0, cap=2)
        assert ray["code"] == 0
        hm[m] = ray["h_max"]
    pairs = [hm[scenes.DOPRI5], hm[scenes.CASH_KARP], hm[scenes.FEHLBERG]]
    assert hm[scenes.GBS] < min(pairs)
    assert max(pairs) < 3 * g["eps_H_max"]
    assert hm[scenes.VERLET] > 10 * max(pairs)
