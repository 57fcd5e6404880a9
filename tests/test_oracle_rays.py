"""Pins for whole rays of the oracle (paper Sec. 3.2 integration and events,
Sec. 4.1 validation rays), against results that need no integrator:

* crossing radii against Carter's separation in Mino time (high-precision
  quadrature), for Henon's refinement and for the paper's Hermite bisection,
  with each of the three 5(4) pairs;
* termination codes against the radial-quartic classifier, and Schwarzschild's
  closed-form shadow radius, outside the +-1e-6 band around the critical curve;
* Bardeen's critical curve sits between captured and escaped rays;
* conservation of E, L (exact) and of Carter's constant;
* the paper's escaping (b = 6) and captured (b = 3) Schwarzschild rays.
"""
import json
import math
import os

import numpy as np
import pytest

import kerr_exact as KE
from paper_2609_08989_gb300 import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _consts(y, inc, a):
    p = -y[4:]                                 # physical momentum
    E, L = -p[0], p[3]
    Q = p[2] ** 2 + math.cos(inc) ** 2 * (-a * a * E * E + L * L / math.sin(inc) ** 2)
    return L / E, Q / E ** 2, p[2]


def _open_disk(sc, rtol):
    return sc.replace(rtol=rtol, atol=rtol, r_in=1e-6, r_out=1e12, max_crossings=3)


@pytest.mark.parametrize("refine,rtol,tol,method", [
    (0, 1e-12, 5e-11, 0), (0, 1e-10, 5e-9, 0), (1, 1e-12, 2e-8, 0),
    (0, 1e-12, 5e-11, 1), (0, 1e-12, 2e-10, 2), (1, 1e-12, 2e-8, 1)])
def test_crossing_radii_vs_mino_time(orc, refine, rtol, tol, method):
    # Fehlberg's error estimate is looser for the propagated fifth-order
    # solution, so at the same rtol its global error sits ~2x higher.
    base = scenes.kerr_disk(64)
    sc = _open_disk(base, rtol).replace(refine=refine, method=method)
    r_stop = orc.rplus(1.0, sc.a) * (1 + sc.horizon_eps)
    rng = np.random.default_rng(21)
    pts = list(rng.uniform(-20, 20, (10, 2))) + [(4.0, 2.0), (-6.1, 0.3), (2.5, -5.5)]
    n_checked = 0
    worst = 0.0
    for al, be in pts:
        y0 = orc.initial_state(sc, al, be)
        xi, eta, pth = _consts(y0, sc.theta_obs, sc.a)
        ray = orc.trace_ray(sc, al, be, cap=2)
        ex = KE.exact_crossings(sc.a, xi, eta, sc.r_obs, sc.theta_obs, -np.sign(pth), 3, r_stop)
        n = min(len(ex), ray["n_cross"], 3)
        assert ray["n_cross"] == len(ex) or abs(len(ex) - ray["n_cross"]) <= 1
        for k in range(n):
            rel = abs(ray["r_cross"][k] - ex[k]) / ex[k]
            worst = max(worst, rel)
            n_checked += 1
    assert n_checked >= 13
    assert worst < tol, worst


def _codes_classifier(orc, sc, pix):
    """Radial-quartic class of each pixel and whether it sits in the +-1e-6 band."""
    r_stop = orc.rplus(1.0, sc.a) * (1 + sc.horizon_eps)
    dx = (sc.alpha_max - sc.alpha_min) / sc.nx
    dy = (sc.beta_max - sc.beta_min) / sc.ny
    cls, band = [], []
    for p in pix:
        i, j = p % sc.nx, p // sc.nx
        al = sc.alpha_min + (i + 0.5) * dx
        be = sc.beta_min + (j + 0.5) * dy

        def klass(a_, b_):
            xi, eta, _ = _consts(orc.initial_state(sc, a_, b_), sc.theta_obs, sc.a)
            return KE.classify(sc.a, xi, eta, r_stop, sc.r_obs)

        c0 = klass(al, be)
        nb = [klass(al + s * 1e-6, be) for s in (-1, 1)] + [klass(al, be + s * 1e-6) for s in (-1, 1)]
        cls.append(c0)
        band.append(any(c != c0 for c in nb))
    return np.array(cls), np.array(band)


def test_schwarzschild_shadow_codes(orc):
    sc = scenes.schwarzschild_shadow(64)
    out = orc.trace(sc)
    D = sc.r_obs
    rho_c = GOLD["b_crit"]["value"] * math.sqrt(1 - 2.0 / D)
    i = np.arange(sc.npix) % sc.nx
    j = np.arange(sc.npix) // sc.nx
    al = sc.alpha_min + (i + 0.5) * (sc.alpha_max - sc.alpha_min) / sc.nx
    be = sc.beta_min + (j + 0.5) * (sc.beta_max - sc.beta_min) / sc.ny
    rho = np.hypot(al, be)
    keep = np.abs(rho - rho_c) > 1e-6
    want = (rho < rho_c).astype(np.int8)
    assert np.array_equal(out["code"][keep], want[keep])
    assert set(np.unique(out["code"])) == {0, 1}


def test_kerr_codes_vs_quartic_classifier(orc):
    sc = scenes.kerr_disk(256)
    pix = scenes.sample_pixels(sc.npix, 600, 4)
    out = orc.trace_list(sc, pix)
    cls, band = _codes_classifier(orc, sc, pix)
    ok = ~band
    assert ok.sum() > 590
    assert np.array_equal(out["code"][ok], cls[ok].astype(np.int8))
    assert 0 < cls.sum() < len(cls)


def test_bardeen_curve_separates_captured_and_escaped(orc):
    a, inc, D = 0.9, math.radians(60), 1e6
    sc = scenes.Scene(a=a, theta_obs=inc, r_obs=D, rtol=1e-11, atol=1e-11)
    rp, rm = KE.photon_orbit_radii(a)
    found = 0
    for r in np.linspace(rp + 1e-3, rm - 1e-3, 9):
        xi, eta = KE.bardeen_curve(a, r)
        b2 = eta + a * a * math.cos(inc) ** 2 - xi * xi / math.tan(inc) ** 2
        if b2 <= 0:
            continue
        al, be = -xi / math.sin(inc), math.sqrt(b2)
        # R(r) has a double root on the curve
        assert abs(KE.R_of(a, xi, eta, r)) < 1e-8 * r ** 4
        cx, cy = 0.0, 0.0                     # scale the image point about the origin
        for f, want in ((0.995, 1), (1.005, 0)):
            ray = orc.trace_ray(sc, cx + f * (al - cx), cy + f * (be - cy), cap=2)
            assert ray["code"] == want, (r, f)
        found += 1
    assert found >= 5


def test_conservation_along_ray(orc):
    sc = scenes.kerr_disk(64)
    for al, be in ((7.0, 3.0), (-3.0, 6.5), (2.0, -9.0)):
        ray = orc.trace_ray(sc, al, be, cap=100000)
        ys = ray["y"]
        assert np.all(ys[:, 4] == ys[0, 4]) and np.all(ys[:, 7] == ys[0, 7])
        E, L = ys[0, 4], ys[0, 7]               # (signs cancel in Q)
        Q = ys[:, 6] ** 2 + np.cos(ys[:, 2]) ** 2 * (L * L / np.sin(ys[:, 2]) ** 2 - sc.a ** 2 * E * E)
        assert np.max(np.abs(Q - Q[0])) < 1e-8 * max(1.0, abs(Q[0]))
        assert ray["h_max"] < 1e-8


def test_paper_escape_ray(orc):
    g = GOLD["escape_ray"]
    D, b = g["D"], g["b"]
    sc = scenes.Scene(a=0.0, r_obs=D, theta_obs=math.pi / 2, rtol=g["rtol"], atol=g["atol"])
    ray = orc.trace_ray(sc, b * math.sqrt(1 - 2.0 / D), 0.0, cap=100000)
    assert ray["code"] == 0
    assert ray["h_max"] <= g["eps_H_max"]
    # periapsis: the largest root of r^3 - b^2 r + 2 b^2 = 0
    roots = np.roots([1.0, 0.0, -b * b, 2 * b * b])
    r_t = max(z.real for z in roots if abs(z.imag) < 1e-12)
    r_min = ray["y"][:, 1].min()
    assert r_t * (1 - 1e-12) <= r_min < r_t * (1 + 1e-3)


def test_paper_capture_ray(orc):
    g = GOLD["capture_ray"]
    D, b = g["D"], g["b"]
    eps = g["r_stop"] / 2.0 - 1.0
    sc = scenes.Scene(a=0.0, r_obs=D, theta_obs=math.pi / 2, horizon_eps=eps)
    ray = orc.trace_ray(sc, b * math.sqrt(1 - 2.0 / D), 0.0, cap=100000)
    assert ray["code"] == 1
    assert 2.0 < ray["y"][-1, 1] < g["r_stop"] <= ray["y"][-2, 1]
    esc = orc.trace_ray(sc, 6 * math.sqrt(1 - 2.0 / D), 0.0, cap=2)
    assert ray["h_max"] > esc["h_max"]         # the residual grows towards the horizon


def test_step_cap_and_underflow_codes(orc):
    sc = scenes.kerr_disk(64)
    r = orc.trace_ray(sc.replace(max_steps=50), 3.0, 4.0, cap=2)
    assert r["code"] == 2 and r["steps"] + r["rejects"] == 50
    r = orc.trace_ray(sc.replace(h_min=1e6), 3.0, 4.0, cap=2)
    assert r["code"] == 3 and r["steps"] == 0
    r = orc.trace_ray(sc.replace(r_obs=10.0), 8.0, 6.0, cap=2)
    assert r["code"] == 5
    r = orc.trace_ray(sc, float("nan"), 0.0, cap=2)
    assert r["code"] == 5


def test_photon_sphere_limit(orc):
    """Schwarzschild rays just outside the critical impact parameter 3 sqrt(3) M
    turn at the largest root of r^3 - b^2 r + 2 b^2 = 0, which tends to the
    photon sphere r = 3M as b -> 3 sqrt(3) M; just inside, they are captured."""
    D = 1000.0
    sc = scenes.Scene(a=0.0, r_obs=D, theta_obs=math.pi / 2, rtol=1e-12, atol=1e-12)
    bc = 3 * math.sqrt(3)
    for eps in (1e-3, 1e-5):
        b = bc * (1 + eps)
        ray = orc.trace_ray(sc, b * math.sqrt(1 - 2.0 / D), 0.0, cap=200000)
        assert ray["code"] == 0
        roots = np.roots([1.0, 0.0, -b * b, 2 * b * b])
        r_t = max(z.real for z in roots if abs(z.imag) < 1e-9)
        r_min = ray["y"][:, 1].min()
        assert 3.0 < r_t < 3.0 + 4 * math.sqrt(eps)
        assert r_t * (1 - 1e-10) <= r_min < r_t * (1 + 2e-3)
        inside = orc.trace_ray(sc, bc * (1 - eps) * math.sqrt(1 - 2.0 / D), 0.0, cap=2)
        assert inside["code"] == 1
