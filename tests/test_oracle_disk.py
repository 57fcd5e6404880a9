"""Pins for the oracle's horizon, ISCO, Page-Thorne flux and redshift
(paper Sec. 2.3-2.4).

* r_+ and the ISCO against published values, and the ISCO against the minimum
  of the circular-orbit energy E(r) found by bisection here.
* The flux as printed equals 4 pi times the Page-Thorne flux obtained by
  quadrature of the conservation-law integral with Kerr circular-orbit E, L,
  Omega (so the roots x_i, logarithms and prefactor are all exercised).
* F(r_isco) = 0, r^3 F -> 3/2, continuity as a -> 0.
* g against the closed-form u^t of circular orbits (BPT 1972).
"""
import json
import math
import os

import mpmath as mp
import numpy as np
import pytest

import kerr_exact as KE
from paper_2609_08989_gb300 import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_horizon_and_isco_published(orc):
    for a, r in zip(GOLD["r_plus"]["a"], GOLD["r_plus"]["r"]):
        assert abs(orc.rplus(1.0, a) - r) < 1e-14
    for a, r in zip(GOLD["isco"]["a"], GOLD["isco"]["r"]):
        assert abs(orc.isco(1.0, a) - r) < 1e-12
    # mass scaling
    assert abs(orc.isco(2.0, 1.8) - 2.0 * orc.isco(1.0, 0.9)) < 1e-13


@pytest.mark.parametrize("a", [0.0, 0.3, 0.9, 0.998])
def test_isco_is_energy_minimum(orc, a):
    r_e = float(KE.isco_by_energy_minimum(a))
    assert abs(orc.isco(1.0, a) - r_e) < 1e-12 * r_e


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, 0.998])
def test_flux_against_page_thorne_quadrature(orc, a):
    r_ms = orc.isco(1.0, a)
    for r in (r_ms * 1.3, 8.0, 30.0, 300.0):
        ref = float(KE.page_thorne_flux(a, r, mp.mpf(r_ms)))
        got = orc.flux(1.0, a, 1.0, r)
        assert abs(got / ref - 4 * math.pi) < 1e-11 * 4 * math.pi
    assert orc.flux(1.0, a, 2.5, 10.0) == pytest.approx(2.5 * orc.flux(1.0, a, 1.0, 10.0), rel=1e-15)


@pytest.mark.parametrize("a", [0.0, 0.9, 0.998])
def test_flux_limits(orc, a):
    r_ms = orc.isco(1.0, a)
    assert orc.flux(1.0, a, 1.0, r_ms) == pytest.approx(0.0, abs=1e-15)
    assert orc.flux(1.0, a, 1.0, 0.99 * r_ms) == 0.0
    rs = np.linspace(r_ms * 1.001, 40, 50)
    assert all(orc.flux(1.0, a, 1.0, r) > 0 for r in rs)
    # r^3 F -> 3/2 with the printed prefactor; the approach is O(r^-1/2)
    v = [r ** 3 * orc.flux(1.0, a, 1.0, r) for r in (1e6, 1e8, 1e10)]
    assert abs(v[2] - 1.5) < abs(v[1] - 1.5) < abs(v[0] - 1.5)
    assert abs(v[2] - 1.5) < 1e-4


def test_flux_continuous_in_spin(orc):
    for r in (7.0, 20.0):
        assert orc.flux(1.0, 1e-9, 1.0, r) == pytest.approx(orc.flux(1.0, 0.0, 1.0, r), rel=1e-7)


@pytest.mark.parametrize("a", [0.0, 0.9, 0.998])
def test_redshift_closed_form(orc, a):
    sc = scenes.Scene(a=a)
    for r in (orc.isco(1.0, a) * 1.01, 6.5, 29.0):
        ut = float(KE.circular_ut(a, r))
        Om = 1.0 / (r ** 1.5 + a)
        for xi in (-7.0, 0.0, 3.3):
            g = orc.redshift(sc, r, -1.0, xi)           # p_t = -E with E = 1, p_phi = xi
            assert g == pytest.approx(1.0 / (ut * (1.0 - Om * xi)), rel=2e-14)
            # homogeneous of degree 0 in p (backward reversal leaves it unchanged)
            assert orc.redshift(sc, r, 2.0, -2.0 * xi) == pytest.approx(g, rel=1e-15)
        off = orc.redshift(sc.replace(doppler=0), r, -1.0, 5.0)
        assert off == pytest.approx(1.0 / ut, rel=2e-14)
