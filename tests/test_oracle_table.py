"""Pins for the oracle's tabulated-metric interpolation.

* Bicubic Hermite patches reproduce any polynomial of degree <= 3 in each of
  (ln r, theta) exactly, with its derivatives -- including outside the node
  range, where the boundary cell's polynomial is extended.
* On sampled Kerr, the interpolation error falls as h^4 when the grid is refined.
* The table-metric flow equals the closed-form Kerr flow to interpolation
  accuracy, and the initial data built from the table is null.
"""
import math

import numpy as np
import pytest

from paper_2609_08989_gb300 import scenes

RMIN, RMAX, NR, NTH = 1.7, 120.0, 24, 19


def _poly_table(coef):
    """Table of five fields f(u, th) = sum c_ij u^i th^j (u = ln r), degree <= 3 each,
    with exact d/dr, d/dth and d2/dr dth at the nodes."""
    u0, u1 = math.log(RMIN), math.log(RMAX)
    tab = np.zeros((NTH, NR, 20))
    for j in range(NTH):
        th = math.pi * j / (NTH - 1)
        for k in range(NR):
            u = u0 + k * (u1 - u0) / (NR - 1)
            r = math.exp(u)
            for f in range(5):
                c = coef[f]
                v = sum(c[i, q] * u ** i * th ** q for i in range(4) for q in range(4))
                vu = sum(i * c[i, q] * u ** (i - 1) * th ** q for i in range(1, 4) for q in range(4))
                vt = sum(q * c[i, q] * u ** i * th ** (q - 1) for i in range(4) for q in range(1, 4))
                vut = sum(i * q * c[i, q] * u ** (i - 1) * th ** (q - 1) for i in range(1, 4) for q in range(1, 4))
                tab[j, k, 4 * f:4 * f + 4] = (v, vu / r, vt, vut / r)
    return tab


def _poly_eval(c, r, th):
    u = math.log(r)
    v = sum(c[i, q] * u ** i * th ** q for i in range(4) for q in range(4))
    vu = sum(i * c[i, q] * u ** (i - 1) * th ** q for i in range(1, 4) for q in range(4))
    vt = sum(q * c[i, q] * u ** i * th ** (q - 1) for i in range(4) for q in range(1, 4))
    return v, vu / r, vt


def test_bicubic_polynomials_reproduced(orc):
    rng = np.random.default_rng(3)
    coef = [rng.normal(size=(4, 4)) * 0.3 for _ in range(5)]
    coef[0][0, 0] = -3.0           # keep the (t, phi) block invertible: g_tt < 0 < g_phiphi
    coef[3][0, 0] = 30.0
    coef[2][0, 0] = 40.0           # g_thth > 0
    coef[1] *= 0.01
    tab = _poly_table(coef)
    sc = scenes.Scene(metric_kind=1, a=0.0, table=tab, r_min=RMIN, r_max=RMAX)
    for r, th in ((2.0, 0.4), (9.7, 1.57), (55.0, 2.9), (RMIN, 0.0), (150.0, 1.0), (1.5, 2.0)):
        g = orc.metric_lower(sc, r, th)
        gi, dgr, dgt = orc.metric_upper(sc, r, th)
        vals = [_poly_eval(c, r, th) for c in coef]
        for (f_idx, (mu, nu)) in enumerate([(0, 0), (0, 3), (2, 2), (3, 3)]):
            assert g[mu, nu] == pytest.approx(vals[f_idx][0], rel=1e-11, abs=1e-11)
        assert gi[1, 1] == pytest.approx(vals[4][0], rel=1e-11, abs=1e-11)
        assert dgr[1, 1] == pytest.approx(vals[4][1], rel=1e-9, abs=1e-10)
        assert dgt[1, 1] == pytest.approx(vals[4][2], rel=1e-9, abs=1e-10)
        # inverse of the (t, phi) block and its derivative, from the exact polynomials
        gtt, gtp, gpp = vals[0][0], vals[1][0], vals[3][0]
        D = gtt * gpp - gtp * gtp
        assert gi[0, 0] == pytest.approx(gpp / D, rel=1e-10)
        dD = vals[0][1] * gpp + gtt * vals[3][1] - 2 * gtp * vals[1][1]
        assert dgr[0, 0] == pytest.approx((vals[3][1] * D - gpp * dD) / D ** 2, rel=1e-8, abs=1e-12)
        assert dgt[2, 2] == pytest.approx(-vals[2][2] / vals[2][0] ** 2, rel=1e-8, abs=1e-12)


def test_fourth_order_convergence_on_kerr(orc):
    a = 0.9
    rh = 1.0 + math.sqrt(1 - a * a)
    rng = np.random.default_rng(5)
    pts = list(zip(np.exp(rng.uniform(math.log(2.5), math.log(60.0), 150)), rng.uniform(0.3, 2.8, 150)))
    errs = []
    for n in (65, 129, 257):                  # spacing halves exactly
        tab = orc.kerr_table(1.0, a, n, n, rh, 1000.0)
        sc = scenes.Scene(metric_kind=1, a=a, table=tab, r_min=rh, r_max=1000.0)
        e2 = 0.0
        for r, th in pts:
            g_t = orc.metric_lower(sc, r, th)
            g_k = orc.kerr_lower(1.0, a, r, th)
            e2 += (np.max(np.abs(g_t - g_k)) / np.max(np.abs(g_k))) ** 2
        errs.append(math.sqrt(e2 / len(pts)))
    for k in range(2):                        # RMS error falls as h^4
        assert 2 ** 3.5 < errs[k] / errs[k + 1] < 2 ** 4.5


def test_table_flow_matches_closed_form(orc):
    a = 0.998
    rh = 1.0 + math.sqrt(1 - a * a)
    tab = orc.kerr_table(1.0, a, 512, 256, rh, 1000.0)
    sc_t = scenes.table_kerr(64, table=tab)
    sc_k = sc_t.replace(metric_kind=0, table=None)
    rng = np.random.default_rng(9)
    for _ in range(10):
        al, be = rng.uniform(-25, 25, 2)
        y_t = orc.initial_state(sc_t, al, be)
        y_k = orc.initial_state(sc_k, al, be)
        assert np.max(np.abs(y_t - y_k)) < 1e-8
        assert abs(orc.hamiltonian(sc_t, y_t)) < 1e-13
        y = y_k.copy()
        y[1], y[2] = rng.uniform(2.0, 30.0), rng.uniform(0.5, 2.6)
        d_t, d_k = orc.rhs(sc_t, y), orc.rhs(sc_k, y)
        assert np.max(np.abs(d_t - d_k)) < 1e-6 * max(1.0, np.max(np.abs(d_k)))


def test_input_module_table_matches_oracle_sampler(orc):
    """The input generator's Kerr table (used by the benchmark) equals the
    oracle's sampler, whose fields are pinned symbolically in test_oracle_metric."""
    a = 0.998
    rh = 1.0 + math.sqrt(1 - a * a)
    t1 = orc.kerr_table(1.0, a, 64, 33, rh, 1000.0)
    t2 = scenes.kerr_table_nodes(1.0, a, 64, 33, rh, 1000.0)
    scale = np.maximum(1.0, np.abs(t1))
    assert np.max(np.abs(t1 - t2) / scale) < 1e-13
