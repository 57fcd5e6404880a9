"""Pins for the oracle's Kerr metric, its inverse, derivatives and Hamiltonian flow.

The reference here is a symbolic Kerr line element that is first checked to be
a vacuum solution (Ricci-flat, evaluated at 40 digits) -- so the oracle is
pinned to Einstein's equations, not to a retyped formula.  The oracle's inverse
and derivatives are then compared with the high-precision inverse and
derivatives of that metric, and its Hamiltonian with Carter's separated form.
"""
import math

import mpmath as mp
import numpy as np
import pytest
import sympy as sp

mp.mp.dps = 40

R_, TH_, M_, A_ = sp.symbols("r theta M a", real=True)
X = (None, R_, TH_, None)            # coordinates t, r, theta, phi; only r and theta appear


def sym_kerr():
    S = R_ ** 2 + A_ ** 2 * sp.cos(TH_) ** 2
    D = R_ ** 2 - 2 * M_ * R_ + A_ ** 2
    s2 = sp.sin(TH_) ** 2
    g = sp.zeros(4, 4)
    g[0, 0] = -(1 - 2 * M_ * R_ / S)
    g[0, 3] = g[3, 0] = -2 * M_ * A_ * R_ * s2 / S
    g[1, 1] = S / D
    g[2, 2] = S
    g[3, 3] = (R_ ** 2 + A_ ** 2 + 2 * M_ * A_ ** 2 * R_ * s2 / S) * s2
    return g


G = sym_kerr()
_f = sp.lambdify((R_, TH_, M_, A_), G, modules="mpmath")
_df = [None, sp.lambdify((R_, TH_, M_, A_), G.diff(R_), modules="mpmath"),
       sp.lambdify((R_, TH_, M_, A_), G.diff(TH_), modules="mpmath"), None]
_ddf = {}
for c in (1, 2):
    for d in (1, 2):
        _ddf[(c, d)] = sp.lambdify((R_, TH_, M_, A_), G.diff(X[c]).diff(X[d]), modules="mpmath")


def hp_metric(r, th, M, a, scale_gtt=1):
    """g, dg[c], ddg[c,d] at 40 digits (c, d in 1=r, 2=theta)."""
    args = (mp.mpf(r), mp.mpf(th), mp.mpf(M), mp.mpf(a))
    g = mp.matrix(_f(*args))
    if scale_gtt != 1:
        g[0, 0] = g[0, 0] * scale_gtt
    dg = {c: mp.matrix(_df[c](*args)) for c in (1, 2)}
    ddg = {k: mp.matrix(f(*args)) for k, f in _ddf.items()}
    return g, dg, ddg


def ricci(g, dg, ddg):
    gi = g ** -1
    z = mp.matrix(4, 4)
    dgf = [z, dg[1], dg[2], z]
    dgi = [z] + [-gi * dgf[c] * gi for c in (1, 2)] + [z]

    def dd(e, c):
        return ddg[(e, c)] if (e in (1, 2) and c in (1, 2)) else z

    Gam = [[[sum(gi[a_, d] * (dgf[b][d, c] + dgf[c][d, b] - dgf[d][b, c]) for d in range(4)) / 2
             for c in range(4)] for b in range(4)] for a_ in range(4)]
    dGam = [[[[sum(dgi[e][a_, d] * (dgf[b][d, c] + dgf[c][d, b] - dgf[d][b, c]) +
                   gi[a_, d] * (dd(e, b)[d, c] + dd(e, c)[d, b] - dd(e, d)[b, c]) for d in range(4)) / 2
               for c in range(4)] for b in range(4)] for a_ in range(4)] for e in range(4)]
    Ric = mp.matrix(4, 4)
    for b in range(4):
        for c in range(4):
            v = 0
            for a_ in range(4):
                v += dGam[a_][a_][b][c] - dGam[c][a_][a_][b]
                for d in range(4):
                    v += Gam[a_][a_][d] * Gam[d][b][c] - Gam[a_][c][d] * Gam[d][a_][b]
            Ric[b, c] = v
    return Ric


POINTS = [(6.3, 0.7, 1.0, 0.9), (3.1, 1.9, 1.0, 0.5), (25.0, 1.2, 1.0, 0.998), (2.7, 2.6, 2.0, 1.3)]


@pytest.mark.parametrize("r,th,M,a", POINTS[:2])
def test_reference_metric_is_vacuum(r, th, M, a):
    g, dg, ddg = hp_metric(r, th, M, a)
    Ric = ricci(g, dg, ddg)
    assert max(abs(Ric[i, j]) for i in range(4) for j in range(4)) < 1e-30
    # the check has teeth: a perturbed g_tt is not a vacuum metric
    g2, dg2, ddg2 = hp_metric(r, th, M, a, scale_gtt=mp.mpf("1.0001"))
    Ric2 = ricci(g2, dg2, ddg2)
    assert max(abs(Ric2[i, j]) for i in range(4) for j in range(4)) > 1e-8


def _rel(a, b, scale):
    return np.max(np.abs(np.asarray(a, float) - np.asarray(b, float))) / scale


@pytest.mark.parametrize("r,th,M,a", POINTS)
def test_lower_upper_and_derivatives(orc, r, th, M, a):
    g, dg, _ = hp_metric(r, th, M, a)
    gi = g ** -1
    g_o = orc.kerr_lower(M, a, r, th)
    gi_o, dr_o, dt_o = orc.kerr_upper(M, a, r, th)
    G_hp = np.array(g.tolist(), dtype=float)
    GI_hp = np.array(gi.tolist(), dtype=float)
    assert _rel(g_o, G_hp, np.abs(G_hp).max()) < 1e-14
    assert _rel(gi_o, GI_hp, np.abs(GI_hp).max()) < 1e-14
    for c, d_o in ((1, dr_o), (2, dt_o)):
        ref = np.array((-gi * dg[c] * gi).tolist(), dtype=float)
        assert _rel(d_o, ref, np.abs(ref).max()) < 1e-13
    # the oracle's two metric routines invert each other
    assert np.max(np.abs(g_o @ gi_o - np.eye(4))) < 1e-13


def _hp_flow(r, th, M, a, p):
    g, dg, _ = hp_metric(r, th, M, a)
    gi = g ** -1
    pv = mp.matrix([mp.mpf(x) for x in p])
    xdot = gi * pv
    pdot = [0, -(pv.T * (-gi * dg[1] * gi) * pv)[0] / 2, -(pv.T * (-gi * dg[2] * gi) * pv)[0] / 2, 0]
    H = (pv.T * gi * pv)[0] / 2
    return [float(xdot[i]) for i in range(4)] + [float(x) for x in pdot], float(H)


@pytest.mark.parametrize("r,th,M,a", POINTS)
def test_hamiltonian_flow(orc, r, th, M, a):
    rng = np.random.default_rng(7)
    p = rng.normal(size=4)
    sc = type("S", (), dict(metric_kind=0, M=M, a=a, table=None, r_min=0.0, r_max=0.0,
                            r_obs=1e3, theta_obs=1.0, nx=1, ny=1, alpha_min=0.0, alpha_max=1.0,
                            beta_min=0.0, beta_max=1.0, rtol=1e-10, atol=1e-10, h0=0.0, h_min=0.0,
                            max_steps=10, horizon_eps=1e-3, escape_factor=1.1, refine=0, method=0,
                            disk_enabled=0, r_in=0.0, r_out=30.0, mdot=1.0, max_crossings=3, doppler=1))
    y = np.array([0.0, r, th, 0.0, *p])
    dy = orc.rhs(sc, y)
    ref, H_ref = _hp_flow(r, th, M, a, p)
    scale = max(1.0, np.abs(ref).max())
    assert np.max(np.abs(dy - np.array(ref))) / scale < 1e-13
    assert dy[4] == 0.0 and dy[7] == 0.0
    # Carter's separated form: 2 Sigma H = Delta p_r^2 + p_th^2 + (L - a E s^2)^2 / s^2
    #                                       - ((r^2 + a^2) E - a L)^2 / Delta
    E, L = -p[0], p[3]
    s2 = math.sin(th) ** 2
    Sig = r * r + a * a * math.cos(th) ** 2
    Del = r * r - 2 * M * r + a * a
    terms = [Del * p[1] ** 2, p[2] ** 2, (L - a * E * s2) ** 2 / s2, ((r * r + a * a) * E - a * L) ** 2 / Del]
    K = terms[0] + terms[1] + terms[2] - terms[3]
    H_o = orc.hamiltonian(sc, y)
    assert abs(2 * Sig * H_o - K) < 1e-14 * max(abs(t) for t in terms) * 8
    assert abs(H_o - H_ref) < 1e-14 * max(abs(t) for t in terms) / Sig * 8


def test_kerr_table_sampler(orc):
    """The Kerr table sampler's fields and derivatives against symbolic differentiation."""
    M, a = 1.0, 0.998
    nr, nth, rmin, rmax = 7, 6, 1.1, 40.0
    tab = orc.kerr_table(M, a, nr, nth, rmin, rmax)
    S = R_ ** 2 + A_ ** 2 * sp.cos(TH_) ** 2
    D = R_ ** 2 - 2 * M_ * R_ + A_ ** 2
    fields = [G[0, 0], G[0, 3], G[2, 2], G[3, 3], D / S]
    fn = []
    for F in fields:
        fn.append([sp.lambdify((R_, TH_, M_, A_), e, modules="mpmath")
                   for e in (F, F.diff(R_), F.diff(TH_), F.diff(R_).diff(TH_))])
    for j in range(1, nth - 1):                   # interior theta nodes (poles are exact zeros)
        th = math.pi * j / (nth - 1)
        for k in range(nr):
            r = math.exp(math.log(rmin) + k * (math.log(rmax) - math.log(rmin)) / (nr - 1))
            for fi in range(5):
                for q in range(4):
                    ref = float(fn[fi][q](mp.mpf(r), mp.mpf(th), M, a))
                    got = tab[j, k, 4 * fi + q]
                    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (j, k, fi, q, got, ref)
