"""Pins for the oracle's initial data (paper Sec. 2.2).

* H(q0) = 0 to rounding.
* The local photon components, recovered by projecting the oracle's momentum on
  a ZAMO frame built here by Gram-Schmidt from the coordinate basis (an
  independent construction, not the paper's tetrad formulas), equal
  (1, sqrt(1 - (alpha^2 + beta^2)/D^2), beta/D, -alpha/D).
* Schwarzschild: impact parameter b = sqrt(alpha^2 + beta^2) / sqrt(1 - 2M/D).
* Far observer: alpha -> -xi / sin(i) and beta^2 -> eta + a^2 cos^2 i - xi^2 cot^2 i
  (Bardeen's celestial coordinates), which fixes the signs of alpha and beta.
"""
import math

import numpy as np
import pytest

from paper_2609_08989_gb300 import scenes


def _scene(a, inc, D=1000.0, M=1.0):
    return scenes.Scene(M=M, a=a, theta_obs=inc, r_obs=D)


def _conserved(y, inc, a):
    """E, L, Q of the physical (future-directed) photon: the state holds -p."""
    p_t, p_th, p_ph = -y[4], -y[6], -y[7]
    E, L = -p_t, p_ph
    Q = p_th ** 2 + math.cos(inc) ** 2 * (-a * a * E * E + L * L / math.sin(inc) ** 2)
    return E, L, Q


CASES = [(0.0, math.pi / 2), (0.9, math.radians(60)), (0.998, math.radians(85)), (0.5, math.radians(17))]


@pytest.mark.parametrize("a,inc", CASES)
def test_null_and_local_components(orc, a, inc):
    D = 1000.0
    sc = _scene(a, inc, D)
    g = orc.metric_lower(sc, D, inc)
    # ZAMO frame by Gram-Schmidt: e_t along the normal to t = const, then the
    # coordinate directions r, theta, phi orthonormalised against it.
    gi = np.linalg.inv(g)
    # future-pointing unit normal: n_mu = -N dt_mu, n^mu = -N g^{mu t}, N = 1/sqrt(-g^tt)
    e_t = -gi[:, 0] / math.sqrt(-gi[0, 0])
    frame = [e_t]
    for k in (1, 2, 3):
        v = np.zeros(4)
        v[k] = 1.0
        for i, e in enumerate(frame):
            eta = -1.0 if i == 0 else 1.0
            v = v - eta * (e @ g @ v) * e
        frame.append(v / math.sqrt(v @ g @ v))
    rng = np.random.default_rng(11)
    for _ in range(20):
        al, be = rng.uniform(-25, 25, 2)
        y = orc.initial_state(sc, al, be)
        H = orc.hamiltonian(sc, y)
        p_phys = -y[4:]                              # undo the backward reversal
        E = -p_phys[0]
        assert abs(H) < 1e-15 * max(1.0, E * E) * 10
        loc = np.array([-(frame[0] @ p_phys)] + [frame[k] @ p_phys for k in (1, 2, 3)])
        want = np.array([1.0, math.sqrt(1 - (al * al + be * be) / D ** 2), be / D, -al / D])
        assert np.max(np.abs(loc - want)) < 1e-13
        # position part of the state
        assert y[1] == D and y[2] == inc and y[0] == 0.0 and y[3] == 0.0
        # backward tracing: moving inward
        assert y[5] < 0


def test_schwarzschild_impact_parameter(orc):
    for D in (100.0, 1000.0, 1e5):
        sc = _scene(0.0, math.pi / 2, D)
        for al, be in ((3.0, 4.0), (-5.19, 0.0), (0.0, 7.5), (-2.0, -9.0)):
            y = orc.initial_state(sc, al, be)
            E, L, Q = _conserved(y, sc.theta_obs, 0.0)
            b = math.sqrt(L * L + Q) / E              # total angular momentum over energy
            want = math.hypot(al, be) / math.sqrt(1 - 2.0 / D)
            assert abs(b - want) < 1e-13 * want


@pytest.mark.parametrize("a,inc", CASES[1:])
def test_far_observer_celestial_coordinates(orc, a, inc):
    D = 1e9
    sc = _scene(a, inc, D)
    for al, be in ((3.0, 4.0), (-6.5, 2.0), (1.25, -7.0)):
        y = orc.initial_state(sc, al, be)
        E, L, Q = _conserved(y, inc, a)
        xi, eta = L / E, Q / E ** 2
        assert abs(al - (-xi / math.sin(inc))) < 1e-6
        b2 = eta + a * a * math.cos(inc) ** 2 - xi * xi / math.tan(inc) ** 2
        assert abs(be * be - b2) < 1e-6 * max(1.0, be * be)


def test_bad_pixel(orc):
    sc = _scene(0.9, 1.0, 10.0)
    with pytest.raises(ValueError):
        orc.initial_state(sc, 8.0, 6.0)          # alpha^2 + beta^2 = D^2
