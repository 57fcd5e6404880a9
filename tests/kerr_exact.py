"""Exact Kerr null-geodesic results used to pin the oracle, computed
independently of any integrator: Carter's separation in Mino time, the
radial quartic R(r), the polar potential, Bardeen's critical curve, and
Bardeen-Press-Teukolsky circular-orbit quantities.  High precision via mpmath.

Conventions: M = 1, constants scaled by the energy, xi = L/E, eta = Q/E^2,
  R(r)   = (r^2 + a^2 - a xi)^2 - Delta (eta + (xi - a)^2),
  U(u)   = eta - (eta + xi^2 - a^2) u^2 - a^2 u^4,   u = cos(theta),
  dr/dtau = +-sqrt(R),  du/dtau = +-sqrt(U)  (Mino time, Sigma dtau = dlambda).
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

mp.mp.dps = 40


def radial_coeffs(a, xi, eta):
    """R(r) = r^4 + (2k - c) r^2 + 2 c r + (k^2 - a^2 c), k = a^2 - a xi, c = eta + (xi - a)^2."""
    k = a * a - a * xi
    c = eta + (xi - a) ** 2
    return [1.0, 0.0, 2 * k - c, 2 * c, k * k - a * a * c]


def R_of(a, xi, eta, r):
    return (r * r + a * a - a * xi) ** 2 - (r * r - 2 * r + a * a) * (eta + (xi - a) ** 2)


def radial_turning_point(a, xi, eta, r_lo, r_hi):
    """Largest real root of R in (r_lo, r_hi), or None (numpy, double precision)."""
    roots = np.roots(radial_coeffs(a, xi, eta))
    real = [z.real for z in roots if abs(z.imag) <= 1e-9 * max(1.0, abs(z))]
    inside = [x for x in real if r_lo < x < r_hi]
    return max(inside) if inside else None


def classify(a, xi, eta, r_stop, D):
    """1 (captured) if an inward ray from D never meets a zero of R above r_stop, else 0."""
    return 1 if radial_turning_point(a, xi, eta, r_stop, D) is None else 0


def bardeen_curve(a, r):
    """Bardeen (1973) critical-curve constants (xi, eta) of the spherical photon
    orbit at radius r (M = 1)."""
    xi = (r * r * (3 - r) - a * a * (r + 1)) / (a * (r - 1))
    eta = r ** 3 * (4 * a * a - r * (r - 3) ** 2) / (a * a * (r - 1) ** 2)
    return xi, eta


def photon_orbit_radii(a):
    """Prograde and retrograde equatorial circular photon orbits."""
    rp = 2 * (1 + np.cos(2.0 / 3.0 * np.arccos(-a)))
    rm = 2 * (1 + np.cos(2.0 / 3.0 * np.arccos(a)))
    return rp, rm


# ---------------------------------------------------------------------------
# Mino-time crossing radii
# ---------------------------------------------------------------------------

def _polar_roots(a, xi, eta):
    """u_+^2 > 0 and u_-^2 < 0 of U(u) = -a^2 (u^2 - u_+^2)(u^2 - u_-^2), eta > 0."""
    a, xi, eta = mp.mpf(a), mp.mpf(xi), mp.mpf(eta)
    if a == 0:
        return eta / (eta + xi * xi), None
    b = eta + xi * xi - a * a
    disc = mp.sqrt(b * b + 4 * a * a * eta)
    up2 = (-b + disc) / (2 * a * a)
    um2 = (-b - disc) / (2 * a * a)
    return up2, um2


def _polar_integral(a, xi, eta, u_from):
    """integral_{u_from}^{u_+} du / sqrt(U(u)), 0 <= u_from <= u_+, via u = u_+ sin(chi)."""
    a, xi, eta = mp.mpf(a), mp.mpf(xi), mp.mpf(eta)
    up2, um2 = _polar_roots(a, xi, eta)
    up = mp.sqrt(up2)
    chi0 = mp.asin(min(mp.mpf(1), mp.mpf(u_from) / up))
    if a == 0:
        return (mp.pi / 2 - chi0) / mp.sqrt(eta + xi * xi)
    f = lambda chi: 1 / (a * mp.sqrt(up2 * mp.sin(chi) ** 2 - um2))
    return mp.quad(f, [chi0, mp.pi / 2])


def mino_times_of_crossings(a, xi, eta, theta0, theta_dot_sign, n):
    """Mino times of the first n passages through u = cos(theta) = 0."""
    u0 = mp.cos(mp.mpf(theta0))
    du_sign = -theta_dot_sign                       # du/dtau = -sin(theta) dtheta/dtau
    K = _polar_integral(a, xi, eta, 0)               # quarter period
    if u0 == 0:
        first = mp.mpf(0)
    elif (u0 > 0 and du_sign < 0) or (u0 < 0 and du_sign > 0):
        first = K - _polar_integral(a, xi, eta, abs(u0))            # straight to the equator
    else:
        first = _polar_integral(a, xi, eta, abs(u0)) + K            # out to the turning point and back
    return [first + 2 * K * k for k in range(n)]


def radius_at_mino_time(a, xi, eta, D, tau, r_stop):
    """Radius on the radial motion that starts at r = D inward, at Mino time tau.
    Returns None if the ray has crossed r_stop (captured) or passed back out beyond D."""
    a, xi, eta, D, tau = mp.mpf(a), mp.mpf(xi), mp.mpf(eta), mp.mpf(D), mp.mpf(tau)
    R = lambda r: (r * r + a * a - a * xi) ** 2 - (r * r - 2 * r + a * a) * (eta + (xi - a) ** 2)
    rt = radial_turning_point(float(a), float(xi), float(eta), float(r_stop), float(D))
    if rt is None:
        # captured: tau(r) = int_r^D dr / sqrt(R), R > 0 on [r_stop, D]
        tin = lambda r: mp.quad(lambda x: 1 / mp.sqrt(R(x)), [r, D])
        if tau >= tin(mp.mpf(r_stop)):
            return None
        return mp.findroot(lambda r: tin(r) - tau, (mp.mpf(r_stop), D), solver="anderson")
    # polish the turning point in high precision, divide it out of R, R = (r - r_t) P3(r),
    # and integrate in s = sqrt(r - r_t): dr / sqrt(R) = 2 ds / sqrt(P3(r_t + s^2))
    rt = mp.re(mp.findroot(R, mp.mpf(rt)))
    c = [mp.mpf(x) for x in radial_coeffs(a, xi, eta)]
    q = [c[0]]
    for ck in c[1:4]:
        q.append(ck + q[-1] * rt)                  # synthetic division by (r - r_t)
    P3 = lambda r: ((q[0] * r + q[1]) * r + q[2]) * r + q[3]
    g = lambda s: 2 / mp.sqrt(P3(rt + s * s))
    S = mp.sqrt(D - rt)
    total_in = mp.quad(g, [0, S])
    if tau <= total_in:
        target = total_in - tau                     # int_{r_t}^{r_c} on the inward leg
    else:
        target = tau - total_in                     # outward leg
        if target >= total_in:
            return None
    sc = mp.findroot(lambda s: mp.quad(g, [0, s]) - target, (mp.mpf(0), S), solver="anderson")
    return rt + sc * sc


def exact_crossings(a, xi, eta, D, theta0, theta_dot_sign, n, r_stop):
    """Radii of the first n equatorial crossings (None once the ray is gone)."""
    out = []
    for tau in mino_times_of_crossings(a, xi, eta, theta0, theta_dot_sign, n):
        r = radius_at_mino_time(a, xi, eta, D, tau, r_stop)
        if r is None:
            break
        out.append(float(r))
    return out


# ---------------------------------------------------------------------------
# circular equatorial orbits (Bardeen, Press & Teukolsky 1972), M = 1
# ---------------------------------------------------------------------------

def circular_E(a, r):
    r = mp.mpf(r)
    return (r ** 1.5 - 2 * mp.sqrt(r) + a) / (r ** 0.75 * mp.sqrt(r ** 1.5 - 3 * mp.sqrt(r) + 2 * a))


def circular_L(a, r):
    r = mp.mpf(r)
    return (r * r - 2 * a * mp.sqrt(r) + a * a) / (r ** 0.75 * mp.sqrt(r ** 1.5 - 3 * mp.sqrt(r) + 2 * a))


def circular_Omega(a, r):
    return 1 / (mp.mpf(r) ** 1.5 + a)


def circular_ut(a, r):
    r = mp.mpf(r)
    return (r ** 1.5 + a) / (r ** 0.75 * mp.sqrt(r ** 1.5 - 3 * mp.sqrt(r) + 2 * a))


def isco_by_energy_minimum(a):
    """ISCO as the minimum of the circular-orbit energy E(r)."""
    dE = lambda r: mp.diff(lambda x: circular_E(a, x), r)
    r_ph = 2 * (1 + mp.cos(mp.mpf(2) / 3 * mp.acos(-mp.mpf(a))))    # prograde photon orbit
    lo, hi = r_ph + (mp.mpf(9) - r_ph) * mp.mpf("1e-3"), mp.mpf(9)
    for _ in range(200):                         # bisection on dE/dr: E falls, then rises
        mid = (lo + hi) / 2
        if dE(mid) < 0:
            lo = mid
        else:
            hi = mid
    return (lo + hi) / 2


def page_thorne_flux(a, r, r_ms):
    """Page & Thorne (1974) flux from the conservation laws, by quadrature:
    F = -(1/(4 pi sqrt(-g))) Omega_r / (E - Omega L)^2 int_{r_ms}^r (E - Omega L) L_r dr,
    sqrt(-g) = r on the equator (M = 1, mdot = 1)."""
    E = lambda x: circular_E(a, x)
    L = lambda x: circular_L(a, x)
    Om = lambda x: circular_Omega(a, x)
    Lr = lambda x: mp.diff(L, x)
    integ = mp.quad(lambda x: (E(x) - Om(x) * L(x)) * Lr(x), [r_ms, r])
    Om_r = mp.diff(Om, r)
    return -Om_r / (4 * mp.pi * r * (E(r) - Om(r) * L(r)) ** 2) * integ
