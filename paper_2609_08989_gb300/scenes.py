"""Seeded synthetic scenes: the camera grids, spacetimes and solver settings that
both the CUDA tracer and the FP64 oracle are run on.

This module holds no arithmetic of the method (no metric, no tetrad, no
integrator, no emission): only parameters, the SplitMix64 generator for drawn
scenes, and seeded pixel samples.  A ``Scene`` carries every field both sides
read, by name.

Workloads (the paper's own scenes are synthetic camera grids too, Sec. 4):
  * ``schwarzschild_shadow`` -- a = 0, 64x64 over [-10, 10]^2, r_obs = 1000,
    theta_obs = 90 deg, rtol = atol = 1e-10, no disk.
  * ``kerr_disk`` -- a = 0.9, theta_obs = 60 deg, r_obs = 1000, 1024x1024 over
    [-20, 20]^2, thin disk from the ISCO to 30 M, up to 3 crossings, FP64.
  * ``kerr_disk_mixed`` -- the same scene at 2048x2048 on the mixed path.
  * ``batch_uneven`` -- 64 images drawn with SplitMix64 (seed 2609).
  * ``table_kerr`` -- a = 0.998 sampled to a 512 x 256 table, 85 deg, 4096^2
    over [-25, 25]^2, rtol = atol = 1e-12.
  * ``osiris_scene`` -- a = 0.98, equatorial observer at 1000 M, [-8, 8]^2.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

FP64, MIXED, MIXED_PAIR, DOUBLE_FLOAT, MIXED_SPLIT = 0, 1, 2, 3, 4
REFINE_HENON, REFINE_HERMITE, REFINE_HENON64 = 0, 1, 2
DOPRI5, CASH_KARP, FEHLBERG, GBS, VERLET = 0, 1, 2, 3, 4
METRIC_KERR, METRIC_TABLE = 0, 1


@dataclass
class Scene:
    # spacetime
    metric_kind: int = METRIC_KERR
    M: float = 1.0
    a: float = 0.0
    table: Optional[np.ndarray] = None      # [nth, nr, 20] tabulated metric (metric_kind 1)
    r_min: float = 0.0
    r_max: float = 0.0
    # observer
    r_obs: float = 1000.0
    theta_obs: float = math.pi / 2
    # camera (cell-centred pixels, p = j*nx + i, j ascending in beta)
    nx: int = 64
    ny: int = 64
    alpha_min: float = -10.0
    alpha_max: float = 10.0
    beta_min: float = -10.0
    beta_max: float = 10.0
    # solver
    precision: int = FP64
    rtol: float = 1e-10
    atol: float = 1e-10
    h0: float = 0.0
    h_min: float = 0.0
    max_steps: int = 1_000_000
    horizon_eps: float = 1e-3
    escape_factor: float = 1.1
    refine: int = REFINE_HENON
    method: int = DOPRI5              # integrator (Verlet: fixed step h0 > 0)
    fp64_radius_factor: float = 0.0   # mixed paths, double-float on a table: extended-precision steps below
                                      # factor * r_h (0: 1.5 mixed, 2 on a table; < 0: none)
    fp64_pole_sin: float = 0.0        # the same, where sin(theta) < this (0 or < 0: none)
    critical_band: float = 0.0        # mixed paths: rays this close to the critical curve (units of M) are traced
                                      # in double-float (0: 0.15, none on the prescribed split; < 0: none)
    critical_rtol: float = 0.0        # their rtol = atol (0: 1e-10)
    # disk
    disk_enabled: int = 0
    r_in: float = 0.0            # <= 0: ISCO
    r_out: float = 30.0
    mdot: float = 1.0
    max_crossings: int = 3
    doppler: int = 1
    name: str = ""

    @property
    def npix(self) -> int:
        return self.nx * self.ny

    def replace(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)


def deg(x: float) -> float:
    return x * math.pi / 180.0


def schwarzschild_shadow(n: int = 64) -> Scene:
    return Scene(name="schwarzschild_shadow_%d" % n, a=0.0, theta_obs=deg(90.0), nx=n, ny=n,
                 alpha_min=-10.0, alpha_max=10.0, beta_min=-10.0, beta_max=10.0)


def kerr_disk(n: int = 1024, precision: int = FP64) -> Scene:
    return Scene(name="kerr_a0.9_i60_disk_%d" % n, a=0.9, theta_obs=deg(60.0), nx=n, ny=n,
                 alpha_min=-20.0, alpha_max=20.0, beta_min=-20.0, beta_max=20.0,
                 precision=precision, disk_enabled=1, r_in=0.0, r_out=30.0, mdot=1.0,
                 max_crossings=3)


# Tolerance of the mixed path; chosen by a sweep so that |H| <= 1e-6 and the
# crossing radii stay within 1e-5 of the FP64 oracle.
MIXED_RTOL = 1e-8


def kerr_disk_mixed(n: int = 2048) -> Scene:
    return kerr_disk(n, MIXED).replace(name="kerr_a0.9_i60_disk_mixed_%d" % n,
                                       rtol=MIXED_RTOL, atol=MIXED_RTOL)


def kerr_e3(n: int = 1024, doppler: int = 1) -> Scene:
    """Paper Sec. 4.2, Fig. 3: Kerr a = 0.5 with a thin disk seen from D = 100 M at
    85 deg, with (panel a) or without (panel b) the Doppler factor.  The paper gives
    no field or disk edge: the field [-32, 32]^2 M holds the whole disk out to 30 M
    (its image spans |alpha| <= 30.3 M)."""
    return Scene(name="kerr_a0.5_i85_d100_disk_%d%s" % (n, "" if doppler else "_nodoppler"), a=0.5,
                 r_obs=100.0, theta_obs=deg(85.0), nx=n, ny=n, alpha_min=-32.0, alpha_max=32.0,
                 beta_min=-32.0, beta_max=32.0, disk_enabled=1, r_in=0.0, r_out=30.0, mdot=1.0,
                 max_crossings=3, doppler=doppler)


def schwarzschild_e5(n: int = 1024) -> Scene:
    """Paper Sec. 4.3, Table 1: Schwarzschild with a thin disk seen from D = 100 M.
    The paper gives no inclination, field or tolerance: those of the Fig. 3 scene
    (85 deg, [-32, 32]^2 M, disk to 30 M) and the tolerance of its Fig. 1 tests (1e-10)."""
    return kerr_e3(n).replace(name="schwarzschild_i85_d100_disk_%d" % n, a=0.0)


def osiris_scene(n: int = 1024) -> Scene:
    """Paper Sec. 4.3, Figs. 5-6: the OSIRIS calibration shadow, Kerr a = 0.98, an
    equatorial observer at 1000 M, field [-8, 8]^2 M, no disk (tolerance not given: 1e-10)."""
    return Scene(name="osiris_a0.98_i90_%d" % n, a=0.98, theta_obs=deg(90.0), nx=n, ny=n,
                 alpha_min=-8.0, alpha_max=8.0, beta_min=-8.0, beta_max=8.0)


def table_kerr(n: int = 4096, table: Optional[np.ndarray] = None, nr: int = 512, nth: int = 256,
               r_max: float = 1000.0) -> Scene:
    """Kerr a = 0.998 as a numerical metric; ``table`` is supplied by the caller
    ([nth, nr, 20]; nodes log-spaced from the horizon to r_max)."""
    a = 0.998
    r_h = 1.0 + math.sqrt(1.0 - a * a)        # nodes start at the horizon of the sampled spacetime
    return Scene(name="table_kerr_a0.998_i85_%d" % n, metric_kind=METRIC_TABLE, a=a, table=table,
                 r_min=r_h, r_max=r_max, theta_obs=deg(85.0), nx=n, ny=n,
                 alpha_min=-25.0, alpha_max=25.0, beta_min=-25.0, beta_max=25.0,
                 rtol=1e-12, atol=1e-12, disk_enabled=1, r_out=30.0)


def kerr_table_nodes(M: float, a: float, nr: int, nth: int, r_min: float, r_max: float) -> np.ndarray:
    """Synthetic numerical metric: the Kerr spacetime sampled onto the table
    format of include/tartarus.h ([nth, nr, 20]: for g_tt, g_tphi, g_thth,
    g_phiphi and g^rr the value, d/dr, d/dth, d2/(dr dth)) -- input data for
    the tabulated-metric path, standing in for a numerically generated metric."""
    u = np.log(r_min) + np.arange(nr) * ((np.log(r_max) - np.log(r_min)) / (nr - 1))
    r = np.exp(u)
    r[0], r[-1] = r_min, r_max
    th = np.pi * np.arange(nth) / (nth - 1)
    s, c = np.sin(th), np.cos(th)
    s[0] = s[-1] = 0.0
    c[0], c[-1] = 1.0, -1.0
    R, S, Cc = r[None, :], s[:, None], c[:, None]
    a2 = a * a
    r2 = R * R
    Sig = r2 + a2 * Cc * Cc
    Del = r2 - 2 * M * R + a2
    q = R / Sig
    q_r = (a2 * Cc * Cc - r2) / Sig ** 2
    q_t = 2 * R * a2 * S * Cc / Sig ** 2
    q_rt = 2 * a2 * S * Cc * (a2 * Cc * Cc - 3 * r2) / Sig ** 3
    s2, sc, s4 = S * S, S * Cc, S ** 4
    s3c = s2 * sc
    out = np.zeros((nth, nr, 20))
    f = [
        (-1 + 2 * M * q, 2 * M * q_r, 2 * M * q_t, 2 * M * q_rt),
        (-2 * M * a * s2 * q, -2 * M * a * s2 * q_r, -2 * M * a * (2 * sc * q + s2 * q_t),
         -2 * M * a * (2 * sc * q_r + s2 * q_rt)),
        (Sig, 2 * R + 0 * S, -2 * a2 * sc + 0 * R, 0 * R * S),
        ((r2 + a2) * s2 + 2 * M * a2 * s4 * q, 2 * R * s2 + 2 * M * a2 * s4 * q_r,
         (r2 + a2) * 2 * sc + 2 * M * a2 * (4 * s3c * q + s4 * q_t),
         4 * R * sc + 2 * M * a2 * (4 * s3c * q_r + s4 * q_rt)),
        (Del / Sig, ((2 * R - 2 * M) * Sig - Del * 2 * R) / Sig ** 2, 2 * a2 * sc * Del / Sig ** 2,
         2 * a2 * sc * ((2 * R - 2 * M) * Sig - 4 * R * Del) / Sig ** 3),
    ]
    for k, comps in enumerate(f):
        for j, v in enumerate(comps):
            out[:, :, 4 * k + j] = np.broadcast_to(v, (nth, nr))
    return out


def table_kerr_with_nodes(n: int = 4096) -> Scene:
    """The tabulated-metric workload with its synthetic Kerr table attached."""
    sc = table_kerr(n)
    return sc.replace(table=kerr_table_nodes(1.0, sc.a, 512, 256, sc.r_min, sc.r_max))


# --------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), for the drawn batch of images.
# --------------------------------------------------------------------------
_MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def batch_uneven(n_images: int = 64, seed: int = 2609, precision: int = MIXED,
                 res_lo: int = 128, res_hi: int = 1024) -> List[Scene]:
    """64 images of uneven resolution, spin and inclination; per image, in this
    order: a ~ U[0, 0.998], theta_obs ~ U[5, 85] deg, N = round(exp(U[ln lo, ln hi])),
    half-field F ~ U[15, 25]."""
    g = SplitMix64(seed)
    out = []
    for k in range(n_images):
        a = g.uniform(0.0, 0.998)
        inc = g.uniform(5.0, 85.0)
        n = int(round(math.exp(g.uniform(math.log(res_lo), math.log(res_hi)))))
        half = g.uniform(15.0, 25.0)
        sc = kerr_disk(n, precision).replace(
            name="batch_%02d" % k, a=a, theta_obs=deg(inc), alpha_min=-half, alpha_max=half,
            beta_min=-half, beta_max=half)
        if precision in (MIXED, MIXED_PAIR):
            sc = sc.replace(rtol=MIXED_RTOL, atol=MIXED_RTOL)
        out.append(sc)
    return out


def sample_pixels(npix: int, n: int, seed: int) -> np.ndarray:
    """A fixed seeded sorted subset of n distinct pixel indices out of npix."""
    rng = np.random.default_rng(seed)
    n = min(n, npix)
    return np.sort(rng.choice(npix, size=n, replace=False)).astype(np.int64)
