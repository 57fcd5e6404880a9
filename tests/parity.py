"""Element-by-element comparison of CUDA outputs with the oracle's.

Rules (FP64 path):
  * termination codes bit-exact, except pixels within the +-1e-6 band around
    the critical curve (classified independently with the radial quartic);
  * crossing counts equal, except band pixels and crossings whose radius lies
    within 1e-8 (relative) of the disk edges;
  * radii and g factors within ``rel`` (relative) -- or ``rel_diverged`` for
    rays whose step counts differ, where a rounding-level accept/reject flip
    made the two sides take different valid step sequences; per-crossing and summed
    intensities within ``rel`` of (value + the image's peak), because F(r)
    vanishes at the ISCO; unused slots exactly 0;
  * |H| maxima (an error measure itself): within 5% on escaped rays; within a
    factor 2 on rays that end at the horizon, where |p_r| ~ 1/(r - r_h) makes
    H sensitive to last-bit differences of the two equivalent flow formulas,
    and on diverged rays when ``rel_diverged`` is given.

Where the step sequence itself is not determined by the method to rounding --
the tabulated metric, whose interpolated flow carries ~1e-12 relative rounding
that moves step sizes, and the extrapolator, whose error estimate is a small
difference of extrapolated values -- two correct integrations at the same
tolerance differ by the integration's own error.  ``tolerance_spread``
measures that error for every crossing with the oracle alone (its change when
the tolerance is halved or doubled), and ``compare(..., spread=...)`` then
allows each crossing max(rel, SPREAD_FACTOR x its spread).
"""
import math

import numpy as np

import kerr_exact as KE

FIELDS = ("r_cross", "g", "I_cross")
# Allowed multiple of the oracle's own tolerance spread.  Largest ratio seen for
# a third valid integration (the oracle with its camera moved by 1e-15 or
# 3e-15): 3.3 on the 40^2 table images at rtol 1e-10 and 1e-12, 18.4 on the
# 1,048,576 rays of the 1024^2 extrapolator image (the tail grows with the
# number of rays: one ray in a million beyond 10).
SPREAD_FACTOR = 30.0


def _rel(x, ref, f):
    ok = ((ref["n_cross"] == x["n_cross"]) & (ref["code"] == x["code"]))[None, :] & (ref[f] != 0)
    den = np.where(ok, np.abs(ref[f]), 1.0)
    return np.where(ok, np.abs(x[f] - ref[f]) / den, 0.0)


SPREAD_TOLERANCES = (0.5, 0.7, 1.4, 2.0)


def tolerance_spread(orc, sc, pix, ref=None):
    """Per crossing (3 x n): the largest relative change of the oracle's r and g
    when its tolerance is scaled by 0.5, 0.7, 1.4 or 2 (0 where a run changes
    the pixel's code or crossing count, or where there is no crossing)."""
    pix = np.asarray(pix, dtype=np.int64)
    if ref is None:
        ref = orc.trace_list(sc, pix)
    sr = np.zeros(ref["r_cross"].shape)
    sg = np.zeros(ref["g"].shape)
    for fac in SPREAD_TOLERANCES:
        x = orc.trace_list(sc.replace(rtol=sc.rtol * fac, atol=sc.atol * fac), pix)
        sr = np.maximum(sr, _rel(x, ref, "r_cross"))
        sg = np.maximum(sg, _rel(x, ref, "g"))
    return sr, sg


def h_image_stats(got, ref, q_rel=0.05, max_ratio=3.0):
    """|H| of the escaped rays compared as image statistics, for an integrator
    whose per-ray maximum is set by single steps whose error estimate cancels
    (the extrapolator: two valid step sequences at the same tolerance put a
    ray's maximum up to ~100x apart): the median, 99th and 99.9th percentiles
    within q_rel (relative) of the oracle's, the image maximum within
    max_ratio.  The oracle against itself (camera moved by 1e-15) keeps them
    within 0.5 % and 0.48-1.23x; at twice its tolerance the median moves 3.2x."""
    def stats(o):
        e = o["h_max"][o["code"] == 0]
        return np.array([np.median(e), np.percentile(e, 99), np.percentile(e, 99.9), e.max()])
    g, r = stats(got), stats(ref)
    q = np.abs(g[:3] / r[:3] - 1.0)
    m = max(g[3] / r[3], r[3] / g[3])
    out = {"h_median_p99_p999_rel": [float(x) for x in q], "h_max_ratio_image": float(m)}
    assert np.all(q <= q_rel), "escaped |H| quantiles off by %s" % q
    assert m <= max_ratio, "escaped |H| image maximum off by %.3g x" % m
    return out


def diverged_spread(orc, sc, pix, got, ref):
    """tolerance_spread on the pixels whose accepted or rejected step counts
    differ between ``got`` and ``ref``, zero on the others.  Given to compare()
    as ``spread``, it leaves the rays that followed the oracle's step sequence
    at ``rel`` and holds each ray that took another valid sequence (an
    accept/reject decision within rounding of err = 1 went the other way) to
    max(rel, SPREAD_FACTOR x its spread), the bar of the tabulated metric."""
    pix = np.asarray(pix, dtype=np.int64)
    sr = np.zeros(ref["r_cross"].shape)
    sg = np.zeros(ref["g"].shape)
    d = np.nonzero((got["steps"] != ref["steps"]) | (got["rejects"] != ref["rejects"]))[0]
    if len(d):
        sub = {k: (v[:, d] if v.ndim == 2 else v[d]) for k, v in ref.items()}
        r, g = tolerance_spread(orc, sc, pix[d], sub)
        sr[:, d] = r
        sg[:, d] = g
    return sr, sg


def pixel_ab(sc, pix):
    i = pix % sc.nx
    j = pix // sc.nx
    al = sc.alpha_min + (i + 0.5) * ((sc.alpha_max - sc.alpha_min) / sc.nx)
    be = sc.beta_min + (j + 0.5) * ((sc.beta_max - sc.beta_min) / sc.ny)
    return al, be


def in_band(orc, sc, pix, width=None):
    """True if the pixel's capture class changes under moves of alpha or beta by
    +-width (1e-6 for the closed-form metric).  A tabulated metric is classified
    with the Kerr spacetime it samples and a band of 1e-4, since interpolation
    (~1e-6 relative) shifts its critical curve."""
    if width is None:
        width = 1e-6 if sc.metric_kind == 0 else 1e-4
    sc = sc.replace(metric_kind=0, table=None) if sc.metric_kind != 0 else sc
    r_stop = orc.rplus(sc.M, sc.a) * (1 + sc.horizon_eps)
    al, be = pixel_ab(sc, pix)

    def klass(a_, b_):
        y = orc.initial_state(sc, a_, b_)
        p = -y[4:]
        E, L = -p[0], p[3]
        Q = p[2] ** 2 + math.cos(sc.theta_obs) ** 2 * (-sc.a ** 2 * E * E + L * L / math.sin(sc.theta_obs) ** 2)
        return KE.classify(sc.a / sc.M, L / E, Q / E ** 2, r_stop, sc.r_obs)

    c0 = klass(al, be)
    return any(klass(al + dx, be + dy) != c0 for dx, dy in ((width, 0), (-width, 0), (0, width), (0, -width)))


def compare(orc, sc, got, ref, pix, rel=1e-9, h_abs=1e-12, h_rel=5e-2, min_same_steps=0.98, report=None,
            rel_diverged=None, h_ratio_only=False, h_ratio=2.0, spread=None, h_per_ray=True):
    """got/ref: dicts of numpy arrays for pixel indices pix (same order).

    h_ratio_only: compare every |H| maximum within a factor 2 (used for the
    tabulated metric, whose C1 interpolant puts kinks in the flow's Jacobian at
    cell edges, where |H| picks up local spikes of the step placement).
    rel_diverged: tolerance for rays whose accepted/rejected step counts differ
    between the two sides (an accept/reject decision taken at err ~ 1 within
    rounding went the other way, so the two are different valid integrations);
    None means such rays get ``rel`` too.
    spread: (r, g) arrays from tolerance_spread; every crossing then gets
    max(rel, SPREAD_FACTOR x its spread) (r and I_cross with the r spread, g
    with the g spread), whatever its step counts.
    h_per_ray: False skips the per-ray |H| comparisons (see h_image_stats)."""
    pix = np.asarray(pix)
    n = len(pix)
    code_bad = np.nonzero(got["code"] != ref["code"])[0]
    band = set(int(q) for q in code_bad if in_band(orc, sc, int(pix[q])))
    unexplained = [int(q) for q in code_bad if int(q) not in band]
    assert not unexplained, "codes differ outside the band at pixels %s" % pix[unexplained[:10]]
    ok = got["code"] == ref["code"]
    r_in = sc.r_in if sc.r_in > 0 else None
    nc_bad = np.nonzero(ok & (got["n_cross"] != ref["n_cross"]))[0]
    for q in nc_bad:
        radii = [x for x in list(ref["r_cross"][:, q]) + list(got["r_cross"][:, q]) if x != 0]
        edges = [sc.r_out] + ([r_in] if r_in else [orc.isco(sc.M, sc.a)])
        near_edge = any(abs(x - e) <= 1e-8 * e for x in radii for e in edges)
        assert near_edge or in_band(orc, sc, int(pix[q])), \
            "crossing count differs at pixel %d: %d vs %d" % (pix[q], got["n_cross"][q], ref["n_cross"][q])
    same = ok & (got["n_cross"] == ref["n_cross"])
    worst = {}
    peak = float(np.abs(ref["I_cross"]).max()) if ref["I_cross"].size else 0.0
    # near-critical rays (photon-ring orbits) amplify last-bit differences
    # exponentially in the number of half-orbits: crossing values of band
    # pixels are exempt, like their codes
    with np.errstate(divide="ignore", invalid="ignore"):
        prel = np.where(ref["r_cross"] != 0, np.abs(got["r_cross"] - ref["r_cross"]) / np.abs(ref["r_cross"]), 0.0)
    diverged = (got["steps"] != ref["steps"]) | (got["rejects"] != ref["rejects"])
    tol_px = np.where(diverged & (rel_diverged is not None), rel_diverged if rel_diverged else rel, rel)
    if spread is not None:
        tol_r = np.maximum(rel, SPREAD_FACTOR * spread[0])
        tol_g = np.maximum(rel, SPREAD_FACTOR * spread[1])
        with np.errstate(divide="ignore", invalid="ignore"):
            grel = np.where(ref["g"] != 0, np.abs(got["g"] - ref["g"]) / np.abs(ref["g"]), 0.0)
        over = ((prel > tol_r) | (grel > tol_g)).any(axis=0)
        for q in np.nonzero(same & over)[0]:
            if in_band(orc, sc, int(pix[q])):
                same[q] = False
                band.add(int(q))
        for f, tol in (("r_cross", tol_r), ("g", tol_g), ("I_cross", tol_r)):
            a, b = got[f][:, same], ref[f][:, same]
            zero = b == 0
            assert np.array_equal(a[zero], b[zero]), "%s: unused slots differ" % f
            den = np.where(zero, 1.0, (np.abs(b) + peak) if f == "I_cross" else np.abs(b))
            ratio = np.where(zero, 0.0, np.abs(a - b) / den) / tol[:, same]
            worst[f + "_over_tol"] = float(ratio.max()) if ratio.size else 0.0
            worst[f] = float((np.where(zero, 0.0, np.abs(a - b) / den)).max()) if ratio.size else 0.0
            assert worst[f + "_over_tol"] <= 1.0, "%s: %.3e of its tolerance max(%.0e, %g x spread)" % (
                f, worst[f + "_over_tol"], rel, SPREAD_FACTOR)
        a, b = got["intensity"][same], ref["intensity"][same]
        nz = b != 0
        assert np.array_equal(a[~nz], b[~nz])
        tol_i = np.maximum(rel, SPREAD_FACTOR * spread[0].max(axis=0))[same]
        di = np.abs(a[nz] - b[nz]) / (np.abs(b[nz]) + peak) / tol_i[nz]
        worst["intensity_over_tol"] = float(di.max()) if di.size else 0.0
        assert worst["intensity_over_tol"] <= 1.0
    for q in np.nonzero(same & (prel.max(axis=0) > tol_px))[0] if spread is None else []:
        if in_band(orc, sc, int(pix[q])):
            same[q] = False
            band.add(int(q))
        else:
            print("crossing mismatch outside the band: pixel", int(pix[q]), "got", got["r_cross"][:, q],
                  "ref", ref["r_cross"][:, q], "steps", got["steps"][q], ref["steps"][q])
    for label, sel, tol in ((("", same & ~diverged, rel), ("_diverged", same & diverged,
                                                             rel_diverged if rel_diverged else rel))
                            if spread is None else ()):
        for f in FIELDS:
            a, b = got[f][:, sel], ref[f][:, sel]
            zero = b == 0
            assert np.array_equal(a[zero], b[zero]), "%s: unused slots differ" % f
            if f == "I_cross":
                # F(r) vanishes at the ISCO, where the relative error of g^4 F is amplified
                # by r F'/F: compare against rel of the value plus rel of the image's peak
                d = np.abs(a[~zero] - b[~zero]) / (np.abs(b[~zero]) + peak)
            else:
                d = np.abs(a[~zero] - b[~zero]) / np.abs(b[~zero])
            worst[f + label] = float(d.max()) if d.size else 0.0
            assert worst[f + label] <= tol, "%s%s: max rel err %.3e > %.1e" % (f, label, worst[f + label], tol)
        a, b = got["intensity"][sel], ref["intensity"][sel]
        nz = b != 0
        assert np.array_equal(a[~nz], b[~nz])
        di = np.abs(a[nz] - b[nz]) / (np.abs(b[nz]) + peak)
        worst["intensity" + label] = float(di.max()) if di.size else 0.0
        assert worst["intensity" + label] <= tol
    # escaped rays end far from the horizon, where H is well conditioned: 5%.
    # Captured rays end at r ~ r_h (1 + 1e-3), where p_r ~ 1/(r - r_h) turns
    # relative state noise of ~1e-13 into ~1e-8 of H: agreement within 2x.
    esc = ok & (ref["code"] == 0) & ~(diverged & (rel_diverged is not None))
    if h_ratio_only or not h_per_ray:
        esc = esc & False
    oth = ok & ~esc
    if not h_per_ray:
        oth = oth & False
    dh = np.abs(got["h_max"][esc] - ref["h_max"][esc])
    lim = h_abs + h_rel * np.abs(ref["h_max"][esc])
    worst["h_max_excess_escaped"] = float((dh / lim).max()) if dh.size else 0.0
    g2, r2 = got["h_max"][oth], ref["h_max"][oth]
    ratio = (np.maximum(g2, r2) + h_abs) / (np.minimum(g2, r2) + h_abs)
    worst["h_max_ratio_other"] = float(ratio.max()) if ratio.size else 1.0
    if dh.size and not np.all(dh <= lim):
        q = int(np.argmax(dh / lim))
        idx = np.nonzero(esc)[0][q]
        raise AssertionError("h_max (escaped) differs by %.3e at pixel %d: got %.6e ref %.6e, steps %d/%d %d/%d"
                             % (dh[q], pix[idx], got["h_max"][idx], ref["h_max"][idx], got["steps"][idx],
                                ref["steps"][idx], got["rejects"][idx], ref["rejects"][idx]))
    assert np.all(ratio <= h_ratio), "h_max (captured) differs by a factor %.2f" % ratio.max()
    same_steps = float(np.mean((got["steps"] == ref["steps"]) & (got["rejects"] == ref["rejects"])))
    worst["same_step_counts"] = same_steps
    assert same_steps >= min_same_steps, same_steps
    worst["band_pixels"] = len(band)
    worst["n"] = n
    if report is not None:
        report.update(worst)
    return worst


def compare_mixed(orc, sc, got, ref, pix, rel=1e-5, band=1e-6):
    """The mixed paths against the FP64 oracle (its own tolerance): codes equal
    outside the +-band around the critical curve; crossing counts equal except
    there or where a crossing lies within ``rel`` of a disk edge; the radius and
    g of every crossing of every other pixel within ``rel`` (relative).
    Returns the largest errors per crossing order."""
    pix = np.asarray(pix)
    code_bad = np.nonzero(got["code"] != ref["code"])[0]
    for q in code_bad:
        assert in_band(orc, sc, int(pix[q]), width=band), "code differs at pixel %d" % pix[q]
    ok = got["code"] == ref["code"]
    r_in = sc.r_in if sc.r_in > 0 else orc.isco(sc.M, sc.a)
    edges = (r_in, sc.r_out)
    skip = np.zeros(len(pix), bool)
    skip[code_bad] = True
    for q in np.nonzero(ok & (got["n_cross"] != ref["n_cross"]))[0]:
        radii = [x for x in list(ref["r_cross"][:, q]) + list(got["r_cross"][:, q]) if x != 0]
        near_edge = any(abs(x - e) <= rel * e for x in radii for e in edges)
        assert near_edge or in_band(orc, sc, int(pix[q]), width=band), \
            "crossing count differs at pixel %d: %d vs %d" % (pix[q], got["n_cross"][q], ref["n_cross"][q])
        skip[q] = True
    er, eg = _rel(got, ref, "r_cross"), _rel(got, ref, "g")
    er[:, skip] = 0.0
    eg[:, skip] = 0.0
    out = {"code_diffs": int(len(code_bad)), "n_cross_diffs": int(skip.sum() - len(code_bad))}
    for k in range(er.shape[0]):
        m = (ref["r_cross"][k] != 0) & ~skip
        out["r%d" % k] = float(er[k][m].max()) if m.any() else 0.0
        out["g%d" % k] = float(eg[k][m].max()) if m.any() else 0.0
        out["n%d" % k] = int(m.sum())
    bad = np.nonzero(((er > rel) | (eg > rel)).any(axis=0))[0]
    assert len(bad) == 0, "crossings off by more than %.0e at pixels %s (r %s, g %s)" % (
        rel, pix[bad[:8]], er[:, bad[:8]].max(axis=0), eg[:, bad[:8]].max(axis=0))
    return out
