"""Parity of the CUDA tracer with the FP64 oracle for the integrators of paper
Sec. 3.2 other than Dormand-Prince, through the C ABI.  Cash-Karp and
Fehlberg: closed-form Kerr at both block sizes, every pixel of the full-size
launch, the Hermite refinement, a tabulated metric and a batch of uneven
images.  Gragg-Bulirsch-Stoer: a Kerr disk image, every pixel of the full-size
launch, a table.
Verlet (fixed step): a Kerr disk image at D = 100 M."""
import math

import numpy as np
import pytest

from paper_2609_08989_gb300 import scenes
import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

METHODS = [scenes.CASH_KARP, scenes.FEHLBERG]


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08989_gb300 import tartarus
    tartarus.lib()
    return tartarus


def run(T, sc, **kw):
    out = T.trace(sc, **kw)
    torch.cuda.synchronize()
    return T.to_numpy(out)


@pytest.mark.parametrize("method", METHODS)
def test_kerr_disk_192(T, orc, method):
    sc = scenes.kerr_disk(192).replace(method=method)
    got = run(T, sc, tune={})
    ref = orc.trace(sc)
    rep = parity.compare(orc, sc, got, ref, np.arange(sc.npix))
    assert (got["n_cross"] > 0).mean() > 0.5
    print("method %d kerr disk 192^2:" % method, rep)
    # the 256-thread build takes the same steps
    wide = run(T, sc, tune=dict(block=256, crossing_batch=16))
    for k in got:
        assert np.array_equal(wide[k], got[k]), k


@pytest.mark.parametrize("method", METHODS)
def test_full_image(T, orc, method):
    """The 1024^2 disk image with the tuned launch shape, every pixel."""
    sc = scenes.kerr_disk(1024).replace(method=method)
    got = run(T, sc)
    rep = parity.compare(orc, sc, got, orc.trace(sc), np.arange(sc.npix))
    assert set(np.unique(got["code"])) <= {0, 1}
    print("method %d kerr disk 1024^2, every pixel:" % method, rep)


@pytest.mark.parametrize("method", METHODS)
def test_hermite_refinement(T, orc, method):
    sc = scenes.kerr_disk(64).replace(method=method, refine=scenes.REFINE_HERMITE)
    parity.compare(orc, sc, run(T, sc), orc.trace(sc), np.arange(sc.npix))


@pytest.mark.parametrize("method", METHODS)
def test_table_metric(T, orc, method):
    a = 0.998
    rh = 1.0 + math.sqrt(1 - a * a)
    nodes = orc.kerr_table(1.0, a, 512, 256, rh, 1000.0)
    sc = scenes.table_kerr(32, table=nodes).replace(method=method)
    got = run(T, sc)
    ref = orc.trace(sc)
    # the bars of the Dormand-Prince table test: max(1e-9, 30 x the oracle's own
    # tolerance spread) per crossing
    spread = parity.tolerance_spread(orc, sc, np.arange(sc.npix), ref)
    rep = parity.compare(orc, sc, got, ref, np.arange(sc.npix), rel=1e-9, min_same_steps=0.0,
                         spread=spread, h_ratio_only=True, h_ratio=10.0)
    print("method %d table 32^2:" % method, rep)


@pytest.mark.parametrize("method", METHODS)
def test_batch_of_uneven_images(T, orc, method):
    imgs = [sc.replace(method=method)
            for sc in scenes.batch_uneven(4, seed=31, precision=scenes.FP64, res_lo=16, res_hi=40)]
    outs = T.trace_batch(imgs)
    torch.cuda.synchronize()
    for sc, o in zip(imgs, outs):
        parity.compare(orc, sc, T.to_numpy(o), orc.trace(sc), np.arange(sc.npix))


def test_methods_take_different_steps(T):
    """The method switch reaches the kernel: four adaptive methods, four step counts."""
    sc = scenes.kerr_disk(32)
    steps = [run(T, sc.replace(method=m))["steps"].sum() for m in (0, 1, 2, 3)]
    assert len(set(steps)) == 4, steps


def test_gbs_kerr_disk_128(T, orc):
    sc = scenes.kerr_disk(128).replace(method=scenes.GBS)
    got = run(T, sc, tune={})
    # the extrapolator's error estimate is a difference of extrapolated values, so a
    # few accept/reject decisions flip on rounding (~5e-4 of rays, also between two
    # oracle runs whose inputs differ by 1e-15); such rays take another valid step
    # sequence -- sometimes with the same totals of accepted and rejected steps, so
    # the flip is not visible in the outputs -- and differ by the integration's own
    # error.  Bar: 1e-9, or 30x the oracle's own change at 0.5 to 2 times the
    # tolerance for the crossings whose integration error is larger (GBS at rtol
    # 1e-10 is within 8.8e-10 of the Mino-time crossings).  A ray's |H| maximum is
    # set by single steps whose error estimate cancels, and two valid sequences
    # put it up to ~100x apart: |H| is compared as image statistics.
    ref = orc.trace(sc)
    spread = parity.tolerance_spread(orc, sc, np.arange(sc.npix), ref)
    rep = parity.compare(orc, sc, got, ref, np.arange(sc.npix), rel=1e-9, spread=spread, h_per_ray=False)
    rep.update(parity.h_image_stats(got, ref))
    print("GBS kerr disk 128^2:", rep)
    wide = run(T, sc, tune=dict(block=256, crossing_batch=16))
    for k in got:
        assert np.array_equal(wide[k], got[k]), k


def test_gbs_full_image(T, orc):
    sc = scenes.kerr_disk(1024).replace(method=scenes.GBS)
    got = run(T, sc)
    pix = np.arange(sc.npix)
    ref = orc.trace(sc)
    spread = parity.tolerance_spread(orc, sc, pix, ref)
    rep = parity.compare(orc, sc, got, ref, pix, rel=1e-9, spread=spread, h_per_ray=False)
    rep.update(parity.h_image_stats(got, ref))
    print("GBS kerr disk 1024^2, every pixel:", rep)
    # the bars hold for a third valid integration: the oracle with its camera moved by 1e-15
    other = orc.trace(sc.replace(alpha_min=sc.alpha_min * (1 + 1e-15), beta_max=sc.beta_max * (1 + 1e-15)))
    cal = parity.compare(orc, sc, other, ref, pix, rel=1e-9, min_same_steps=0.0, spread=spread, h_per_ray=False)
    cal.update(parity.h_image_stats(other, ref))
    print("the oracle against itself (camera moved by 1e-15):", cal)


def test_gbs_table_metric(T, orc):
    a = 0.998
    rh = 1.0 + math.sqrt(1 - a * a)
    nodes = orc.kerr_table(1.0, a, 512, 256, rh, 1000.0)
    sc = scenes.table_kerr(32, table=nodes).replace(method=scenes.GBS)
    ref = orc.trace(sc)
    spread = parity.tolerance_spread(orc, sc, np.arange(sc.npix), ref)
    rep = parity.compare(orc, sc, run(T, sc), ref, np.arange(sc.npix), rel=1e-9, min_same_steps=0.0,
                         spread=spread, h_ratio_only=True, h_ratio=10.0)
    print("GBS table 32^2:", rep)


def verlet_scene(n, h0=0.01):
    # the capture radius of the paper's Fig. 2 test (2.05 M at a = 0: eps = 0.025); closer
    # in, p_r ~ 1/Delta outruns the fixed step and the implicit half steps diverge
    return scenes.kerr_disk(n).replace(method=scenes.VERLET, h0=h0, r_obs=100.0, horizon_eps=0.025,
                                       name="kerr_disk_verlet")


def test_verlet_kerr_disk(T, orc):
    sc = verlet_scene(40)
    got = run(T, sc)
    ref = orc.trace(sc)
    rep = parity.compare(orc, sc, got, ref, np.arange(sc.npix))
    assert np.all(got["rejects"] == 0)
    assert set(np.unique(got["code"])) == {0, 1}
    print("Verlet kerr disk 40^2 (D = 100, h = 0.01):", rep)
    # second order: halving the step moves the crossing radii by ~1/4 as much
    half = run(T, sc.replace(h0=0.005))
    quarter = run(T, sc.replace(h0=0.0025))
    m = (got["n_cross"] == half["n_cross"]) & (half["n_cross"] == quarter["n_cross"]) & (got["n_cross"] > 0)
    d1 = np.abs(got["r_cross"][0, m] - half["r_cross"][0, m])
    d2 = np.abs(half["r_cross"][0, m] - quarter["r_cross"][0, m])
    ratio = np.median(d1[d2 > 0] / d2[d2 > 0])
    assert 3.0 < ratio < 5.0, ratio
