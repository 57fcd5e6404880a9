"""The paper's Fig. 3 image (Sec. 4.2, Kerr a = 0.5, D = 100 M, 85 deg) from
the oracle, against what the figure shows: the approaching (left) side of the
disk outshines the receding side with the Doppler factor, the emission is left-
right symmetric without it (up to frame dragging), and lensed secondary images
appear above and below the shadow.  Also the host logic of the image products."""
import json

import numpy as np
import pytest

from paper_2609_08989_gb300 import products, scenes

N = 64


@pytest.fixture(scope="module")
def e3(orc):
    on = scenes.kerr_e3(N)
    return on, orc.trace(on), orc.trace(on.replace(doppler=0))


def test_doppler_breaks_left_right_symmetry(e3):
    sc, on, off = e3
    lr_on = products.left_right_ratio(products.image(on, sc), sc)
    lr_off = products.left_right_ratio(products.image(off, sc), sc)
    assert lr_on > 2.0, lr_on                  # approaching side (alpha < 0) beamed
    assert abs(lr_off - 1.0) < 0.1, lr_off     # intrinsic emission symmetric


def test_redshift_factors(e3):
    sc, on, off = e3
    m = on["n_cross"] > 0
    g_on, g_off = on["g"][0, m], off["g"][0, m]
    assert np.all(g_off < 1.0)                 # gravitational and transverse redshift only
    assert g_on.max() > 1.0                    # blueshift on the approaching side
    assert np.array_equal(on["code"], off["code"]) and np.array_equal(on["r_cross"], off["r_cross"])


def test_lensed_images_above_and_below_shadow(e3):
    """Unlensed, a flat disk out to r_out seen at 85 deg projects into
    |beta| <= r_out cos(85 deg) ~ 2.6 M; the lensed images of its far side reach
    well beyond that on both sides of the shadow."""
    sc, on, _ = e3
    nc = products.image(on, sc, "n_cross")
    beta = sc.beta_min + (np.arange(sc.ny) + 0.5) * (sc.beta_max - sc.beta_min) / sc.ny
    flat = sc.r_out * np.cos(sc.theta_obs)
    rows = beta[np.nonzero((nc >= 1).any(axis=1))[0]]
    assert rows.max() > 2 * flat and rows.min() < -2 * flat
    assert (products.image(on, sc, "code") == 1).sum() > 0
    assert (nc >= 2).sum() > 0                 # rays that cross the disk twice (higher-order images)


def test_image_products_host_logic(tmp_path):
    sc = scenes.kerr_e3(4).replace(ny=3)
    out = {"intensity": np.arange(12.0), "r_cross": np.arange(36.0).reshape(3, 12)}
    img = products.image(out, sc)
    assert img.shape == (3, 4) and img[1, 2] == 6.0          # p = j * nx + i
    assert products.image(out, sc, "r_cross", 1)[0, 0] == 12.0
    with pytest.raises(ValueError):
        products.image(out, sc, "r_cross")
    with pytest.raises(ValueError):
        products.image({"intensity": np.zeros(5)}, sc)
    lr = products.left_right_ratio(np.array([[1.0, 2.0, 3.0, 4.0]] * 3), sc)
    assert lr == pytest.approx(3.0 / 7.0)
    path = str(tmp_path / "m.npz")
    products.save_npz(path, sc, {"intensity": img})
    z = np.load(path)
    assert np.array_equal(z["intensity"], img)
    meta = json.loads(str(z["scene"]))
    assert meta["a"] == 0.5 and meta["nx"] == 4 and meta["name"] == sc.name
