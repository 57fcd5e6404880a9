"""The paper's own scenes traced on the GPU through the C ABI, against the
oracle: the Fig. 3 Kerr disk image with and without the Doppler factor
(Sec. 4.2), the Table 1 Schwarzschild disk (Sec. 4.3) and the OSIRIS
calibration shadow (Sec. 4.3), small and at the benchmark's 1024^2 (every
pixel); plus the image-product helpers on a GPU render."""
import json

import numpy as np
import pytest

from paper_2609_08989_gb300 import products, scenes
import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08989_gb300 import tartarus
    tartarus.lib()
    return tartarus


def run(T, sc):
    out = T.trace(sc)
    torch.cuda.synchronize()
    return T.to_numpy(out)


@pytest.mark.parametrize("doppler", [1, 0])
def test_e3_parity(T, orc, doppler):
    sc = scenes.kerr_e3(96, doppler=doppler)
    rep = parity.compare(orc, sc, run(T, sc), orc.trace(sc), np.arange(sc.npix))
    print("E3 96^2 doppler=%d:" % doppler, rep)


def test_e5_and_osiris_parity(T, orc):
    for sc in (scenes.schwarzschild_e5(64), scenes.osiris_scene(64)):
        rep = parity.compare(orc, sc, run(T, sc), orc.trace(sc), np.arange(sc.npix))
        print(sc.name, rep)


@pytest.mark.parametrize("make", [scenes.kerr_e3, scenes.schwarzschild_e5, scenes.osiris_scene],
                         ids=["e3", "e5", "osiris"])
def test_scene_full_image_1024(T, orc, make):
    """The scenes at the 1024^2 size the benchmark times them at, every pixel."""
    sc = make(1024)
    got = run(T, sc)
    rep = parity.compare(orc, sc, got, orc.trace(sc), np.arange(sc.npix))
    print(sc.name, "1024^2, every pixel:", rep)


def test_e3_products(T, tmp_path):
    sc = scenes.kerr_e3(256)
    pair = products.doppler_pair(sc)
    on, off = pair["doppler"], pair["no_doppler"]
    assert on["intensity"].shape == (256, 256)
    assert products.left_right_ratio(on["intensity"], sc) > 2.0
    assert abs(products.left_right_ratio(off["intensity"], sc) - 1.0) < 0.1
    assert np.array_equal(on["code"], off["code"])
    path = str(tmp_path / "e3.npz")
    products.save_npz(path, sc, on)
    z = np.load(path)
    assert np.array_equal(z["intensity"], on["intensity"])
    assert json.loads(str(z["scene"]))["theta_obs"] == sc.theta_obs
