"""The remaining launches at their full sizes, against the oracle on sampled
pixels: the 4096^2 tabulated-metric image (the benchmark's table workload, one
launch), and a camera of 2.5e9 pixels -- beyond 32-bit pixel indices -- traced
over its last rows only."""
import math

import numpy as np
import pytest

from paper_2609_08989_gb300 import scenes
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


def test_table_4096_sampled(T, orc):
    sc = scenes.table_kerr_with_nodes(4096)
    table = T.Table(sc.table, sc.r_min, sc.r_max)
    try:
        out = T.trace(sc, table=table)
        torch.cuda.synchronize()
        got = T.to_numpy(out)
    finally:
        table.destroy()
    assert set(np.unique(got["code"])) <= {0, 1}
    pix = scenes.sample_pixels(sc.npix, 600, 59)
    ref = orc.trace_list(sc, pix)
    sub = {k: (v[:, pix] if v.ndim == 2 else v[pix]) for k, v in got.items()}
    # the bars of the small table test: max(1e-9, 30 x the oracle's own tolerance
    # spread) per crossing
    spread = parity.tolerance_spread(orc, sc, pix, ref)
    rep = parity.compare(orc, sc, sub, ref, pix, rel=1e-9, min_same_steps=0.0, spread=spread,
                         h_ratio_only=True, h_ratio=10.0)
    print("table 4096^2 sampled:", rep)


def test_camera_beyond_32bit_indices(T, orc):
    n = 50000                                   # 2.5e9 pixels
    sc = scenes.kerr_disk(n)
    assert sc.npix > 2 ** 31
    begin = sc.npix - 777
    out = T.trace(sc, pix_begin=begin, pix_count=777)
    torch.cuda.synchronize()
    got = T.to_numpy(out)
    ref = orc.trace(sc, pix_begin=begin, npix=777)
    parity.compare(orc, sc, got, ref, np.arange(begin, begin + 777))
    # the last pixel sits at the top-right corner of the field
    al, be = parity.pixel_ab(sc, sc.npix - 1)
    assert math.isclose(al, sc.alpha_max - 0.5 * (sc.alpha_max - sc.alpha_min) / n)
    assert math.isclose(be, sc.beta_max - 0.5 * (sc.beta_max - sc.beta_min) / n)
