"""The autotuner on the device: a coordinate-descent search over launch shapes
times real launches, keeps the fastest, and every shape it tries gives the
same results (bit for bit on the FP64 path; on the mixed paths all but the
sampled |H| maxima, whose sampling follows the warps' iterations)."""
import numpy as np
import pytest

from paper_2609_08989_gb300 import autotune, scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08989_gb300 import tartarus
    tartarus.lib()
    return tartarus


def _search(T, sc, space):
    out = T.alloc_outputs(sc.npix)
    results = []

    def run(tune):
        T.trace(sc, out=out, tune=tune)
        torch.cuda.synchronize()
        results.append((dict(tune), T.to_numpy(out)))

    best, ms, hist = autotune.search(run, space, reps=1, sweeps=1)
    return best, ms, hist, results


def test_search_fp64_shapes_identical(T):
    sc = scenes.kerr_disk(96)
    space = {"block": [128, 256], "refill": [4, 32], "crossing_batch": [8, 32]}
    best, ms, hist, results = _search(T, sc, space)
    assert len(hist) >= 1 + sum(len(v) - 1 for v in space.values()) - 1
    assert ms <= hist[0][1] * 1.0001
    ref = results[0][1]
    for tune, got in results:
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (tune, k)


def test_search_mixed_pair_shapes_agree(T):
    sc = scenes.kerr_disk(128).replace(precision=scenes.MIXED_PAIR, rtol=scenes.MIXED_RTOL, atol=scenes.MIXED_RTOL)
    space = {"crit_stride": [1, 2], "crit_refill": [8, 32], "refill": [16, 32], "fp64_batch": [8, 16]}
    best, ms, hist, results = _search(T, sc, space)
    ref = results[0][1]
    for tune, got in results:
        for k in ref:
            if k != "h_max":
                assert np.array_equal(got[k], ref[k]), (tune, k)
