"""The no-allocation batch entry point against the ordinary one.

tartarus_trace_batch_noalloc serves callers that may not allocate device
memory while they run (they budget all GPU memory up front and own every
buffer); it keeps its work-queue counters in a fixed array inside the library.
This file is named to run last: it checks that two calls in a row, through the
C ABI, reproduce tartarus_trace_batch's outputs within the parity tolerances,
both in a fresh process and after the other tests have used the library --
with one launch, with the 65-to-1024-image batches that take one counter
slot per chunk of 64 images, and at the 1024-image limit.
"""
import ctypes as C

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


def poisoned(T, imgs):
    outs = [T.alloc_outputs(s.npix) for s in imgs]
    for o in outs:                                 # every pixel must be rewritten
        for v in o.values():
            v.fill_(-7)
    return outs


def test_noalloc_batch_matches_batch(T, orc):
    imgs = [scenes.kerr_disk(40), scenes.schwarzschild_shadow(24), scenes.kerr_disk(33).replace(a=0.5, ny=17)]
    ref = [T.to_numpy(o) for o in T.trace_batch(imgs)]
    torch.cuda.synchronize()
    for call in range(2):                              # the array keeps the last call's counts
        outs = poisoned(T, imgs)
        status = []
        T.trace_batch_noalloc(imgs, outs, status_out=status)
        torch.cuda.synchronize()
        assert status == [0, 0, 0]
        for sc, o, r in zip(imgs, outs, ref):
            got = T.to_numpy(o)
            parity.compare(orc, sc, got, r, np.arange(sc.npix))
            assert np.array_equal(got["code"], r["code"]) and np.array_equal(got["steps"], r["steps"])


def tiny_images(n, seed):
    """n Kerr-disk images of 1 to 4 pixels (1x1 .. 2x2 cameras), seeded spins."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(rng.integers(1, 3))
        out.append(scenes.kerr_disk(side).replace(
            name="tiny_%d" % k, a=float(rng.uniform(0.0, 0.95)), alpha_min=-8.0 + k % 7, alpha_max=9.0 + k % 5,
            beta_min=-7.0 - k % 3, beta_max=6.0 + k % 4))
    return out


@pytest.mark.parametrize("n", [130, 1024])
def test_noalloc_many_launches(T, orc, n):
    """130 images span three launches (counter slots 0-2), 1024 all sixteen; each
    chunk's counters are zeroed on the stream before its launch, so two calls in
    a row give the same results as tartarus_trace_batch, and as the oracle."""
    imgs = tiny_images(n, seed=n)
    ref = [T.to_numpy(o) for o in T.trace_batch(imgs)]
    torch.cuda.synchronize()
    n0 = T.launch_count()
    for call in range(2):
        outs = poisoned(T, imgs)
        status = []
        T.trace_batch_noalloc(imgs, outs, status_out=status)
        torch.cuda.synchronize()
        assert status == [0] * n
        for o, r in zip(outs, ref):
            got = T.to_numpy(o)
            for k in got:
                assert np.array_equal(got[k], r[k]), k
    assert T.launch_count() - n0 == 2 * ((n + 63) // 64)
    # the oracle on every pixel of a few of them (one per chunk)
    for sc, r in list(zip(imgs, ref))[::64]:
        parity.compare(orc, sc, r, orc.trace(sc), np.arange(sc.npix))


def test_noalloc_rejects_too_many_images(T):
    sc = scenes.kerr_disk(1)
    out = T.alloc_outputs(1)
    n = 1025
    imgs = (T.TTImage * n)()
    for i in range(n):
        imgs[i].metric = T.TTMetric(kind=0, M=1.0, a=0.9, table=None)
        imgs[i].obs = T.TTObserver(sc.r_obs, sc.theta_obs)
        imgs[i].cam = T._camera(sc, 0, 0)
        imgs[i].disk = T._disk(sc)
        imgs[i].out = T._out_struct(out)
    n0 = T.launch_count()
    st = T.lib().tartarus_trace_batch_noalloc(imgs, n, C.byref(T.solver_struct(sc)), None, None, None)
    assert st == T.TT_EINVAL and T.launch_count() == n0


def test_noalloc_reports_every_bad_image_before_launching(T):
    """An invalid image in the third chunk is reported, the others traced."""
    imgs = tiny_images(150, seed=5)
    imgs[140] = imgs[140].replace(r_obs=-1.0)
    outs = poisoned(T, imgs)
    status = []
    T.trace_batch_noalloc(imgs, outs, status_out=status)
    torch.cuda.synchronize()
    assert status[140] == T.TT_EINVAL and status.count(0) == 149
    ref = [T.to_numpy(o) for o in T.trace_batch(imgs[:140])]
    for o, r in zip(outs[:140], ref):
        assert np.array_equal(T.to_numpy(o)["code"], r["code"])
