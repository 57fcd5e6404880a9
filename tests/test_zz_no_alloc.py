"""The no-allocation batch entry point against the ordinary one.

tartarus_trace_batch_noalloc serves callers that may not allocate device
memory while they run (they budget all GPU memory up front and own every
buffer); it keeps its work-queue counters in a fixed array inside the library.
This file is named to run last: it checks that two calls in a row, through the
C ABI, reproduce tartarus_trace_batch's outputs within the parity tolerances,
both in a fresh process and after the other tests have used the library.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2609_08989_gb300 import scenes
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_batch_matches_batch(orc):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08989_gb300 import tartarus as T
    imgs = [scenes.kerr_disk(40), scenes.schwarzschild_shadow(24), scenes.kerr_disk(33).replace(a=0.5, ny=17)]
    ref = [T.to_numpy(o) for o in T.trace_batch(imgs)]
    torch.cuda.synchronize()
    for call in range(2):                              # the array keeps the last call's counts
        outs = [T.alloc_outputs(s.npix) for s in imgs]
        for o in outs:                                 # poison the outputs: every pixel must be rewritten
            for v in o.values():
                v.fill_(-7)
        status = []
        T.trace_batch_noalloc(imgs, outs, status_out=status)
        torch.cuda.synchronize()
        assert status == [0, 0, 0]
        for sc, o, r in zip(imgs, outs, ref):
            got = T.to_numpy(o)
            parity.compare(orc, sc, got, r, np.arange(sc.npix))
            assert np.array_equal(got["code"], r["code"]) and np.array_equal(got["steps"], r["steps"])


def test_noalloc_rejects_too_many_images():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08989_gb300 import tartarus as T
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
