"""Run by tests/test_gpu_bounds_check.py in a process of its own: every kernel
family through the bounds-checking build of the library (every output store
checked against its buffer; an out-of-range one skipped and counted), on small
cases that cover ragged pixel ranges, single pixels, batches and every
precision and integrator.  Prints one JSON line: per case the fault count and
the parity result against the oracle."""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import parity  # noqa: E402
from paper_2609_08989_gb300 import scenes, tartarus as T  # noqa: E402


def poisoned(n):
    out = T.alloc_outputs(n)
    for v in out.values():
        v.fill_(-9)
    return out


def main():
    T.use_bounds_check_build(True)
    assert "bounds-checking" in T.version(), T.version()
    assert T.bounds_faults() == 0
    a = 0.998
    rh = 1.0 + math.sqrt(1 - a * a)
    table = scenes.table_kerr(24, table=oracle.kerr_table(1.0, a, 512, 256, rh, 1000.0))
    cases = [
        ("fp64_kerr_64", scenes.kerr_disk(64), {}),
        ("fp64_ragged", scenes.kerr_disk(97).replace(ny=83), dict(pix_begin=1234, pix_count=2345)),
        ("fp64_last_pixel", scenes.kerr_disk(33), dict(pix_begin=33 * 33 - 1, pix_count=1)),
        ("fp64_badpixels", scenes.kerr_disk(40).replace(r_obs=15.0), {}),
        ("mixed_64", scenes.kerr_disk(64).replace(precision=scenes.MIXED, rtol=1e-8, atol=1e-8), {}),
        ("mixed_pair_ragged", scenes.kerr_disk(72).replace(precision=scenes.MIXED_PAIR, rtol=1e-8, atol=1e-8),
         dict(pix_begin=100, pix_count=3001)),
        ("mixed_split_48", scenes.kerr_disk(48).replace(precision=scenes.MIXED_SPLIT, rtol=1e-8, atol=1e-8), {}),
        ("double_float_64", scenes.kerr_disk(64).replace(precision=scenes.DOUBLE_FLOAT), {}),
        ("cash_karp_48", scenes.kerr_disk(48).replace(method=scenes.CASH_KARP), {}),
        ("fehlberg_48", scenes.kerr_disk(48).replace(method=scenes.FEHLBERG), {}),
        ("gbs_32", scenes.kerr_disk(32).replace(method=scenes.GBS), {}),
        ("verlet_16", scenes.kerr_disk(16).replace(method=scenes.VERLET, h0=0.01, r_obs=100.0, horizon_eps=0.025), {}),
        ("table_fp64_24", table, {}),
        ("table_df_24", table.replace(precision=scenes.DOUBLE_FLOAT), {}),
    ]
    res = {}
    for name, sc, kw in cases:
        n = kw.get("pix_count", sc.npix)
        out = poisoned(n)
        T.trace(sc, out=out, **kw)
        torch.cuda.synchronize()
        got = T.to_numpy(out)
        faults = T.bounds_faults()
        unwritten = int((got["code"] == -9).sum())
        begin = kw.get("pix_begin", 0)
        pix = np.arange(begin, begin + n)
        ref = oracle.trace(sc.replace(precision=scenes.FP64) if sc.precision != scenes.DOUBLE_FLOAT else sc,
                           pix_begin=begin, npix=n)
        same_codes = float(np.mean(got["code"] == ref["code"]))
        res[name] = {"faults": faults, "unwritten": unwritten, "same_codes": same_codes}
    # a batch of uneven images in one launch, and the no-allocation entry point
    imgs = scenes.batch_uneven(6, seed=3, precision=scenes.MIXED_PAIR, res_lo=8, res_hi=40)
    outs = [poisoned(s.npix) for s in imgs]
    T.trace_batch(imgs, outs)
    outs2 = [poisoned(s.npix) for s in imgs]
    T.trace_batch_noalloc(imgs, outs2)
    torch.cuda.synchronize()
    res["batch_and_noalloc"] = {"faults": T.bounds_faults(),
                                "unwritten": int(sum((o["code"] == -9).sum().item() for o in outs + outs2)),
                                "same_codes": 1.0}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
