"""Multi-rank host logic on CPU (gloo, world size 2): pixel ranges partition
the image exactly, weighted ranges balance work, and gathering the ranks'
outputs reproduces the single-process image bit for bit.  The tracer here is
the oracle (no GPU); the GPU path calls the same functions with the C ABI's
pixel range."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_08989_gb300 import distributed as D, scenes


def test_pixel_ranges_partition():
    for npix in (1, 7, 100, 4096):
        for world in (1, 2, 3, 8):
            ranges = [D.pixel_range(npix, r, world) for r in range(world)]
            assert ranges[0][0] == 0
            for (b0, n0), (b1, _) in zip(ranges, ranges[1:]):
                assert b0 + n0 == b1
            assert sum(n for _, n in ranges) == npix
            assert max(n for _, n in ranges) - min(n for _, n in ranges) <= 1
    w = np.ones(100)
    w[:10] = 10.0                      # the first tenth carries half the work
    b, n = D.pixel_range(100, 0, 2, w)
    assert b == 0 and n == 10
    with pytest.raises(ValueError):
        D.pixel_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, result_path):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = scenes.kerr_disk(24)
    begin, out = D.trace_shard(lambda s, b, n: oracle.trace(s, pix_begin=b, npix=n, nthreads=1), sc, rank, world)
    full = D.gather_image(begin, out, sc.npix)
    if rank == 0:
        np.savez(result_path, **full)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_matches_single_process(orc, tmp_path):
    path = str(tmp_path / "img.npz")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, path)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(np.load(path))
    ref = orc.trace(scenes.kerr_disk(24))
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


def _weighted_worker(rank, world, port, result_path):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = scenes.kerr_disk(32).replace(beta_min=-6.0, beta_max=34.0)      # the shadow near the bottom rows
    # the step map of a previous trace of the image (here: the oracle's) as weights
    prev = oracle.trace(sc, nthreads=1)
    weights = (prev["steps"] + prev["rejects"]).astype(np.float64)
    begin, out = D.trace_shard(lambda s, b, n: oracle.trace(s, pix_begin=b, npix=n, nthreads=1), sc, rank, world,
                               weights=weights, align=4 * sc.nx)
    work = [None] * world
    dist.all_gather_object(work, (begin, len(out["code"]), int((out["steps"] + out["rejects"]).sum())))
    full = D.gather_image(begin, out, sc.npix)
    if rank == 0:
        np.savez(result_path, work=np.array(work), **full)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_step_weighted_split(orc, tmp_path):
    """Ranges of whole 4-row bands balanced by a real step map: the two ranks get
    nearly equal work (closer than an equal-pixel split), and the gathered image
    is the single-process one bit for bit."""
    path = str(tmp_path / "img_w.npz")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_weighted_worker, args=(r, 2, port, path)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(np.load(path))
    work = res.pop("work")
    sc = scenes.kerr_disk(32).replace(beta_min=-6.0, beta_max=34.0)      # the shadow near the bottom rows
    ref = orc.trace(sc)
    for k in ref:
        assert np.array_equal(res[k], ref[k]), k
    assert all(b % (4 * sc.nx) == 0 for b, _, _ in work)
    att = ref["steps"].astype(np.int64) + ref["rejects"]
    half = sc.npix // 2
    equal_split = abs(int(att[:half].sum()) - int(att[half:].sum())) / att.sum()
    weighted = abs(int(work[0][2]) - int(work[1][2])) / att.sum()
    print("work imbalance: equal-pixel split %.3f, step-weighted split %.3f" % (equal_split, weighted))
    assert weighted <= equal_split
    # one 4-row band holds at most this share of the work: the balance is within it
    band_share = max(att[k:k + 4 * sc.nx].sum() for k in range(0, sc.npix, 4 * sc.nx)) / att.sum()
    assert weighted <= band_share
