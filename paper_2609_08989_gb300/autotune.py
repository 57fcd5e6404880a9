"""Autotuner for the persistent tracer's launch shape.

The tracer's speed depends on knobs the hardware decides, not the physics:
threads per block, the register cap, and the warp-phase thresholds of the
persistent loop (how many idle lanes trigger a refill -- the compaction
period -- and how many lanes a batched FP64 phase waits for).  This module
times them on the current GPU with CUDA events (coordinate descent from the
built-in defaults, two sweeps), and keeps the winners per workload class in
``tuned.json`` next to this file, keyed by the device name.  ``tartarus.trace``
and ``trace_batch`` use the cached shape when no explicit ``tune`` is given.

Workload classes: "fp64" (closed-form Kerr, FP64), "mixed" (FP32 stages with
FP64 accumulation), "mixed_pair" (FP32-pair accumulation), "mixed_split" (the
prescribed FP64 split), "double_float"
(every step in double-float), "table" (FP64 on a tabulated metric),
"table_double_float" (double-float on a tabulated metric).  Results are
identical for every shape; only time changes.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Callable, Dict, List, Optional, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tuned.json")
_lock = threading.Lock()
_cache: Optional[dict] = None

# search space per class (0 = the kernel's default)
SPACE: Dict[str, Dict[str, List[int]]] = {
    "fp64": {"block": [128, 256, 384], "reg_variant": [0, 1, 2], "refill": [1, 2, 4, 8, 16, 32],
             "crossing_batch": [2, 4, 8, 16, 24, 32], "blocks_per_sm": [0, 1, 2]},
    "table": {"refill": [1, 2, 4, 8, 16], "crossing_batch": [2, 4, 8, 16, 24], "blocks_per_sm": [0, 1, 2]},
    "mixed": {"refill": [8, 16, 24, 32], "crossing_batch": [8, 16, 24, 32], "fp64_batch": [8, 16, 24, 32],
              "fp64_wait": [64, 256, 1024], "monitor_period": [16, 32, 64], "blocks_per_sm": [0, 1, 2],
              "crit_stride": [1, 2, 4], "crit_refill": [8, 16, 32]},
}
SPACE["mixed_pair"] = SPACE["mixed"]
SPACE["mixed_split"] = SPACE["mixed"]
SPACE["mixed_pair_batch"] = SPACE["mixed"]
SPACE["double_float"] = {"refill": [2, 4, 8, 16, 32], "crossing_batch": [4, 8, 16, 32], "blocks_per_sm": [0, 1, 2]}
SPACE["table_double_float"] = {"refill": [2, 4, 8, 16, 32], "crossing_batch": [4, 8, 16, 32], "fp64_batch": [1, 4, 16]}


def workload_class(sc, batch: bool = False) -> str:
    """The class of a scene; batch: one of several images traced in one launch
    (the mixed-pair batch has a class of its own, its images being uneven)."""
    if sc.metric_kind == 1:
        return "table_double_float" if sc.precision == 3 else "table"
    cls = {0: "fp64", 1: "mixed", 2: "mixed_pair", 3: "double_float", 4: "mixed_split"}[sc.precision]
    if batch and cls == "mixed_pair":
        return "mixed_pair_batch"
    return cls


def _device_key() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def load() -> dict:
    global _cache
    with _lock:
        if _cache is None:
            try:
                with open(CACHE) as f:
                    _cache = json.load(f)
            except (OSError, ValueError):
                _cache = {}
        return _cache


def cached(sc, batch: bool = False) -> Optional[dict]:
    """The tuned shape for this scene's class on the current device, or None."""
    try:
        dev = _device_key()
    except Exception:
        return None
    entry = load().get(dev, {}).get(workload_class(sc, batch))
    if entry is None and batch:
        entry = load().get(dev, {}).get(workload_class(sc))
    return dict(entry["tune"]) if entry else None


def _time(run: Callable[[dict], None], tune: dict, reps: int) -> float:
    import torch
    run(tune)                       # warm-up (and first-touch of outputs)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run(tune)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def search(run: Callable[[dict], None], space: Dict[str, List[int]], reps: int = 2, sweeps: int = 2,
           start: Optional[dict] = None, log: Optional[Callable[[str], None]] = None) -> Tuple[dict, float, list]:
    """Coordinate descent: for each knob in turn keep the fastest value with the
    others fixed; repeat ``sweeps`` times.  Returns (best tune, ms, history)."""
    best = dict(start or {})
    best_ms = _time(run, best, reps)
    history = [(dict(best), best_ms)]
    for _ in range(sweeps):
        improved = False
        for knob, values in space.items():
            for v in values:
                if best.get(knob, 0) == v:
                    continue
                cand = dict(best)
                cand[knob] = v
                ms = _time(run, cand, reps)
                history.append((dict(cand), ms))
                if log:
                    log("%s -> %.2f ms" % (cand, ms))
                if ms < best_ms * 0.995:
                    best, best_ms, improved = cand, ms, True
        if not improved:
            break
    return best, best_ms, history


def tune_scene(sc, reps: int = 2, sweeps: int = 2, save: bool = True, log=None) -> Tuple[dict, float]:
    """Tune the launch shape for scenes like ``sc`` and record it in the cache."""
    from . import tartarus as T
    out = T.alloc_outputs(sc.npix)
    table = T.Table(sc.table, sc.r_min, sc.r_max) if sc.metric_kind == 1 else None
    cls = workload_class(sc)

    def run(tune):
        T.trace(sc, out=out, tune=tune, table=table)

    base_ms = _time(run, {}, reps)
    best, ms, _ = search(run, SPACE[cls], reps=reps, sweeps=sweeps, log=log)
    if table is not None:
        table.destroy()
    if save:
        record(cls, best, ms, base_ms, sc.name)
    return best, ms


def tune_batch(imgs, reps: int = 2, sweeps: int = 2, save: bool = True, log=None) -> Tuple[dict, float]:
    """Tune the launch shape of one batch call over ``imgs`` (closed-form Kerr)."""
    from . import tartarus as T
    outs = [T.alloc_outputs(s.npix) for s in imgs]
    cls = workload_class(imgs[0], batch=True)

    def run(tune):
        T.trace_batch(imgs, outs, tune=tune)

    base_ms = _time(run, {}, reps)
    best, ms, _ = search(run, SPACE[cls], reps=reps, sweeps=sweeps, log=log)
    if save:
        record(cls, best, ms, base_ms, "batch_uneven_%d_images" % len(imgs))
    return best, ms


def record(cls: str, tune: dict, ms: float, base_ms: float, workload: str) -> None:
    data = load()
    dev = _device_key()
    data.setdefault(dev, {})[cls] = {"tune": tune, "ms": ms, "default_ms": base_ms, "workload": workload}
    tmp = CACHE + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


if __name__ == "__main__":
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2609_08989_gb300 import scenes
    which = sys.argv[1:] or ["fp64", "mixed", "mixed_pair", "double_float"]
    todo = {"fp64": lambda: scenes.kerr_disk(1024),
            "mixed": lambda: scenes.kerr_disk_mixed(2048),
            "mixed_pair": lambda: scenes.kerr_disk_mixed(2048).replace(precision=scenes.MIXED_PAIR),
            "mixed_split": lambda: scenes.kerr_disk_mixed(2048).replace(precision=scenes.MIXED_SPLIT),
            "double_float": lambda: scenes.kerr_disk(1024).replace(precision=scenes.DOUBLE_FLOAT),
            "table": lambda: scenes.table_kerr_with_nodes(1024),
            "table_double_float": lambda: scenes.table_kerr_with_nodes(2048).replace(precision=scenes.DOUBLE_FLOAT)}
    for name in which:
        if name == "mixed_pair_batch":
            best, ms = tune_batch(scenes.batch_uneven(64, seed=2609, precision=scenes.MIXED_PAIR),
                                  log=lambda m: print("  " + m, flush=True))
        else:
            best, ms = tune_scene(todo[name](), log=lambda m: print("  " + m, flush=True))
        print("%s: %s  %.2f ms" % (name, best, ms), flush=True)
