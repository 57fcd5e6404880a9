"""Benchmark: geodesics/s of the GB300 tracer on the Kerr thin-disk scene
(a = 0.9, theta_obs = 60 deg, r_obs = 1000 M, 1024 x 1024 camera over
[-20, 20]^2 M, Dormand-Prince 5(4) at rtol = atol = 1e-10, FP64, disk from the
ISCO to 30 M with up to 3 crossings).

One step = one full image traced by one persistent launch of the tracer
(every pixel: initial data, integration, events, crossing refinement,
emission, constraint monitor).  Rank r of N traces its own image (weak
scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tartarus|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "geodesics/sec (Kerr a=0.9, 1024², rtol 1e-10) FP64 vs mixed at |H|≤1e-6; % FP peak"
UNIT = "geodesics/s"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# FP64 pipe: 2 DFMA per clock per SM (measured 1.185 TFLOP/s at 1995 MHz with an FMA-chain probe)
FP64_PEAK_TFLOPS = SM_COUNT * SM_MAX_MHZ * 1e6 * 2 * 2 / 1e12
# Algorithmic FP64 flops of one Dormand-Prince step attempt on the Kerr FP64 path,
# counted from the kernel source of this build (FMA = 2; add, mul, reciprocal and
# sqrt 1 each, the reciprocal's Newton refinement not counted; sin and cos 1 each,
# however they are evaluated -- here by angle addition from the step start):
# 6 flow evaluations x 56 + stage combinations 226 (stages 2-4 with h-scaled
# coefficients) + error norm 30 (one shared reciprocal) + step control 5.
FLOW_FLOPS, NORM_FLOPS, CONTROL_FLOPS = 56, 30, 5
FLOPS_PER_STEP = 6 * FLOW_FLOPS + 226 + NORM_FLOPS + CONTROL_FLOPS
# Cash-Karp and Fehlberg also evaluate the flow six times per step attempt (five
# stages and the new point); their stage sums have one (Fehlberg: e_7 = 0) or two
# (Cash-Karp: b_5 = e_7 = 0) fewer FMA per state component.
# Gragg-Bulirsch-Stoer macro-step (6 columns, 2..12 sub-steps): 36 chain flows + the flow at
# the new point, 12 flops per chain sub-step (y + d, d0 + 2h f), 6 x (4 + 1) to start the
# chains, 15 Aitken-Neville updates x 4 components x 3, the new point and the error (8),
# norm and control.
FLOPS_PER_GBS_STEP = 37 * FLOW_FLOPS + 36 * 12 + 6 * 5 + 15 * 4 * 3 + 8 + NORM_FLOPS + CONTROL_FLOPS
FLOPS_PER_STEP_METHOD = {0: FLOPS_PER_STEP, 1: FLOPS_PER_STEP - 2 * 2 * 4, 2: FLOPS_PER_STEP - 2 * 4,
                         3: FLOPS_PER_GBS_STEP}
METHODS = {"dopri5": 0, "cash_karp": 1, "fehlberg": 2, "gbs": 3, "verlet": 4}
# Verlet's fixed step (the paper gives none) and its capture radius: the paper's own
# stop of its Fig. 2 test (2.05 M at a = 0, eps = 0.025); closer in, p_r ~ 1/Delta
# outruns any fixed step and the implicit half steps diverge
VERLET_H, VERLET_EPS, VERLET_N = 0.01, 0.025, 128
METHOD_NAMES = {v: k for k, v in METHODS.items()}
# The same count for an FP32 step of the mixed paths (the rearranged FP32 flow is 72;
# its stages, norm and control as in the FP64 step before the h-scaling above).
FLOPS_PER_STEP_F32 = 6 * 72 + 232 + 20 + 5
FP32_PEAK_TFLOPS = SM_COUNT * SM_MAX_MHZ * 1e6 * 128 * 2 / 1e12
# FP64 thread instructions per Dormand-Prince step attempt of the FP64 kernel, measured by ncu on
# the 512^2 image (profiles/trace_kernel64_kerr_disk_1024.md): DFMA, DMUL, DADD
FP64_ISSUED_PER_STEP = (281.2, 208.6, 19.5)
# FP32 thread instructions (FFMA + FMUL + FADD) per double-float step attempt, measured by ncu
# on the 512^2 image (profiles/trace_kernel_df_kerr_disk_1024.md)
DF_FP32_INST_PER_STEP = 4693
BYTES_OUT_PER_PIXEL = 3 * 3 * 8 + 8 + 8 + 4 + 4 + 1 + 1
# DRAM traffic of the FP64 tracer per ray: ncu's dram__bytes_read.sum + dram__bytes_write.sum of
# the 512^2 capture (profiles/trace_kernel64_kerr_disk_1024.md) divided by its 262,144 rays
TRAFFIC_BYTES_PER_RAY = (440320.0 + 0.0) / 262144.0
# host-to-device input of one step: the image descriptor (sizeof(tt::ImageDesc)) and the queue reset
DESC_BYTES = 384 + 8


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="tartarus", choices=["tartarus", "reference"])
    p.add_argument("--n", type=int, default=1024, help="camera resolution (default: the 1024^2 workload)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget per measurement")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_pair", "double_float"],
                   help="path of the main measurement (default: the FP64 headline)")
    p.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision objects")
    p.add_argument("--method", default="dopri5", choices=list(METHODS),
                   help="integrator of the FP64 run (default: Dormand-Prince, the headline)")
    p.add_argument("--no-pairs", action="store_true",
                   help="skip the objects of the other four integrators in the default line")
    p.add_argument("--workload", default="kerr_disk", choices=["kerr_disk", "batch", "table", "e3", "e5", "osiris"],
                   help="kerr_disk: the 1024^2 headline image (default); batch: 64 uneven images in one "
                        "persistent launch, replayed from a CUDA graph; table: the 4096^2 tabulated-metric image")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_pair": 2, "double_float": 3}


def workload(n, precision="fp64", method="dopri5"):
    from paper_2609_08989_gb300 import scenes
    if precision == "double_float":
        if method != "dopri5":
            raise SystemExit("the double-float path steps with Dormand-Prince only")
        return scenes.kerr_disk(n).replace(precision=PRECISIONS[precision])
    if precision == "fp64":
        sc = scenes.kerr_disk(n).replace(method=METHODS[method])
        if method == "verlet":
            sc = sc.replace(h0=VERLET_H, horizon_eps=VERLET_EPS, name=sc.name + "_verlet")
        return sc
    if method != "dopri5":
        raise SystemExit("the mixed-precision paths step with Dormand-Prince only")
    return scenes.kerr_disk_mixed(n).replace(precision=PRECISIONS[precision])


def time_variant(T, sc, steps, warmup, flush, tune=None):
    """Device time per image of one scene (CUDA events, L2 flushed between images)."""
    import torch
    out = T.alloc_outputs(sc.npix)
    stream = torch.cuda.current_stream()
    for k in range(max(warmup, 1)):
        flush.fill_(k & 0xFF)
        T.trace(sc, out=out, tune=tune)
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        T.trace(sc, out=out, stream=stream, tune=tune)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return sum(ms) / len(ms), out


def config_dict(sc, world):
    return {"workload": sc.name, "nx": sc.nx, "ny": sc.ny, "a": sc.a, "theta_obs_deg": 60.0,
            "r_obs": sc.r_obs, "field": [sc.alpha_min, sc.alpha_max], "rtol": sc.rtol, "atol": sc.atol,
            "integrator": METHOD_NAMES[sc.method], "disk": ["isco", sc.r_out], "max_crossings": sc.max_crossings,
            "global_batch": sc.npix * world, "per_gpu_rays": sc.npix, "parallelism": "dp%d" % world,
            "l2": "flushed between timed steps (256 MiB write); working set is a few MB of state + outputs"}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object)
# ---------------------------------------------------------------------------

def time_oracle(sc, seconds, seed=7):
    """Trace seeded random pixels of the scene with the oracle on all host cores
    until about ``seconds`` of wall time have passed; returns (rays/s, rays, cores)."""
    import numpy as np
    import oracle
    from paper_2609_08989_gb300 import scenes
    oracle.build()
    cores = os.cpu_count() or 1
    rng_seed = seed
    done, t_used = 0, 0.0
    chunk = 4096
    while t_used < seconds:
        pix = scenes.sample_pixels(sc.npix, chunk, rng_seed)
        t0 = time.perf_counter()
        oracle.trace_list(sc, pix, nthreads=cores)
        dt = time.perf_counter() - t0
        t_used += dt
        done += len(pix)
        rng_seed += 1
        if dt < 0.5 * seconds:
            chunk = min(chunk * 2, 1 << 18)
    return done / t_used, done, cores, t_used


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sc = workload(args.n)
    vals = []
    for _ in range(args.warmup):
        time_oracle(sc, min(2.0, args.cpu_seconds / 4))
    tot_rays, tot_t = 0, 0.0
    for _ in range(args.steps):
        v, rays, cores, t = time_oracle(sc, args.cpu_seconds / max(1, args.steps) * 2)
        vals.append(v)
        tot_rays += rays
        tot_t += t
    value = tot_rays / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sc.npix / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(sc, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "%d seeded random pixels of the %dx%d image, all host cores"
                                       % (tot_rays, sc.nx, sc.ny)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        import statistics
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_tartarus(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2609_08989_gb300 import tartarus as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc = workload(args.n, args.precision, args.method)
    T.lib()
    out = T.alloc_outputs(sc.npix)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    for k in range(max(args.warmup, 0)):
        flush.fill_(k & 0xFF)                     # first touch of the flush buffer stays out of the timing
        T.trace(sc, out=out)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = T.launch_count()
    step_attempts = 0
    barrier()
    clocks.start()
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                     # L2 flush between timed steps
        ev[k][0].record(stream)
        T.trace(sc, out=out, stream=stream)
        ev[k][1].record(stream)
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    launches = T.launch_count() - launches0
    step_attempts = int(out["steps"].sum().item() + out["rejects"].sum().item())
    total_ms = t_begin.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = world * sc.npix * args.steps / (total_ms / 1e3)
    mean_kern = sum(kern_ms) / len(kern_ms)

    # end to end through the host-buffer entry point (outputs copied to pinned host memory)
    host = T.alloc_host_outputs(sc.npix)
    T.trace_host(sc, out=host)
    barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        T.trace_host(sc, out=host)
        _ = float(host["intensity"][0])           # the host reads the result
    barrier()
    e2e_s = time.perf_counter() - e0
    tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    e2e_value = world * sc.npix * args.steps / float(tt.item())

    mixed = {}
    if not args.no_mixed and args.precision == "fp64":
        # the double-float path on the headline image itself (same tolerance, FP64-class results)
        dsc = workload(args.n, "double_float")
        ms, dout = time_variant(T, dsc, max(2, args.steps // 2), 1, flush)
        h = dout["h_max"].cpu().numpy()
        esc = dout["code"].cpu().numpy() == 0
        att = int(dout["steps"].sum().item() + dout["rejects"].sum().item())
        eq = FLOPS_PER_STEP * att / (ms / 1e3) / 1e12
        mixed["double_float"] = {
            "value": dsc.npix / (ms / 1e3), "unit": UNIT, "ms_per_image": ms, "workload": dsc.name,
            "rtol": dsc.rtol, "arithmetic": "every stage in FP32-pair (double-float, ~48-bit) on the FP32 pipe",
            "h_max_escaped": float(h[esc].max()) if esc.any() else None,
            "h_max_escaped_p99": float(np.percentile(h[esc], 99)) if esc.any() else None,
            "rk_step_attempts_per_image": att,
            "fp64_equivalent_tflops": eq, "fp64_equivalent_vs_fp64_peak": eq / FP64_PEAK_TFLOPS,
            "fp32_pipe": {"instructions_per_step": DF_FP32_INST_PER_STEP,
                          "achieved_ginst_per_s": DF_FP32_INST_PER_STEP * att / (ms / 1e3) / 1e9,
                          "peak_ginst_per_s": FP32_PEAK_TFLOPS / 2 * 1e3,
                          "frac": DF_FP32_INST_PER_STEP * att / (ms / 1e3) / (FP32_PEAK_TFLOPS / 2 * 1e12),
                          "source": "FP32 thread instructions per step from the 512^2 ncu capture "
                                    "(profiles/trace_kernel_df_kerr_disk_1024.md)"}}
        # the mixed-precision paths on the same Kerr disk scene at 2048^2, each at
        # the tolerance that keeps |H| <= 1e-6 on escaped rays
        for name in ("mixed", "mixed_pair"):
            msc = workload(2 * args.n, name)
            ms, mout = time_variant(T, msc, max(2, args.steps // 2), 1, flush)
            h = mout["h_max"].cpu().numpy()
            code = mout["code"].cpu().numpy()
            esc = code == 0
            mixed[name] = {"value": msc.npix / (ms / 1e3), "unit": UNIT, "ms_per_image": ms,
                           "workload": msc.name, "rtol": msc.rtol,
                           "accumulation": "fp64" if name == "mixed" else "compensated fp32 pair",
                           "h_max_escaped": float(h[esc].max()) if esc.any() else None,
                           "h_max_escaped_p99": float(np.percentile(h[esc], 99)) if esc.any() else None,
                           "h_max_captured": float(h[~esc].max()) if (~esc).any() else None,
                           "rk_step_attempts_per_image": int(mout["steps"].sum().item() + mout["rejects"].sum().item())}
    pairs = {}
    if not args.no_pairs and args.precision == "fp64" and args.method == "dopri5":
        # the other four integrators of Sec. 3.2 on the same scene and tolerance
        # (Verlet: fixed step VERLET_H on a VERLET_N^2 camera, which it needs ~10^5 steps per ray for)
        for name in ("cash_karp", "fehlberg", "gbs", "verlet"):
            psc = workload(VERLET_N if name == "verlet" else args.n, "fp64", name)
            ms, pout = time_variant(T, psc, max(2, args.steps // 2), 1, flush)
            h = pout["h_max"].cpu().numpy()
            code = pout["code"].cpu().numpy()
            esc = code == 0
            att = int(pout["steps"].sum().item() + pout["rejects"].sum().item())
            pairs[name] = {"value": psc.npix / (ms / 1e3), "unit": UNIT, "ms_per_image": ms,
                           "workload": psc.name, "step_attempts_per_image": att,
                           "steps_per_ray": att / psc.npix,
                           "h_max_escaped_median": float(np.median(h[esc])) if esc.any() else None,
                           "h_max_escaped": float(h[esc].max()) if esc.any() else None,
                           "captured": int((code == 1).sum()), "other_codes": int((code > 1).sum())}
            if psc.method in FLOPS_PER_STEP_METHOD:
                pach = FLOPS_PER_STEP_METHOD[psc.method] * att / (ms / 1e3) / 1e12
                pairs[name].update({"fp64_tflops": pach, "frac": pach / FP64_PEAK_TFLOPS})
            else:
                pairs[name].update({"h0": psc.h0, "horizon_eps": psc.horizon_eps,
                                    "note": "flops per step vary with the fixed-point iterations: no roofline"})
    if rank == 0:
        fpu = FLOPS_PER_STEP_METHOD.get(sc.method, 0)
        achieved = fpu * step_attempts / (mean_kern / 1e3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(sc, world),
            "rk_steps_per_s": world * step_attempts * args.steps / (total_ms / 1e3),
            "rk_step_attempts_per_image": step_attempts,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS,
                         "traffic": (TRAFFIC_BYTES_PER_RAY * sc.npix
                                     if args.precision == "fp64" and sc.method == 0 else None),
                         "traffic_note": "bytes per launch, scaled from a 512^2 ncu capture by rays",
                         "kernel": ("trace_kernel64_b256<0,1>" if sc.method == 0
                                    else "trace_kernel_rk<%d,0,1,256>" % sc.method), "kernel_ms": mean_kern,
                         "peak_source": "FP64 pipe: 152 SMs x 2070 MHz x 2 DFMA/clk (derived)",
                         "flops_per_unit": fpu,
                         "unit_of_work": "%s step attempt" % METHOD_NAMES[sc.method],
                         "issued": ({"fp64_flops_per_unit": 2 * FP64_ISSUED_PER_STEP[0] + sum(FP64_ISSUED_PER_STEP[1:]),
                                     "tflops": (2 * FP64_ISSUED_PER_STEP[0] + sum(FP64_ISSUED_PER_STEP[1:]))
                                               * step_attempts / (mean_kern / 1e3) / 1e12,
                                     "frac": (2 * FP64_ISSUED_PER_STEP[0] + sum(FP64_ISSUED_PER_STEP[1:]))
                                             * step_attempts / (mean_kern / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                                     "source": "DFMA x 2 + DMUL + DADD per step from the 512^2 ncu capture"}
                                    if sc.method == 0 else None)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": DESC_BYTES,
                    "d2h_bytes_per_step": BYTES_OUT_PER_PIXEL * sc.npix},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if args.precision != "fp64":
            line["dtype"] = {"mixed": "f32 stages / f64 state", "mixed_pair": "f32 stages / f32-pair state",
                             "double_float": "f32 pair (double-float)"}[args.precision]
            line["roofline"] = None          # the FP64 flop count does not describe the mixed step
        if sc.method not in FLOPS_PER_STEP_METHOD:
            line["roofline"] = None          # Verlet: flops per step vary with its fixed-point iterations
        line.update(mixed)
        if pairs:
            line["integrators"] = pairs
        if not args.no_cpu_baseline:
            v, rays, cores, tsec = time_oracle(sc, args.cpu_seconds)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": "%d seeded random pixels of the %dx%d image (%.1f s)"
                                              % (rays, sc.nx, sc.ny, tsec)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_workload(args):
    """The batched (C4) and tabulated-metric (C5) workloads: same JSON line format."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2609_08989_gb300 import scenes, tartarus as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    T.lib()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    table = None
    if args.workload == "batch":
        imgs = scenes.batch_uneven(64, seed=2609, precision=scenes.MIXED_PAIR)
        rays = sum(s.npix for s in imgs)
        graph = T.TraceGraph(imgs)
        step = graph.replay
        launches_per_step = graph.launches_per_replay
        outs = graph.outs
        name = "batch_uneven_64_images_seed2609_mixed_pair"
        dtype = "f32 stages / f32-pair state"
        cfg = {"workload": name, "images": 64, "rays": rays, "res": [min(s.nx for s in imgs), max(s.nx for s in imgs)],
               "rtol": imgs[0].rtol, "precision": "mixed_pair", "launch": "CUDA graph replay of one batch call"}
        direct = lambda: T.trace_batch(imgs, outs)
    elif args.workload == "table":
        sc = scenes.table_kerr_with_nodes(args.n if args.n != 1024 else 4096)
        if args.precision not in ("fp64", "double_float"):
            raise SystemExit("tabulated metrics are traced in FP64 or double-float")
        sc = sc.replace(precision=PRECISIONS[args.precision])
        table = T.Table(sc.table, sc.r_min, sc.r_max)
        out = T.alloc_outputs(sc.npix)
        rays = sc.npix
        step = lambda: T.trace(sc, out=out, table=table, stream=stream)
        launches_per_step = 1
        outs = [out]
        name = sc.name
        dtype = "f64" if args.precision == "fp64" else "f32 pair (double-float)"
        cfg = {"workload": name, "nx": sc.nx, "ny": sc.ny, "a": sc.a, "table": [512, 256], "rtol": sc.rtol,
               "precision": args.precision}
        direct = None
    else:
        # the paper's own scenes: Fig. 3 (e3), Table 1 (e5), the OSIRIS shadow of Figs. 5-6
        make = {"e3": scenes.kerr_e3, "e5": scenes.schwarzschild_e5, "osiris": scenes.osiris_scene}
        sc = make[args.workload](args.n).replace(method=METHODS[args.method])
        if args.method == "verlet":
            sc = sc.replace(h0=VERLET_H, horizon_eps=VERLET_EPS)
        out = T.alloc_outputs(sc.npix)
        rays = sc.npix
        step = lambda: T.trace(sc, out=out, stream=stream)
        launches_per_step = 1
        outs = [out]
        name = sc.name
        dtype = "f64"
        cfg = {"workload": name, "nx": sc.nx, "ny": sc.ny, "a": sc.a, "r_obs": sc.r_obs,
               "theta_obs_deg": round(sc.theta_obs * 180.0 / math.pi, 6),
               "field": [sc.alpha_min, sc.alpha_max], "disk": bool(sc.disk_enabled), "doppler": sc.doppler,
               "rtol": sc.rtol, "integrator": args.method, "precision": "fp64"}
        direct = None
    for k in range(max(args.warmup, 0)):
        flush.fill_(k & 0xFF)
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    tt = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    total_ms = float(tt.item())
    kern_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    attempts = int(sum(o["steps"].sum().item() + o["rejects"].sum().item() for o in outs))
    if rank == 0:
        fpu = None
        if args.workload == "batch":
            fpu, flops = FLOPS_PER_STEP_F32, FLOPS_PER_STEP_F32 * attempts
            peak, unit = FP32_PEAK_TFLOPS, "TFLOP/s"
            work = "FP32 Dormand-Prince step attempt (FP64 side work not counted)"
            src = "FP32 pipe: 152 SMs x 2070 MHz x 128 FFMA/clk (derived)"
        elif args.workload in ("e3", "e5", "osiris") and sc.method in FLOPS_PER_STEP_METHOD:
            fpu = FLOPS_PER_STEP_METHOD[sc.method]
            flops, peak, unit = fpu * attempts, FP64_PEAK_TFLOPS, "TFLOP/s"
            work = "%s step attempt" % args.method
            src = "FP64 pipe: 152 SMs x 2070 MHz x 2 DFMA/clk (derived)"
        else:
            flops, peak, unit = None, FP64_PEAK_TFLOPS, "TFLOP/s"
        line = {"metric": METRIC, "value": world * rays * args.steps / (total_ms / 1e3), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
                "data": "synthetic", "config": cfg, "rk_step_attempts_per_step": attempts,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk,
                "e2e": None}
        if flops is not None:
            ach = flops / (kern_ms / 1e3) / 1e12
            line["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                                "traffic": None, "flops_per_unit": fpu, "unit_of_work": work,
                                "peak_source": src}
        if args.workload in ("e3", "e5", "osiris"):
            # the paper's hardware-independent figure: wall time per photon per integration step
            line["ns_per_photon_step"] = total_ms / args.steps * 1e6 / max(attempts, 1)
        if direct is not None:
            direct()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            direct()
            b.record(stream)
            torch.cuda.synchronize()
            line["direct_call"] = {"value": rays / (a.elapsed_time(b) / 1e3), "unit": UNIT,
                                   "ms": a.elapsed_time(b)}
        print(json.dumps(line), flush=True)
    if table is not None:
        table.destroy()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "kerr_disk":
        run_workload(args)
    else:
        run_tartarus(args)


if __name__ == "__main__":
    main()
