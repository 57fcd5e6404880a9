"""Benchmark: geodesics/s of the GB300 tracer on the Kerr thin-disk scene
(a = 0.9, theta_obs = 60 deg, r_obs = 1000 M, 1024 x 1024 camera over
[-20, 20]^2 M, Dormand-Prince 5(4) at rtol = atol = 1e-10, FP64, disk from the
ISCO to 30 M with up to 3 crossings).

One step = one full image traced by one persistent launch of the tracer
(every pixel: initial data, integration, events, crossing refinement,
emission, constraint monitor).  Rank r of N traces its own image (weak
scaling, no collective on the data path); with --shard the N ranks split one
image into pixel ranges of whole 4-row bands balanced by the step counts of a
previous trace of it (strong scaling; each rank keeps its slice, which
distributed.gather_image can assemble on the host).

Besides the headline, the line carries the other paths on the same scene:
double-float at the headline's tolerance, the mixed paths on the 2048^2 image
(with their FP32-pipe fraction), the prescribed FP64 split, the 64-image
batch, the FP64 and double-float paths at the loosest tolerance that also
meets the mixed path's accuracy (the equal-accuracy comparison), and the
paper's other four integrators.  The roofline denominators are the FP64 and
FP32 FMA rates measured by an FMA-chain probe at the start of the run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tartarus|reference] [--shard]
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
# Unit-count peaks at the maximum SM clock, for reference beside the measured ones:
# 2 DFMA and 128 FFMA per clock per SM.
FP64_PEAK_DERIVED = SM_COUNT * SM_MAX_MHZ * 1e6 * 2 * 2 / 1e12
FP32_PEAK_DERIVED = SM_COUNT * SM_MAX_MHZ * 1e6 * 128 * 2 / 1e12
# Algorithmic FP64 flops of one Dormand-Prince step attempt on the Kerr FP64 path,
# counted from the kernel source of this build (FMA = 2; add, mul, reciprocal and
# sqrt 1 each, the reciprocal's Newton refinement not counted; sin and cos 1 each,
# however they are evaluated -- here by angle addition from the step start):
# 6 flow evaluations x 55 + stage combinations and error sum 222 (stages 2-4 with
# h-scaled coefficients; the error vector without its factor h) + error norm 30 (one
# shared reciprocal) + 1 (h applied to that reciprocal) + step control 5.
FLOW_FLOPS, NORM_FLOPS, CONTROL_FLOPS = 55, 30, 5
FLOPS_PER_STEP = 6 * FLOW_FLOPS + 222 + NORM_FLOPS + 1 + CONTROL_FLOPS
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
# FP64 thread instructions per Dormand-Prince step attempt of the FP64 kernel, from ncu's
# instruction counts on the 512^2 image (7.02e7 attempts): DFMA, DMUL, DADD
FP64_ISSUED_PER_STEP = (260.8, 199.6, 19.5)
# FP32 thread instructions (FFMA + FMUL + FADD) per double-float step attempt, from ncu's
# instruction counts on the 512^2 image
DF_FP32_INST_PER_STEP = 4693
# the same for the double-float kernel on the tabulated metric (256^2 image of its scene)
TABLE_DF_FP32_INST_PER_STEP = 15398
# the same per step attempt of the mixed-pair kernel on the 1024^2 image (its FP32 steps with
# the zone and near-critical double-float steps amortised over all attempts)
MIXED_FP32_INST_PER_STEP = 889
BYTES_OUT_PER_PIXEL = 3 * 3 * 8 + 8 + 8 + 4 + 4 + 1 + 1
# DRAM traffic of the FP64 tracer per launch on the 1024^2 image: ncu's
# dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch (2.6 MB read,
# 51.2 MB written: part of the 103 MB of outputs leaves the L2 during the kernel)
TRAFFIC_BYTES_1024 = 2555392 + 51188480
# host-to-device input of one step: the launch's parameter block (sizeof(tt::LaunchParams<1>):
# solver settings, launch shape and the image descriptor)
DESC_BYTES = 728
# The tolerance of the equal-accuracy comparison: the mixed paths' own, at which the FP64
# and double-float paths also keep |H| <= 1e-6 on every escaped ray of the 2048^2 disk
# image (the next looser ones measured there, 2e-8 and 3e-8, give 1.1e-6 and more) and
# their crossings within 1e-6 of the rtol-1e-10 oracle
EQUAL_ACCURACY_RTOL = 1e-8


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="tartarus", choices=["tartarus", "reference"])
    p.add_argument("--n", type=int, default=1024, help="camera resolution (default: the 1024^2 workload)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget per measurement")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_pair", "double_float",
                                                            "mixed_split"],
                   help="path of the main measurement (default: the FP64 headline)")
    p.add_argument("--no-mixed", action="store_true", help="skip the objects of the other paths")
    p.add_argument("--method", default="dopri5", choices=list(METHODS),
                   help="integrator of the FP64 run (default: Dormand-Prince, the headline)")
    p.add_argument("--no-pairs", action="store_true",
                   help="skip the objects of the other four integrators in the default line")
    p.add_argument("--shard", action="store_true",
                   help="N ranks split one image by pixel ranges balanced by a previous trace's step counts")
    p.add_argument("--critical-band", type=float, default=None,
                   help="mixed paths: near-critical band in M (negative: no escalation; default: the library's)")
    p.add_argument("--zone-factor", type=float, default=None,
                   help="mixed paths: extended-precision zone radius in r_+ (negative: none; default: the library's)")
    p.add_argument("--workload", default="kerr_disk", choices=["kerr_disk", "batch", "table", "e3", "e5", "osiris"],
                   help="kerr_disk: the 1024^2 headline image (default); batch: 64 uneven images in one "
                        "persistent launch, replayed from a CUDA graph; table: the 4096^2 tabulated-metric image")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_pair": 2, "double_float": 3, "mixed_split": 4}


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


def config_dict(sc, world, shard=False):
    extra = {k: v for k, v in (("critical_band", sc.critical_band), ("zone_factor", sc.fp64_radius_factor)) if v != 0.0}
    return {**extra, "workload": sc.name, "nx": sc.nx, "ny": sc.ny, "a": sc.a,
            "theta_obs_deg": round(math.degrees(sc.theta_obs), 6),
            "r_obs": sc.r_obs, "field": [sc.alpha_min, sc.alpha_max], "rtol": sc.rtol, "atol": sc.atol,
            "integrator": METHOD_NAMES[sc.method], "disk": ["isco", sc.r_out], "max_crossings": sc.max_crossings,
            "global_batch": sc.npix * (1 if shard else world), "per_gpu_rays": (sc.npix // world if shard else sc.npix),
            "parallelism": ("shard%d" % world) if shard else ("dp%d" % world),
            "l2": "flushed between timed steps (256 MiB write); working set is a few MB of state + outputs"}


def kernel_name(sc):
    """The tracing kernel the FP64 launch of this scene runs (its tuned block size)."""
    from paper_2609_08989_gb300 import autotune
    block = (autotune.cached(sc) or {}).get("block", 0)
    if sc.method == 0:
        return {256: "trace_kernel64_b256<0,1>", 384: "trace_kernel64_b384<0,1>"}.get(block, "trace_kernel64<0,1>")
    return "trace_kernel_rk<%d,0,1,%d>" % (sc.method, 256 if block in (256, 384) else 128)


def h_stats(out):
    """|H| maxima of escaped and captured rays of a device output dict."""
    import numpy as np
    h = out["h_max"].cpu().numpy()
    esc = out["code"].cpu().numpy() == 0
    r = {}
    if esc.any():
        r.update({"h_max_escaped": float(h[esc].max()), "h_max_escaped_p99": float(np.percentile(h[esc], 99)),
                  "h_max_escaped_median": float(np.median(h[esc]))})
    if (~esc).any():
        r.update({"h_max_captured": float(h[~esc].max()), "h_max_captured_median": float(np.median(h[~esc]))})
    return r


def attempts_of(out):
    return int(out["steps"].sum().item() + out["rejects"].sum().item())


def fp32_roofline(attempts, ms, peaks):
    """Algorithmic FP32 flops of the mixed step over the kernel time, against the
    measured FP32 FMA rate."""
    ach = FLOPS_PER_STEP_F32 * attempts / (ms / 1e3) / 1e12
    inst = MIXED_FP32_INST_PER_STEP * attempts / (ms / 1e3)
    return {"bound": "alu", "achieved": ach, "peak": peaks["fp32"], "unit": "TFLOP/s",
            "frac": ach / peaks["fp32"], "peak_source": peaks["fp32_source"],
            "issued": {"fp32_instructions_per_unit": MIXED_FP32_INST_PER_STEP,
                       "frac_of_fp32_instruction_peak": inst / (peaks["fp32"] / 2 * 1e12),
                       "source": "FFMA + FMUL + FADD per attempt from ncu's counts (mixed pair, 1024^2)"},
            "peak_derived": FP32_PEAK_DERIVED, "frac_of_derived": ach / FP32_PEAK_DERIVED,
            "flops_per_unit": FLOPS_PER_STEP_F32, "traffic": None,
            "unit_of_work": "step attempt, each counted as one FP32 Dormand-Prince step (the double-float "
                            "steps of the zones and of near-critical rays, ~7x the FP32 work, are not "
                            "counted extra)"}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object)
# ---------------------------------------------------------------------------

def time_oracle(sc, seconds, seed=7, nthreads=None):
    """Trace seeded random pixels of the scene with the oracle (all host cores, or
    nthreads) until about ``seconds`` of wall time have passed; returns
    (rays/s, rays, threads, seconds)."""
    import oracle
    from paper_2609_08989_gb300 import scenes
    oracle.build()
    cores = nthreads or os.cpu_count() or 1
    rng_seed = seed
    done, t_used = 0, 0.0
    chunk = 4096 if cores > 1 else 256
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


def cpu_baseline(sc, seconds):
    """The oracle on all host cores: the whole image when a short probe predicts
    it within twice ``seconds``, else seeded random pixels for about ``seconds``;
    and one thread on seeded random pixels."""
    import oracle
    v, rays, cores, tsec = time_oracle(sc, min(1.0, seconds))
    if sc.npix / v <= 2.0 * seconds:
        t0 = time.perf_counter()
        oracle.trace(sc, nthreads=cores)
        tsec = time.perf_counter() - t0
        rays, v = sc.npix, sc.npix / tsec
        sample = "the whole %dx%d image (%.1f s, all %d host cores)" % (sc.nx, sc.ny, tsec, cores)
    else:
        v, rays, cores, tsec = time_oracle(sc, seconds)
        sample = ("%d seeded random pixels of the %dx%d image, in chunks of distinct pixels (%.1f s, all %d host "
                  "cores)" % (rays, sc.nx, sc.ny, tsec, cores))
    v1, rays1, _, t1 = time_oracle(sc, max(2.0, seconds / 3), seed=1007, nthreads=1)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": "%d seeded random pixels in chunks of distinct pixels (%.1f s, one thread)"
                                        % (rays1, t1)}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sc = workload(args.n)
    for _ in range(args.warmup):
        time_oracle(sc, min(2.0, args.cpu_seconds / 4))
    tot_rays, tot_t = 0, 0.0
    for k in range(args.steps):
        v, rays, cores, t = time_oracle(sc, args.cpu_seconds / max(1, args.steps) * 2, seed=7 + 1000 * k)
        tot_rays += rays
        tot_t += t
    value = tot_rays / tot_t
    cfg = config_dict(sc, 1)
    cfg["step"] = "one seeded sample of the image's pixels per step (%d pixels in all)" % tot_rays
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "ms_per_step_note": "wall time per step; each step traces a bounded seeded sample of the image's "
                                "pixels, and value = sampled pixels / wall time",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "%d seeded random pixels of the %dx%d image in chunks of distinct pixels, "
                                       "all host cores" % (tot_rays, sc.nx, sc.ny)},
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


def measure_peaks(local):
    """FP64 and FP32 FMA rates from the FMA-chain probe, with the SM clock seen meanwhile."""
    from paper_2609_08989_gb300 import peaks
    clocks = ClockSampler(local)
    clocks.start()
    p64 = peaks.measure(True, seconds=0.5)
    p32 = peaks.measure(False, seconds=0.5)
    clk = clocks.stop()
    src = "FMA-chain probe in this run (best of 3 launches of ~0.5 s; median SM clock %s MHz)" % (
        clk["sm_mhz"] if clk else "not sampled")
    return {"fp64": p64["tflops"], "fp32": p32["tflops"], "fp64_source": "FP64 " + src, "fp32_source": "FP32 " + src,
            "clocks": clk}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def other_paths(T, args, flush, peaks, main_sc):
    """The double-float, mixed, prescribed-split, batch and equal-accuracy objects."""
    import torch
    from paper_2609_08989_gb300 import scenes
    objs = {}
    reps = max(2, args.steps // 2)
    # the double-float path on the headline image itself (same tolerance, FP64-class results)
    dsc = workload(args.n, "double_float")
    ms, dout = time_variant(T, dsc, reps, 1, flush)
    att = attempts_of(dout)
    eq = FLOPS_PER_STEP * att / (ms / 1e3) / 1e12
    inst = DF_FP32_INST_PER_STEP * att / (ms / 1e3)
    objs["double_float"] = dict(
        {"value": dsc.npix / (ms / 1e3), "unit": UNIT, "ms_per_image": ms, "workload": dsc.name,
         "rtol": dsc.rtol, "arithmetic": "every stage in FP32-pair (double-float, ~48-bit) on the FP32 pipe",
         "rk_step_attempts_per_image": att,
         "fp64_equivalent_tflops": eq, "fp64_equivalent_vs_fp64_peak": eq / peaks["fp64"],
         "fp32_pipe": {"instructions_per_step": DF_FP32_INST_PER_STEP, "achieved_ginst_per_s": inst / 1e9,
                       "peak_ginst_per_s": peaks["fp32"] / 2 * 1e3, "frac": inst / (peaks["fp32"] / 2 * 1e12),
                       "source": "FP32 thread instructions per step from ncu's instruction counts (512^2 image) "
                                 "over the FMA rate measured in this run"}}, **h_stats(dout))
    # the mixed paths on the same scene at 2048^2 (rtol 1e-8, |H| <= 1e-6 on escaped rays)
    for name in ("mixed", "mixed_pair", "mixed_split"):
        msc = workload(2 * args.n, name)
        ms, mout = time_variant(T, msc, reps, 1, flush)
        att = attempts_of(mout)
        objs[name] = dict({"value": msc.npix / (ms / 1e3), "unit": UNIT, "ms_per_image": ms,
                           "workload": msc.name, "rtol": msc.rtol, "rk_step_attempts_per_image": att,
                           "roofline": fp32_roofline(att, ms, peaks)}, **h_stats(mout))
    objs["mixed"]["arithmetic"] = ("FP32 stages (theta relative to the nearest axis crossing), norm and control; "
                                   "FP64 state; double-float steps within 1.5 r_+; rays within 0.15 M of the "
                                   "critical curve traced in double-float at rtol 1e-10")
    objs["mixed_pair"]["arithmetic"] = objs["mixed"]["arithmetic"].replace("FP64 state", "compensated FP32-pair state")
    objs["mixed_split"]["arithmetic"] = ("the prescribed split: FP32 stages; FP64 state, error norm and step "
                                         "control; FP64 steps within 1.5 r_+; FP64 crossing refinement")
    # mixed pair without the near-critical escalation (every ray in FP32 stages)
    msc = workload(2 * args.n, "mixed_pair").replace(critical_band=-1.0)
    ms, mout = time_variant(T, msc, reps, 1, flush)
    objs["mixed_pair_no_escalation"] = {
        "value": msc.npix / (ms / 1e3), "unit": UNIT, "ms_per_image": ms, "workload": msc.name,
        "rk_step_attempts_per_image": attempts_of(mout), "roofline": fp32_roofline(attempts_of(mout), ms, peaks),
        "note": "primary crossings within 1e-5 of the oracle; photon-ring crossings up to ~1e-4"}
    # the 64-image batch (C4): one persistent launch, replayed from a CUDA graph
    imgs = scenes.batch_uneven(64, seed=2609, precision=scenes.MIXED_PAIR)
    rays = sum(s.npix for s in imgs)
    graph = T.TraceGraph(imgs)
    graph.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    bms = []
    for k in range(reps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay()
        b.record(stream)
        torch.cuda.synchronize()
        bms.append(a.elapsed_time(b))
    ms = sum(bms) / len(bms)
    batt = sum(attempts_of(o) for o in graph.outs)
    hesc = max(float(o["h_max"][o["code"] == 0].max().item()) for o in graph.outs)
    objs["batch"] = {"value": rays / (ms / 1e3), "unit": UNIT, "ms_per_replay": ms, "rays": rays,
                     "workload": "batch_uneven_64_images_seed2609_mixed_pair", "images": 64,
                     "res": [min(s.nx for s in imgs), max(s.nx for s in imgs)], "rtol": imgs[0].rtol,
                     "launch": "CUDA graph replay of one tartarus_trace_batch call (%d launch)"
                               % graph.launches_per_replay,
                     "rk_step_attempts": batt, "h_max_escaped": hesc,
                     "roofline": fp32_roofline(batt, ms, peaks)}
    # the tabulated-metric image (C5): Kerr a = 0.998 sampled on a 512 x 256 grid, the
    # 4096^2 camera at rtol 1e-12, traced in double-float (one warm-up, one timed launch)
    tsc = scenes.table_kerr_with_nodes(4 * args.n).replace(precision=scenes.DOUBLE_FLOAT)
    table = T.Table(tsc.table, tsc.r_min, tsc.r_max)
    tout = T.alloc_outputs(tsc.npix)
    T.trace(tsc, out=tout, table=table, stream=stream)
    torch.cuda.synchronize()
    flush.fill_(3)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    T.trace(tsc, out=tout, table=table, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    tms = a.elapsed_time(b)
    tatt = attempts_of(tout)
    tinst = TABLE_DF_FP32_INST_PER_STEP * tatt / (tms / 1e3)
    objs["table"] = dict({"value": tsc.npix / (tms / 1e3), "unit": UNIT, "ms_per_image": tms, "workload": tsc.name,
                          "a": tsc.a, "table": [512, 256], "rtol": tsc.rtol, "precision": "double_float",
                          "rk_step_attempts_per_image": tatt,
                          "fp32_pipe": {"instructions_per_step": TABLE_DF_FP32_INST_PER_STEP,
                                        "frac": tinst / (peaks["fp32"] / 2 * 1e12),
                                        "source": "FP32 thread instructions per step from ncu's instruction counts "
                                                  "(256^2 image of this scene) over the FMA rate measured in this run"},
                          "note": "one timed launch after one warm-up; the FP64 path on this image: "
                                  "bench.py --workload table"}, **h_stats(tout))
    del tout, table
    # equal accuracy: the FP64 and double-float paths on the mixed paths' 2048^2 image at the
    # loosest tolerance that also keeps |H| <= 1e-6 on escaped rays and crossings within 1e-5
    eqa = {}
    for name in ("fp64", "double_float"):
        esc = workload(2 * args.n, name).replace(rtol=EQUAL_ACCURACY_RTOL, atol=EQUAL_ACCURACY_RTOL,
                                                 name="kerr_a0.9_i60_disk_%d_rtol%g" % (2 * args.n,
                                                                                          EQUAL_ACCURACY_RTOL))
        ms, eout = time_variant(T, esc, 2, 1, flush)
        eqa[name] = dict({"value": esc.npix / (ms / 1e3), "unit": UNIT, "ms_per_image": ms,
                          "workload": esc.name, "rtol": esc.rtol, "rk_step_attempts_per_image": attempts_of(eout)},
                         **h_stats(eout))
    mp = objs["mixed_pair"]["value"]
    eqa["mixed_pair_over_fp64"] = mp / eqa["fp64"]["value"]
    eqa["mixed_pair_over_double_float"] = mp / eqa["double_float"]["value"]
    eqa["note"] = ("the FP64 and double-float paths at the mixed paths' rtol 1e-8, where they also keep |H| <= 1e-6 "
                   "on every escaped ray (2e-8 gives 1.1e-6 on this image) and their crossings within 1e-6 of the "
                   "rtol-1e-10 oracle; the mixed pair's crossings are within 1e-5")
    objs["equal_accuracy"] = eqa
    return objs


def integrator_objects(T, args, flush, peaks):
    """The other four integrators of Sec. 3.2 on the same scene and tolerance
    (Verlet: fixed step VERLET_H on a VERLET_N^2 camera, which it needs ~10^5 steps per ray for)."""
    import numpy as np
    pairs = {}
    for name in ("cash_karp", "fehlberg", "gbs", "verlet"):
        psc = workload(VERLET_N if name == "verlet" else args.n, "fp64", name)
        ms, pout = time_variant(T, psc, 1 if name == "verlet" else 2, 1, flush)
        h = pout["h_max"].cpu().numpy()
        code = pout["code"].cpu().numpy()
        esc = code == 0
        att = attempts_of(pout)
        pairs[name] = {"value": psc.npix / (ms / 1e3), "unit": UNIT, "ms_per_image": ms,
                       "workload": psc.name, "step_attempts_per_image": att,
                       "steps_per_ray": att / psc.npix,
                       "h_max_escaped_median": float(np.median(h[esc])) if esc.any() else None,
                       "h_max_escaped": float(h[esc].max()) if esc.any() else None,
                       "captured": int((code == 1).sum()), "other_codes": int((code > 1).sum())}
        if psc.method in FLOPS_PER_STEP_METHOD:
            pach = FLOPS_PER_STEP_METHOD[psc.method] * att / (ms / 1e3) / 1e12
            pairs[name].update({"fp64_tflops": pach, "frac": pach / peaks["fp64"]})
        else:
            pairs[name].update({"h0": psc.h0, "horizon_eps": psc.horizon_eps,
                                "note": "flops per step vary with the fixed-point iterations: no roofline"})
    return pairs


def run_tartarus(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2609_08989_gb300 import distributed as D, tartarus as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc = workload(args.n, args.precision, args.method)
    if args.critical_band is not None:
        sc = sc.replace(critical_band=args.critical_band)
    if args.zone_factor is not None:
        sc = sc.replace(fp64_radius_factor=args.zone_factor)
    T.lib()
    peaks = measure_peaks(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    shard = args.shard and world > 1
    if shard:
        # one image split over the ranks by pixel ranges, balanced by the step counts
        # of a previous trace of the same image (each rank traces it once, in full)
        probe = T.trace(sc)
        torch.cuda.synchronize()
        weights = (probe["steps"] + probe["rejects"]).to(torch.float64)
        if world > 1:
            dist.all_reduce(weights)                   # identical on every rank; makes the split agree
            weights /= world
        begin, count = D.pixel_range(sc.npix, rank, world, weights=weights.cpu().numpy(), align=4 * sc.nx)
        del probe
    else:
        begin, count = 0, sc.npix
    out = T.alloc_outputs(max(count, 1))

    def trace_step(s=stream):
        T.trace(sc, out=out, stream=s, pix_begin=begin, pix_count=count)

    for k in range(max(args.warmup, 0)):
        flush.fill_(k & 0xFF)                     # first touch of the flush buffer stays out of the timing
        trace_step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = T.launch_count()
    barrier()
    clocks.start()
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                     # L2 flush between timed steps
        ev[k][0].record(stream)
        trace_step()
        ev[k][1].record(stream)
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    launches = T.launch_count() - launches0
    step_attempts = attempts_of(out)
    total_ms = t_begin.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    rays_per_step = sc.npix if shard else world * sc.npix
    value = rays_per_step * args.steps / (total_ms / 1e3)
    mean_kern = sum(kern_ms) / len(kern_ms)
    att_all = torch.tensor([step_attempts], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(att_all)
    attempts_total = float(att_all.item())
    hst = h_stats(out)
    spread = None
    if shard:
        # per-rank work spread of the balanced split: attempts and kernel time
        w = torch.tensor([float(step_attempts), mean_kern], dtype=torch.float64, device="cuda")
        allw = [torch.zeros_like(w) for _ in range(world)]
        dist.all_gather(allw, w)
        spread = {"attempts_per_rank": [float(x[0]) for x in allw], "kernel_ms_per_rank": [float(x[1]) for x in allw]}

    # end to end through the host-buffer entry point (outputs copied to pinned host memory)
    host = T.alloc_host_outputs(max(count, 1))
    T.trace_host(sc, out=host, pix_begin=begin, pix_count=count)
    barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        T.trace_host(sc, out=host, pix_begin=begin, pix_count=count)
        _ = float(host["intensity"][0])           # the host reads the result
    barrier()
    e2e_s = time.perf_counter() - e0
    tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    e2e_value = rays_per_step * args.steps / float(tt.item())

    objs = {}
    if not args.no_mixed and args.precision == "fp64" and not shard:
        objs = other_paths(T, args, flush, peaks, sc)
    pairs = {}
    if not args.no_pairs and args.precision == "fp64" and args.method == "dopri5" and not shard:
        pairs = integrator_objects(T, args, flush, peaks)
    if rank == 0:
        fpu = FLOPS_PER_STEP_METHOD.get(sc.method, 0)
        achieved = fpu * step_attempts / (mean_kern / 1e3) / 1e12
        issued = 2 * FP64_ISSUED_PER_STEP[0] + sum(FP64_ISSUED_PER_STEP[1:])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(sc, world, shard),
            "rk_steps_per_s": attempts_total * args.steps / (total_ms / 1e3),
            "rk_step_attempts_per_image": step_attempts if not shard else attempts_total,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fp64"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["fp64"], "peak_source": peaks["fp64_source"],
                         "peak_derived": FP64_PEAK_DERIVED, "frac_of_derived": achieved / FP64_PEAK_DERIVED,
                         "traffic": (TRAFFIC_BYTES_1024 * count / (1024 * 1024)
                                     if TRAFFIC_BYTES_1024 and args.precision == "fp64" and sc.method == 0 else None),
                         "traffic_note": "DRAM bytes of one full-size launch (ncu), scaled by the pixels traced",
                         "kernel": kernel_name(sc), "kernel_ms": mean_kern,
                         "flops_per_unit": fpu,
                         "unit_of_work": "%s step attempt" % METHOD_NAMES[sc.method],
                         "issued": ({"fp64_flops_per_unit": issued,
                                     "tflops": issued * step_attempts / (mean_kern / 1e3) / 1e12,
                                     "frac": issued * step_attempts / (mean_kern / 1e3) / 1e12 / peaks["fp64"],
                                     "source": "DFMA x 2 + DMUL + DADD per step from ncu's instruction counts "
                                               "(512^2 image)"}
                                    if sc.method == 0 else None)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": DESC_BYTES,
                    "d2h_bytes_per_step": BYTES_OUT_PER_PIXEL * count},
            "gpu_launches": launches,
            "clocks": clk,
            "peaks": {"fp64_tflops": peaks["fp64"], "fp32_tflops": peaks["fp32"], "clocks": peaks["clocks"],
                      "fp64_derived": FP64_PEAK_DERIVED, "fp32_derived": FP32_PEAK_DERIVED},
        }
        line.update(hst)
        if spread:
            line["shard"] = spread
        if args.precision != "fp64":
            line["dtype"] = {"mixed": "f32 stages / f64 state", "mixed_pair": "f32 stages / f32-pair state",
                             "double_float": "f32 pair (double-float)",
                             "mixed_split": "f32 stages / f64 state, norm, zones"}[args.precision]
            if args.precision == "double_float":
                line["roofline"] = None
            else:
                line["roofline"] = fp32_roofline(step_attempts, mean_kern, peaks)
        if sc.method not in FLOPS_PER_STEP_METHOD:
            line["roofline"] = None          # Verlet: flops per step vary with its fixed-point iterations
        line.update(objs)
        if pairs:
            line["integrators"] = pairs
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(sc, args.cpu_seconds)
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
    peaks = measure_peaks(local)
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
    attempts = int(sum(attempts_of(o) for o in outs))
    if rank == 0:
        roof = None
        if args.workload == "batch":
            roof = fp32_roofline(attempts, kern_ms, peaks)
        elif args.workload in ("e3", "e5", "osiris") and sc.method in FLOPS_PER_STEP_METHOD:
            fpu = FLOPS_PER_STEP_METHOD[sc.method]
            ach = fpu * attempts / (kern_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": peaks["fp64"], "unit": "TFLOP/s",
                    "frac": ach / peaks["fp64"], "traffic": None, "flops_per_unit": fpu,
                    "unit_of_work": "%s step attempt" % args.method, "peak_source": peaks["fp64_source"]}
        line = {"metric": METRIC, "value": world * rays * args.steps / (total_ms / 1e3), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
                "data": "synthetic", "config": cfg, "rk_step_attempts_per_step": attempts,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk,
                "e2e": None, "roofline": roof}
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
