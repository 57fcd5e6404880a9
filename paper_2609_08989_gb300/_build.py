"""Build the CUDA libraries in-tree (nvcc, sm_103a only): libtartarus.so (the
tracer behind include/tartarus.h) and libtt_peaks.so (the FMA-chain probe of
the FP64 and FP32 pipes that the benchmark's roofline divides by).

The translation units are compiled in parallel and linked with the static CUDA
runtime; the results land in paper_2609_08989_gb300/_build/.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libtartarus.so")
DEBUG_BUILD = os.path.join(BUILD, "bounds_check")
DEBUG_SO = os.path.join(BUILD, "libtartarus_debug.so")
PEAKS_SRC = "tt_peaks.cu"
PEAKS_SO = os.path.join(BUILD, "libtt_peaks.so")
SOURCES = ["tt_capi.cu", "tt_kernel64.cu", "tt_kernel_mixed.cu", "tt_kernel_split.cu", "tt_kernel_ck.cu", "tt_kernel_f.cu",
           "tt_kernel_gbs.cu", "tt_kernel_verlet.cu", "tt_kernel_df.cu"]
HEADERS = ["tt_internal.h", "tt_device.cuh", "tt_df.cuh", "tt_trace.cuh", "tt_kernel_rk.cuh", os.path.join("..", "..", "include", "tartarus.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
# The FP64 kernels write every fused multiply-add explicitly; without contraction
# by the compiler each build (block size, batch width) rounds alike, so results
# do not depend on the launch shape.
NO_CONTRACT = {"tt_kernel64.cu", "tt_kernel_ck.cu", "tt_kernel_f.cu", "tt_kernel_gbs.cu", "tt_kernel_verlet.cu"}


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def build_peaks(force: bool = False) -> str:
    """Compile (if stale) and return the path of libtt_peaks.so."""
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(CSRC, PEAKS_SRC)
    if not force and os.path.exists(PEAKS_SO) and os.path.getmtime(PEAKS_SO) >= os.path.getmtime(src):
        return PEAKS_SO
    tmp = PEAKS_SO + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), *ARCH, *FLAGS, "-shared", "-cudart", "static", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (PEAKS_SRC, r.stdout, r.stderr))
    os.replace(tmp, PEAKS_SO)
    return PEAKS_SO


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) both libraries and return the path of libtartarus.so."""
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(1) as side:
        peaks = side.submit(build_peaks, force)
        so = _build_tracer(force, verbose)
        peaks.result()
    return so


def build_debug(force: bool = False) -> str:
    """The bounds-checking build (TT_BOUNDS_CHECK: every output store checked
    and an out-of-range one counted): libtartarus_debug.so, a test artefact
    compiled on demand."""
    return _build_tracer(force, False, debug=True)


def _build_tracer(force: bool, verbose: bool, debug: bool = False) -> str:
    so = DEBUG_SO if debug else SO
    odir = DEBUG_BUILD if debug else BUILD
    os.makedirs(odir, exist_ok=True)
    if not force and os.path.exists(so) and os.path.getmtime(so) >= _newest_input():
        return so
    objs = []

    def compile_one(src):
        obj = os.path.join(odir, src.replace(".cu", ".o"))
        extra = ["-fmad=false"] if src in NO_CONTRACT else []
        if debug:
            extra.append("-DTT_BOUNDS_CHECK")
        cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = so + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
