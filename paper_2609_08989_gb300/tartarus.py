"""Python binding of the C ABI in include/tartarus.h (ctypes; argument
marshalling only -- every step of the tracer runs in the CUDA library).

PyTorch supplies device memory and streams.  If libtartarus.so is missing or
cannot be loaded, every entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import _build
from .scenes import Scene

TT_OK, TT_EINVAL, TT_ENOMEM, TT_ECUDA, TT_EUNSUPPORTED = 0, -1, -2, -3, -4
CODE_ESCAPED, CODE_CAPTURED, CODE_MAXSTEPS, CODE_UNDERFLOW, CODE_NONFINITE, CODE_BADPIXEL = range(6)
MAX_CROSSINGS = 3
TABLE_NF = 20

EXPORTS = ["tartarus_trace", "tartarus_trace_host", "tartarus_trace_batch", "tartarus_trace_batch_noalloc",
           "tartarus_table_create", "tartarus_table_destroy", "tartarus_table_coefficients",
           "tartarus_error_string", "tartarus_launch_count", "tartarus_debug_faults", "tartarus_version"]


class TTMetric(C.Structure):
    _fields_ = [("kind", C.c_int), ("M", C.c_double), ("a", C.c_double), ("table", C.c_void_p)]


class TTObserver(C.Structure):
    _fields_ = [("r_obs", C.c_double), ("theta_obs", C.c_double)]


class TTCamera(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("alpha_min", C.c_double), ("alpha_max", C.c_double),
                ("beta_min", C.c_double), ("beta_max", C.c_double), ("pix_begin", C.c_longlong),
                ("pix_count", C.c_longlong)]


class TTSolver(C.Structure):
    _fields_ = [("method", C.c_int), ("precision", C.c_int), ("rtol", C.c_double), ("atol", C.c_double),
                ("h0", C.c_double), ("h_min", C.c_double), ("max_steps", C.c_longlong),
                ("horizon_eps", C.c_double), ("escape_factor", C.c_double), ("refine", C.c_int),
                ("fp64_radius_factor", C.c_double), ("fp64_pole_sin", C.c_double),
                ("critical_band", C.c_double), ("critical_rtol", C.c_double)]


class TTDisk(C.Structure):
    _fields_ = [("enabled", C.c_int), ("r_in", C.c_double), ("r_out", C.c_double), ("mdot", C.c_double),
                ("max_crossings", C.c_int), ("doppler", C.c_int)]


class TTOutputs(C.Structure):
    _fields_ = [("code", C.c_void_p), ("n_cross", C.c_void_p), ("r_cross", C.c_void_p), ("g", C.c_void_p),
                ("I_cross", C.c_void_p), ("intensity", C.c_void_p), ("h_max", C.c_void_p),
                ("steps", C.c_void_p), ("rejects", C.c_void_p)]


class TTTune(C.Structure):
    _fields_ = [("block", C.c_int), ("reg_variant", C.c_int), ("refill", C.c_int), ("blocks_per_sm", C.c_int),
                ("crossing_batch", C.c_int), ("fp64_batch", C.c_int), ("monitor_period", C.c_int),
                ("fp64_wait", C.c_int), ("crit_stride", C.c_int), ("crit_refill", C.c_int)]


class TTImage(C.Structure):
    _fields_ = [("metric", TTMetric), ("obs", TTObserver), ("cam", TTCamera), ("disk", TTDisk),
                ("out", TTOutputs)]


OUTPUT_FIELDS = [f for f, _ in TTOutputs._fields_]

_lock = threading.Lock()
_lib = None


class TartarusError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__("%s: %s (status %d)" % (what or "tartarus", error_string(status), status))
        self.status = status


_bounds_check = False


def library_path() -> str:
    return _build.DEBUG_SO if _bounds_check else _build.SO


def use_bounds_check_build(enable: bool = True) -> None:
    """Route every entry point to the bounds-checking build of the library
    (libtartarus_debug.so, compiled with TT_BOUNDS_CHECK: every output store is
    checked and an out-of-range one counted, see bounds_faults).  A test
    artefact; takes effect before the first call that loads the library."""
    global _bounds_check, _lib
    with _lock:
        if _lib is not None and enable != _bounds_check:
            raise RuntimeError("the library is already loaded; choose the build before the first call")
        _bounds_check = enable


def bounds_faults() -> int:
    """tartarus_debug_faults: out-of-range output stores since the last call
    (bounds-checking build only)."""
    n = C.c_longlong()
    st = lib().tartarus_debug_faults(C.byref(n))
    _check(st, "tartarus_debug_faults")
    return n.value


def lib():
    """Load libtartarus.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build_debug() if _bounds_check else _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libtartarus.so is not built: run paper_2609_08989_gb300._build.build()")
            L = C.CDLL(path)
            P = C.POINTER
            common = [P(TTMetric), P(TTObserver), P(TTCamera), P(TTSolver), P(TTDisk), P(TTOutputs),
                      P(TTTune), C.c_void_p]
            L.tartarus_trace.argtypes = common
            L.tartarus_trace.restype = C.c_int
            L.tartarus_trace_host.argtypes = common
            L.tartarus_trace_host.restype = C.c_int
            L.tartarus_trace_batch.argtypes = [P(TTImage), C.c_int, P(TTSolver), P(TTTune), P(C.c_int), C.c_void_p]
            L.tartarus_trace_batch.restype = C.c_int
            L.tartarus_trace_batch_noalloc.argtypes = [P(TTImage), C.c_int, P(TTSolver), P(TTTune), P(C.c_int),
                                                       C.c_void_p]
            L.tartarus_trace_batch_noalloc.restype = C.c_int
            L.tartarus_table_create.argtypes = [P(C.c_double), C.c_int, C.c_int, C.c_double, C.c_double,
                                                P(C.c_void_p)]
            L.tartarus_table_create.restype = C.c_int
            L.tartarus_table_destroy.argtypes = [C.c_void_p]
            L.tartarus_table_destroy.restype = C.c_int
            L.tartarus_table_coefficients.argtypes = [P(C.c_double), C.c_int, C.c_int, C.c_double, C.c_double,
                                                      P(C.c_double)]
            L.tartarus_table_coefficients.restype = C.c_int
            L.tartarus_error_string.argtypes = [C.c_int]
            L.tartarus_error_string.restype = C.c_char_p
            L.tartarus_launch_count.argtypes = []
            L.tartarus_launch_count.restype = C.c_longlong
            L.tartarus_debug_faults.argtypes = [P(C.c_longlong)]
            L.tartarus_debug_faults.restype = C.c_int
            L.tartarus_version.argtypes = []
            L.tartarus_version.restype = C.c_char_p
            _lib = L
    return _lib


def error_string(status: int) -> str:
    return lib().tartarus_error_string(status).decode()


def launch_count() -> int:
    return int(lib().tartarus_launch_count())


def version() -> str:
    return lib().tartarus_version().decode()


def _check(status: int, what: str):
    if status != TT_OK:
        raise TartarusError(status, what)


def table_coefficients(nodes: np.ndarray, r_min: float, r_max: float) -> np.ndarray:
    """tartarus_table_coefficients (host only): the per-cell patch coefficients,
    shaped [nth - 1, nr - 1, 5, 4, 4] (cell j, k; field; power of t; power of w)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    if nodes.ndim != 3 or nodes.shape[2] != TABLE_NF:
        raise ValueError("table nodes must have shape [nth, nr, 20]")
    nth, nr = nodes.shape[0], nodes.shape[1]
    out = np.empty((max(nth - 1, 0), max(nr - 1, 0), 5, 4, 4))
    P = C.POINTER(C.c_double)
    _check(lib().tartarus_table_coefficients(nodes.ctypes.data_as(P), nr, nth, float(r_min), float(r_max),
                                             out.ctypes.data_as(P)), "tartarus_table_coefficients")
    return out


class Table:
    """Device copy of a tabulated metric ([nth, nr, 20] nodes, see include/tartarus.h)."""

    def __init__(self, nodes: np.ndarray, r_min: float, r_max: float):
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        if nodes.ndim != 3 or nodes.shape[2] != TABLE_NF:
            raise ValueError("table nodes must have shape [nth, nr, 20]")
        self.nth, self.nr = nodes.shape[0], nodes.shape[1]
        self.r_min, self.r_max = float(r_min), float(r_max)
        h = C.c_void_p()
        _check(lib().tartarus_table_create(nodes.ctypes.data_as(C.POINTER(C.c_double)), self.nr, self.nth,
                                           self.r_min, self.r_max, C.byref(h)), "tartarus_table_create")
        self.handle = h

    def destroy(self):
        if self.handle:
            _check(lib().tartarus_table_destroy(self.handle), "tartarus_table_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.tartarus_table_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


# ---------------------------------------------------------------------------
# scene -> structs
# ---------------------------------------------------------------------------

def _metric(sc: Scene, table: Optional[Table]) -> TTMetric:
    m = TTMetric(kind=sc.metric_kind, M=sc.M, a=sc.a, table=None)
    if sc.metric_kind == 1:
        if table is None:
            raise ValueError("a tabulated-metric scene needs a Table")
        m.table = table.handle
    return m


def _camera(sc: Scene, pix_begin: int, pix_count: int) -> TTCamera:
    return TTCamera(nx=sc.nx, ny=sc.ny, alpha_min=sc.alpha_min, alpha_max=sc.alpha_max, beta_min=sc.beta_min,
                    beta_max=sc.beta_max, pix_begin=pix_begin, pix_count=pix_count)


def solver_struct(sc: Scene) -> TTSolver:
    return TTSolver(method=sc.method, precision=sc.precision, rtol=sc.rtol, atol=sc.atol, h0=sc.h0, h_min=sc.h_min,
                    max_steps=sc.max_steps, horizon_eps=sc.horizon_eps, escape_factor=sc.escape_factor,
                    refine=sc.refine, fp64_radius_factor=sc.fp64_radius_factor,
                    fp64_pole_sin=sc.fp64_pole_sin, critical_band=sc.critical_band,
                    critical_rtol=sc.critical_rtol)


def _disk(sc: Scene) -> TTDisk:
    return TTDisk(enabled=sc.disk_enabled, r_in=sc.r_in, r_out=sc.r_out, mdot=sc.mdot,
                  max_crossings=sc.max_crossings, doppler=sc.doppler)


def _tune(tune, sc: Optional[Scene] = None, batch: bool = False) -> Optional[TTTune]:
    """Explicit shape, else the autotuned shape cached for this device and
    workload class, else the library's built-in defaults (None)."""
    if tune is None and sc is not None:
        from . import autotune
        tune = autotune.cached(sc, batch)
    if tune is None:
        return None
    if isinstance(tune, TTTune):
        return tune
    return TTTune(**{f: int(tune.get(f, 0)) for f, _ in TTTune._fields_})


def _tune_ref(tune, sc, batch: bool = False):
    t = _tune(tune, sc, batch)
    return C.byref(t) if t is not None else None


def _npix(sc: Scene, pix_begin: int, pix_count: int) -> int:
    return pix_count if pix_count > 0 else sc.nx * sc.ny - pix_begin


def alloc_outputs(n: int, device="cuda"):
    """Torch output tensors for n pixels on a device (crossing arrays are [3, n])."""
    import torch
    dev = torch.device(device)
    return {
        "code": torch.empty(n, dtype=torch.int8, device=dev),
        "n_cross": torch.empty(n, dtype=torch.int8, device=dev),
        "r_cross": torch.empty((MAX_CROSSINGS, n), dtype=torch.float64, device=dev),
        "g": torch.empty((MAX_CROSSINGS, n), dtype=torch.float64, device=dev),
        "I_cross": torch.empty((MAX_CROSSINGS, n), dtype=torch.float64, device=dev),
        "intensity": torch.empty(n, dtype=torch.float64, device=dev),
        "h_max": torch.empty(n, dtype=torch.float64, device=dev),
        "steps": torch.empty(n, dtype=torch.int32, device=dev),
        "rejects": torch.empty(n, dtype=torch.int32, device=dev),
    }


def alloc_host_outputs(n: int, pinned: bool = True):
    """Pinned host tensors (torch) for n pixels."""
    import torch
    kw = dict(pin_memory=pinned)
    return {
        "code": torch.empty(n, dtype=torch.int8, **kw),
        "n_cross": torch.empty(n, dtype=torch.int8, **kw),
        "r_cross": torch.empty((MAX_CROSSINGS, n), dtype=torch.float64, **kw),
        "g": torch.empty((MAX_CROSSINGS, n), dtype=torch.float64, **kw),
        "I_cross": torch.empty((MAX_CROSSINGS, n), dtype=torch.float64, **kw),
        "intensity": torch.empty(n, dtype=torch.float64, **kw),
        "h_max": torch.empty(n, dtype=torch.float64, **kw),
        "steps": torch.empty(n, dtype=torch.int32, **kw),
        "rejects": torch.empty(n, dtype=torch.int32, **kw),
    }


def _out_struct(out) -> TTOutputs:
    o = TTOutputs()
    for f in OUTPUT_FIELDS:
        t = out[f]
        if not t.is_contiguous():
            raise ValueError("output %s must be contiguous" % f)
        setattr(o, f, t.data_ptr())
    return o


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def trace(sc: Scene, out=None, stream=None, tune=None, table: Optional[Table] = None,
          pix_begin: int = 0, pix_count: int = 0):
    """tartarus_trace: trace the scene's camera (or a pixel range) into device tensors.
    Asynchronous on ``stream`` (default: torch's current stream)."""
    n = _npix(sc, pix_begin, pix_count)
    if out is None:
        out = alloc_outputs(n)
    own = None
    if sc.metric_kind == 1 and table is None:
        own = table = Table(sc.table, sc.r_min, sc.r_max)
    st = lib().tartarus_trace(C.byref(_metric(sc, table)), C.byref(TTObserver(sc.r_obs, sc.theta_obs)),
                              C.byref(_camera(sc, pix_begin, pix_count)), C.byref(solver_struct(sc)),
                              C.byref(_disk(sc)), C.byref(_out_struct(out)), _tune_ref(tune, sc), _stream_ptr(stream))
    if own is not None:
        import torch
        torch.cuda.synchronize()
        own.destroy()
    _check(st, "tartarus_trace")
    return out


def trace_host(sc: Scene, out=None, stream=None, tune=None, table: Optional[Table] = None,
               pix_begin: int = 0, pix_count: int = 0):
    """tartarus_trace_host: outputs in (pinned) host tensors; synchronous."""
    n = _npix(sc, pix_begin, pix_count)
    if out is None:
        out = alloc_host_outputs(n)
    own = None
    if sc.metric_kind == 1 and table is None:
        own = table = Table(sc.table, sc.r_min, sc.r_max)
    st = lib().tartarus_trace_host(C.byref(_metric(sc, table)), C.byref(TTObserver(sc.r_obs, sc.theta_obs)),
                                   C.byref(_camera(sc, pix_begin, pix_count)), C.byref(solver_struct(sc)),
                                   C.byref(_disk(sc)), C.byref(_out_struct(out)), _tune_ref(tune, sc),
                                   _stream_ptr(stream))
    if own is not None:
        own.destroy()
    _check(st, "tartarus_trace_host")
    return out


def trace_batch(scenes: Sequence[Scene], outs=None, stream=None, tune=None,
                tables: Optional[Sequence[Optional[Table]]] = None, status_out: Optional[List[int]] = None):
    """tartarus_trace_batch: all images in one persistent launch sharing one ray queue.
    The solver settings of scenes[0] apply to every image."""
    n = len(scenes)
    if outs is None:
        outs = [alloc_outputs(s.npix) for s in scenes]
    imgs = (TTImage * max(n, 1))()
    for i, s in enumerate(scenes):
        tb = tables[i] if tables is not None else None
        imgs[i].metric = _metric(s, tb)
        imgs[i].obs = TTObserver(s.r_obs, s.theta_obs)
        imgs[i].cam = _camera(s, 0, 0)
        imgs[i].disk = _disk(s)
        imgs[i].out = _out_struct(outs[i])
    status = (C.c_int * max(n, 1))()
    st = lib().tartarus_trace_batch(imgs, n, C.byref(solver_struct(scenes[0])),
                                    _tune_ref(tune, scenes[0] if n else None, n > 1), status, _stream_ptr(stream))
    if status_out is not None:
        status_out[:] = list(status)[:n]
    if st != TT_OK and status_out is None:
        _check(st, "tartarus_trace_batch")
    return outs


def trace_batch_noalloc(scenes: Sequence[Scene], outs, stream=None, tune=None,
                        tables: Optional[Sequence[Optional[Table]]] = None,
                        status_out: Optional[List[int]] = None):
    """tartarus_trace_batch_noalloc: like trace_batch, but the library allocates
    nothing (its work-queue counters sit in a fixed array inside the library).
    The caller supplies the output tensors; at most 1024 images per call, and
    calls that overlap on the GPU race on the shared counters."""
    n = len(scenes)
    imgs = (TTImage * max(n, 1))()
    for i, s in enumerate(scenes):
        tb = tables[i] if tables is not None else None
        imgs[i].metric = _metric(s, tb)
        imgs[i].obs = TTObserver(s.r_obs, s.theta_obs)
        imgs[i].cam = _camera(s, 0, 0)
        imgs[i].disk = _disk(s)
        imgs[i].out = _out_struct(outs[i])
    status = (C.c_int * max(n, 1))()
    st = lib().tartarus_trace_batch_noalloc(imgs, n, C.byref(solver_struct(scenes[0])),
                                            _tune_ref(tune, scenes[0] if n else None, n > 1), status,
                                            _stream_ptr(stream))
    if status_out is not None:
        status_out[:] = list(status)[:n]
    if st != TT_OK and status_out is None:
        _check(st, "tartarus_trace_batch_noalloc")
    return outs


class TraceGraph:
    """A batch render captured once into a CUDA graph and replayed.

    For repeated renders of the same images into the same output buffers (an
    animation loop, a parameter scan that rewrites one set of outputs): the
    descriptors are built and validated once, and each replay is one graph
    launch.  The first (uncaptured) call also performs the library's one-time
    per-device set-up, so capture itself makes no allocation."""

    def __init__(self, scenes: Sequence[Scene], outs=None, tune=None,
                 tables: Optional[Sequence[Optional[Table]]] = None):
        import torch
        self.scenes = list(scenes)
        self.outs = outs if outs is not None else [alloc_outputs(s.npix) for s in self.scenes]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            trace_batch(self.scenes, self.outs, stream=side, tune=tune, tables=tables)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            trace_batch(self.scenes, self.outs, stream=torch.cuda.current_stream(), tune=tune, tables=tables)
        self.launches_per_replay = (len(self.scenes) + 63) // 64

    def replay(self):
        self.graph.replay()
        return self.outs


def to_numpy(out) -> Dict[str, np.ndarray]:
    return {k: v.cpu().numpy() for k, v in out.items()}
