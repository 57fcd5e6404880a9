"""FP64 CPU oracle for backward null-geodesic ray tracing (TARTARUS, arXiv 2609.08989).

TEST INFRASTRUCTURE ONLY.  The plain C oracle in ``tt_oracle.c`` is what the
CUDA library is checked against; this module compiles it with gcc and wraps it
with ctypes.  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import it.  It does not import the CUDA package and the CUDA
package does not import it: scenes are passed in as plain objects whose
attributes name the scene fields (duck typing), so the two share no code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tt_oracle.c")
_HDR = os.path.join(_HERE, "tt_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtt_oracle.so")
_lock = threading.Lock()
_lib = None

ESCAPED, CAPTURED, MAXSTEPS, UNDERFLOW, NONFINITE, BADPIXEL = range(6)
MAXCROSS = 3
TABLE_NF = 20


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libtt_oracle.so (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wno-unknown-pragmas", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Scene(C.Structure):
    _fields_ = [
        ("metric_kind", C.c_int), ("M", C.c_double), ("a", C.c_double),
        ("table", C.POINTER(C.c_double)), ("nr", C.c_int), ("nth", C.c_int),
        ("r_min", C.c_double), ("r_max", C.c_double),
        ("r_obs", C.c_double), ("theta_obs", C.c_double),
        ("nx", C.c_int), ("ny", C.c_int),
        ("alpha_min", C.c_double), ("alpha_max", C.c_double),
        ("beta_min", C.c_double), ("beta_max", C.c_double),
        ("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double), ("h_min", C.c_double),
        ("max_steps", C.c_longlong), ("horizon_eps", C.c_double), ("escape_factor", C.c_double),
        ("refine", C.c_int), ("method", C.c_int),
        ("disk_enabled", C.c_int), ("r_in", C.c_double), ("r_out", C.c_double), ("mdot", C.c_double),
        ("max_crossings", C.c_int), ("doppler", C.c_int),
    ]


class Outputs(C.Structure):
    _fields_ = [
        ("code", C.POINTER(C.c_int8)), ("n_cross", C.POINTER(C.c_int8)),
        ("r_cross", C.POINTER(C.c_double)), ("g", C.POINTER(C.c_double)),
        ("I_cross", C.POINTER(C.c_double)), ("intensity", C.POINTER(C.c_double)),
        ("h_max", C.POINTER(C.c_double)), ("steps", C.POINTER(C.c_int32)),
        ("rejects", C.POINTER(C.c_int32)),
    ]


_D = C.POINTER(C.c_double)
_FN = C.CFUNCTYPE(None, C.c_void_p, _D, _D)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            SP = C.POINTER(Scene)
            L.orc_kerr_lower.argtypes = [C.c_double] * 4 + [_D]
            L.orc_kerr_upper.argtypes = [C.c_double] * 4 + [_D, _D, _D]
            L.orc_metric_upper.argtypes = [SP, C.c_double, C.c_double, _D, _D, _D]
            L.orc_metric_lower.argtypes = [SP, C.c_double, C.c_double, _D]
            L.orc_hamiltonian.argtypes = [SP, _D]
            L.orc_hamiltonian.restype = C.c_double
            L.orc_rhs.argtypes = [SP, _D, _D]
            L.orc_initial_state.argtypes = [SP, C.c_double, C.c_double, _D]
            L.orc_rplus.argtypes = [C.c_double, C.c_double]
            L.orc_rplus.restype = C.c_double
            L.orc_isco.argtypes = [C.c_double, C.c_double]
            L.orc_isco.restype = C.c_double
            L.orc_flux.argtypes = [C.c_double] * 4
            L.orc_flux.restype = C.c_double
            L.orc_redshift.argtypes = [SP, C.c_double, C.c_double, C.c_double]
            L.orc_redshift.restype = C.c_double
            L.orc_dp5_step.argtypes = [C.c_int, _FN, C.c_void_p, _D, _D, C.c_double, _D, _D, _D]
            L.orc_dp5_tableau.argtypes = [_D, _D, _D, _D]
            L.orc_rk_step.argtypes = [C.c_int, C.c_int, _FN, C.c_void_p, _D, _D, C.c_double, _D, _D, _D]
            L.orc_rk_tableau.argtypes = [C.c_int, _D, _D, _D, _D]
            L.orc_rk_tableau.restype = C.c_int
            L.orc_gbs_step.argtypes = [C.c_int, _FN, C.c_void_p, _D, _D, C.c_double, C.c_int, _D, _D, _D]
            L.orc_verlet_step.argtypes = [C.c_int, _FN, C.c_void_p, _D, C.c_double, _D, _D]
            i8 = C.POINTER(C.c_int8)
            i32 = C.POINTER(C.c_int32)
            L.orc_trace_ray.argtypes = [SP, C.c_double, C.c_double, C.c_int, _D, _D, _D,
                                        i8, i8, _D, _D, _D, _D, _D, i32, i32]
            L.orc_trace_ray.restype = C.c_int
            L.orc_kerr_table.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int,
                                         C.c_double, C.c_double, _D]
            L.orc_kerr_table.restype = C.c_int
            OP = C.POINTER(Outputs)
            L.orc_trace.argtypes = [SP, C.c_longlong, C.c_longlong, OP, C.c_int]
            L.orc_trace_list.argtypes = [SP, C.POINTER(C.c_int64), C.c_longlong, OP, C.c_int]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def scene_struct(sc):
    """Fill the C scene from any object carrying the scene fields as attributes."""
    s = Scene()
    table = getattr(sc, "table", None)
    for name, _ in Scene._fields_:
        if name in ("table", "nr", "nth"):
            continue
        setattr(s, name, getattr(sc, name))
    keep = None
    if table is not None:
        keep = np.ascontiguousarray(table, dtype=np.float64)
        assert keep.ndim == 3 and keep.shape[2] == TABLE_NF
        s.table = _dp(keep)
        s.nth, s.nr = keep.shape[0], keep.shape[1]
    s._keep = keep     # keep the table alive as long as the struct
    return s


def alloc_outputs(n: int) -> dict:
    return {
        "code": np.zeros(n, np.int8), "n_cross": np.zeros(n, np.int8),
        "r_cross": np.zeros((MAXCROSS, n)), "g": np.zeros((MAXCROSS, n)),
        "I_cross": np.zeros((MAXCROSS, n)), "intensity": np.zeros(n),
        "h_max": np.zeros(n), "steps": np.zeros(n, np.int32), "rejects": np.zeros(n, np.int32),
    }


def _out_struct(o: dict) -> Outputs:
    s = Outputs()
    for name, ctype in Outputs._fields_:
        setattr(s, name, o[name].ctypes.data_as(ctype))
    return s


def trace(sc, pix_begin: int = 0, npix: int | None = None, nthreads: int = 0) -> dict:
    """Trace pixels [pix_begin, pix_begin + npix) of the scene's camera."""
    if npix is None:
        npix = sc.nx * sc.ny - pix_begin
    o = alloc_outputs(npix)
    s = scene_struct(sc)
    lib().orc_trace(C.byref(s), pix_begin, npix, C.byref(_out_struct(o)), nthreads)
    return o


def trace_list(sc, pix, nthreads: int = 0) -> dict:
    """Trace an explicit list of pixel indices (p = j*nx + i)."""
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    o = alloc_outputs(len(pix))
    s = scene_struct(sc)
    lib().orc_trace_list(C.byref(s), pix.ctypes.data_as(C.POINTER(C.c_int64)), len(pix),
                         C.byref(_out_struct(o)), nthreads)
    return o


def trace_ray(sc, alpha: float, beta: float, cap: int = 200000) -> dict:
    """One ray with its accepted-step trajectory (lambda, y[8]) for the pins."""
    lam = np.zeros(cap)
    ys = np.zeros((cap, 8))
    lamc = np.zeros(3)
    code, nc = C.c_int8(), C.c_int8()
    rc, g, I = np.zeros(3), np.zeros(3), np.zeros(3)
    inten, hmax = C.c_double(), C.c_double()
    st, rj = C.c_int32(), C.c_int32()
    s = scene_struct(sc)
    n = lib().orc_trace_ray(C.byref(s), alpha, beta, cap, _dp(lam), _dp(ys), _dp(lamc),
                            C.byref(code), C.byref(nc), _dp(rc), _dp(g), _dp(I),
                            C.byref(inten), C.byref(hmax), C.byref(st), C.byref(rj))
    return {"lam": lam[:n], "y": ys[:n], "lam_cross": lamc, "code": code.value,
            "n_cross": nc.value, "r_cross": rc, "g": g, "I_cross": I,
            "intensity": inten.value, "h_max": hmax.value, "steps": st.value, "rejects": rj.value}


def kerr_lower(M, a, r, th):
    g = np.zeros(16)
    lib().orc_kerr_lower(M, a, r, th, _dp(g))
    return g.reshape(4, 4)


def kerr_upper(M, a, r, th):
    gi, dr, dt = np.zeros(16), np.zeros(16), np.zeros(16)
    lib().orc_kerr_upper(M, a, r, th, _dp(gi), _dp(dr), _dp(dt))
    return gi.reshape(4, 4), dr.reshape(4, 4), dt.reshape(4, 4)


def metric_upper(sc, r, th):
    gi, dr, dt = np.zeros(16), np.zeros(16), np.zeros(16)
    s = scene_struct(sc)
    lib().orc_metric_upper(C.byref(s), r, th, _dp(gi), _dp(dr), _dp(dt))
    return gi.reshape(4, 4), dr.reshape(4, 4), dt.reshape(4, 4)


def metric_lower(sc, r, th):
    g = np.zeros(16)
    s = scene_struct(sc)
    lib().orc_metric_lower(C.byref(s), r, th, _dp(g))
    return g.reshape(4, 4)


def hamiltonian(sc, y) -> float:
    y = np.ascontiguousarray(y, dtype=np.float64)
    s = scene_struct(sc)
    return lib().orc_hamiltonian(C.byref(s), _dp(y))


def rhs(sc, y) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float64)
    dy = np.zeros(8)
    s = scene_struct(sc)
    lib().orc_rhs(C.byref(s), _dp(y), _dp(dy))
    return dy


def initial_state(sc, alpha, beta) -> np.ndarray:
    y = np.zeros(8)
    s = scene_struct(sc)
    rc = lib().orc_initial_state(C.byref(s), alpha, beta, _dp(y))
    if rc != 0:
        raise ValueError("pixel outside the observer's sky (alpha^2 + beta^2 >= r_obs^2)")
    return y


def rplus(M, a):
    return lib().orc_rplus(M, a)


def isco(M, a):
    return lib().orc_isco(M, a)


def flux(M, a, mdot, r):
    return lib().orc_flux(M, a, mdot, r)


def redshift(sc, r, p_t, p_phi):
    s = scene_struct(sc)
    return lib().orc_redshift(C.byref(s), r, p_t, p_phi)


def tableau(method: int = 0):
    """(c, A, b, bhat, stages) of a 5(4) pair: 0 Dormand-Prince, 1 Cash-Karp, 2 Fehlberg."""
    c, a, b, bh = np.zeros(7), np.zeros(49), np.zeros(7), np.zeros(7)
    st = lib().orc_rk_tableau(method, _dp(c), _dp(a), _dp(b), _dp(bh))
    return c[:st], a.reshape(7, 7)[:st, :st], b[:st], bh[:st]


def _callback(f, n):
    def cb(_ctx, yp, dyp):
        yy = np.ctypeslib.as_array(yp, shape=(n,)).copy()
        d = np.asarray(f(yy), dtype=np.float64)
        for i in range(n):
            dyp[i] = d[i]
    return _FN(cb)


def dp5_step(f, y, h, method: int = 0):
    """One step of the oracle's generic 5(4) stepper (default Dormand-Prince) on dy/dx = f(y)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = len(y)
    fn = _callback(f, n)
    f0 = np.asarray(f(y.copy()), dtype=np.float64)
    yn, fnew, err = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_rk_step(method, n, fn, None, _dp(y), _dp(f0), h, _dp(yn), _dp(fnew), _dp(err))
    return yn, fnew, err


def gbs_step(f, y, H, k):
    """One Gragg-Bulirsch-Stoer macro-step with k extrapolation columns: (T_kk, f(T_kk), T_kk - T_k,k-1)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = len(y)
    fn = _callback(f, n)
    f0 = np.asarray(f(y.copy()), dtype=np.float64)
    yn, fnew, err = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_gbs_step(n, fn, None, _dp(y), _dp(f0), H, k, _dp(yn), _dp(fnew), _dp(err))
    return yn, fnew, err


def verlet_step(f, y, h):
    """One Stormer-Verlet step; y = (q, p), f(y) = (dH/dp, -dH/dq).  Returns (y_new, f(y_new))."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = len(y)
    fn = _callback(f, n)
    yn, fnew = np.zeros(n), np.zeros(n)
    lib().orc_verlet_step(n, fn, None, _dp(y), h, _dp(yn), _dp(fnew))
    return yn, fnew


def kerr_table(M, a, nr, nth, r_min, r_max) -> np.ndarray:
    """Kerr sampled onto the tabulated-metric format: array [nth, nr, 20]."""
    nodes = np.zeros((nth, nr, TABLE_NF))
    rc = lib().orc_kerr_table(M, a, nr, nth, r_min, r_max, _dp(nodes))
    if rc != 0:
        raise ValueError("bad table geometry")
    return nodes
