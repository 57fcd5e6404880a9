"""The C ABI library loads, exports every entry point include/tartarus.h
declares, its struct layouts match the binding, and argument validation
rejects bad input before touching the GPU (no GPU needed)."""
import ctypes as C
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2609_08989_gb300 import _build, scenes, tartarus as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tartarus.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tartarus_\w+)\s*\(", src)))


def test_library_builds_and_exports_header():
    path = _build.build()
    lib = C.CDLL(path)
    names = declared_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(T.EXPORTS) == names


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "tartarus.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(tt_metric), sizeof(tt_observer), sizeof(tt_camera),
         sizeof(tt_solver), sizeof(tt_disk), sizeof(tt_outputs), sizeof(tt_tune), sizeof(tt_image));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(tt_solver, fp64_radius_factor), offsetof(tt_camera, pix_count),
         offsetof(tt_image, out), offsetof(tt_solver, critical_rtol), offsetof(tt_tune, crit_refill));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    assert sizes == [C.sizeof(s) for s in (T.TTMetric, T.TTObserver, T.TTCamera, T.TTSolver, T.TTDisk,
                                           T.TTOutputs, T.TTTune, T.TTImage)]
    offs = [int(x) for x in lines[1].split()]
    assert offs == [T.TTSolver.fp64_radius_factor.offset, T.TTCamera.pix_count.offset, T.TTImage.out.offset,
                    T.TTSolver.critical_rtol.offset, T.TTTune.crit_refill.offset]


def _args(sc, **over):
    m = T.TTMetric(kind=sc.metric_kind, M=sc.M, a=sc.a, table=None)
    o = T.TTObserver(sc.r_obs, sc.theta_obs)
    cam = T.TTCamera(nx=sc.nx, ny=sc.ny, alpha_min=sc.alpha_min, alpha_max=sc.alpha_max,
                     beta_min=sc.beta_min, beta_max=sc.beta_max, pix_begin=0, pix_count=0)
    s = T.solver_struct(sc)
    d = T.TTDisk(enabled=sc.disk_enabled, r_in=sc.r_in, r_out=sc.r_out, mdot=sc.mdot,
                 max_crossings=sc.max_crossings, doppler=sc.doppler)
    out = T.TTOutputs(*([8] * 9))                 # non-null dummies: never dereferenced on these paths
    for k, v in over.items():
        obj, field = k.split("__")
        setattr({"m": m, "o": o, "cam": cam, "s": s, "d": d}[obj], field, v)
    return m, o, cam, s, d, out


BAD = [
    dict(m__M=0.0), dict(m__M=float("nan")), dict(m__a=1.0), dict(m__kind=7),
    dict(o__r_obs=-1.0), dict(o__theta_obs=0.0), dict(o__theta_obs=3.2),
    dict(cam__nx=0), dict(cam__alpha_min=float("inf")), dict(cam__pix_begin=-1),
    dict(cam__pix_count=10 ** 9),
    dict(s__rtol=0.0), dict(s__atol=-1.0), dict(s__max_steps=0), dict(s__escape_factor=1.0),
    dict(s__refine=3), dict(s__horizon_eps=-0.1), dict(s__precision=5), dict(s__method=5), dict(s__method=-1), dict(s__method=4),
    dict(d__max_crossings=4), dict(d__r_out=0.0),
]


@pytest.mark.parametrize("over", BAD)
def test_validation_rejects_without_gpu(over):
    sc = scenes.kerr_disk(16)
    m, o, cam, s, d, out = _args(sc, **over)
    st = T.lib().tartarus_trace(C.byref(m), C.byref(o), C.byref(cam), C.byref(s), C.byref(d),
                                C.byref(out), None, None)
    assert st == T.TT_EINVAL, over


def test_unsupported_and_null_arguments():
    sc = scenes.kerr_disk(16)
    L = T.lib()
    for method in (1, 2, 3, 4):         # every integrator but Dormand-Prince runs in FP64 only
        for prec in (1, 2, 3):
            m, o, cam, s, d, out = _args(sc, s__method=method, s__precision=prec)
            assert L.tartarus_trace(C.byref(m), C.byref(o), C.byref(cam), C.byref(s), C.byref(d),
                                    C.byref(out), None, None) == T.TT_EUNSUPPORTED
    m, o, cam, s, d, out = _args(sc)
    assert L.tartarus_trace(None, C.byref(o), C.byref(cam), C.byref(s), C.byref(d), C.byref(out),
                            None, None) == T.TT_EINVAL
    nul = T.TTOutputs()
    assert L.tartarus_trace(C.byref(m), C.byref(o), C.byref(cam), C.byref(s), C.byref(d), C.byref(nul),
                            None, None) == T.TT_EINVAL
    bad_tune = T.TTTune(block=100)
    assert L.tartarus_trace(C.byref(m), C.byref(o), C.byref(cam), C.byref(s), C.byref(d), C.byref(out),
                            C.byref(bad_tune), None) == T.TT_EUNSUPPORTED
    h = C.c_void_p()
    assert L.tartarus_table_create(None, 4, 4, 1.0, 2.0, C.byref(h)) == T.TT_EINVAL
    assert L.tartarus_table_destroy(None) == T.TT_EINVAL
    assert T.error_string(T.TT_EINVAL) == "invalid argument"


def test_batch_reports_bad_image_without_gpu():
    sc = scenes.kerr_disk(16)
    imgs = (T.TTImage * 2)()
    for i in range(2):
        m, o, cam, s, d, out = _args(sc, **({"o__r_obs": -5.0} if i == 1 else {"cam__nx": 0}))
        imgs[i].metric, imgs[i].obs, imgs[i].cam, imgs[i].disk, imgs[i].out = m, o, cam, d, out
    status = (C.c_int * 2)()
    st = T.lib().tartarus_trace_batch(imgs, 2, C.byref(T.solver_struct(sc)), None, status, None)
    assert st == T.TT_EINVAL and list(status) == [T.TT_EINVAL, T.TT_EINVAL]


def test_batch_mixing_metric_kinds_refused_for_one_kind_kernels():
    sc = scenes.kerr_disk(16)
    imgs = (T.TTImage * 2)()
    for i in range(2):
        m, o, cam, s, d, out = _args(sc, **({"m__kind": 1} if i == 1 else {}))
        imgs[i].metric, imgs[i].obs, imgs[i].cam, imgs[i].disk, imgs[i].out = m, o, cam, d, out
    status = (C.c_int * 2)(-7, -7)
    # the other integrators, and the double-float path, take one metric kind per launch
    solvers = [sc.replace(method=method, h0=0.01) for method in (1, 2, 3, 4)]
    solvers.append(sc.replace(precision=scenes.DOUBLE_FLOAT))
    for sv in solvers:
        s = T.solver_struct(sv)
        for fn in (T.lib().tartarus_trace_batch, T.lib().tartarus_trace_batch_noalloc):
            assert fn(imgs, 2, C.byref(s), None, status, None) == T.TT_EUNSUPPORTED
            assert list(status) == [-7, -7]          # refused before any image was looked at


def test_table_coefficients_reproduce_the_oracle_interpolant(orc):
    """The per-cell monomial coefficients the library uploads (formed on the
    host from the Hermite node data) evaluate to the oracle's bicubic Hermite
    interpolant: values of the five fields, and derivatives through the
    oracle's inverse metric -- inside the table and beyond its radial range."""
    a, nr, nth, rmax = 0.9, 40, 25, 200.0
    rh = orc.rplus(1.0, a)
    nodes = orc.kerr_table(1.0, a, nr, nth, rh, rmax)
    cf = T.table_coefficients(nodes, rh, rmax)
    assert cf.shape == (nth - 1, nr - 1, 5, 4, 4)
    sc = scenes.Scene(metric_kind=1, a=a, table=nodes, r_min=rh, r_max=rmax)
    u0 = math.log(rh)
    du = (math.log(rmax) - u0) / (nr - 1)
    dth = math.pi / (nth - 1)
    rng = np.random.default_rng(17)
    pts = [(rh * (rmax * 1.2 / rh) ** rng.uniform(0.02, 1.0), rng.uniform(0.05, math.pi - 0.05)) for _ in range(60)]
    pts += [(rmax * 1.15, 1.0), (rh * 1.001, 2.0)]
    ip = np.arange(4.0)
    for r, th in pts:
        tu, tw = (math.log(r) - u0) / du, th / dth
        k, j = min(max(int(math.floor(tu)), 0), nr - 2), min(max(int(math.floor(tw)), 0), nth - 2)
        t, w = tu - k, tw - j
        T4, W4 = t ** ip, w ** ip
        dT4 = np.array([0.0, 1.0, 2 * t, 3 * t * t])
        dW4 = np.array([0.0, 1.0, 2 * w, 3 * w * w])
        val = [T4 @ cf[j, k, f] @ W4 for f in range(5)]
        dr = [dT4 @ cf[j, k, f] @ W4 / (du * r) for f in range(5)]
        dt = [T4 @ cf[j, k, f] @ dW4 / dth for f in range(5)]
        g = orc.metric_lower(sc, r, th)
        gi, dgr, dgt = orc.metric_upper(sc, r, th)
        for f, (mu, nu) in enumerate([(0, 0), (0, 3), (2, 2), (3, 3)]):
            assert val[f] == pytest.approx(g[mu, nu], rel=1e-12, abs=1e-12 * abs(g[3, 3])), (r, th, f)
        assert val[4] == pytest.approx(gi[1, 1], rel=1e-12), (r, th)
        # derivatives: of g^rr directly, of g_thth through g^thth = 1/g_thth, of the
        # (t, phi) block through g^tt = g_phiphi / D, D = g_tt g_phiphi - g_tphi^2
        D = val[0] * val[3] - val[1] ** 2
        for dv, dg in ((dr, dgr), (dt, dgt)):
            assert dv[4] == pytest.approx(dg[1, 1], rel=1e-9, abs=1e-12)
            assert -dv[2] / val[2] ** 2 == pytest.approx(dg[2, 2], rel=1e-9, abs=1e-14)
            dD = dv[0] * val[3] + val[0] * dv[3] - 2 * val[1] * dv[1]
            dgtt = (dv[3] * D - val[3] * dD) / D ** 2
            assert dgtt == pytest.approx(dg[0, 0], rel=1e-8, abs=1e-12 * abs(gi[0, 0])), (r, th)


def test_table_coefficients_validation():
    L = T.lib()
    P = C.POINTER(C.c_double)
    out = np.zeros(80)
    nodes = np.ones((2, 2, 20))
    assert L.tartarus_table_coefficients(None, 2, 2, 1.0, 2.0, out.ctypes.data_as(P)) == T.TT_EINVAL
    assert L.tartarus_table_coefficients(nodes.ctypes.data_as(P), 2, 2, 1.0, 2.0, None) == T.TT_EINVAL
    assert L.tartarus_table_coefficients(nodes.ctypes.data_as(P), 1, 2, 1.0, 2.0, out.ctypes.data_as(P)) == T.TT_EINVAL
    assert L.tartarus_table_coefficients(nodes.ctypes.data_as(P), 2, 2, 2.0, 1.0, out.ctypes.data_as(P)) == T.TT_EINVAL
    nodes[1, 1, 7] = np.nan
    assert L.tartarus_table_coefficients(nodes.ctypes.data_as(P), 2, 2, 1.0, 2.0, out.ctypes.data_as(P)) == T.TT_EINVAL
    # a constant field: c_00 = the value, every other coefficient zero
    nodes = np.zeros((2, 2, 20))
    nodes[:, :, 0] = 2.5
    assert L.tartarus_table_coefficients(nodes.ctypes.data_as(P), 2, 2, 1.0, 2.0, out.ctypes.data_as(P)) == T.TT_OK
    assert out[0] == 2.5 and np.all(out[1:] == 0.0)
