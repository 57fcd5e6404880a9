"""The C ABI library loads, exports every entry point include/tartarus.h
declares, its struct layouts match the binding, and argument validation
rejects bad input before touching the GPU (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

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
  printf("%zu %zu %zu\\n", offsetof(tt_solver, fp64_radius_factor), offsetof(tt_camera, pix_count),
         offsetof(tt_image, out));
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
    assert offs == [T.TTSolver.fp64_radius_factor.offset, T.TTCamera.pix_count.offset, T.TTImage.out.offset]


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
