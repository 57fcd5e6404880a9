"""Accuracy of the double-float arithmetic the double-float path and the mixed
paths' zone steps use: a small CUDA program (tests/cuda/df_accuracy.cu, built
here with nvcc for sm_103a against the library's own device headers) compares
double-float sin/cos, reciprocal, logarithm, Kerr flow and Hamiltonian with
their FP64 values on 8192 seeded inputs, including polar angles beyond (0, pi)
and arguments of the logarithm from 2^-30 to 2^30, and the double-float
tabulated-metric patches (value and both derivatives of five fields) with the
FP64 ones on a random coefficient table, inside and just outside its range."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2609_08989_gb300", "csrc")

# double-float carries ~48 bits (2^-48 = 3.6e-15; the reciprocal within 2^-46): sin/cos to the absolute precision of theta
# itself (|theta| <= 8 here: 2^-48 x 8 ~ 3e-14); the flow components relative
# to their own size except where they are a cancelled difference
BOUNDS = {"sin": 1e-13, "cos": 1e-13, "rcp": 5e-14, "flow_th": 1e-12, "flow_r": 1e-11,
          "log": 5e-13,      # |ln x| <= 21 here: 21 x 2^-48 = 7.5e-14 per rounding
          # the table patches against the size of their terms: the evaluation point
          # t = (ln r - u0)/du - k carries the pair's rounding of ln r (~2e-14 here),
          # which moves the patch by v_t dt (~2.5e-13 seen); the Horner chains
          # themselves add a few units of 2^-48
          "table_value": 1e-12, "table_dr": 1e-12, "table_dth": 1e-12}


def test_double_float_accuracy(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08989_gb300 import _build
    exe = str(tmp_path / "df_accuracy")
    cmd = [_build.nvcc(), *_build.ARCH, "-std=c++17", "-O3", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "cuda", "df_accuracy.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    res = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120)
    got = {}
    for line in res.stdout.splitlines():
        name, val, _ = line.split()
        got[name] = float(val)
    print(got)
    for name, bound in BOUNDS.items():
        assert got[name] < bound, (name, got[name])
    # H: a sum of terms that cancel (up to ~1e8 near the axis here), measured
    # against the size of those terms.  Within 1 % of r_+ Delta = r (r - 2M) + a^2
    # itself cancels ~10^3-fold, so the pair's 2^-48 becomes ~1e-11 there
    # (FP64 loses the same factor, from 2^-53)
    assert got["H"] < 1e-10
