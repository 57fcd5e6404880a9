"""The bounds-checking build (TT_BOUNDS_CHECK): every output store of every
kernel family is checked against its buffer's length, and an out-of-range one
would be skipped and counted instead of made.  Run on small cases (ragged
pixel ranges, a single last pixel, pixels outside the sky, batches, the
no-allocation entry point, every precision and integrator, both metric kinds)
in a process of its own: no store may fall outside its buffer, every pixel is
written, and the codes agree with the oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_store_out_of_bounds():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_check_run.py")], capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    print(res)
    for name, v in res.items():
        assert v["faults"] == 0, name
        assert v["unwritten"] == 0, name
        assert v["same_codes"] >= 0.99, name
