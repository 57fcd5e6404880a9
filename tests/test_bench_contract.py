"""bench.py's output contract, on the CPU: the reference arm (the oracle on the
host cores) prints one JSON line with the keys and types the benchmark's
consumers read; the workload and config helpers describe the headline scene."""
import json
import math
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--cpu-seconds", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key, typ in (("impl", str), ("metric", str), ("value", float), ("unit", str), ("n_gpus", int),
                     ("steps", int), ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool),
                     ("scaling", str), ("dtype", str), ("data", str), ("config", dict), ("cpu_baseline", dict),
                     ("e2e", dict)):
        assert isinstance(d[key], typ), key
    assert d["impl"] == "reference" and d["unit"] == "geodesics/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and math.isfinite(d["value"])
    assert d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "kerr_a0.9_i60_disk_1024"


def test_headline_workload_and_config():
    sys.path.insert(0, ROOT)
    import bench
    sc = bench.workload(1024)
    assert (sc.nx, sc.ny, sc.a, sc.rtol, sc.atol, sc.r_obs) == (1024, 1024, 0.9, 1e-10, 1e-10, 1000.0)
    assert abs(math.degrees(sc.theta_obs) - 60.0) < 1e-12 and (sc.alpha_min, sc.alpha_max) == (-20.0, 20.0)
    cfg = bench.config_dict(sc, 1)
    assert cfg["workload"] == sc.name and cfg["theta_obs_deg"] == 60.0 and cfg["parallelism"] == "dp1"
    assert "critical_band" not in cfg
    m = bench.workload(2048, "mixed_pair").replace(critical_band=-1.0)
    assert bench.config_dict(m, 1)["critical_band"] == -1.0
