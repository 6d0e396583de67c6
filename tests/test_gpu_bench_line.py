"""The benchmark's GPU line (a short run without the comparison rows): the
contract's keys, the same config as the reference arm, host copies counted
in the end-to-end figure, the dominant kernel's roofline against the
measured float64 peak, the clocks sampled during the timed solves, and the
measured DRAM figures whenever the committed ncu summaries match the
library sources."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line():
    r = subprocess.run([sys.executable, "bench.py", "--steps", "3", "--warmup", "3",
                        "--no-extras", "--no-cpu-baseline"], cwd=ROOT, capture_output=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr.decode()[-2000:]
    lines = [l for l in r.stdout.decode().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
                "gpu_launches", "roofline", "clocks"):
        assert key in d, key
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "DOF/s" and d["dtype"] == "f64"
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == json.loads(json.dumps(bench.bench_config(1)))
    cells = 256 ** 3
    assert d["e2e"]["h2d_bytes_per_step"] == 8 * cells
    assert d["e2e"]["d2h_bytes_per_step"] == 8 * cells
    assert d["e2e"]["value"] > 0
    assert d["gpu_launches"] > 0 and d["gpu_launches"] % 3 == 0
    rf = d["roofline"]
    assert rf["bound"] == "alu" and rf["peak"] > 0
    assert 0.3 < rf["frac"] < 1.2
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    if bench.ncu_traffic(rf["kernel"]) is not None:
        assert rf["traffic"] == bench.ncu_traffic(rf["kernel"])
    if bench.ncu_dram_per_solve():
        assert d["hbm"]["dram_bytes_per_solve"] == bench.ncu_dram_per_solve()["sr_fmg_fp64_256"]
