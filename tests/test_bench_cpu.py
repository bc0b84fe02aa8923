"""CPU checks of bench.py's host-side pieces: the host record, the
sparse-direct sample, the C oracle's timed V-cycle and the reference arm's
JSON line (the oracle timed on the host: no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_host_record():
    h = bench.host_info()
    assert h["nproc"] >= 1 and h["machine"]
    assert "cpu_model" in h


def test_sparse_direct_sample_small():
    r = bench.sparse_direct_sample(64)
    assert r["N"] == 64 and r["n_dof"] > 0 and r["value"] > 0 and r["seconds"] > 0


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--N", "512"], capture_output=True,
                         text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
                "ms_per_step", "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["config"]["N"] == 512
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_cpu_vcycle_timing():
    p, s, lev, F = bench.oracle_hierarchy(64)
    sec, cyc, used, u = bench.cpu_vcycle(lev, F, 2, steps=1, warmup=0)
    assert sec > 0 and 0 < cyc < 30 and used == 2
    r = F - s.A @ u
    assert abs(r[s.dof]).max() <= 1e-10 * abs(F).max()
