"""bench.py's reference arm on CPU: the JSON line it prints carries the keys the
measurement contract asks for (the arm times the oracle; no GPU is involved)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--scale", "12", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("rmat12_")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_cpu_baseline_blocks_and_rate():
    """bench.cpu_baseline times the oracle in blocks of one realization per core: with no
    time floor it runs one block, with a floor it stops at R at the latest, and its rate
    is arcs x realizations x steps over the seconds it reports."""
    import re
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import bench
    import workloads as W
    g = W.rmat(12, 8, seed=11)
    s = W.seed_set(g.n, 20, seed=12)
    cores = os.cpu_count() or 1
    one = bench.cpu_baseline(g, s, min_seconds=0.0)
    m = re.match(r"SIR, (\d+) realizations x 1 steps on the full graph, ([0-9.]+) s", one["sample"])
    assert m and int(m.group(1)) == min(cores, bench.R)
    assert one["cores"] == cores and one["kind"] == "oracle" and one["value"] > 0
    full = bench.cpu_baseline(g, s, min_seconds=1e9)
    assert full["sample"].startswith(f"SIR, {bench.R} realizations")
