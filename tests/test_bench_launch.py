"""bench.py --gpus N starts N ranks by itself (torch.distributed.run on 127.0.0.1) when it
is not already running under torchrun.  On a machine without GPUs the ranks join a gloo
group; --dry-run makes each take its realization shard and rank 0 report them."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(n):
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", str(n), "--dry-run"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_two_ranks_start_and_shard_lanes():
    d = _run(2)
    assert d["n_gpus"] == 2 and d["backend"] == "gloo"
    ranks = sorted(d["ranks"], key=lambda x: x["rank"])
    assert [r["rank"] for r in ranks] == [0, 1]
    R = d["lanes_per_rank"]
    # weak scaling: rank i runs lanes [i R, (i+1) R) of a 2R-lane job
    assert [(r["r_offset"], r["R"]) for r in ranks] == [(0, R), (R, R)]


def test_one_rank_needs_no_launcher():
    d = _run(1)
    assert d["n_gpus"] == 1 and d["ranks"][0]["r_offset"] == 0
