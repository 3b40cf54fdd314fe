"""Realization sharding on CPU ranks (gloo, world size 2): disjoint lane ranges, merged
by the package's host logic, equal one run over every lane.  Each rank computes its
lanes with the oracle (the CPU stand-in for a GPU), so no GPU is involved."""
import os
import socket
import traceback

import numpy as np
import pytest

from paper_2603_14895_gb300.shard import lane_shard


def test_lane_shard_covers_every_lane_once():
    for R in (1, 20, 31, 32, 33, 64, 72, 256, 1000, 4096):
        for world in (1, 2, 3, 4, 8):
            seen = []
            prev_end = 0
            for rank in range(world):
                r0, rl = lane_shard(R, world, rank)
                assert r0 == prev_end
                assert r0 % 32 == 0 or rl == 0
                # only the job's last group may be ragged
                if rl and r0 + rl < R:
                    assert rl % 32 == 0
                seen.extend(range(r0, r0 + rl))
                prev_end = r0 + rl
            assert seen == list(range(R)), (R, world)
    # whole groups are spread as evenly as possible
    sizes = [lane_shard(32 * 10, 4, r)[1] // 32 for r in range(4)]
    assert sizes == [3, 3, 2, 2]
    with pytest.raises(ValueError):
        lane_shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = {
    # model, R_total, T, params: rank 0 gets two groups, rank 1 one ragged group
    "sir_ragged": (0, 72, 12, dict(beta=0.2, gamma=0.15)),
    # rank 1 gets no lanes
    "ic_one_group": (2, 20, 10, dict(ic_mode=0)),
    "lt_even": (3, 64, 10, dict(ic_mode=0)),
    "sis_even": (1, 64, 8, dict(beta=0.1, gamma=0.3)),
}


def _worker(rank, world, port, case, q):
    try:
        import torch
        import torch.distributed as dist
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import oracle as O
        import workloads as W
        from paper_2603_14895_gb300.shard import merge_results
        model, R_total, T, prm = CASES[case]
        g = W.er(300, 5.0, seed=31)
        seeds = W.seed_set(g.n, 6, seed=32)
        r0, rl = lane_shard(R_total, world, rank)
        if rl:
            res = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=r0 + rl, T=T, rng_seed=9,
                             r_lo=r0, n_real=rl, outputs=("counts", "per_real", "freq"), **prm)
            local = {"counts": torch.from_numpy(res.counts.astype(np.int64))[None],
                     "freq": torch.from_numpy(res.freq.astype(np.int64))[None],
                     "per_real": torch.from_numpy(res.per_real.astype(np.int64))[None],
                     "steps_run": torch.tensor([int(res.quiet_step.max())], dtype=torch.int32)}
        else:
            local = {"counts": torch.zeros((1, T + 1, 3), dtype=torch.int64),
                     "freq": torch.zeros((1, 3, g.n), dtype=torch.int64),
                     "per_real": torch.zeros((1, 0, T + 1, 3), dtype=torch.int64),
                     "steps_run": torch.zeros((1,), dtype=torch.int32)}
        merged = merge_results(local, R_total, world, rank)
        full = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=R_total, T=T, rng_seed=9,
                          outputs=("counts", "per_real", "freq"), **prm)
        ok = (np.array_equal(merged["counts"][0].numpy(), full.counts.astype(np.int64))
              and np.array_equal(merged["freq"][0].numpy(), full.freq.astype(np.int64))
              and np.array_equal(merged["per_real"][0].numpy(), full.per_real.astype(np.int64)))
        if model in (2, 3):
            ok = ok and int(merged["steps_run"][0]) == int(full.quiet_step.max())
        dist.destroy_process_group()
        q.put((rank, "ok" if ok else "mismatch"))
    except Exception:
        q.put((rank, traceback.format_exc()))


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_cpu_ranks_merge_to_the_single_run(case):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in procs:
            rank, msg = q.get(timeout=180)
            out[rank] = msg
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert out == {0: "ok", 1: "ok"}, out
