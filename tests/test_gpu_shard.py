"""run_sharded on the GPU: one NCCL rank, and two ranks' lane ranges run one after the
other on the same GPU (no kernel waits on another rank) and summed on the host, against
one run over every lane."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from paper_2603_14895_gb300.shard import lane_shard

pytestmark = pytest.mark.gpu


def test_run_sharded_single_rank_and_two_lane_ranges(cuda_lib):
    import torch
    import torch.distributed as dist
    from paper_2603_14895_gb300.shard import run_sharded
    f = cuda_lib
    g = W.er(5000, 8.0, seed=41)
    seeds = W.seed_set(g.n, 20, seed=42)
    graph = f.Graph(g.row_ptr, g.col_idx)
    R_total, T = 72, 30
    full = f.simulate(graph, 0, [seeds], R_total, T, 5, beta=0.1, gamma=0.1, per_real=True)
    # two ranks' lane ranges, summed on the host
    parts = []
    for rank in range(2):
        r0, rl = lane_shard(R_total, 2, rank)
        parts.append(f.simulate(graph, 0, [seeds], rl, T, 5, beta=0.1, gamma=0.1, per_real=True,
                                options=dict(r_offset=r0)))
    assert torch.equal(parts[0]["counts"] + parts[1]["counts"], full["counts"])
    assert torch.equal(parts[0]["freq"] + parts[1]["freq"], full["freq"])
    assert torch.equal(torch.cat([parts[0]["per_real"], parts[1]["per_real"]], 1), full["per_real"])
    # the public helper through a one-rank NCCL group
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        m = run_sharded(graph, 0, [seeds], R_total, T, 5, world=1, rank=0, per_real=True,
                        beta=0.1, gamma=0.1)
    finally:
        dist.destroy_process_group()
    assert torch.equal(m["counts"], full["counts"].to(torch.int64))
    assert torch.equal(m["freq"], full["freq"].to(torch.int64))
    assert torch.equal(m["per_real"], full["per_real"].to(torch.int64))
