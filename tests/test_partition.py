"""Target-node partitioning (Sec. 3.2) on CPU: the load-balance proposition, exact
coverage of targets and arcs, and the distributed step protocol of Sec. 3.2 emulated by
gloo ranks that update only their own targets (with the oracle's per-node rule) and sum
their new target states after every step."""
import os
import socket
import traceback

import numpy as np
import pytest

import workloads as W
from paper_2603_14895_gb300.partition import partition_graph, target_partition


def _graphs():
    yield W.rmat(12, 16, seed=61)
    yield W.ba(3000, 4, seed=62)
    yield W.er(2000, 5.0, seed=63)
    yield W.from_arcs(40, [0] * 30 + [1, 2, 3], [5] * 30 + [6, 7, 8])      # one heavy row
    yield W.from_arcs(10, [], [])                                          # no arcs


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 13])
def test_load_balance_and_coverage(d):
    for g in _graphs():
        deg = np.diff(g.row_ptr.astype(np.int64))
        q = target_partition(deg, d)
        assert q.shape == (g.n,) and q.min() >= 0 and q.max() < d
        Wt = int(deg.sum())
        wmax = int(deg.max()) if g.n else 0
        loads = np.bincount(q, weights=deg, minlength=d)
        if Wt > 0:
            # the proposition: |load_q - W/d| < w_max for every partition
            assert (np.abs(loads - Wt / d) < wmax).all(), (g.name, d, loads, Wt / d, wmax)
        parts = partition_graph(g.row_ptr, g.col_idx, d, q)
        # every target in exactly one partition, every arc in the partition of its target
        allt = np.concatenate([p.targets for p in parts])
        assert np.array_equal(np.sort(allt), np.arange(g.n))
        assert sum(p.load for p in parts) == g.nnz
        for p in parts:
            for k in range(0, len(p.targets), max(1, len(p.targets) // 50)):
                v = p.targets[k]
                a, b = g.row_ptr[v], g.row_ptr[v + 1]
                assert p.arc_begin[k] == a
                assert np.array_equal(p.col_idx[p.row_ptr[k]:p.row_ptr[k + 1]], g.col_idx[a:b])


def test_partition_follows_the_sorted_prefix_rule():
    # degrees 5, 3, 3, 1, 0 (node order 2, 0, 4, 1, 3 after the stable sort), d = 2:
    # C = 5, 8, 11, 12, 12; q = ceil(2 C / 12) = 1, 2, 2, 2, 2
    deg = np.array([3, 1, 5, 0, 3])
    q = target_partition(deg, 2)
    assert q.tolist() == [1, 1, 0, 1, 1]
    # d = 4: q = ceil(4 C / 12) = 2, 3, 4, 4, 4
    assert target_partition(deg, 4).tolist() == [2, 3, 1, 3, 3]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, model, q_out):
    try:
        import torch
        import torch.distributed as dist
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import oracle as O
        g = W.rmat(8, 6, seed=64)
        seeds = W.seed_set(g.n, 5, seed=65)
        prm = dict(beta=0.3, gamma=0.2) if model in (O.SIR, O.SIS) else dict(ic_mode=O.IC_WEIGHTED_CASCADE)
        T, r, seed = 8, 3, 17
        part = partition_graph(g.row_ptr, g.col_idx, world)[rank]
        # this rank's view: only its targets' rows, at their global arc positions
        col_local = np.zeros(g.nnz, dtype=np.int32)
        for k, v in enumerate(part.targets):
            a = int(part.arc_begin[k])
            col_local[a:a + part.row_ptr[k + 1] - part.row_ptr[k]] = part.col_idx[part.row_ptr[k]:part.row_ptr[k + 1]]
        X = np.zeros(g.n, dtype=np.uint8)
        X[seeds] = 1
        rows = []
        for t in range(1, T + 1):
            Y = np.zeros(g.n, dtype=np.int64)
            for v in part.targets:
                Y[v] = O.node_step(model, g.row_ptr, col_local, int(v), X, t=t, r=r, rng_seed=seed, **prm)
            Yt = torch.from_numpy(Y)
            dist.all_reduce(Yt, op=dist.ReduceOp.SUM)   # each node comes from exactly one rank
            X = Yt.numpy().astype(np.uint8)
            rows.append(np.bincount(X, minlength=3)[:3])
        full = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=r + 1, T=T, rng_seed=seed,
                          r_lo=r, n_real=1, outputs=("per_real", "final_state"), **prm)
        ok = (np.array_equal(X, full.final_state[0])
              and np.array_equal(np.array(rows), full.per_real[0, 1:].astype(np.int64)))
        dist.destroy_process_group()
        q_out.put((rank, "ok" if ok else "mismatch"))
    except Exception:
        q_out.put((rank, traceback.format_exc()))


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_distributed_step_protocol_matches_single_run(model):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_worker, args=(r, world, port, model, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in procs:
            rank, msg = q.get(timeout=300)
            out[rank] = msg
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert out == {r: "ok" for r in range(world)}, out
