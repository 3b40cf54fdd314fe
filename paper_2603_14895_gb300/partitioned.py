"""Partitioned execution of the propagation step (Sec. 3.2): the graph is split into
target-node partitions (partition.target_partition), each partition's row kernels
update only its own targets from the previous step's full state, and the partitions' new
target states are combined before the next step (the exchange of the distributed step;
every node is written by exactly one partition).

Each partition is a graph handle of its own: the in-CSR of all n nodes in which only the
partition's targets keep their in-arcs.  The partitions run one after another on the
current GPU, each for one step from the combined state (fsgp_simulate with t0 and
init_planes); on several devices each would run on its own.  Draws are keyed by node,
realization and step, so the combined run equals the unpartitioned one bit for bit for
every model whose draws are keyed by node: SIR, SIS, SI, LT, SEIR, SEIS, SWIR.  IC and
weighted runs key their draws by the arc's position in the caller's col_idx, which a
partition's own CSR renumbers, so they are not supported here.
"""
from __future__ import annotations

import numpy as np

from . import fsgp
from .partition import partition_graph

_NODE_KEYED = (fsgp.SIR, fsgp.SIS, fsgp.SI, fsgp.LT, fsgp.SEIR, fsgp.SEIS, fsgp.SWIR)


class PartitionedGraph:
    """d target partitions of an in-CSR graph, each as a device graph handle."""

    def __init__(self, row_ptr, col_idx, d: int):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.n = int(row_ptr.shape[0] - 1)
        self.parts = partition_graph(row_ptr, col_idx, d)
        deg = np.diff(row_ptr.astype(np.int64))
        self.graphs = []
        for p in self.parts:
            keep = np.zeros(self.n, dtype=np.int64)
            keep[p.targets] = deg[p.targets]
            rp = np.zeros(self.n + 1, dtype=np.int64)
            np.cumsum(keep, out=rp[1:])
            # targets are increasing node ids, so the partition's arcs are in CSR order
            self.graphs.append(fsgp.Graph(rp.astype(np.int32), np.ascontiguousarray(p.col_idx)))

    def close(self):
        for g in self.graphs:
            g.close()


def run_partitioned(pg: PartitionedGraph, model: int, seeds, R: int, T: int, rng_seed: int, **params):
    """T steps of `model` from the seed set, partition by partition each step.  Returns
    (counts [T+1][C] int64 over all realizations, final planes [P][n][ceil(R/32)] int32),
    both torch tensors on the current device."""
    import torch
    if model not in _NODE_KEYED:
        raise ValueError("partitioned runs need node-keyed draws (not IC or weighted graphs)")
    if params.get("weighted"):
        raise ValueError("weighted runs key their draws by arc position")
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    empty = seeds[:0]
    # step 0: the seeded state (any partition's handle has all n nodes)
    out = fsgp.simulate(pg.graphs[0], model, [seeds], R, 0, rng_seed, freq=False, final_planes=True, **params)
    state = out["final_planes"][0].clone()
    counts = [out["counts"][0, 0].clone()]
    targets = [torch.from_numpy(p.targets.astype(np.int64)).to(state.device) for p in pg.parts]
    for t in range(1, T + 1):
        new = torch.empty_like(state)
        for g, tg in zip(pg.graphs, targets):
            o = fsgp.simulate(g, model, [empty], R, 1, rng_seed, freq=False, final_planes=True,
                              options=dict(t0=t - 1, init_planes=state), **params)
            new[:, tg, :] = o["final_planes"][0][:, tg, :]
        state = new
        # the step's compartment counts, from the combined state (a zero-step run)
        c = fsgp.simulate(pg.graphs[0], model, [empty], R, 0, rng_seed, freq=False,
                          options=dict(t0=t, init_planes=state), **params)
        counts.append(c["counts"][0, 0].clone())
    return torch.stack(counts), state
