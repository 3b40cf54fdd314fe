"""Target-node partitioning (Sec. 3.2, the partitioning definition and its load-balance
proposition), for graphs beyond one device's memory.

Nodes are sorted by non-increasing in-degree (ties by node id), the prefix sums C_i of
their weights w = in-degree are taken, and node pi_i goes to partition
q(i) = ceil(d C_i / W) (W = C_N).  Every target node lands in exactly one partition, so
its in-arcs E_q = {(u, v) : v in P_q} are all local and its update needs no partial
messages; after each step the partitions' new target states are combined (one sum over
partitions, every node contributed by exactly one of them).  The load of every
partition is within w_max of W / d.

Host logic only (numpy).  One GB300 holds graphs of a billion arcs (an R-MAT scale-26
graph with its tables takes 14.7 GB of 288), so the propagation kernels normally run
unpartitioned; this module is the partitioner and its subgraph extraction, and
partitioned.py runs the step partition by partition.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def target_partition(in_degree, d: int) -> np.ndarray:
    """Partition id (0-based) of every node.  With no arcs at all (W = 0) the nodes are
    split into d runs of equal size in the sorted order (the definition divides by W)."""
    w = np.asarray(in_degree, dtype=np.int64)
    n = w.shape[0]
    if d < 1:
        raise ValueError("need at least one partition")
    order = np.argsort(-w, kind="stable")            # non-increasing, ties by node id
    C = np.cumsum(w[order])
    W = int(C[-1]) if n else 0
    if W == 0:
        q_sorted = (np.arange(n, dtype=np.int64) * d) // max(n, 1)
    else:
        q_sorted = (d * C + W - 1) // W - 1          # ceil(d C_i / W), made 0-based
        np.clip(q_sorted, 0, d - 1, out=q_sorted)
    q = np.empty(n, dtype=np.int32)
    q[order] = q_sorted.astype(np.int32)
    return q


@dataclass
class Partition:
    """One partition's targets and their in-arcs.  Row k of the local CSR is target
    targets[k]; its arcs are the global arcs arc_begin[k] .. arc_begin[k] + deg, kept in
    order (IC draws are keyed by the global arc position)."""
    targets: np.ndarray      # int32, increasing node ids
    row_ptr: np.ndarray      # int32 [len(targets) + 1], local
    col_idx: np.ndarray      # int32 sources (global ids)
    arc_begin: np.ndarray    # int64 global position of each target's first arc
    sources: np.ndarray      # int32 distinct sources: the states this partition reads

    @property
    def load(self) -> int:
        return int(self.col_idx.shape[0])


def partition_graph(row_ptr, col_idx, d: int, q=None) -> list[Partition]:
    """Split an in-CSR into d target partitions (q from target_partition if not given)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int32)
    deg = np.diff(row_ptr)
    if q is None:
        q = target_partition(deg, d)
    parts = []
    for p in range(d):
        in_p = q == p
        t = np.nonzero(in_p)[0].astype(np.int32)
        dt = deg[t]
        rp = np.zeros(t.shape[0] + 1, dtype=np.int64)
        np.cumsum(dt, out=rp[1:])
        # the arcs of this partition's rows, in CSR order (rows are contiguous arc ranges)
        cols = col_idx[np.repeat(in_p, deg)]
        seen = np.zeros(deg.shape[0], dtype=bool)   # distinct sources by marking, not sorting
        seen[cols] = True
        parts.append(Partition(targets=t, row_ptr=rp.astype(np.int32), col_idx=cols,
                               arc_begin=row_ptr[t].astype(np.int64),
                               sources=np.nonzero(seen)[0].astype(np.int32)))
    return parts
