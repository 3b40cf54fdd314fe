"""Partitioned execution on the GPU (Sec. 3.2): the graph split into target-node
partitions, each partition's row kernels updating only its targets from the previous
step's full state, the new target states combined after every step, equals the
unpartitioned run bit for bit (states and per-step counts) for the node-keyed models."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

PRM = {O.SIR: dict(beta=0.15, gamma=0.2), O.SIS: dict(beta=0.15, gamma=0.2), O.LT: {},
       O.SEIR: dict(beta=0.2, alpha=0.3, gamma=0.15), O.SWIR: dict(beta=0.15, mu=0.25, nu=0.4),
       O.SI: dict(beta=0.1)}


@pytest.mark.parametrize("model", [O.SIR, O.SIS, O.LT, O.SEIR, O.SWIR, O.SI])
@pytest.mark.parametrize("d", [2, 3, 5])
def test_partitioned_equals_single(cuda_lib, model, d):
    import torch
    from paper_2603_14895_gb300.partitioned import PartitionedGraph, run_partitioned
    f = cuda_lib
    g = W.ba(3000, 3, seed=951)
    seeds = W.seed_set(g.n, 10, seed=952)
    pg = PartitionedGraph(g.row_ptr, g.col_idx, d)
    loads = [p.load for p in pg.parts]
    assert sum(loads) == g.nnz and max(loads) - min(loads) <= 2 * int(np.diff(g.row_ptr).max())
    counts, planes = run_partitioned(pg, model, seeds, 96, 12, 17, **PRM[model])
    graph = f.Graph(g.row_ptr, g.col_idx)
    one = f.simulate(graph, model, [seeds], 96, 12, 17, final_planes=True, **PRM[model])
    torch.cuda.synchronize()
    assert torch.equal(planes, one["final_planes"][0])
    assert torch.equal(counts, one["counts"][0])
    pg.close()


def test_partitioned_rejects_arc_keyed_models(cuda_lib):
    from paper_2603_14895_gb300.partitioned import PartitionedGraph, run_partitioned
    g = W.er(500, 3.0, seed=953)
    pg = PartitionedGraph(g.row_ptr, g.col_idx, 2)
    with pytest.raises(ValueError):
        run_partitioned(pg, O.IC, W.seed_set(g.n, 3, seed=954), 32, 3, 1)
    with pytest.raises(ValueError):
        run_partitioned(pg, O.SIR, W.seed_set(g.n, 3, seed=954), 32, 3, 1, beta=0.1, weighted=True)
    pg.close()
