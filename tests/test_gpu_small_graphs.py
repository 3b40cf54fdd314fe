"""Small graphs: the fused launch (every row in one warp-per-row kernel, dense steps) and
the reuse of captured step-loop graphs across runs give the same bits as the degree-class
kernels and as the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model", [O.SIR, O.SIS, O.IC, O.LT, O.SEIR, O.SWIR])
def test_fused_rows_equal_classes_and_oracle(cuda_lib, model):
    import torch
    f = cuda_lib
    g = W.ba(3000, 4, seed=701)        # hub rows of a few hundred in-arcs
    seeds = W.seed_set(g.n, 15, seed=702)
    prm = dict(beta=0.1, gamma=0.1, alpha=0.3, mu=0.2, nu=0.3) if model not in (O.IC, O.LT) else {}
    graph = f.Graph(g.row_ptr, g.col_idx)
    outs = {}
    for fuse in (1, -1):
        o = f.simulate(graph, model, [seeds], 96, 20, 13, per_real=True, final_planes=True,
                       options=dict(fuse_rows=fuse), **prm)
        torch.cuda.synchronize()
        outs[fuse] = {k: v.cpu().numpy() for k, v in o.items()}
    for k in outs[1]:
        assert np.array_equal(outs[1][k], outs[-1][k]), k
    orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=96, T=20, rng_seed=13, **prm)
    assert np.array_equal(outs[1]["per_real"][0].view(np.uint32), orc.per_real)
    assert np.array_equal(outs[1]["counts"][0].astype(np.uint64), orc.counts)


def test_captured_graph_reused_across_runs(cuda_lib):
    """Repeated captured runs (same launch sequence: the cached executable graph is
    relaunched) with changing seeds and parameters equal fresh uncaptured runs."""
    import torch
    f = cuda_lib
    wl = W.er10k_sir()
    g = wl.graph
    graph = f.Graph(g.row_ptr, g.col_idx)
    st = torch.cuda.Stream()
    for i, (beta, k) in enumerate([(0.05, 100), (0.08, 100), (0.05, 37), (0.02, 100)]):
        seeds = W.seed_set(g.n, k, seed=900 + i)
        with torch.cuda.stream(st):
            a = f.simulate(graph, O.SIR, [seeds], wl.R, wl.T, 1 + i, beta=beta, gamma=wl.gamma,
                           per_real=True, options=dict(capture_graph=1), stream=st)
        st.synchronize()
        b = f.simulate(graph, O.SIR, [seeds], wl.R, wl.T, 1 + i, beta=beta, gamma=wl.gamma, per_real=True)
        torch.cuda.synchronize()
        for key in a:
            assert np.array_equal(a[key].cpu().numpy(), b[key].cpu().numpy()), (i, key)
        if i == 3:
            orc = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, beta=beta, gamma=wl.gamma, R=wl.R, T=wl.T,
                             rng_seed=1 + i)
            assert np.array_equal(a["per_real"][0].cpu().numpy().view(np.uint32), orc.per_real)
