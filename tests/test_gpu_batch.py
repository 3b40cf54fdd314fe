"""Batched requests (fsgp_batch_run) and the autotuner, through the C ABI.

Every request of a batch must equal an fsgp_simulate call for it alone (bit for bit),
whatever the stacking, streams, CUDA-graph capture or tuning; a few requests are also
checked against the CPU oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _pool():
    return W.batch_pool(n_graphs=6, n_requests=60, n_min=500, n_max=20_000, seed=77, T=25)


def _single(f, graphs, gobjs, q):
    out = f.simulate(gobjs[q.graph_index], q.model, [q.seeds], q.R, q.T, q.rng_seed, beta=q.beta,
                     gamma=q.gamma, ic_mode=O.IC_WEIGHTED_CASCADE, freq=True, device=True)
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("capture,streams", [(0, 4), (-1, 1), (0, 1)])
def test_batch_equals_single_requests(cuda_lib, capture, streams):
    import torch
    f = cuda_lib
    graphs, reqs = _pool()
    gobjs = [f.Graph(g.row_ptr, g.col_idx) for g in graphs]
    spec = [dict(graph=gobjs[q.graph_index], model=q.model, seeds=q.seeds, R=q.R, T=q.T,
                 rng_seed=q.rng_seed, beta=q.beta, gamma=q.gamma, freq=True) for q in reqs]
    outs = f.batch_run(spec, n_streams=streams, capture_graph=capture)
    torch.cuda.synchronize()
    for i, q in enumerate(reqs):
        ref = _single(f, graphs, gobjs, q)
        got = {k: v.cpu().numpy() for k, v in outs[i].items()}
        assert np.array_equal(got["counts"], ref["counts"]), i
        assert np.array_equal(got["freq"], ref["freq"]), i
        assert np.array_equal(got["steps_run"], ref["steps_run"]), i
    # and a few against the oracle
    for i in (0, 7, 33):
        q = reqs[i]
        g = graphs[q.graph_index]
        orc = O.simulate(q.model, g.row_ptr, g.col_idx, q.seeds, beta=q.beta, gamma=q.gamma,
                         R=q.R, T=q.T, rng_seed=q.rng_seed)
        assert np.array_equal(outs[i]["counts"][0].cpu().numpy().astype(np.uint64), orc.counts), i
        assert np.array_equal(outs[i]["freq"][0].cpu().numpy().view(np.uint32), orc.freq), i


def test_autotune_picks_valid_and_identical(cuda_lib):
    f = cuda_lib
    g = W.rmat(14, 12, seed=301)
    seeds = W.seed_set(g.n, 30, seed=302)
    graph = f.Graph(g.row_ptr, g.col_idx)
    opts = f.fsgp_options()
    prm = f.fsgp_params(beta=0.05, gamma=0.1, ic_mode=0, ic_p=0.0)
    f.fsgp_autotune(graph.handle, 0, prm, seeds, len(seeds), 256, 4, 9, opts)
    # either the automatic defaults won (fields left at 0) or one explicit candidate did
    if (opts.vector_words, opts.small_max_deg, opts.hub_min_deg, opts.hub_chunk) != (0, 0, 0, 0):
        assert opts.vector_words in (1, 2, 4)
        assert opts.small_max_deg in (63, 255) and opts.hub_min_deg in (4096, 8192, 16384)
    a = f.simulate(graph, 0, [seeds], 256, 30, 9, beta=0.05, gamma=0.1, per_real=True)
    b = f.simulate(graph, 0, [seeds], 256, 30, 9, beta=0.05, gamma=0.1, per_real=True, options=opts)
    for k in a:
        assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), k


def test_batch_rejects_bad_request(cuda_lib):
    f = cuda_lib
    g = W.er(300, 3.0, seed=303)
    graph = f.Graph(g.row_ptr, g.col_idx)
    with pytest.raises(f.FsgpError):
        f.batch_run([dict(graph=graph, model=0, seeds=np.array([1], np.int32), R=5000, T=3,
                          rng_seed=1, beta=0.1, gamma=0.1)])
