"""Weighted graphs on the GPU (SIR, SIS and SI with per-arc probability beta * w_e): every
row class and path equals the oracle element by element (counts, per-realization counts,
frequencies, final states), device and host weights agree, batched weighted requests
equal single calls, the certain-arc limit equals the unweighted BFS run, and bad
requests are rejected."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

MODELS = [O.SIR, O.SIS, O.SI]


def _weights(g, seed, hi=2.0):
    return np.random.default_rng(seed).uniform(0.0, hi, size=g.nnz).astype(np.float32)


def _run(f, graph, model, sets, R, T, rng, options=None, **prm):
    import torch
    out = f.simulate(graph, model, sets, R, T, rng, weighted=True, freq=True, per_real=True,
                     final_planes=True, options=options, **prm)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["counts"] = res["counts"].astype(np.uint64)
    for k in ("freq", "per_real", "final_planes"):
        res[k] = res[k].view(np.uint32)
    return res


def _states(model, planes, R):
    I = ((planes[0][:, None, :] >> np.arange(32, dtype=np.uint32)[None, :, None]) & 1)
    I = I.transpose(0, 2, 1).reshape(planes.shape[1], -1)[:, :R]
    if model == O.SIR:
        Rp = ((planes[1][:, None, :] >> np.arange(32, dtype=np.uint32)[None, :, None]) & 1)
        Rp = Rp.transpose(0, 2, 1).reshape(planes.shape[1], -1)[:, :R]
        return np.where(I == 1, 1, np.where(Rp == 1, 2, 0)).T.astype(np.uint8)
    return I.T.astype(np.uint8)


def _check(f, g, w, model, seeds, R, T, rng, options=None, **prm):
    graph = f.Graph(g.row_ptr, g.col_idx)
    graph.set_arc_weights(w)
    gr = _run(f, graph, model, [seeds], R, T, rng, options=options, **prm)
    orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=R, T=T, rng_seed=rng, arc_weights=w, **prm)
    ctx = f"model {model} R={R} opts={options}"
    assert np.array_equal(gr["counts"][0], orc.counts), ctx + " counts"
    assert np.array_equal(gr["per_real"][0], orc.per_real), ctx + " per_real"
    assert np.array_equal(gr["freq"][0], orc.freq), ctx + " freq"
    assert np.array_equal(_states(model, gr["final_planes"][0], R), orc.final_state), ctx + " state"
    return gr


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("R", [1, 31, 32, 33, 256, 1024])
def test_weighted_matches_oracle(cuda_lib, model, R):
    g = W.rmat(11, 8, seed=601)
    w = _weights(g, 602)
    seeds = W.seed_set(g.n, 10, seed=603)
    _check(cuda_lib, g, w, model, seeds, R, 16, 70 + R, beta=0.15, gamma=0.2)


@pytest.mark.parametrize("model", [O.SIR, O.SIS])
@pytest.mark.parametrize("opts", [
    dict(small_max_deg=3, hub_min_deg=16, hub_chunk=7, sparse_frac=-1.0),   # split hub rows
    dict(small_max_deg=1, hub_min_deg=4, hub_chunk=1, sparse_frac=1.0),     # frontier steps
    dict(vector_words=1, sparse_frac=1.0),
    dict(vector_words=4, lane_words=2),
    dict(fuse_rows=1, persistent=-1),
    dict(fuse_rows=1, persistent=1),
])
def test_weighted_every_path_matches_oracle(cuda_lib, model, opts):
    g = W.ba(3000, 3, seed=611)          # hubs of a few hundred in-arcs
    w = _weights(g, 612)
    seeds = W.seed_set(g.n, 6, seed=613)
    _check(cuda_lib, g, w, model, seeds, 96, 14, 9, options=opts, beta=0.2, gamma=0.25)


def test_device_weights_and_reattach(cuda_lib):
    import torch
    f = cuda_lib
    g = W.er(2000, 6.0, seed=621)
    w = _weights(g, 622)
    seeds = W.seed_set(g.n, 8, seed=623)
    graph = f.Graph(g.row_ptr, g.col_idx)
    graph.set_arc_weights(torch.from_numpy(w).cuda())
    a = _run(f, graph, O.SIR, [seeds], 64, 20, 5, beta=0.2, gamma=0.1)
    graph.set_arc_weights(w)
    b = _run(f, graph, O.SIR, [seeds], 64, 20, 5, beta=0.2, gamma=0.1)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    w2 = _weights(g, 624)
    graph.set_arc_weights(w2)
    c = _run(f, graph, O.SIR, [seeds], 64, 20, 5, beta=0.2, gamma=0.1)
    orc = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, R=64, T=20, rng_seed=5, beta=0.2, gamma=0.1,
                     arc_weights=w2)
    assert np.array_equal(c["counts"][0], orc.counts)
    graph.set_arc_weights(None)
    with pytest.raises(f.FsgpError):
        _run(f, graph, O.SIR, [seeds], 64, 5, 5, beta=0.2, gamma=0.1)


def test_certain_arcs_equal_unweighted_bfs(cuda_lib):
    """beta * w >= 1 on every arc: every infectious in-arc transmits, as the unweighted
    rule does at beta = 1; with gamma = 1 both runs are deterministic and equal."""
    import torch
    f = cuda_lib
    g = W.rmat(10, 6, seed=631)
    seeds = W.seed_set(g.n, 4, seed=632)
    graph = f.Graph(g.row_ptr, g.col_idx)
    graph.set_arc_weights(np.full(g.nnz, 3.0, np.float32))
    a = f.simulate(graph, O.SIR, [seeds], 100, 12, 1, beta=0.5, gamma=1.0, weighted=True, final_planes=True)
    b = f.simulate(graph, O.SIR, [seeds], 100, 12, 2, beta=1.0, gamma=1.0, final_planes=True)
    torch.cuda.synchronize()
    for k in ("counts", "freq", "final_planes"):
        assert torch.equal(a[k], b[k]), k


def test_weighted_batch_equals_single(cuda_lib):
    import torch
    f = cuda_lib
    g = W.ba(1500, 4, seed=641)
    w = _weights(g, 642)
    graph = f.Graph(g.row_ptr, g.col_idx)
    graph.set_arc_weights(w)
    sets = [W.seed_set(g.n, k, seed=643 + k) for k in (1, 7, 20)]
    spec = [dict(graph=graph, model=m, seeds=sets[j], R=R, T=10, rng_seed=80 + j, beta=0.1 + 0.05 * j,
                 gamma=0.2, weighted=wt, freq=True)
            for j, (m, R, wt) in enumerate([(O.SIR, 64, True), (O.SIS, 200, True), (O.SIR, 64, False)])]
    outs = f.batch_run(spec)
    torch.cuda.synchronize()
    for q, o in zip(spec, outs):
        one = f.simulate(graph, q["model"], [q["seeds"]], q["R"], 10, q["rng_seed"], beta=q["beta"],
                         gamma=0.2, weighted=q["weighted"])
        torch.cuda.synchronize()
        assert torch.equal(o["counts"], one["counts"])
        assert torch.equal(o["freq"], one["freq"])


def test_weighted_rejections(cuda_lib):
    f = cuda_lib
    g = W.er(300, 3.0, seed=651)
    graph = f.Graph(g.row_ptr, g.col_idx)
    seeds = W.seed_set(g.n, 3, seed=652)
    bad = np.ones(g.nnz, np.float32)
    bad[3] = np.nan
    with pytest.raises(f.FsgpError):
        graph.set_arc_weights(bad)
    bad[3] = -0.5
    with pytest.raises(f.FsgpError):
        graph.set_arc_weights(bad)
    graph.set_arc_weights(np.ones(g.nnz, np.float32))
    with pytest.raises(f.FsgpError):       # IC has its own arc rule
        f.simulate(graph, O.IC, [seeds], 32, 4, 1, weighted=True)
    with pytest.raises(f.FsgpError):       # the single-instance path has no weights
        f.simulate_single(graph, O.SIR, seeds, 0, 4, 1, beta=0.1, gamma=0.1, weighted=True)
