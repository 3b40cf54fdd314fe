"""The plain single-instance path (one realization, one byte per node) against the
oracle's lane r, and against lane r of the packed path."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

MODELS = [O.SIR, O.SIS, O.IC, O.LT]


def _prm(model):
    if model in (O.SIR, O.SIS):
        return dict(beta=0.12, gamma=0.2)
    return dict(ic_mode=O.IC_WEIGHTED_CASCADE)


def _check(f, g, model, seeds, r, T, rng, graph=None, **prm):
    graph = graph or f.Graph(g.row_ptr, g.col_idx)
    out = f.simulate_single(graph, model, seeds, r, T, rng, **prm)
    orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=r + 1, T=T, rng_seed=rng, r_lo=r, n_real=1,
                     outputs=("counts", "final_state"), **prm)
    assert np.array_equal(out["counts"].cpu().numpy().astype(np.uint64), orc.counts), (model, r)
    assert np.array_equal(out["final_state"].cpu().numpy(), orc.final_state[0]), (model, r)
    if model in (O.IC, O.LT):
        assert int(out["steps_run"][0]) == int(orc.quiet_step[0])
    return out


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("r", [0, 37, 1000])
def test_single_matches_oracle_lane(cuda_lib, model, r):
    g = W.er(3000, 6.0, seed=51)
    seeds = W.seed_set(g.n, 15, seed=52)
    _check(cuda_lib, g, model, seeds, r, 25, 11, **_prm(model))


@pytest.mark.parametrize("model", MODELS)
def test_single_big_rows(cuda_lib, model):
    """R-MAT scale 14, edge factor 16: rows of several thousand in-arcs go to the
    CTA-per-row kernel."""
    g = W.rmat(14, 16, seed=53)
    assert np.diff(g.row_ptr).max() >= 4096
    seeds = W.seed_set(g.n, 10, seed=54)
    prm = dict(beta=0.02, gamma=0.3) if model in (O.SIR, O.SIS) else dict(ic_mode=O.IC_WEIGHTED_CASCADE)
    _check(cuda_lib, g, model, seeds, 5, 12, 12, **prm)


@pytest.mark.parametrize("model", MODELS)
def test_single_equals_packed_lane(cuda_lib, model):
    import torch
    f = cuda_lib
    g = W.ba(5000, 3, seed=55)
    seeds = W.seed_set(g.n, 8, seed=56)
    graph = f.Graph(g.row_ptr, g.col_idx)
    prm = _prm(model)
    packed = f.simulate(graph, model, [seeds], 96, 30, 13, per_real=True, final_planes=False, **prm)
    for r in (3, 64, 95):
        s = f.simulate_single(graph, model, seeds, r, 30, 13, **prm)
        assert torch.equal(s["counts"], packed["per_real"][0, r].to(torch.int64)), (model, r)


def test_single_edge_cases(cuda_lib):
    f = cuda_lib
    g = W.er(500, 4.0, seed=57)
    graph = f.Graph(g.row_ptr, g.col_idx)
    # no seeds: IC is quiet from the start, SIR stays all-S
    out = f.simulate_single(graph, O.IC, np.zeros(0, np.int32), 0, 5, 1, ic_mode=0)
    assert int(out["steps_run"][0]) == 0
    assert (out["counts"][:, 0] == g.n).all()
    _check(f, g, O.SIR, np.zeros(0, np.int32), 4, 3, 2, graph=graph, beta=0.5, gamma=0.5)
    # T = 0, duplicate seeds, beta = 1 / gamma = 0
    _check(f, g, O.SIR, np.array([3, 3, 7], np.int32), 9, 0, 2, graph=graph, beta=1.0, gamma=0.0)
    _check(f, g, O.SIS, np.array([3, 3, 7], np.int32), 9, 6, 2, graph=graph, beta=1.0, gamma=0.0)
    with pytest.raises(f.FsgpError):
        f.simulate_single(graph, O.SIR, np.array([g.n], np.int32), 0, 3, 1, beta=0.1, gamma=0.1)
    with pytest.raises(f.FsgpError):
        f.simulate_single(graph, O.SIR, np.array([1], np.int32), -1, 3, 1, beta=0.1, gamma=0.1)
    # the library stays usable after the rejected calls
    _check(f, g, O.LT, np.array([1, 2], np.int32), 0, 4, 3, graph=graph, ic_mode=0)
