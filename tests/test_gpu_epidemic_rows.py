"""GPU parity of the discrete-time epidemic rows of Table 1 (SI, SEIR(DT), SEIS(DT), SWIR)
against the oracle, element by element: per-realization and total compartment counts,
per-node frequencies and final states, through every row class (thread, team, warp and
CTA-split rows), dense and frontier steps, ragged and wide lane counts, stacked seed sets
and batched requests."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

MODELS = [O.SI, O.SEIR, O.SEIS, O.SWIR]
PRM = {O.SI: dict(beta=0.2), O.SEIR: dict(beta=0.2, alpha=0.3, gamma=0.15),
       O.SEIS: dict(beta=0.2, alpha=0.35, gamma=0.2), O.SWIR: dict(beta=0.15, mu=0.25, nu=0.4)}


def _states(model, planes, lanes):
    """Oracle state codes from the GPU planes [P][n][W]."""
    planes = planes.astype(np.uint32)

    def bit(p, r):
        return ((planes[p][:, r >> 5] >> np.uint32(r & 31)) & 1).astype(np.uint8)

    out = np.zeros((len(lanes), planes.shape[1]), np.uint8)
    for i, r in enumerate(lanes):
        I = bit(0, r)
        if model == O.SI:
            out[i] = I
        elif model == O.SEIS:                 # planes I, E -> 0 S, 1 E, 2 I
            out[i] = np.where(I == 1, 2, np.where(bit(1, r) == 1, 1, 0))
        else:                                 # SEIR I, R, E / SWIR I, R, W -> 0, 1 (E/W), 2 I, 3 R
            out[i] = np.where(I == 1, 2, np.where(bit(1, r) == 1, 3, np.where(bit(2, r) == 1, 1, 0)))
    return out


def _run(f, g, model, sets, R, T, rng, options=None, graph=None, **prm):
    import torch
    graph = graph or f.Graph(g.row_ptr, g.col_idx)
    out = f.simulate(graph, model, sets, R, T, rng, freq=True, per_real=True, final_planes=True,
                     options=options, **prm)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["counts"] = res["counts"].astype(np.uint64)
    for k in ("freq", "per_real", "final_planes"):
        res[k] = res[k].view(np.uint32)
    return res


def _check(f, g, model, seeds, R, T, rng, options=None, **prm):
    gr = _run(f, g, model, [seeds], R, T, rng, options=options, **prm)
    orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=R, T=T, rng_seed=rng, **prm)
    ctx = f"model {model} R={R} T={T} opts={options}"
    assert gr["counts"].shape[2] == O.compartments(model)
    assert np.array_equal(gr["per_real"][0], orc.per_real), ctx + " per_real"
    assert np.array_equal(gr["counts"][0], orc.counts), ctx + " counts"
    assert np.array_equal(gr["freq"][0], orc.freq), ctx + " freq"
    assert np.array_equal(_states(model, gr["final_planes"][0], range(R)), orc.final_state), ctx + " state"
    assert gr["steps_run"][0] == T


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("R", [31, 256, 1024])
def test_models_match_oracle(cuda_lib, model, R):
    g = W.rmat(11, 8, seed=501)
    seeds = W.seed_set(g.n, 10, seed=502)
    _check(cuda_lib, g, model, seeds, R, 18, 40 + R, **PRM[model])


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("opts", [
    dict(small_max_deg=3, hub_min_deg=16, hub_chunk=7, sparse_frac=-1.0),
    dict(small_max_deg=1, hub_min_deg=4, hub_chunk=1, sparse_frac=1.0),
    dict(vector_words=1, sparse_frac=1.0),
    dict(lane_words=2, small_max_deg=7, hub_min_deg=64, hub_chunk=33),
])
def test_row_classes_and_paths(cuda_lib, model, opts):
    g = W.rmat(12, 12, seed=503)   # skewed in-degrees: thread, team, warp and split rows
    seeds = W.seed_set(g.n, 20, seed=504)
    _check(cuda_lib, g, model, seeds, 96, 14, 9, options=opts, **PRM[model])


@pytest.mark.parametrize("model", [O.SEIR, O.SWIR])
def test_degenerate_parameters(cuda_lib, model):
    g = W.ba(1200, 3, seed=505)
    seeds = W.seed_set(g.n, 6, seed=506)
    for prm in ([dict(beta=1.0, alpha=1.0, gamma=1.0), dict(beta=0.0, alpha=0.0, gamma=0.0),
                 dict(beta=0.5, alpha=0.0, gamma=1.0)] if model == O.SEIR else
                [dict(beta=1.0, mu=0.0, nu=0.0), dict(beta=0.0, mu=1.0, nu=1.0), dict(beta=0.0, mu=0.0, nu=0.0)]):
        _check(cuda_lib, g, model, seeds, 64, 10, 3, **prm)


def test_stacked_sets_and_batch(cuda_lib):
    import torch
    f = cuda_lib
    g = W.ba(2500, 3, seed=507)
    graph = f.Graph(g.row_ptr, g.col_idx)
    sets = [W.seed_set(g.n, 1 + i, seed=600 + i) for i in range(5)]
    for model in MODELS:
        gr = _run(f, g, model, sets, 64, 9, 51, graph=graph, **PRM[model])
        for i in (0, 4):
            orc = O.simulate(model, g.row_ptr, g.col_idx, sets[i], R=64, T=9, rng_seed=51, **PRM[model])
            assert np.array_equal(gr["per_real"][i], orc.per_real), (model, i)
    spec = [dict(graph=graph, model=m, seeds=sets[j], R=96, T=8, rng_seed=70 + j, freq=True, **PRM[m])
            for j, m in enumerate(MODELS)]
    outs = f.batch_run(spec)
    torch.cuda.synchronize()
    for j, m in enumerate(MODELS):
        orc = O.simulate(m, g.row_ptr, g.col_idx, sets[j], R=96, T=8, rng_seed=70 + j, **PRM[m])
        assert np.array_equal(outs[j]["counts"][0].cpu().numpy().astype(np.uint64), orc.counts), m
        assert np.array_equal(outs[j]["freq"][0].cpu().numpy().view(np.uint32), orc.freq), m


def test_import_exposed_and_weakened_states(cuda_lib):
    """Start planes given by the caller with exposed (SEIR) / weakened (SWIR) lanes."""
    import torch
    f = cuda_lib
    g = W.er(800, 5.0, seed=508)
    R, T = 40, 7
    rng = np.random.default_rng(3)
    for model in (O.SEIR, O.SEIS, O.SWIR):
        ns = 3 if model == O.SEIS else 4
        st = rng.choice(range(ns), size=(R, g.n), p=[0.85, 0.08, 0.07] if ns == 3 else [0.8, 0.08, 0.07, 0.05])
        st = st.astype(np.uint8)
        W_ = (R + 31) // 32
        P = 2 if model == O.SEIS else 3
        planes = np.zeros((P, g.n, W_), np.uint64)
        for r in range(R):
            s = st[r]
            sh = np.uint64(r & 31)
            planes[0, :, r >> 5] |= (s == 2).astype(np.uint64) << sh          # I
            if model == O.SEIS:
                planes[1, :, r >> 5] |= (s == 1).astype(np.uint64) << sh      # E
            else:
                planes[1, :, r >> 5] |= (s == 3).astype(np.uint64) << sh      # R
                planes[2, :, r >> 5] |= (s == 1).astype(np.uint64) << sh      # E / W
        dev = torch.from_numpy(planes.astype(np.uint32).view(np.int32)).cuda()
        gr = _run(f, g, model, [np.zeros(0, np.int32)], R, T, 31, options=dict(t0=3, init_planes=dev), **PRM[model])
        orc = O.simulate(model, g.row_ptr, g.col_idx, np.zeros(0, np.int32), R=R, T=T, rng_seed=31,
                         init_state=st, t0=3, **PRM[model])
        assert np.array_equal(gr["per_real"][0], orc.per_real), model
        assert np.array_equal(_states(model, gr["final_planes"][0], range(R)), orc.final_state), model


def test_other_entry_points_refuse_new_models(cuda_lib):
    f = cuda_lib
    g = W.er(100, 3.0, seed=509)
    graph = f.Graph(g.row_ptr, g.col_idx)
    with pytest.raises(f.FsgpError) as e:
        f.simulate_single(graph, O.SEIR, np.array([1], np.int32), 0, 3, 1, beta=0.1)
    assert e.value.code == f.FSGP_EUNSUPPORTED
