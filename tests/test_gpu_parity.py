"""GPU path vs the CPU oracle, element by element (bit-exact: all outputs are integers).

Runs through the C ABI (libfsgp.so via its ctypes binding).  Sizes span several
tiles, ragged lane tails (R not a multiple of 32), every row class (team rows, warp
rows, CTA-split hub rows), dense and frontier steps, and the degenerate cases.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.planes import states_from_planes, planes_from_states

pytestmark = pytest.mark.gpu

MODELS = [O.SIR, O.SIS, O.IC, O.LT]
MNAME = {O.SIR: "SIR", O.SIS: "SIS", O.IC: "IC", O.LT: "LT"}


def gpu_run(fsgp, g, model, seed_sets, R, T, rng_seed, options=None, graph_obj=None, **prm):
    import torch
    graph = graph_obj or fsgp.Graph(g.row_ptr, g.col_idx)
    out = fsgp.simulate(graph, model, seed_sets, R, T, rng_seed, freq=True, per_real=True,
                        final_planes=True, steps_run=True, device=True, options=options, **prm)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["counts"] = res["counts"].astype(np.uint64)
    for k in ("freq", "per_real", "final_planes"):
        res[k] = res[k].view(np.uint32)
    return res


def assert_parity(fsgp, g, model, seeds, R, T, rng_seed, options=None, r_offset=0, **prm):
    """One seed set: every output of the GPU equals the oracle's."""
    gr = gpu_run(fsgp, g, model, [seeds], R, T, rng_seed, options=options, **prm)
    orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=R + r_offset, T=T, rng_seed=rng_seed,
                     r_lo=r_offset, n_real=R, **prm)
    ctx = f"{MNAME[model]} R={R} T={T} opts={options}"
    assert np.array_equal(gr["per_real"][0], orc.per_real), ctx + " per_real"
    assert np.array_equal(gr["counts"][0], orc.counts), ctx + " counts"
    assert np.array_equal(gr["freq"][0], orc.freq), ctx + " freq"
    st = states_from_planes(model, gr["final_planes"][0], range(R))
    assert np.array_equal(st, orc.final_state), ctx + " final state"
    if model in (O.IC, O.LT):
        assert gr["steps_run"][0] == (orc.quiet_step.max() if R else 0), ctx + " steps_run"
    else:
        assert gr["steps_run"][0] == T
    return gr, orc


def _prm(model):
    if model in (O.SIR, O.SIS):
        return dict(beta=0.15, gamma=0.2)
    return dict(ic_mode=O.IC_WEIGHTED_CASCADE)


# ----------------------------------------------------------------- workloads

def test_er10k_sir_full(cuda_lib):
    """ER n=10,000 mean degree 10, SIR beta=0.05 gamma=0.1, 1% seeds, R=64, T=50."""
    wl = W.er10k_sir()
    assert_parity(cuda_lib, wl.graph, O.SIR, wl.seed_sets[0], wl.R, wl.T, wl.rng_seed,
                  beta=wl.beta, gamma=wl.gamma)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("R", [1, 31, 32, 33, 100, 256])
def test_models_ragged_lanes(cuda_lib, model, R):
    g = W.rmat(11, 8, seed=101)
    seeds = W.seed_set(g.n, 12, seed=102)
    assert_parity(cuda_lib, g, model, seeds, R, 20, 7 + R, **_prm(model))


@pytest.mark.parametrize("model", MODELS)
def test_wide_lanes_1024(cuda_lib, model):
    g = W.ba(3000, 3, seed=103)
    seeds = W.seed_set(g.n, 5, seed=104)
    assert_parity(cuda_lib, g, model, seeds, 1024, 12, 99, **_prm(model))


@pytest.mark.parametrize("model", MODELS)
def test_max_lanes_4096(cuda_lib, model):
    g = W.er(600, 4.0, seed=105)
    seeds = W.seed_set(g.n, 4, seed=106)
    assert_parity(cuda_lib, g, model, seeds, 4096, 6, 5, **_prm(model))


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("opts", [
    dict(small_max_deg=3, hub_min_deg=16, hub_chunk=7, sparse_frac=-1.0),
    dict(small_max_deg=1, hub_min_deg=4, hub_chunk=1, sparse_frac=1.0),
    dict(small_max_deg=255, hub_min_deg=65536, sparse_frac=-1.0),
    dict(vector_words=1, sparse_frac=1.0),
    dict(vector_words=2, small_max_deg=7, hub_min_deg=64, hub_chunk=33),
])
def test_row_classes_and_paths_bit_identical(cuda_lib, model, opts):
    """Every tuning choice (team / warp / CTA-split rows, dense or frontier steps,
    words per thread) gives the oracle's results bit for bit."""
    g = W.rmat(12, 12, seed=107)       # skewed in-degrees: all three row classes
    seeds = W.seed_set(g.n, 20, seed=108)
    assert_parity(cuda_lib, g, model, seeds, 96, 15, 11, options=opts, **_prm(model))


@pytest.mark.parametrize("model", MODELS)
def test_realization_offset_matches_oracle_lanes(cuda_lib, model):
    """Lanes of a shard with r_offset = 64 are the oracle's realizations 64..64+R-1."""
    g = W.ba(2000, 4, seed=109)
    seeds = W.seed_set(g.n, 6, seed=110)
    assert_parity(cuda_lib, g, model, seeds, 70, 10, 12, options=dict(r_offset=64), r_offset=64,
                  **_prm(model))


@pytest.mark.parametrize("model", MODELS)
def test_resume_from_planes(cuda_lib, model):
    """T steps in one call == t steps, export planes, resume for T-t steps (t0 = t)."""
    g = W.rmat(10, 8, seed=111)
    seeds = W.seed_set(g.n, 8, seed=112)
    R, T, t = 80, 14, 6
    full = gpu_run(cuda_lib, g, model, [seeds], R, T, 21, **_prm(model))
    a = gpu_run(cuda_lib, g, model, [seeds], R, t, 21, **_prm(model))
    b = gpu_run(cuda_lib, g, model, [seeds], R, T - t, 21,
                options=dict(t0=t, init_planes=_dev(a["final_planes"][0])), **_prm(model))
    assert np.array_equal(full["final_planes"][0], b["final_planes"][0])
    assert np.array_equal(full["per_real"][0][:, t:], b["per_real"][0])
    # and the oracle resumed from the same states agrees
    st = states_from_planes(model, a["final_planes"][0], range(R))
    orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=R, T=T - t, rng_seed=21,
                     init_state=st, t0=t, **_prm(model))
    assert np.array_equal(b["per_real"][0], orc.per_real)


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).cuda()


@pytest.mark.parametrize("model", MODELS)
def test_import_arbitrary_start_state(cuda_lib, model):
    """Start planes given by the caller (random states) instead of seeds."""
    g = W.er(700, 5.0, seed=113)
    R, T = 40, 8
    rng = np.random.default_rng(5)
    if model in (O.IC, O.LT):
        st = rng.choice([0, 1, 2], size=(R, g.n), p=[0.9, 0.05, 0.05]).astype(np.uint8)
    elif model == O.SIS:
        st = (rng.random((R, g.n)) < 0.1).astype(np.uint8)
    else:
        st = rng.choice([0, 1, 2], size=(R, g.n), p=[0.85, 0.1, 0.05]).astype(np.uint8)
    planes = planes_from_states(model, st)
    gr = gpu_run(cuda_lib, g, model, [np.zeros(0, np.int32)], R, T, 31,
                 options=dict(t0=3, init_planes=_dev(planes)), **_prm(model))
    orc = O.simulate(model, g.row_ptr, g.col_idx, np.zeros(0, np.int32), R=R, T=T, rng_seed=31,
                     init_state=st, t0=3, **_prm(model))
    assert np.array_equal(gr["per_real"][0], orc.per_real)
    assert np.array_equal(states_from_planes(model, gr["final_planes"][0], range(R)), orc.final_state)


def test_multiple_seed_sets(cuda_lib):
    g = W.ba(1500, 3, seed=114)
    sets = [W.seed_set(g.n, k, seed=115 + k) for k in (1, 7, 30)]
    for model in MODELS:
        gr = gpu_run(cuda_lib, g, model, sets, 64, 10, 41, **_prm(model))
        for i, s in enumerate(sets):
            orc = O.simulate(model, g.row_ptr, g.col_idx, s, R=64, T=10, rng_seed=41, **_prm(model))
            assert np.array_equal(gr["per_real"][i], orc.per_real), (model, i)
            assert np.array_equal(gr["freq"][i], orc.freq), (model, i)


@pytest.mark.parametrize("model", MODELS)
def test_special_parameters(cuda_lib, model):
    g = W.rmat(10, 6, seed=116)
    seeds = W.seed_set(g.n, 5, seed=117)
    if model in (O.SIR, O.SIS):
        for beta, gamma in ((0.0, 0.3), (1.0, 1.0), (1.0, 0.0), (0.5, 0.0), (1e-12, 0.5)):
            assert_parity(cuda_lib, g, model, seeds, 45, 9, 3, beta=beta, gamma=gamma)
    elif model == O.IC:
        for p in (0.0, 1.0, 0.37):
            assert_parity(cuda_lib, g, model, seeds, 45, 30, 3, ic_mode=O.IC_CONSTANT, ic_p=p)
    else:
        assert_parity(cuda_lib, g, model, seeds, 45, 30, 3)


@pytest.mark.parametrize("model", MODELS)
def test_edge_cases(cuda_lib, model):
    # empty seed set
    g = W.er(300, 3.0, seed=118)
    assert_parity(cuda_lib, g, model, np.zeros(0, np.int32), 33, 5, 1, **_prm(model))
    # T = 0
    assert_parity(cuda_lib, g, model, W.seed_set(g.n, 3, seed=119), 33, 0, 1, **_prm(model))
    # no arcs at all
    empty = W.from_arcs(50, [], [])
    assert_parity(cuda_lib, empty, model, np.array([1, 2], np.int32), 40, 4, 1, **_prm(model))
    # self-loops, duplicate arcs, duplicate seeds
    g2 = W.from_arcs(6, [0, 0, 0, 1, 2, 2, 3, 4, 5, 5], [0, 1, 1, 2, 3, 3, 4, 5, 5, 0])
    assert_parity(cuda_lib, g2, model, np.array([0, 0, 2], np.int32), 64, 8, 2, **_prm(model))


def test_invalid_arguments_rejected(cuda_lib):
    f = cuda_lib
    g = W.er(100, 3.0, seed=120)
    graph = f.Graph(g.row_ptr, g.col_idx)
    with pytest.raises(f.FsgpError):
        f.simulate(graph, O.SIR, [np.array([5], np.int32)], 0, 3, 1, beta=0.1, gamma=0.1)
    with pytest.raises(f.FsgpError):
        f.simulate(graph, O.SIR, [np.array([5], np.int32)], 4097, 3, 1, beta=0.1, gamma=0.1)
    with pytest.raises(f.FsgpError):
        f.simulate(graph, O.SIR, [np.array([100], np.int32)], 32, 3, 1, beta=0.1, gamma=0.1)
    with pytest.raises(f.FsgpError):
        f.simulate(graph, O.SIR, [np.array([5], np.int32)], 32, 3, 1, beta=1.5, gamma=0.1)
    with pytest.raises(f.FsgpError):
        f.simulate(graph, 9, [np.array([5], np.int32)], 32, 3, 1)
    with pytest.raises(f.FsgpError):
        f.simulate(graph, O.SIR, [np.array([5], np.int32)], 32, 3, 1, beta=0.1,
                   options=dict(r_offset=5))
    bad_rp = g.row_ptr.copy()
    bad_rp[5] = bad_rp[6] + 1
    with pytest.raises(f.FsgpError):
        f.Graph(bad_rp, g.col_idx)
    bad_col = g.col_idx.copy()
    bad_col[3] = g.n
    with pytest.raises(f.FsgpError):
        f.Graph(g.row_ptr, bad_col)


def test_host_result_buffers(cuda_lib):
    """Results in host memory (the end-to-end path) equal the device-memory results."""
    wl = W.er10k_sir()
    graph = cuda_lib.Graph(wl.graph.row_ptr, wl.graph.col_idx)
    h = cuda_lib.simulate(graph, O.SIR, wl.seed_sets, wl.R, wl.T, wl.rng_seed, beta=wl.beta,
                          gamma=wl.gamma, per_real=True, final_planes=True, device=False)
    d = gpu_run(cuda_lib, wl.graph, O.SIR, wl.seed_sets, wl.R, wl.T, wl.rng_seed, beta=wl.beta,
                gamma=wl.gamma)
    for k in ("counts", "freq", "per_real", "final_planes", "steps_run"):
        assert np.array_equal(np.asarray(h[k]).view(d[k].dtype), d[k]), k


def test_trim_frees_workspace_and_keeps_results(cuda_lib):
    """fsgp_graph_trim drops the cached workspace; the next run re-allocates it and gives
    the same bits."""
    wl = W.er10k_sir()
    graph = cuda_lib.Graph(wl.graph.row_ptr, wl.graph.col_idx)
    a = gpu_run(cuda_lib, wl.graph, O.SIR, wl.seed_sets, wl.R, wl.T, wl.rng_seed, graph_obj=graph,
                beta=wl.beta, gamma=wl.gamma)
    grown = graph.info()["device_bytes"]
    graph.trim()
    assert graph.info()["device_bytes"] < grown
    graph.trim()                       # idempotent
    b = gpu_run(cuda_lib, wl.graph, O.SIR, wl.seed_sets, wl.R, wl.T, wl.rng_seed, graph_obj=graph,
                beta=wl.beta, gamma=wl.gamma)
    assert graph.info()["device_bytes"] == grown
    for k in ("counts", "freq", "per_real", "final_planes"):
        assert np.array_equal(a[k], b[k]), k


# ---------------------------------------------------------- larger workloads

@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_ba1m_r1024_lane_subset(cuda_lib, model):
    """BA n=1,000,000 m=5, R=1024, weighted cascade / LT 1/d_in, to quiescence (T<=100):
    the oracle runs lanes 0..31 and 992..1023 and must match those lanes exactly."""
    g = W.ba1m_graph()
    wl = W.ba1m(model, g)
    gr = gpu_run(cuda_lib, g, model, wl.seed_sets, wl.R, wl.T, wl.rng_seed)
    for lo in (0, 992):
        orc = O.simulate(model, g.row_ptr, g.col_idx, wl.seed_sets[0], R=wl.R, T=wl.T,
                         rng_seed=wl.rng_seed, r_lo=lo, n_real=32)
        assert np.array_equal(gr["per_real"][0][lo:lo + 32], orc.per_real), lo
        st = states_from_planes(model, gr["final_planes"][0], range(lo, lo + 32))
        assert np.array_equal(st, orc.final_state), lo
    pr = gr["per_real"][0].astype(np.int64)
    assert np.all(pr.sum(axis=2) == g.n)
    assert np.array_equal(gr["counts"][0].astype(np.int64), pr.sum(axis=0))


def test_rmat20_sir_sis_lane_subset(cuda_lib):
    """R-MAT scale 20 (16M arcs, hub rows present), SIR and SIS beta=0.01 gamma=0.05,
    R=256, T=100, lanes 0..7 and 250..255 against the oracle."""
    g = W.rmat(20, 16, seed=12345 + 3)
    seeds = W.seed_set(g.n, max(1, g.n // 10000), seed=22345 + 3)
    for model in (O.SIR, O.SIS):
        gr = gpu_run(cuda_lib, g, model, [seeds], 256, 100, 3, beta=0.01, gamma=0.05)
        for lo, cnt in ((0, 8), (250, 6)):
            orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=256, T=100, rng_seed=3,
                             beta=0.01, gamma=0.05, r_lo=lo, n_real=cnt)
            assert np.array_equal(gr["per_real"][0][lo:lo + cnt], orc.per_real), (model, lo)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("R,n_sets", [(32, 5), (64, 130), (100, 3)])
def test_stacked_seed_sets(cuda_lib, model, R, n_sets):
    """Many seed sets run side by side in one launch sequence (waves of up to 128 sets,
    odd set counts, 1-word sets): every set equals the oracle run of that set alone."""
    g = W.ba(2500, 3, seed=121)
    sets = [W.seed_set(g.n, 1 + (i % 7), seed=1000 + i) for i in range(n_sets)]
    gr = gpu_run(cuda_lib, g, model, sets, R, 9, 51, **_prm(model))
    check = sorted({0, 1, n_sets // 2, n_sets - 1})
    for i in check:
        orc = O.simulate(model, g.row_ptr, g.col_idx, sets[i], R=R, T=9, rng_seed=51, **_prm(model))
        assert np.array_equal(gr["per_real"][i], orc.per_real), (model, i)
        assert np.array_equal(gr["freq"][i], orc.freq), (model, i)
        st = states_from_planes(model, gr["final_planes"][i], range(R))
        assert np.array_equal(st, orc.final_state), (model, i)
        if model in (O.IC, O.LT):
            assert gr["steps_run"][i] == orc.quiet_step.max(), (model, i)
