"""Small graphs: the persistent step loop (all T steps of the fused team-per-row mode in one
cooperative launch, steps separated by bounded grid barriers) gives the same bits as the
launched step loop and as the oracle, and its barrier reports a wait that runs out
instead of hanging."""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

PRM = dict(beta=0.12, gamma=0.15, alpha=0.35, mu=0.25, nu=0.4)


def _run(f, graph, model, sets, R, T, rng, pers, **kw):
    import torch
    prm = {} if model in (O.IC, O.LT) else PRM
    o = f.simulate(graph, model, sets, R, T, rng, freq=True, final_planes=True,
                   options=dict(fuse_rows=1, persistent=pers, **kw.pop("options", {})), **prm, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in o.items()}


@pytest.mark.parametrize("model", [O.SIR, O.SIS, O.IC, O.LT, O.SEIR, O.SEIS, O.SWIR, O.SI])
@pytest.mark.parametrize("R", [1, 64, 100, 1024])
def test_persistent_equals_launched_and_oracle(cuda_lib, model, R):
    f = cuda_lib
    g = W.er(3000, 6.0, seed=811)          # every in-degree well below 256: team kernel
    seeds = W.seed_set(g.n, 12, seed=812)
    graph = f.Graph(g.row_ptr, g.col_idx)
    T = 40
    a = _run(f, graph, model, [seeds], R, T, 21, 1)
    b = _run(f, graph, model, [seeds], R, T, 21, -1)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    if R <= 100:
        prm = {} if model in (O.IC, O.LT) else PRM
        orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=R, T=T, rng_seed=21, **prm)
        assert np.array_equal(a["counts"][0].astype(np.uint64), orc.counts)
        assert np.array_equal(a["freq"][0].astype(np.uint32), orc.freq)


def test_persistent_stacked_sets_resume_and_stop(cuda_lib):
    """Three seed sets side by side; IC stops at quiescence inside the loop (later rows
    repeat); a run resumed from exported planes continues the same realizations."""
    f = cuda_lib
    g = W.er(2000, 3.0, seed=821)
    graph = f.Graph(g.row_ptr, g.col_idx)
    sets = [W.seed_set(g.n, k, seed=822 + k) for k in (1, 5, 30)]
    for model in (O.IC, O.SIR):
        a = _run(f, graph, model, sets, 96, 80, 5, 1)
        b = _run(f, graph, model, sets, 96, 80, 5, -1)
        for k in a:
            assert np.array_equal(a[k], b[k]), (model, k)
    a = _run(f, graph, O.IC, sets, 96, 80, 5, 1)
    assert (a["steps_run"] < 80).all()           # the cascades stopped inside the loop
    # resume: 15 steps, then 25 more from the exported planes == 40 steps at once
    import torch
    first = _run(f, graph, O.SIR, sets, 96, 15, 6, 1)
    planes = torch.from_numpy(first["final_planes"]).cuda()
    o = f.simulate(graph, O.SIR, [s[:0] for s in sets], 96, 25, 6, freq=True, final_planes=True,
                   options=dict(fuse_rows=1, persistent=1, t0=15, init_planes=planes), **PRM)
    torch.cuda.synchronize()
    whole = _run(f, graph, O.SIR, sets, 96, 40, 6, 1)
    assert np.array_equal(o["final_planes"].cpu().numpy(), whole["final_planes"])
    assert np.array_equal(o["counts"].cpu().numpy()[:, -1], whole["counts"][:, -1])


def test_persistent_host_results(cuda_lib):
    """Host result buffers through the persistent loop equal the device results."""
    f = cuda_lib
    g = W.er(1500, 5.0, seed=831)
    graph = f.Graph(g.row_ptr, g.col_idx)
    seeds = W.seed_set(g.n, 8, seed=832)
    d = _run(f, graph, O.SIS, [seeds], 64, 30, 9, 1)
    h = f.simulate(graph, O.SIS, [seeds], 64, 30, 9, freq=True, device=False,
                   options=dict(fuse_rows=1, persistent=1), **PRM)
    assert np.array_equal(np.asarray(h["counts"]).astype(np.uint64), d["counts"].astype(np.uint64))
    assert np.array_equal(np.asarray(h["freq"]).astype(np.uint32), d["freq"].astype(np.uint32))


def test_grid_barrier_completes_and_times_out(cuda_lib):
    """The barrier passes when every CTA arrives, and a barrier that waits for a CTA that
    never comes (a flag nothing sets) ends each wait after its cycle limit with
    FSGP_ETIMEOUT; the device stays usable."""
    import torch
    f = cuda_lib
    assert f.fsgp_selftest_barrier(16, 0, 500, 2_000_000_000) == f.FSGP_OK
    t = time.perf_counter()
    assert f.fsgp_selftest_barrier(16, 1, 3, 20_000_000) == f.FSGP_ETIMEOUT
    assert time.perf_counter() - t < 10.0
    g = W.er(500, 4.0, seed=841)
    graph = f.Graph(g.row_ptr, g.col_idx)
    o = f.simulate(graph, O.SIR, [W.seed_set(g.n, 5, seed=842)], 32, 5, 1, beta=0.3, gamma=0.2)
    torch.cuda.synchronize()
    assert int(o["counts"][0, 0].sum().item()) == g.n * 32
