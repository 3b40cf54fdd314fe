"""The benchmark workload at full size: R-MAT scale 26 (67,108,864 nodes, 1,073,741,824
arcs), SIR and SIS, beta=0.01, gamma=0.05, 6,710 seeds, R=256, T=100.

Checked in the benchmark's launch configuration (no per-realization outputs) by what
holds at any size, and against the oracle on sampled outputs it can compute: the first
two steps of realizations 0 and 1 (a second run with per-realization rows, whose totals
must equal the first run's)."""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def test_rmat26_sir_sis_full_size(cuda_lib):
    import torch
    f = cuda_lib
    g = W.rmat26_graph(26)
    wl = W.rmat26(O.SIR, g, 26)
    seeds = wl.seed_sets[0]
    graph = f.Graph(g.row_ptr, g.col_idx)
    n, R, T = g.n, wl.R, wl.T
    for model in (O.SIR, O.SIS):
        prm = dict(beta=wl.beta, gamma=wl.gamma)
        # the benchmark's configuration
        bench = f.simulate(graph, model, [seeds], R, T, wl.rng_seed, freq=False, **prm)
        counts = bench["counts"][0].cpu().numpy().astype(np.int64)      # [T+1][3]
        assert (counts.sum(axis=1) == n * R).all()
        assert counts[0, 1] == len(np.unique(seeds)) * R
        if model == O.SIR:
            assert (np.diff(counts[:, 2]) >= 0).all()                    # R never shrinks
            assert (np.diff(counts[:, 0]) <= 0).all()                    # S never grows
        else:
            assert (counts[:, 2] == 0).all()
        # per-realization rows: totals equal, every row sums to n
        out = f.simulate(graph, model, [seeds], R, T, wl.rng_seed, freq=False, per_real=True, **prm)
        pr = out["per_real"][0].cpu().numpy().astype(np.int64)          # [R][T+1][3]
        assert np.array_equal(pr.sum(axis=0), counts)
        assert (pr.sum(axis=2) == n).all()
        # realizations 0 and 1, first two steps, against the oracle
        orc = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=2, T=2, rng_seed=wl.rng_seed,
                         r_lo=0, n_real=2, nthreads=min(2, os.cpu_count() or 1),
                         outputs=("counts", "per_real"), **prm)
        assert np.array_equal(pr[:2, :3], orc.per_real.astype(np.int64))
        del bench, out
        torch.cuda.synchronize()


def _lane_states(model, planes, r):
    """0/1/2 states of lane r from device planes [P][n][W] (computed on the device)."""
    import torch
    b0 = ((planes[0, :, r >> 5] >> (r & 31)) & 1).to(torch.uint8)
    if model == O.SIS:
        return b0.cpu().numpy()
    b1 = ((planes[1, :, r >> 5] >> (r & 31)) & 1).to(torch.uint8)
    return (b0 + 2 * b1 * (1 - b0)).cpu().numpy()     # SIR: I -> 1, R -> 2


def test_rmat26_mid_epidemic_step_matches_oracle(cuda_lib):
    """Step 51 of the benchmark workload, deep in the epidemic (SIS endemic, hub rows
    hot): the GPU runs to t = 50 and to t = 51 in the benchmark's configuration; the
    oracle takes the GPU's t = 50 states of lanes {0, 1, 31, 32, 255} and computes one
    step (Algorithm 1 with the draws of those realizations, Sec. 3.1 Eq. batch), which
    must equal the GPU's t = 51 states element by element."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    f = cuda_lib
    g = W.rmat26_graph(26)
    wl = W.rmat26(O.SIR, g, 26)
    seeds = wl.seed_sets[0]
    graph = f.Graph(g.row_ptr, g.col_idx)
    lanes = (0, 1, 31, 32, 255)
    t_mid = 50
    for model in (O.SIR, O.SIS):
        prm = dict(beta=wl.beta, gamma=wl.gamma)
        a = f.simulate(graph, model, [seeds], wl.R, t_mid, wl.rng_seed, freq=False,
                       final_planes=True, **prm)
        st50 = {r: _lane_states(model, a["final_planes"][0], r) for r in lanes}
        del a
        b = f.simulate(graph, model, [seeds], wl.R, t_mid + 1, wl.rng_seed, freq=False,
                       final_planes=True, **prm)
        st51 = {r: _lane_states(model, b["final_planes"][0], r) for r in lanes}
        del b
        torch.cuda.synchronize()
        infected = sum(int((st50[r] == 1).sum()) for r in lanes)
        assert infected > 1000, infected         # mid-epidemic: many infected nodes

        def one(r):
            return O.simulate(model, g.row_ptr, g.col_idx, seeds, R=r + 1, T=1,
                              rng_seed=wl.rng_seed, r_lo=r, n_real=1, nthreads=1,
                              init_state=st50[r][None, :], t0=t_mid,
                              outputs=("counts", "final_state"), **prm)

        with ThreadPoolExecutor(max_workers=len(lanes)) as ex:
            res = list(ex.map(one, lanes))
        for r, orc in zip(lanes, res):
            assert np.array_equal(orc.final_state[0], st51[r]), (model, r)
    graph.close()
