"""Pins of the oracle's weighted graphs (SIR, SIS and SI with a weight w_e per arc: arc e
infects with probability beta * w_e per step, independently over arcs), against what
that definition fixes without the oracle's own loop: deterministic limits that reduce to
breadth-first search layers, the no-weight limit, and the exact synchronous Markov chain
over 3^N states on a tiny graph with unequal weights (chi-square over 2^14
realizations), which also rejects the unweighted model of the same mean rate."""
import itertools
from collections import defaultdict

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle as O
import workloads as W
from tests.exact_models import chi_square_gof


def _bfs_layers(g, seeds):
    n = g.n
    dst = np.repeat(np.arange(n), np.diff(g.row_ptr))
    A = csr_matrix((np.ones(g.nnz), (g.col_idx, dst)), shape=(n, n))   # u -> v
    return shortest_path(A, indices=np.unique(seeds), unweighted=True).min(axis=0)


def _weights(g, seed, lo=0.0, hi=2.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=g.nnz).astype(np.float32)


@pytest.mark.parametrize("beta,w", [(1.0, 1.0), (0.5, 5.0)])
def test_certain_arcs_give_bfs_layers(beta, w):
    """beta * w >= 1 on every arc: every infectious in-arc transmits, so SIR with
    gamma = 1 infects BFS layer t at step t and removes it at t + 1."""
    g = W.er(300, 3.0, seed=51)
    seeds = W.seed_set(g.n, 3, seed=52)
    T = 12
    res = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, beta=beta, gamma=1.0, R=40, T=T, rng_seed=3,
                     arc_weights=np.full(g.nnz, w, np.float32))
    d = _bfs_layers(g, seeds)
    for t in range(T + 1):
        I = int((d == t).sum())
        Rm = int((d < t).sum())
        assert np.array_equal(res.counts[t].astype(np.int64), np.array([g.n - I - Rm, I, Rm]) * 40), t


def test_zero_weights_infect_nobody():
    g = W.ba(200, 3, seed=53)
    seeds = W.seed_set(g.n, 5, seed=54)
    for model in (O.SIR, O.SIS, O.SI):
        res = O.simulate(model, g.row_ptr, g.col_idx, seeds, beta=0.9, gamma=0.3, R=33, T=10, rng_seed=4,
                         arc_weights=np.zeros(g.nnz, np.float32))
        S = res.counts[:, 0].astype(np.int64)
        assert (S == (g.n - len(np.unique(seeds))) * 33).all() if model != O.SIS else (S >= S[0]).all()
        assert res.counts[0, 1] == len(np.unique(seeds)) * 33


def test_weights_need_a_supported_model_and_valid_values():
    g = W.er(50, 2.0, seed=55)
    seeds = W.seed_set(g.n, 2, seed=56)
    with pytest.raises(ValueError):
        O.simulate(O.IC, g.row_ptr, g.col_idx, seeds, R=4, T=3, arc_weights=np.ones(g.nnz, np.float32))
    bad = np.ones(g.nnz, np.float32)
    bad[0] = -1.0
    with pytest.raises(ValueError):
        O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, beta=0.2, R=4, T=3, arc_weights=bad)


def _exact_weighted(row_ptr, col_idx, p_arc, g_rec, init, T, mode):
    """Distribution of (S, I, R) after T synchronous steps: a susceptible node escapes
    with prod over infectious in-arcs (1 - p_e); an infected one recovers with g_rec
    (to R for SIR, to S for SIS; SI: never)."""
    n = len(row_ptr) - 1
    cur = {tuple(init): 1.0}
    for _ in range(T):
        nxt = defaultdict(float)
        for st, p in cur.items():
            opts = []
            for v in range(n):
                s = st[v]
                if s == 0:
                    esc = 1.0
                    for e in range(row_ptr[v], row_ptr[v + 1]):
                        if st[col_idx[e]] == 1:
                            esc *= 1.0 - p_arc[e]
                    opts.append([(1, 1.0 - esc), (0, esc)])
                elif s == 1:
                    back = 2 if mode == "sir" else 0
                    opts.append([(back, g_rec), (1, 1.0 - g_rec)] if mode != "si" else [(1, 1.0)])
                else:
                    opts.append([(2, 1.0)])
            for combo in itertools.product(*[[o for o in op if o[1] > 0] for op in opts]):
                q = p
                for _, w in combo:
                    q *= w
                if q > 0:
                    nxt[tuple(s for s, _ in combo)] += q
        cur = nxt
    out = defaultdict(float)
    for st, p in cur.items():
        out[(st.count(0), st.count(1), st.count(2))] += p
    return out


def _tiny():
    # 5 nodes: 0->1, 0->2, 1->2, 2->3, 1->3, 3->4, 4->3, 2->4, and a duplicate 0->1
    return W.from_arcs(5, [0, 0, 1, 2, 1, 3, 4, 2, 0], [1, 2, 2, 3, 3, 4, 3, 4, 1])


@pytest.mark.parametrize("model,mode", [(O.SIR, "sir"), (O.SIS, "sis"), (O.SI, "si")])
def test_exact_weighted_chain_chi_square(model, mode):
    g = _tiny()
    w = np.array([0.3, 1.7, 0.9, 2.5, 0.0, 1.2, 0.6, 1.0, 0.8], np.float32)[: g.nnz]
    beta, gamma = 0.35, 0.3
    R, T = 1 << 14, 5
    seeds = np.array([0], np.int32)
    res = O.simulate(model, g.row_ptr, g.col_idx, seeds, beta=beta, gamma=gamma, R=R, T=T, rng_seed=91,
                     arc_weights=w)
    obs = defaultdict(int)
    for row in res.per_real[:, -1, :]:
        obs[tuple(int(x) for x in row[:3])] += 1
    p_arc = np.minimum(1.0, beta * w.astype(np.float64))
    init = [1, 0, 0, 0, 0]
    exact = _exact_weighted(g.row_ptr, g.col_idx, p_arc, gamma, init, T, mode)
    stat, thr, _ = chi_square_gof(obs, exact, R)
    assert stat < thr, (stat, thr)
    # the same counts reject the model whose arcs all carry the mean rate
    flat = _exact_weighted(g.row_ptr, g.col_idx, np.full(g.nnz, p_arc.mean()), gamma, init, T, mode)
    if all(k in flat and flat[k] > 0 for k in obs):
        stat2, thr2, _ = chi_square_gof(obs, flat, R)
        assert stat2 > thr2, (stat2, thr2)
