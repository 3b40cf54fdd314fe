"""Pins of the oracle's discrete-time epidemic rows of Table 1 (SI, SEIR(DT), SEIS(DT),
SWIR), against what the definitions fix without running the oracle's own loop:
identities with the SIR / SIS rows, deterministic limits that reduce to breadth-first
search layers, and exact synchronous Markov chains over 4^N states on tiny graphs
(chi-square over 2^14 realizations)."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle as O
import workloads as W
from tests.exact_models import SeirRule, SwirRule, chain_state_distribution, chi_square_gof


def _graphs():
    return [W.er(200, 3.0, seed=11), W.ba(150, 2, seed=12), W.rmat(8, 4, seed=13)]


def _bfs_layers(g, seeds):
    n = g.n
    dst = np.repeat(np.arange(n), np.diff(g.row_ptr))
    A = csr_matrix((np.ones(g.nnz), (g.col_idx, dst)), shape=(n, n))   # u -> v
    d = shortest_path(A, indices=np.unique(seeds), unweighted=True).min(axis=0)
    return d


@pytest.mark.parametrize("gi", range(3))
def test_si_equals_sis_and_sir_without_recovery(gi):
    g = _graphs()[gi]
    seeds = W.seed_set(g.n, 4, seed=20 + gi)
    kw = dict(beta=0.2, R=70, T=15, rng_seed=5 + gi)
    si = O.simulate(O.SI, g.row_ptr, g.col_idx, seeds, **kw)
    sis = O.simulate(O.SIS, g.row_ptr, g.col_idx, seeds, gamma=0.0, **kw)
    sir = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, gamma=0.0, **kw)
    assert np.array_equal(si.per_real, sis.per_real)
    assert np.array_equal(si.per_real, sir.per_real)
    assert np.array_equal(si.final_state, sir.final_state)
    assert (np.diff(si.counts[:, 1].astype(np.int64)) >= 0).all()


@pytest.mark.parametrize("gi", range(3))
def test_seir_deterministic_limit_is_bfs_with_period_two(gi):
    """beta = alpha = gamma = 1: a node at distance d >= 1 from the seeds is exposed at
    step 2d-1, infectious at 2d and removed at 2d+1; seeds are removed at step 1."""
    g = _graphs()[gi]
    seeds = W.seed_set(g.n, 3, seed=30 + gi)
    T = 14
    res = O.simulate(O.SEIR, g.row_ptr, g.col_idx, seeds, beta=1.0, alpha=1.0, gamma=1.0,
                     R=33, T=T, rng_seed=1)
    d = _bfs_layers(g, seeds)
    L = {k: int((d == k).sum()) for k in range(0, T + 2)}
    for t in range(T + 1):
        E = L.get((t + 1) // 2, 0) if t % 2 == 1 else 0
        I = L.get(t // 2, 0) if t % 2 == 0 else 0
        Rm = sum(L[k] for k in L if 2 * k + 1 <= t)
        want = np.array([g.n - E - I - Rm, E, I, Rm]) * 33
        assert np.array_equal(res.counts[t].astype(np.int64), want), t


@pytest.mark.parametrize("gi", range(3))
def test_swir_deterministic_limits(gi):
    g = _graphs()[gi]
    seeds = W.seed_set(g.n, 3, seed=40 + gi)
    T = 10
    d = _bfs_layers(g, seeds)
    L = {k: int((d == k).sum()) for k in range(0, T + 2)}
    # kappa = 1: infected at distance d at step d, removed at d + 1, nobody weakened
    res = O.simulate(O.SWIR, g.row_ptr, g.col_idx, seeds, beta=1.0, mu=0.7, nu=0.3, R=32, T=T,
                     rng_seed=2)
    for t in range(T + 1):
        I = L.get(t, 0)
        Rm = sum(L[k] for k in L if k < t)
        assert np.array_equal(res.counts[t].astype(np.int64), np.array([g.n - I - Rm, 0, I, Rm]) * 32), t
    # kappa = 0, mu = 1: the seeds' out-neighbours are weakened at step 1; the seeds are
    # removed then, so nothing is infectious afterwards and the weakened stay weakened
    res = O.simulate(O.SWIR, g.row_ptr, g.col_idx, seeds, beta=0.0, mu=1.0, nu=1.0, R=32, T=T,
                     rng_seed=3)
    for t in range(1, T + 1):
        want = np.array([g.n - L[0] - L[1], L[1], 0, L[0]]) * 32
        assert np.array_equal(res.counts[t].astype(np.int64), want), t


def _tiny(model):
    if model == O.SWIR:
        # layered: every node after the first two layers has two sources that become
        # infectious one step apart, so weakened nodes meet a second infectious source
        return W.from_arcs(5, [0, 0, 1, 2, 1, 3, 2], [1, 2, 2, 3, 3, 4, 4])
    # 5 nodes: a directed triangle 0->1->2->0, 1->3, 3->4, 4->3, a self-loop on 2,
    # a duplicate arc 0->1
    return W.from_arcs(5, [0, 1, 2, 1, 3, 4, 2, 0], [1, 2, 0, 3, 4, 3, 2, 1])


def _mc_counts(res, C):
    out = {}
    for row in res.per_real[:, -1, :]:
        key = tuple(int(x) for x in row[:C])
        out[key] = out.get(key, 0) + 1
    return out


@pytest.mark.parametrize("model,kw", [
    (O.SEIR, dict(beta=0.45, alpha=0.5, gamma=0.35)),
    (O.SEIS, dict(beta=0.45, alpha=0.6, gamma=0.4)),
    (O.SWIR, dict(beta=0.2, mu=0.7, nu=0.95)),
])
def test_exact_markov_chain_chi_square(model, kw):
    g = _tiny(model)
    seeds = np.array([0], np.int32)
    T, R = 5, 1 << 14
    res = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=R, T=T, rng_seed=77, **kw)
    init = [0] * g.n
    init[0] = 2
    if model == O.SWIR:
        rule = SwirRule(kw["beta"], kw["mu"], kw["nu"])
        C = 4
    else:
        rule = SeirRule(kw["beta"], kw["alpha"], kw["gamma"], sis=model == O.SEIS)
        C = 4 if model == O.SEIR else 3
    exact = chain_state_distribution(g.row_ptr, g.col_idx, init, T, rule, 4)
    if C == 3:   # SEIS reports S, E, I
        red = {}
        for k, p in exact.items():
            assert k[3] == 0
            red[k[:3]] = red.get(k[:3], 0.0) + p
        exact = red
    stat, thr, df = chi_square_gof(_mc_counts(res, C), exact, R)
    assert stat < thr, (stat, thr, df)


@pytest.mark.parametrize("model", [O.SI, O.SEIR, O.SEIS, O.SWIR])
def test_invariants_and_resume(model):
    g = W.ba(300, 3, seed=50)
    seeds = W.seed_set(g.n, 5, seed=51)
    kw = dict(beta=0.25, gamma=0.2, alpha=0.4, mu=0.3, nu=0.5, rng_seed=9)
    C = O.compartments(model)
    full = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=40, T=12, **kw)
    pr = full.per_real.astype(np.int64)
    assert pr.shape[2] == C and (pr.sum(axis=2) == g.n).all()
    if model in (O.SEIR, O.SWIR):
        assert (np.diff(pr[:, :, 3], axis=1) >= 0).all()          # R never shrinks
        assert (np.diff(pr[:, :, 0], axis=1) <= 0).all()          # S never grows
    a = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=40, T=5, **kw)
    b = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=40, T=7, init_state=a.final_state, t0=5, **kw)
    assert np.array_equal(b.per_real, full.per_real[:, 5:])
    assert np.array_equal(b.final_state, full.final_state)
