"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something it does not compute itself: a library
routine (cuRAND's host Philox generator, scipy's graph BFS, sparse mat-vec), an exact
rational bound, a closed-form probability, or an exact enumeration (exact_models).
"""
import ctypes
import ctypes.util
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import sparse, stats
from scipy.sparse import csgraph

import oracle as O
import workloads as W
from tests import exact_models as X

TWO32 = 1 << 32


# ----------------------------------------------------------------------------- Philox

def _curand_host():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) if cand.startswith("/") else cand:
            try:
                return ctypes.CDLL(cand)
            except OSError:
                continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host-side PHILOX4_32_10 generator emits block i of its stream as
    Philox4x32-10(counter=(0,0,i,0), key=(lo32(seed), hi32(seed))).  The oracle's own
    Philox (written from Salmon et al., SC'11) must reproduce those blocks."""
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not found")
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161  # curand.h enum value
    for seed in (0, 1, 0x0123456789ABCDEF, 0xFEDCBA9876543210, 2**63 + 12345):
        gen = ctypes.c_void_p()
        assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        nblk = 64
        buf = (ctypes.c_uint * (4 * nblk))()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(4 * nblk)) == 0
        lib.curandDestroyGenerator(gen)
        ref = np.frombuffer(buf, dtype=np.uint32).reshape(nblk, 4)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i in range(nblk):
            got = O.philox4x32_10([0, 0, i, 0], key)
            assert np.array_equal(got, ref[i]), (seed, i, got, ref[i])


def test_uniform_is_uniform_and_lane_independent():
    """u(tag, a, t, r) over many subjects: 16-bin chi-square for uniformity, and the
    bits of neighbouring lanes r, r+1 (same Philox words) are uncorrelated."""
    us = np.array([O.uniform(7, 1, a, 3, r) for a in range(64) for r in range(64)], dtype=np.uint64)
    hist = np.bincount((us >> 28).astype(np.int64), minlength=16)
    chi = ((hist - us.size / 16) ** 2 / (us.size / 16)).sum()
    assert chi < stats.chi2.ppf(0.999, 15)
    u2 = us.reshape(64, 64)
    a = (u2[:, 0::2] >> 31).astype(float).ravel()
    b = (u2[:, 1::2] >> 31).astype(float).ravel()
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.1
    # different tags and steps give different streams
    assert O.uniform(7, 1, 5, 3, 9) != O.uniform(7, 2, 5, 3, 9)
    assert O.uniform(7, 1, 5, 3, 9) != O.uniform(7, 1, 5, 4, 9)
    assert O.uniform(7, 1, 5, 3, 9) != O.uniform(8, 1, 5, 3, 9)


# --------------------------------------------------------------------- survival table

@pytest.mark.parametrize("beta", [0.0, 1e-6, 0.005, 0.01, 0.05, 0.2, 0.5, 0.999, 1.0])
def test_survival_table_exact_bound(beta):
    """surv[k] is within k units (of 2^-32) below the exact 2^32 (1-b/2^32)^k, with
    b = round(beta 2^32): each of the k floors loses less than one unit."""
    kmax = 600
    surv = O.survival_table(beta, kmax)
    b = int(round(beta * TWO32))
    q = TWO32 - b
    assert int(surv[0]) == TWO32
    qk = 1
    for k in range(1, kmax + 1):
        qk *= q
        exact = Fraction(qk, TWO32 ** (k - 1))   # = 2^32 (q/2^32)^k
        s = int(surv[k])
        assert s <= exact
        assert exact - s <= k
        assert s <= int(surv[k - 1])
    if beta == 0.0:
        assert np.all(surv == TWO32)
    if beta == 1.0:
        assert np.all(surv[1:] == 0)


def test_survival_probability_close_to_paper_rule():
    """1 - surv[k]/2^32 approximates the paper's 1-(1-beta)^k within k 2^-32 + rounding
    of beta (Appendix A.1, infection probability m_i)."""
    for beta in (0.01, 0.05, 0.3):
        surv = O.survival_table(beta, 300)
        for k in range(1, 301):
            p_int = 1.0 - int(surv[k]) / TWO32
            p_paper = 1.0 - (1.0 - beta) ** k
            assert abs(p_int - p_paper) <= (k + 1) * 2.0 ** -31


# ------------------------------------------------------------------ deterministic pins

def _bfs_dist(g, seeds):
    """Forward BFS distance from the seed set (scipy), arcs u -> v from the in-CSR."""
    n = g.n
    indptr, indices = g.row_ptr, g.col_idx
    # in-CSR row v holds sources u: matrix M[v, u]; forward adjacency is M^T
    M = sparse.csr_matrix((np.ones(len(indices)), indices, indptr), shape=(n, n))
    F = M.T.tocsr()
    # super-source BFS: distance to nearest seed
    d = csgraph.shortest_path(F, method="D", unweighted=True, indices=np.unique(seeds))
    return np.min(np.atleast_2d(d), axis=0)


def _graphs():
    yield W.er(300, 4.0, seed=5)
    yield W.ba(400, 2, seed=6)
    yield W.rmat(9, 4, seed=7)


@pytest.mark.parametrize("gi", range(3))
def test_sir_beta1_reproduces_bfs_layers(gi):
    """beta=1, gamma=1: every S node with an infected in-neighbour is infected and
    every I node recovers, so I_t is exactly BFS layer t and R_t the layers < t."""
    g = list(_graphs())[gi]
    seeds = W.seed_set(g.n, 3, seed=11 + gi)
    T = 12
    res = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, beta=1.0, gamma=1.0, R=37, T=T,
                     rng_seed=99)
    dist = _bfs_dist(g, seeds)
    for t in range(T + 1):
        n_layer = int(np.sum(dist == t))
        n_before = int(np.sum(dist < t))
        assert np.all(res.per_real[:, t, 1] == n_layer), t
        assert np.all(res.per_real[:, t, 2] == n_before), t


@pytest.mark.parametrize("gi", range(3))
def test_si_limit_gamma0(gi):
    """beta=1, gamma=0 (SI): I_t = nodes within distance t, R = 0."""
    g = list(_graphs())[gi]
    seeds = W.seed_set(g.n, 2, seed=21 + gi)
    res = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, beta=1.0, gamma=0.0, R=5, T=8,
                     rng_seed=3)
    dist = _bfs_dist(g, seeds)
    for t in range(9):
        assert np.all(res.per_real[:, t, 1] == int(np.sum(dist <= t)))
        assert np.all(res.per_real[:, t, 2] == 0)


@pytest.mark.parametrize("gi", range(3))
def test_ic_p1_is_reachability(gi):
    """IC with constant p=1: F_t = BFS layer t, final active set = reachable set, and
    the run stops at the first empty frontier."""
    g = list(_graphs())[gi]
    seeds = W.seed_set(g.n, 2, seed=31 + gi)
    T = 40
    res = O.simulate(O.IC, g.row_ptr, g.col_idx, seeds, ic_mode=O.IC_CONSTANT, ic_p=1.0,
                     R=4, T=T, rng_seed=5)
    dist = _bfs_dist(g, seeds)
    reach = np.isfinite(dist)
    maxd = int(dist[reach].max())
    for t in range(1, T + 1):
        assert np.all(res.per_real[:, t, 1] == int(np.sum(dist == t)))
    assert np.all(res.final_state[:, reach] != 0)
    assert np.all(res.final_state[:, ~reach] == 0)
    assert np.all(res.quiet_step == maxd + 1)


def test_lt_in_degree_one_is_bfs():
    """LT on a graph where every node has in-degree <= 1: an inactive node with its
    single in-neighbour active has k = d = 1 and activates surely, so LT = BFS."""
    n = 200
    rng = np.random.default_rng(1)
    parent = [-1] + [int(rng.integers(0, v)) for v in range(1, n)]
    src = [parent[v] for v in range(1, n)]
    dst = list(range(1, n))
    g = W.from_arcs(n, src, dst)
    seeds = np.array([0, 5], dtype=np.int32)
    res = O.simulate(O.LT, g.row_ptr, g.col_idx, seeds, R=3, T=60, rng_seed=4)
    dist = _bfs_dist(g, seeds)
    for t in range(1, 61):
        assert np.all(res.per_real[:, t, 1] == int(np.sum(dist == t)))


def test_sis_deterministic_limit_matches_sparse_matvec():
    """SIS with beta=1, gamma=1: I_t = {v not in I_{t-1} with an in-neighbour in
    I_{t-1}}, computed independently with a sparse mat-vec."""
    g = W.er(250, 3.0, seed=8)
    n = g.n
    M = sparse.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(n, n))
    seeds = W.seed_set(n, 4, seed=9)
    I = np.zeros(n, dtype=bool)
    I[seeds] = True
    T = 15
    res = O.simulate(O.SIS, g.row_ptr, g.col_idx, seeds, beta=1.0, gamma=1.0, R=3, T=T,
                     rng_seed=2)
    for t in range(1, T + 1):
        I = (M @ I.astype(float) > 0) & ~I
        assert np.all(res.per_real[:, t, 1] == int(I.sum())), t
        assert np.all(res.per_real[:, t, 2] == 0)


# ------------------------------------------------------------------ invariants, means

@pytest.mark.parametrize("model", [O.SIR, O.SIS, O.IC, O.LT])
def test_invariants(model):
    g = W.rmat(10, 6, seed=12)
    seeds = W.seed_set(g.n, 10, seed=13)
    T = 25
    res = O.simulate(model, g.row_ptr, g.col_idx, seeds, beta=0.1, gamma=0.2, R=40, T=T,
                     rng_seed=77)
    pr = res.per_real.astype(np.int64)
    assert np.all(pr.sum(axis=2) == g.n)
    assert np.array_equal(res.counts.astype(np.int64), pr.sum(axis=0))
    if model == O.SIR:
        assert np.all(np.diff(pr[:, :, 2], axis=1) >= 0)
        assert np.all(np.diff(pr[:, :, 0], axis=1) <= 0)
    if model == O.SIS:
        assert np.all(pr[:, :, 2] == 0)
    if model in (O.IC, O.LT):
        active = pr[:, :, 1] + pr[:, :, 2]
        assert np.all(np.diff(active, axis=1) >= 0)
        # frontier at t = newly active at t
        assert np.all(np.diff(active, axis=1) == pr[:, 1:, 1])
    fs = res.final_state
    for c in range(3):
        assert np.array_equal(res.freq[c], (fs == c).sum(axis=0))


def test_beta0_recovery_is_geometric():
    """beta=0: only recovery acts; each seed stays infected a geometric time, so
    E[I_t] = I_0 (1-gamma)^t (z-test over many realizations)."""
    g = W.er(500, 4.0, seed=14)
    seeds = W.seed_set(g.n, 50, seed=15)
    gamma, T, R = 0.2, 6, 2000
    res = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, beta=0.0, gamma=gamma, R=R, T=T,
                     rng_seed=16)
    for t in range(T + 1):
        p = (1 - gamma) ** t
        mean = res.counts[t, 1] / R
        sd = np.sqrt(50 * p * (1 - p) / R)
        assert abs(mean - 50 * p) <= 5 * sd + 1e-9
        assert np.all(res.per_real[:, t, 1] + res.per_real[:, t, 2] == 50)


def test_lt_star_exact_probability():
    """Centre with d in-arcs, k of them from seeds: the integer rule activates it at
    t=1 with probability (floor(k 2^32/d)+1)/2^32; checked with a binomial z-test."""
    d, k = 7, 3
    src = list(range(1, d + 1))
    g = W.from_arcs(d + 1, src, [0] * d)
    seeds = np.arange(1, k + 1, dtype=np.int32)
    R = 20000
    res = O.simulate(O.LT, g.row_ptr, g.col_idx, seeds, R=R, T=1, rng_seed=21)
    p = ((k * TWO32) // d + 1) / TWO32
    hits = int(res.freq[1][0])
    assert abs(hits - R * p) <= 5 * np.sqrt(R * p * (1 - p))


def test_ic_star_weighted_cascade_probability():
    d = 5
    g = W.from_arcs(d + 1, list(range(1, d + 1)), [0] * d)
    seeds = np.arange(1, d + 1, dtype=np.int32)
    R = 20000
    res = O.simulate(O.IC, g.row_ptr, g.col_idx, seeds, R=R, T=1, rng_seed=22)
    pe = ((TWO32 - 1) // d + 1) / TWO32
    p = 1 - (1 - pe) ** d
    hits = int(res.freq[1][0])
    assert abs(hits - R * p) <= 5 * np.sqrt(R * p * (1 - p))


# ------------------------------------------------------------ exact distributions

def _tiny_graph():
    # 6 nodes, 11 arcs, one duplicated arc (2->3 twice) and a 2-cycle
    arcs = [(0, 1), (0, 2), (1, 2), (2, 3), (2, 3), (1, 3), (3, 4), (4, 5), (2, 5), (5, 1), (1, 5)]
    src, dst = zip(*arcs)
    return W.from_arcs(6, src, dst)


def _mc_keys_layers(res, horizon):
    keys = {}
    pr = res.per_real
    T = pr.shape[1] - 1
    for r in range(pr.shape[0]):
        key = tuple(int(pr[r, t, 1]) for t in range(1, horizon + 1))
        key = key + (int(pr[r, T, 1] + pr[r, T, 2]),)
        keys[key] = keys.get(key, 0) + 1
    return keys


def test_ic_exact_distribution_chi_square():
    g = _tiny_graph()
    seeds = np.array([0], dtype=np.int32)
    deg = g.in_degree()
    exact = X.ic_layer_distribution(g.row_ptr, g.col_idx, seeds,
                                    lambda u, v: 1.0 / deg[v], horizon=3)
    R = 1 << 14
    res = O.simulate(O.IC, g.row_ptr, g.col_idx, seeds, R=R, T=10, rng_seed=31)
    stat, thr, df = X.chi_square_gof(_mc_keys_layers(res, 3), exact, R)
    assert stat < thr, (stat, thr, df)


def test_ic_constant_p_exact_distribution_chi_square():
    g = _tiny_graph()
    seeds = np.array([0, 4], dtype=np.int32)
    exact = X.ic_layer_distribution(g.row_ptr, g.col_idx, seeds, lambda u, v: 0.35, horizon=2)
    R = 1 << 14
    res = O.simulate(O.IC, g.row_ptr, g.col_idx, seeds, ic_mode=O.IC_CONSTANT, ic_p=0.35,
                     R=R, T=10, rng_seed=32)
    stat, thr, df = X.chi_square_gof(_mc_keys_layers(res, 2), exact, R)
    assert stat < thr, (stat, thr, df)


def test_lt_exact_distribution_chi_square():
    g = _tiny_graph()
    seeds = np.array([0], dtype=np.int32)
    exact = X.lt_layer_distribution(g.row_ptr, g.col_idx, seeds, horizon=3)
    R = 1 << 14
    res = O.simulate(O.LT, g.row_ptr, g.col_idx, seeds, R=R, T=10, rng_seed=33)
    stat, thr, df = X.chi_square_gof(_mc_keys_layers(res, 3), exact, R)
    assert stat < thr, (stat, thr, df)


@pytest.mark.parametrize("sis", [False, True])
def test_sir_sis_exact_markov_chain_chi_square(sis):
    arcs = [(0, 1), (1, 0), (1, 2), (2, 1), (2, 3), (3, 2), (0, 3), (3, 4), (4, 3), (4, 4)]
    src, dst = zip(*arcs)
    g = W.from_arcs(5, src, dst)
    seeds = np.array([0], dtype=np.int32)
    beta, gamma, T = 0.45, 0.3, 4
    exact = X.sir_state_distribution(g.row_ptr, g.col_idx, seeds, beta, gamma, T, sis=sis)
    R = 1 << 14
    res = O.simulate(O.SIS if sis else O.SIR, g.row_ptr, g.col_idx, seeds, beta=beta,
                     gamma=gamma, R=R, T=T, rng_seed=34)
    obs = {}
    for r in range(R):
        key = tuple(int(x) for x in res.per_real[r, T])
        obs[key] = obs.get(key, 0) + 1
    stat, thr, df = X.chi_square_gof(obs, exact, R)
    assert stat < thr, (stat, thr, df)


# ------------------------------------------------------------- oracle self-consistency

@pytest.mark.parametrize("model", [O.SIR, O.IC, O.LT, O.SIS])
def test_resume_equals_uninterrupted(model):
    g = W.ba(300, 3, seed=41)
    seeds = W.seed_set(g.n, 5, seed=42)
    kw = dict(beta=0.2, gamma=0.1, R=33, rng_seed=43)
    full = O.simulate(model, g.row_ptr, g.col_idx, seeds, T=12, **kw)
    a = O.simulate(model, g.row_ptr, g.col_idx, seeds, T=5, **kw)
    b = O.simulate(model, g.row_ptr, g.col_idx, seeds, T=7, init_state=a.final_state, t0=5, **kw)
    assert np.array_equal(full.per_real[:, 5:], b.per_real)
    assert np.array_equal(full.final_state, b.final_state)


def test_realization_subset_matches_full_run():
    g = W.er(400, 5.0, seed=44)
    seeds = W.seed_set(g.n, 4, seed=45)
    kw = dict(beta=0.15, gamma=0.1, R=100, T=10, rng_seed=46)
    full = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, **kw)
    sub = O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, r_lo=37, n_real=20, **kw)
    assert np.array_equal(full.per_real[37:57], sub.per_real)


def test_node_step_agrees_with_simulate():
    g = W.er(200, 6.0, seed=47)
    seeds = W.seed_set(g.n, 5, seed=48)
    for model in (O.SIR, O.SIS, O.IC, O.LT):
        kw = dict(beta=0.3, gamma=0.2)
        a = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=4, T=3, rng_seed=49, **kw)
        b = O.simulate(model, g.row_ptr, g.col_idx, seeds, R=4, T=4, rng_seed=49, **kw)
        for r in range(4):
            for v in range(0, g.n, 7):
                s = O.node_step(model, g.row_ptr, g.col_idx, v, a.final_state[r], t=4, r=r,
                                rng_seed=49, **kw)
                if model in (O.IC, O.LT) and a.quiet_step[r] < 4:
                    continue
                assert s == b.final_state[r, v]
