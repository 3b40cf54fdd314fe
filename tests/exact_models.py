"""Exact distributions of the propagation models on tiny graphs.

These are independent first-principles computations used to pin the Monte Carlo
oracle (they do not call it):

* IC: enumerate all 2^|E| live-edge worlds (Kempe, Kleinberg, Tardos, KDD 2003,
  Claim 2.3): the set activated by step t equals the set within live-path distance t
  of the seeds.
* LT: enumerate the worlds in which every node picks at most one in-arc with
  probability equal to its weight (Kempe et al., Claim 2.6); with weights 1/d_in every
  node of positive in-degree picks exactly one in-arc.
* SIR/SIS: the synchronous chain factorises over nodes given the current state, so
  the exact distribution over 3^N states is propagated step by step.

Probabilities here use the paper's real-valued rules (1-(1-beta)^k, gamma, 1/d), not
the library's 32-bit integer thresholds; the two differ by at most k*2^-32, far below
what a chi-square test at these sample sizes can see.
"""
from __future__ import annotations

import itertools
from collections import defaultdict

import numpy as np
from scipy import stats


def arcs_of(row_ptr, col_idx):
    """List of (src, dst) for the in-CSR."""
    out = []
    for v in range(len(row_ptr) - 1):
        for e in range(row_ptr[v], row_ptr[v + 1]):
            out.append((int(col_idx[e]), v))
    return out


def _layers(n, live_arcs, seeds):
    """BFS layer index of each node (None if unreachable) over live arcs."""
    adj = defaultdict(list)
    for u, v in live_arcs:
        adj[u].append(v)
    dist = [None] * n
    frontier = sorted(set(int(s) for s in seeds))
    for s in frontier:
        dist[s] = 0
    d = 0
    while frontier:
        d += 1
        nxt = []
        for u in frontier:
            for v in adj[u]:
                if dist[v] is None:
                    dist[v] = d
                    nxt.append(v)
        frontier = nxt
    return dist


def ic_layer_distribution(row_ptr, col_idx, seeds, p_of_arc, horizon):
    """Exact distribution of (|F_1|, ..., |F_horizon|, |A_final|) for IC."""
    n = len(row_ptr) - 1
    arcs = arcs_of(row_ptr, col_idx)
    probs = [p_of_arc(u, v) for (u, v) in arcs]
    dist = defaultdict(float)
    for mask in range(1 << len(arcs)):
        pw = 1.0
        live = []
        for i, a in enumerate(arcs):
            if (mask >> i) & 1:
                pw *= probs[i]
                live.append(a)
            else:
                pw *= 1.0 - probs[i]
        if pw == 0.0:
            continue
        d = _layers(n, live, seeds)
        key = tuple(sum(1 for x in d if x == t) for t in range(1, horizon + 1))
        key = key + (sum(1 for x in d if x is not None),)
        dist[key] += pw
    return dict(dist)


def lt_layer_distribution(row_ptr, col_idx, seeds, horizon):
    """Exact distribution of (|F_1|, ..., |F_horizon|, |A_final|) for LT with weights
    1/d_in (every in-arc, counted with multiplicity, is picked with probability 1/d)."""
    n = len(row_ptr) - 1
    choices = []
    for v in range(n):
        b, e = int(row_ptr[v]), int(row_ptr[v + 1])
        if e > b:
            choices.append([(int(col_idx[k]), v, 1.0 / (e - b)) for k in range(b, e)])
    dist = defaultdict(float)
    for pick in itertools.product(*choices):
        pw = 1.0
        live = []
        for (u, v, p) in pick:
            pw *= p
            live.append((u, v))
        d = _layers(n, live, seeds)
        key = tuple(sum(1 for x in d if x == t) for t in range(1, horizon + 1))
        key = key + (sum(1 for x in d if x is not None),)
        dist[key] += pw
    return dict(dist)


def sir_state_distribution(row_ptr, col_idx, seeds, beta, gamma, T, sis=False):
    """Exact distribution of (S, I, R) counts after T synchronous steps."""
    n = len(row_ptr) - 1
    in_nb = [[int(col_idx[e]) for e in range(row_ptr[v], row_ptr[v + 1])] for v in range(n)]
    init = tuple(1 if v in set(int(s) for s in seeds) else 0 for v in range(n))
    cur = {init: 1.0}
    for _ in range(T):
        nxt = defaultdict(float)
        for st, p in cur.items():
            opts = []
            for v in range(n):
                if st[v] == 0:
                    k = sum(1 for u in in_nb[v] if st[u] == 1)
                    pi = 1.0 - (1.0 - beta) ** k if k > 0 else 0.0
                    opts.append([(0, 1.0 - pi), (1, pi)])
                elif st[v] == 1:
                    opts.append([(1, 1.0 - gamma), (0 if sis else 2, gamma)])
                else:
                    opts.append([(2, 1.0)])
            for combo in itertools.product(*opts):
                q = p
                for (_, w) in combo:
                    q *= w
                if q > 0.0:
                    nxt[tuple(s for (s, _) in combo)] += q
        cur = nxt
    out = defaultdict(float)
    for st, p in cur.items():
        out[(st.count(0), st.count(1), st.count(2))] += p
    return dict(out)


def chi_square_gof(observed: dict, expected_prob: dict, n_samples: int, alpha=1e-3):
    """Pearson chi-square; bins with expected count < 5 are pooled into one bin.
    Returns (stat, threshold, df).  Every observed key must be possible."""
    for k in observed:
        assert k in expected_prob and expected_prob[k] > 0, f"impossible outcome {k}"
    keys = sorted(expected_prob)
    big = [k for k in keys if expected_prob[k] * n_samples >= 5]
    small = [k for k in keys if expected_prob[k] * n_samples < 5]
    obs, exp = [], []
    for k in big:
        obs.append(observed.get(k, 0))
        exp.append(expected_prob[k] * n_samples)
    if small:
        obs.append(sum(observed.get(k, 0) for k in small))
        exp.append(sum(expected_prob[k] for k in small) * n_samples)
    obs = np.array(obs, dtype=float)
    exp = np.array(exp, dtype=float)
    stat = float(((obs - exp) ** 2 / exp).sum())
    df = max(1, len(obs) - 1)
    return stat, float(stats.chi2.ppf(1 - alpha, df)), df


def chain_state_distribution(row_ptr, col_idx, init, T, transitions, n_states):
    """Exact distribution of the compartment counts after T synchronous steps of a model
    whose per-node transition depends only on the node's state and on k, the number of
    its in-arcs (with multiplicity) whose source is infectious.  transitions(state, k)
    returns [(new_state, probability), ...]; init is the tuple of start states; the
    infectious state is given by transitions.infectious."""
    n = len(row_ptr) - 1
    in_nb = [[int(col_idx[e]) for e in range(row_ptr[v], row_ptr[v + 1])] for v in range(n)]
    inf = transitions.infectious
    cur = {tuple(init): 1.0}
    for _ in range(T):
        nxt = defaultdict(float)
        for st, p in cur.items():
            opts = []
            for v in range(n):
                k = sum(1 for u in in_nb[v] if st[u] == inf)
                opts.append([o for o in transitions(st[v], k) if o[1] > 0.0])
            for combo in itertools.product(*opts):
                q = p
                for (_, w) in combo:
                    q *= w
                if q > 0.0:
                    nxt[tuple(s for (s, _) in combo)] += q
        cur = nxt
    out = defaultdict(float)
    for st, p in cur.items():
        out[tuple(st.count(c) for c in range(n_states))] += p
    return dict(out)


class SeirRule:
    """SEIR / SEIS (discrete time): S -> E with 1-(1-beta)^k, E -> I with alpha, I -> R
    (SEIS: S) with gamma.  States 0 S, 1 E, 2 I, 3 R."""
    infectious = 2

    def __init__(self, beta, alpha, gamma, sis=False):
        self.b, self.a, self.g, self.sis = beta, alpha, gamma, sis

    def __call__(self, s, k):
        if s == 0:
            p = 1.0 - (1.0 - self.b) ** k if k > 0 else 0.0
            return [(1, p), (0, 1.0 - p)]
        if s == 1:
            return [(2, self.a), (1, 1.0 - self.a)]
        if s == 2:
            return [(0 if self.sis else 3, self.g), (2, 1.0 - self.g)]
        return [(3, 1.0)]


class SwirRule:
    """SWIR: S -> I with 1-(1-kappa)^k, else S -> W with 1-(1-mu)^k; W -> I with
    1-(1-nu)^k; I -> R after one step.  States 0 S, 1 W, 2 I, 3 R."""
    infectious = 2

    def __init__(self, kappa, mu, nu):
        self.k, self.m, self.n = kappa, mu, nu

    def __call__(self, s, k):
        def p_of(x):
            return 1.0 - (1.0 - x) ** k if k > 0 else 0.0
        if s == 0:
            pi, pw = p_of(self.k), p_of(self.m)
            return [(2, pi), (1, (1.0 - pi) * pw), (0, (1.0 - pi) * (1.0 - pw))]
        if s == 1:
            pi = p_of(self.n)
            return [(2, pi), (1, 1.0 - pi)]
        return [(3, 1.0)]
