"""Input generators: determinism and structural properties (CPU only)."""
import numpy as np

import workloads as W


def _csr_ok(g):
    assert g.row_ptr[0] == 0 and g.row_ptr[-1] == g.nnz
    assert np.all(np.diff(g.row_ptr) >= 0)
    assert g.col_idx.min() >= 0 and g.col_idx.max() < g.n
    for v in range(0, g.n, max(1, g.n // 50)):
        row = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert np.all(np.diff(row) >= 0)


def test_rmat_shape_and_determinism():
    a = W.rmat(12, 8, seed=3, nthreads=3)
    b = W.rmat(12, 8, seed=3, nthreads=5)
    assert a.n == 4096 and a.nnz == 8 * 4096
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    _csr_ok(a)
    # skew: node 0 (all-zero bits) gets ~ E * (a+c)^scale arcs
    expect = a.nnz * 0.76 ** 12
    assert 0.5 * expect < a.in_degree()[0] < 2 * expect
    c = W.rmat(12, 8, seed=4)
    assert not np.array_equal(a.col_idx, c.col_idx)


def test_ba_symmetric_degrees():
    g = W.ba(2000, 3, seed=1)
    _csr_ok(g)
    assert g.nnz == 2 * (3 * 4 // 2 + (2000 - 4) * 3)
    # symmetric: the arc multiset equals its reverse
    dst = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    fwd = np.sort(g.col_idx.astype(np.int64) * g.n + dst)
    rev = np.sort(dst.astype(np.int64) * g.n + g.col_idx)
    assert np.array_equal(fwd, rev)
    assert g.in_degree().min() >= 3
    assert np.array_equal(W.ba(2000, 3, seed=1).col_idx, g.col_idx)


def test_er_simple_symmetric():
    g = W.er(3000, 6.0, seed=2)
    _csr_ok(g)
    dst = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    assert np.all(dst != g.col_idx)
    keys = g.col_idx.astype(np.int64) * g.n + dst
    assert np.unique(keys).size == keys.size
    assert abs(g.nnz / g.n - 6.0) < 0.5
    big = W.er(200_000, 4.0, seed=2)
    _csr_ok(big)
    assert big.nnz == 2 * int(4.0 * 200_000 / 2 + 0.5)


def test_seed_sets():
    s = W.seed_set(1000, 100, seed=5)
    assert s.size == 100 and np.unique(s).size == 100
    assert s.min() >= 0 and s.max() < 1000
    assert np.array_equal(s, W.seed_set(1000, 100, seed=5))
    assert not np.array_equal(s, W.seed_set(1000, 100, seed=6))


def test_surrogate_pool_and_candidates_are_seeded_and_shaped():
    import numpy as np
    import workloads as W
    gs = W.surrogate_pool(4, n_min=2000, n_max=4000, threads=2)
    gs2 = W.surrogate_pool(4, n_min=2000, n_max=4000, threads=1)
    for a, b in zip(gs, gs2):          # a pure function of the seed, not of the thread count
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    assert gs[0].name.startswith("ba") and gs[1].name.startswith("rmat")
    assert 2000 <= gs[0].n <= 4000 and gs[1].n in (1 << 17, 1 << 18, 1 << 19)
    sets = W.surrogate_sets(gs[0], 0)
    assert len(sets) == 8 and all(len(s) == 20 and 0.01 <= b <= 0.1 for s, b in sets)
    c = W.surrogate_candidates(gs[0], 50, 20, seed=3)
    assert c.shape == (50, 20) and c.dtype == np.int32
    assert c.min() >= 0 and c.max() < gs[0].n
    assert np.array_equal(c, W.surrogate_candidates(gs[0], 50, 20, seed=3))
