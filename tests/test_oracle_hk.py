"""Pins of the oracle's Hegselmann-Krause opinion dynamics (Appendix A.2), against what the
definition fixes without the oracle's loop: no update at eps = 0, linear in-neighbour
averaging (DeGroot without self-weight) when eps exceeds every distance, the closed form
on a complete graph, the strict "< eps" reading at an exact tie, multiplicity of
duplicate arcs, separated opinion clusters that never mix, and nodes without in-arcs."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _h0(R, n, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(R, n)).astype(np.float32)


def test_eps_zero_changes_nothing():
    g = W.er(300, 4.0, seed=71)
    h0 = _h0(5, g.n, 72)
    h, ch = O.hk(g.row_ptr, g.col_idx, h0, T=6, eps=0.0)
    assert np.array_equal(h, h0)
    assert (ch == 0).all()


@pytest.mark.parametrize("gi", range(2))
def test_wide_eps_is_linear_in_neighbour_averaging(gi):
    g = [W.er(200, 5.0, seed=73), W.ba(150, 3, seed=74)][gi]
    h0 = _h0(3, g.n, 75)
    T = 8
    h, _ = O.hk(g.row_ptr, g.col_idx, h0, T=T, eps=3.0)    # every distance is < 2
    deg = np.diff(g.row_ptr)
    dst = np.repeat(np.arange(g.n), deg)
    for r in range(3):
        x = h0[r].astype(np.float64)
        for _ in range(T):
            s = np.bincount(dst, weights=x[g.col_idx], minlength=g.n)
            x = np.where(deg > 0, s / np.maximum(deg, 1), x)
        assert np.abs(h[r] - x).max() < 2e-5


def test_complete_graph_closed_form():
    n, T = 7, 6
    src = [u for v in range(n) for u in range(n) if u != v]
    dst = [v for v in range(n) for u in range(n) if u != v]
    g = W.from_arcs(n, src, dst)
    h0 = _h0(2, n, 76)
    h, _ = O.hk(g.row_ptr, g.col_idx, h0, T=T, eps=5.0)
    for r in range(2):
        m = h0[r].astype(np.float64).mean()
        want = m + (-1.0 / (n - 1)) ** T * (h0[r].astype(np.float64) - m)
        assert np.abs(h[r] - want).max() < 1e-5


def test_strict_inequality_at_an_exact_tie():
    g = W.from_arcs(2, [0], [1])
    h0 = np.array([[0.0, 0.5]], np.float32)
    h, ch = O.hk(g.row_ptr, g.col_idx, h0, T=1, eps=0.5)           # |0.5 - 0| == eps: not a neighbour
    assert h[0, 1] == np.float32(0.5) and ch[1] == 0
    h, ch = O.hk(g.row_ptr, g.col_idx, h0, T=1, eps=np.nextafter(np.float32(0.5), np.float32(1)))
    assert h[0, 1] == np.float32(0.0) and ch[1] == 1


def test_duplicate_arcs_count_with_multiplicity_and_sourceless_nodes_stay():
    g = W.from_arcs(4, [0, 0, 1], [2, 2, 2])         # node 3 has no in-arcs
    h0 = np.array([[0.1, 0.4, -0.2, 0.7]], np.float32)
    h, _ = O.hk(g.row_ptr, g.col_idx, h0, T=1, eps=1.5)
    a, b = np.float32(0.1), np.float32(0.4)
    assert h[0, 2] == np.float32((a + a + b) / np.float32(3))
    assert h[0, 3] == np.float32(0.7) and h[0, 0] == np.float32(0.1)


def test_separated_clusters_never_mix():
    g = W.er(400, 6.0, seed=77)
    rng = np.random.default_rng(78)
    grp = rng.random(g.n) < 0.5
    h0 = np.where(grp, rng.uniform(0.0, 0.1, g.n), rng.uniform(0.9, 1.0, g.n)).astype(np.float32)[None]
    h, _ = O.hk(g.row_ptr, g.col_idx, h0, T=20, eps=0.5)
    assert h[0, grp].min() >= 0.0 and h[0, grp].max() <= np.float32(0.1)
    assert h[0, ~grp].min() >= np.float32(0.9) and h[0, ~grp].max() <= 1.0


def test_rejects_bad_inputs():
    g = W.er(20, 2.0, seed=79)
    with pytest.raises(ValueError):
        O.hk(g.row_ptr, g.col_idx, _h0(1, g.n, 1), T=2, eps=-0.1)
    bad = _h0(1, g.n, 2)
    bad[0, 3] = np.inf
    with pytest.raises(ValueError):
        O.hk(g.row_ptr, g.col_idx, bad, T=2, eps=0.3)
