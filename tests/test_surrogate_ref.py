"""Pins of the CPU surrogate reference (CPU only): analytic gradients against central
finite differences of the float64 function, closed forms, and the bfloat16 rounding."""
import numpy as np
import pytest

import workloads as W
from oracle import surrogate_ref as S


def _tiny():
    g = W.ba(60, 2, seed=5)
    seeds = np.array([0, 7, 13], dtype=np.int32)
    x = S.features(g.row_ptr, g.col_idx, seeds, 0.07, 0.1)
    y = np.random.default_rng(1).random(g.n)
    return g, x, y


def test_gradient_matches_finite_differences():
    g, x, y = _tiny()
    theta = S.init_params(3)
    loss, grad = S.loss_and_grad(theta, g.row_ptr, g.col_idx, x, y, bf16=False)
    rng = np.random.default_rng(2)
    idx = rng.choice(S.N_PARAMS, 60, replace=False)
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        lp = S.loss_and_grad(tp, g.row_ptr, g.col_idx, x, y, bf16=False)[0]
        lm = S.loss_and_grad(tm, g.row_ptr, g.col_idx, x, y, bf16=False)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, grad[i])


def test_closed_forms():
    g, x, y = _tiny()
    theta = np.zeros(S.N_PARAMS)
    P = S.unflatten(theta)
    P["bo"][0] = 0.3
    theta = S.flatten(P)
    p, _ = S.forward(theta, g.row_ptr, g.col_idx, x, bf16=False)
    assert np.allclose(p, 1 / (1 + np.exp(-0.3)))
    # a node with no in-arcs aggregates zeros
    iso = W.from_arcs(3, [0], [1])
    m = S._mean_agg(iso.row_ptr, iso.col_idx, np.arange(6.0).reshape(3, 2))
    assert np.array_equal(m, np.array([[0, 0], [0, 1], [0, 0]], dtype=float))
    # the adjoint of the mean aggregation: <A h, g> = <h, A^T g>
    rng = np.random.default_rng(4)
    h = rng.random((g.n, 5))
    gg = rng.random((g.n, 5))
    lhs = np.sum(S._mean_agg(g.row_ptr, g.col_idx, h) * gg)
    rhs = np.sum(h * S._mean_agg_T(g.row_ptr, g.col_idx, gg))
    assert abs(lhs - rhs) < 1e-9 * abs(lhs)


def test_seed_in_arc_feature_brute_force():
    """Feature 5 is log(1 + number of in-arcs from seeds), counted arc by arc."""
    g = W.from_arcs(5, [0, 0, 1, 2, 3, 0, 4], [1, 1, 2, 1, 4, 3, 0])
    seeds = np.array([0, 2], dtype=np.int32)
    x = S.features(g.row_ptr, g.col_idx, seeds, 0.1, 0.2)
    want = np.zeros(5)
    for u, v in zip([0, 0, 1, 2, 3, 0, 4], [1, 1, 2, 1, 4, 3, 0]):
        if u in (0, 2):
            want[v] += 1
    assert np.array_equal(want, [0, 3, 0, 1, 0])
    assert np.allclose(x[:, 5], np.log1p(want))
    assert np.array_equal(x[:, 0], [1, 0, 1, 0, 0])
    assert np.allclose(x[:, 3], np.log1p([1, 3, 1, 1, 1]))   # in-degrees
    assert np.allclose(x[:, 4], np.log1p([3, 1, 1, 1, 1]))   # out-degrees
    # a seed listed twice counts twice
    x2 = S.features(g.row_ptr, g.col_idx, np.array([0, 2, 0], dtype=np.int32), 0.1, 0.2)
    assert np.allclose(x2[:, 5], np.log1p([0, 5, 0, 2, 0]))
    assert np.array_equal(x2[:, 0], x[:, 0])


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.001953125, 1.005859375, -2.5, 3.0e-3, 65504.0,
                     1.01171875])
    r = S.bf16_round(vals)
    # bfloat16 keeps 8 significant bits: spacing 2^-7 at 1.0
    assert r[0] == 1.0
    assert r[1] == 1.0                       # 1 + 2^-8: tie, to the even neighbour 1.0
    assert r[2] == 1.0                       # below the half-way point
    assert r[3] == 1.0078125                 # above it
    assert r[7] == 1.015625                  # 1 + 1.5 * 2^-7: tie, to the even 1 + 2^-6
    assert r[6] == 65536.0
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 3.0e-3 * 2 ** -8
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2 ** -8)


def test_adam_first_step_moves_by_lr():
    theta = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    t2, m, v = S.adam_step(theta, g, np.zeros(5), np.zeros(5), 1, lr=0.01)
    nz = g != 0
    assert np.allclose(np.abs(t2[nz]), 0.01, rtol=1e-6)
    assert np.all(np.sign(t2[nz]) == -np.sign(g[nz]))
