"""Hegselmann-Krause opinion dynamics on the GPU (fsgp_hk) equals the oracle bit for bit:
final opinions of every realization and the per-step change counts, for several graphs,
R not a multiple of 32, eps from 0 to wider than every distance, host and device buffers,
exact ties, T = 0, and the rejected inputs."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _h0(R, n, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(R, n)).astype(np.float32)


def _graphs():
    return [W.er(3000, 8.0, seed=901), W.ba(4000, 4, seed=902), W.rmat(12, 8, seed=903)]


@pytest.mark.parametrize("gi", range(3))
@pytest.mark.parametrize("R,eps", [(1, 0.3), (31, 0.2), (32, 0.5), (33, 0.05), (100, 3.0), (64, 0.0)])
def test_hk_matches_oracle(cuda_lib, gi, R, eps):
    f = cuda_lib
    g = _graphs()[gi]
    graph = f.Graph(g.row_ptr, g.col_idx)
    h0 = _h0(R, g.n, 910 + R)
    T = 15
    h, ch = f.hk(graph, h0, T, eps)
    oh, och = O.hk(g.row_ptr, g.col_idx, h0, T=T, eps=eps)
    assert np.array_equal(h.view(np.uint32), oh.view(np.uint32))
    assert np.array_equal(ch.astype(np.uint64), och)


def test_hk_max_realizations(cuda_lib):
    """R = 4096 (128 realization groups, two per warp) on a small graph."""
    f = cuda_lib
    g = W.ba(300, 3, seed=941)
    graph = f.Graph(g.row_ptr, g.col_idx)
    h0 = _h0(4096, g.n, 942)
    h, ch = f.hk(graph, h0, 10, 0.3)
    oh, och = O.hk(g.row_ptr, g.col_idx, h0, T=10, eps=0.3)
    assert np.array_equal(h.view(np.uint32), oh.view(np.uint32))
    assert np.array_equal(ch.astype(np.uint64), och)


def test_hk_device_buffers_and_t0(cuda_lib):
    import torch
    f = cuda_lib
    g = W.ba(2000, 3, seed=921)
    graph = f.Graph(g.row_ptr, g.col_idx)
    h0 = _h0(40, g.n, 922)
    hd, chd = f.hk(graph, torch.from_numpy(h0).cuda(), 12, 0.25)
    torch.cuda.synchronize()
    hh, chh = f.hk(graph, h0, 12, 0.25)
    assert np.array_equal(hd.cpu().numpy().view(np.uint32), hh.view(np.uint32))
    assert np.array_equal(chd.cpu().numpy().astype(np.uint64), chh.astype(np.uint64))
    h, ch = f.hk(graph, h0, 0, 0.25)
    assert np.array_equal(h, h0) and ch.tolist() == [0]


def test_hk_exact_tie_and_multiplicity(cuda_lib):
    f = cuda_lib
    g = W.from_arcs(5, [0, 0, 1, 3], [1, 2, 2, 4])
    graph = f.Graph(g.row_ptr, g.col_idx)
    h0 = np.array([[0.0, 0.5, 0.25, 1.0, 0.5]], np.float32)
    for eps in (0.5, float(np.nextafter(np.float32(0.5), np.float32(1))), 0.25):
        h, ch = f.hk(graph, h0, 3, eps)
        oh, och = O.hk(g.row_ptr, g.col_idx, h0, T=3, eps=eps)
        assert np.array_equal(h.view(np.uint32), oh.view(np.uint32)), eps
        assert np.array_equal(ch.astype(np.uint64), och), eps


def test_hk_rejects_bad_inputs(cuda_lib):
    f = cuda_lib
    g = W.er(100, 3.0, seed=931)
    graph = f.Graph(g.row_ptr, g.col_idx)
    h0 = _h0(3, g.n, 932)
    with pytest.raises(f.FsgpError):
        f.hk(graph, h0, 3, -0.1)
    with pytest.raises(f.FsgpError):
        f.hk(graph, h0, 3, float("nan"))
    bad = h0.copy()
    bad[1, 5] = np.nan
    with pytest.raises(f.FsgpError):
        f.hk(graph, bad, 3, 0.2)
