"""fsgp_step_noalloc: the step for callers that cannot allocate device memory.

A serving process that has handed its free device memory to its own pool, or a runtime
that forbids allocation on its hot path, cannot call cudaMalloc; fsgp_step_noalloc
serves them with a fixed scratch array inside the library.  Its output must equal that
of the ordinary entry point (fsgp_simulate run for one step from the same planes), bit
for bit, on two calls in a row (the second call reuses the scratch the first one left
behind).  Lane widths cover one padded word (R = 20), padded words within a power-of-two
set (R = 96: 3 words used of 4) and full words (R = 256); one SIR case has a survival
table that reaches zero below the graph's largest in-degree (beta = 0.9), so lanes at
and above K_sat are decided without draws.  Collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _popcounts(planes):
    bits = np.unpackbits(planes.view(np.uint8), axis=None)
    P = planes.shape[0]
    per = bits.reshape(P, -1).sum(axis=1)
    return [int(x) for x in per] + [0] * (2 - P)


def _pad_words(planes, Ws):
    """[P][n][W] -> [P][n][Ws] with zero padding words (the entry point's layout)."""
    import torch
    P, n, W = planes.shape
    if W == Ws:
        return planes.contiguous()
    out = torch.zeros((P, n, Ws), dtype=planes.dtype, device=planes.device)
    out[:, :, :W] = planes
    return out


CASES = [(m, R, None) for m in (0, 1, 2, 3) for R in (20, 96, 256)] + [(0, 256, 0.9)]


@pytest.mark.parametrize("model,R,beta", CASES)
def test_step_noalloc_matches_simulate(cuda_lib, model, R, beta):
    import torch
    f = cuda_lib
    # R-MAT scale 14: rows up to ~5,000 in-arcs, so long rows span several CTA chunks
    g = W.rmat(14, 16, seed=201)
    seeds = W.seed_set(g.n, 40, seed=202)
    t0 = 4
    Wd = (R + 31) // 32
    Ws = 1 << (Wd - 1).bit_length()
    if model in (0, 1):
        prm = dict(beta=0.2 if beta is None else beta, gamma=0.1)
    else:
        prm = dict()
    if beta is not None:
        from oracle import survival_table
        ksat = int(np.argmax(survival_table(beta, 64) == 0))
        assert 0 < ksat < int(np.diff(g.row_ptr).max())
    graph = f.Graph(g.row_ptr, g.col_idx)
    start = f.simulate(graph, model, [seeds], R, t0, 17, final_planes=True, **prm)
    cur = _pad_words(start["final_planes"][0], Ws)       # [P][n][Ws]
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    params = f.fsgp_params(beta=prm.get("beta", 0.0), gamma=prm.get("gamma", 0.0),
                           ic_mode=f.IC_WEIGHTED_CASCADE, ic_p=0.0)
    ref_planes = start["final_planes"][0].contiguous()   # [P][n][W]
    for call in range(2):
        t = t0 + 1 + call
        nxt = torch.full_like(cur, -1)                   # garbage the step must overwrite
        counts = torch.zeros(2, dtype=torch.int64, device="cuda")
        f.fsgp_step_noalloc(model, params, rp, ci, g.n, g.nnz, R, t, 17, cur, nxt, counts)
        ref = f.simulate(graph, model, [np.zeros(0, np.int32)], R, 1, 17, final_planes=True,
                         options=dict(t0=t - 1, init_planes=ref_planes), **prm)
        torch.cuda.synchronize()
        got = nxt.cpu().numpy().view(np.uint32)
        want = ref["final_planes"][0].cpu().numpy().view(np.uint32)
        assert np.array_equal(got[:, :, :Wd], want), (model, R, call)
        assert not got[:, :, Wd:].any(), (model, R, call)     # padding words stay zero
        assert counts.cpu().tolist() == _popcounts(want), (model, R, call)
        cur, ref_planes = nxt, ref["final_planes"][0].contiguous()
    graph.close()


def test_step_noalloc_rejects_oversized(cuda_lib):
    import torch
    f = cuda_lib
    n = 300_000                      # 300k rows x 1 KiB of per-lane counts > 32 MiB
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    planes = torch.zeros((2, n, 8), dtype=torch.int32, device="cuda")
    out = torch.empty_like(planes)
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    params = f.fsgp_params(beta=0.1, gamma=0.1, ic_mode=0, ic_p=0.0)
    with pytest.raises(f.FsgpError, match="too large"):
        f.fsgp_step_noalloc(0, params, rp, None, n, 0, 256, 1, 1, planes, out, counts)
