"""fsgp_step_noalloc: the step for callers that cannot allocate device memory.

Callers inside a stream capture, or whose device memory is fully budgeted, cannot call
cudaMalloc; fsgp_step_noalloc serves them with a fixed scratch array inside the
library.  Its output must equal that of the ordinary entry point (fsgp_simulate run
for one step from the same planes), bit for bit, on two calls in a row (the second call
reuses the scratch the first one left behind).  Collected last on purpose.
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


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_step_noalloc_matches_simulate(cuda_lib, model):
    import torch
    f = cuda_lib
    # R-MAT scale 14: rows up to ~5,000 in-arcs, so long rows span several CTA chunks
    g = W.rmat(14, 16, seed=201)
    seeds = W.seed_set(g.n, 40, seed=202)
    R, t0 = 256, 4
    prm = dict(beta=0.2, gamma=0.1) if model in (0, 1) else dict()
    graph = f.Graph(g.row_ptr, g.col_idx)
    start = f.simulate(graph, model, [seeds], R, t0, 17, final_planes=True, **prm)
    cur = start["final_planes"][0].contiguous()          # [P][n][8], 8 words = 2^3
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    params = f.fsgp_params(beta=prm.get("beta", 0.0), gamma=prm.get("gamma", 0.0),
                           ic_mode=f.IC_WEIGHTED_CASCADE, ic_p=0.0)
    ref_planes = cur
    for call in range(2):
        t = t0 + 1 + call
        nxt = torch.empty_like(cur)
        counts = torch.zeros(2, dtype=torch.int64, device="cuda")
        f.fsgp_step_noalloc(model, params, rp, ci, g.n, g.nnz, R, t, 17, cur, nxt, counts)
        ref = f.simulate(graph, model, [np.zeros(0, np.int32)], R, 1, 17, final_planes=True,
                         options=dict(t0=t - 1, init_planes=ref_planes), **prm)
        torch.cuda.synchronize()
        got = nxt.cpu().numpy().view(np.uint32)
        want = ref["final_planes"][0].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), (model, call)
        assert counts.cpu().tolist() == _popcounts(want), (model, call)
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
