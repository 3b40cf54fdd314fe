"""Realization sharding over ranks (one process per GPU).

Realizations are independent, and every random draw is keyed by the global realization
index (the lane), so ranks that run disjoint lane ranges of one job reproduce, lane for
lane, what one GPU running every lane computes.  The state never crosses ranks: the only
exchange is one sum of the result arrays when the run ends (Sec. 3.1 batches
realizations; this splits that batch dimension across devices instead of partitioning
the graph, which a graph that fits one GPU does not need).

Host logic only; the simulation itself is `fsgp.simulate` with `r_offset`.
"""
from __future__ import annotations

LANE_GROUP = 32


def lane_shard(R_total: int, world: int, rank: int, align: int = LANE_GROUP) -> tuple[int, int]:
    """(r_offset, R_local) of `rank`: contiguous runs of whole `align`-lane groups, the
    first ranks taking one group more when the groups do not divide evenly.  Only the
    job's last group may be ragged.  A rank may get no lanes (R_local = 0)."""
    if R_total < 0 or world < 1 or not 0 <= rank < world or align < 1:
        raise ValueError("bad shard request")
    groups = (R_total + align - 1) // align
    base, extra = divmod(groups, world)
    g0 = rank * base + min(rank, extra)
    g1 = g0 + base + (1 if rank < extra else 0)
    r0 = min(g0 * align, R_total)
    r1 = min(g1 * align, R_total)
    return r0, r1 - r0


def merge_results(result: dict, R_total: int, world: int, rank: int, group=None) -> dict:
    """Combine one rank's results into the job's, on every rank.

    counts and freq are sums over lanes, so they add; steps_run takes the maximum (a
    rank whose lanes went quiet earlier repeats its last row, which the sum keeps
    right); per_real (one row per lane) is assembled in lane order.  Tensors must live
    where the process group's backend can reduce them (CPU for gloo, CUDA for nccl)."""
    import torch
    import torch.distributed as dist
    out = {}
    if "counts" in result:
        c = result["counts"].to(torch.int64).clone()
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
        out["counts"] = c
    if "freq" in result:
        f = result["freq"].to(torch.int64).clone()
        dist.all_reduce(f, op=dist.ReduceOp.SUM, group=group)
        out["freq"] = f
    if "steps_run" in result:
        s = result["steps_run"].to(torch.int32).clone()
        dist.all_reduce(s, op=dist.ReduceOp.MAX, group=group)
        out["steps_run"] = s
    if "per_real" in result:
        pr = result["per_real"]
        n_sets, _, tp1, three = pr.shape
        full = torch.zeros((n_sets, R_total, tp1, three), dtype=torch.int64, device=pr.device)
        r0, rl = lane_shard(R_total, world, rank)
        full[:, r0:r0 + rl] = pr[:, :rl].to(torch.int64)
        dist.all_reduce(full, op=dist.ReduceOp.SUM, group=group)   # disjoint lanes: sum = gather
        out["per_real"] = full
    return out


def run_sharded(graph, model: int, seed_sets, R_total: int, T: int, rng_seed: int, *,
                world: int, rank: int, group=None, per_real: bool = False, **params) -> dict:
    """Run this rank's lanes of an R_total-realization job on the current GPU and merge
    the job's results on every rank (one all-reduce per result array at the end)."""
    import torch
    from . import fsgp
    r0, rl = lane_shard(R_total, world, rank)
    n_sets = 1 if (hasattr(seed_sets, "ndim") and seed_sets.ndim == 1) else len(seed_sets)
    dev = torch.device("cuda", torch.cuda.current_device())
    opts = params.pop("options", None)
    if rl > 0:
        if opts is None or isinstance(opts, dict):
            opts = dict(opts or {}, r_offset=r0)
        else:
            opts.r_offset = r0
        res = fsgp.simulate(graph, model, seed_sets, rl, T, rng_seed, freq=True, per_real=per_real,
                            steps_run=True, device=True, options=opts, **params)
    else:
        res = {"counts": torch.zeros((n_sets, T + 1, 3), dtype=torch.int64, device=dev),
               "freq": torch.zeros((n_sets, 3, graph.n), dtype=torch.int32, device=dev),
               "steps_run": torch.zeros((n_sets,), dtype=torch.int32, device=dev)}
        if per_real:
            res["per_real"] = torch.zeros((n_sets, 0, T + 1, 3), dtype=torch.int32, device=dev)
    keep = {k: res[k] for k in ("counts", "freq", "steps_run", "per_real") if k in res}
    return merge_results(keep, R_total, world, rank, group=group)
