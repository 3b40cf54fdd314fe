#!/usr/bin/env python
"""Benchmark: full Monte Carlo SIR and SIS on the web-scale R-MAT graph.

Workload (one bench step = one full Monte Carlo run of SIR and one of SIS):
  R-MAT scale 26 (67,108,864 nodes), edge factor 16 (1,073,741,824 arcs, duplicates and
  self-loops kept), (a, b, c) = (0.57, 0.19, 0.19); beta = 0.01, gamma = 0.05; 0.01%
  uniformly random seeds (6,710 nodes); R = 256 realizations; T = 100 steps; rng seed 3.
Metric: edge-realization-steps per second (E * R * T per model, summed), whole job.

Timing: W untimed warm-up steps, then K timed steps bracketed by a barrier and
cudaDeviceSynchronize, CUDA events on the launching stream, max over ranks.  The graph
(4.3 GB of arcs) and the state planes (8.6 GB) are far larger than L2, so no flush is
needed.  SM clocks and throttle reasons are sampled with nvidia-smi during the timed
region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fsgp|reference]

With --gpus N > 1 and no torchrun environment (WORLD_SIZE unset), bench.py starts the N
ranks itself (torch.distributed.run on 127.0.0.1, one process per GPU) and exits with
their status; under torchrun it is one of the ranks.  --dry-run checks the launch: every
rank joins the process group (NCCL with GPUs, gloo without), takes its realization shard,
and rank 0 prints the ranks' lane ranges; nothing is simulated.

--impl reference times the CPU oracle (test infrastructure) on a bounded sample of the
same workload: the paper's method has no runnable reference implementation here.
Multi-GPU (torchrun): realization sharding, rank i runs lanes with r_offset = 256 i
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE = 26
R = 256
T = 100
BETA, GAMMA = 0.01, 0.05
RNG_SEED = 3
MODELS = (0, 1)   # SIR, SIS


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ clocks sampler

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------ helpers

def gpu_selector(torch) -> str:
    """nvidia-smi -i argument for the current CUDA device (its UUID when known)."""
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        first = vis.split(",")[torch.cuda.current_device()] if vis else str(torch.cuda.current_device())
        return first

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


PROPAGATION_SOURCES = ("fsgp_internal.cuh", "step.cuh", "rows.cuh", "model_sir.cu", "model_sis.cu",
                       "model_ic.cu", "model_lt.cu", "simulate.cu", "graph.cu")


def kernel_source_hash() -> str:
    """Hash of the sources of the propagation kernels (the ones the traffic figures cover)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_14895_gb300", "csrc")
    for f in PROPAGATION_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic_ratios():
    """DRAM bytes over algorithmic bytes per kernel kind and model, from the committed
    summary of small ncu captures (one kernel, one mid-run step, R-MAT scale 23), or None
    if absent or taken on different kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic_step_rmat23.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    return {m: {k: float(v["dram_over_alg"]) for k, v in kinds.items()}
            for m, kinds in d.get("models", {}).items()}


def build_workload(scale: int):
    import workloads as W
    t0 = time.time()
    g = W.rmat26_graph(scale)
    wl = W.rmat26(W.SIR, g, scale)
    log(f"[bench] graph R-MAT scale {scale}: n={g.n} nnz={g.nnz} in {time.time() - t0:.1f}s")
    return g, wl.seed_sets[0]


# -------------------------------------------------------------------- reference arm

def run_reference(args, g, seeds, rank):
    """The CPU oracle on a bounded sample of the workload: n_real realizations of SIR
    for T_s steps on the full graph, one realization per host core."""
    import oracle as O
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    n_real = cores
    T_s = 1

    def one_step():
        t = time.perf_counter()
        O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, beta=BETA, gamma=GAMMA, R=R, T=T_s,
                   rng_seed=RNG_SEED, r_lo=0, n_real=n_real, nthreads=cores,
                   outputs=("counts",))
        return time.perf_counter() - t

    for _ in range(args.warmup):
        one_step()
    times = [one_step() for _ in range(args.steps)]
    units = float(g.nnz) * n_real * T_s
    sec = sum(times) / len(times)
    value = units / sec
    sample = (f"SIR, {n_real} realizations x {T_s} steps on the full R-MAT scale-{SCALE} graph "
              f"({g.nnz} arcs) per step, {cores} threads")
    return {"impl": "reference", "metric": "edge-realization-steps/sec", "value": value,
            "unit": "edge-realization-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(g, seeds),
            "cpu_baseline": {"value": value, "unit": "edge-realization-steps/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "edge-realization-steps/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def workload_config(g, seeds):
    return {"workload": f"rmat{SCALE}_sir_sis_full_mc_R{R}_T{T}",
            "graph": f"R-MAT scale {SCALE}, edge factor 16, (a,b,c)=(0.57,0.19,0.19), "
                     "duplicates and self-loops kept",
            "n": g.n, "nnz": g.nnz, "R": R, "T": T, "beta": BETA, "gamma": GAMMA,
            "seeds": int(len(seeds)), "models": ["SIR", "SIS"], "rng_seed": RNG_SEED,
            "l2": "inputs larger than L2 (4.3 GB arcs, 8.6 GB state planes); no flush"}


def cpu_baseline(g, seeds, min_seconds=10.0):
    """The oracle's first SIR step on the full graph, in blocks of one realization per
    core: at least one block, then more until min_seconds of CPU work or all R
    realizations are done."""
    import oracle as O
    cores = os.cpu_count() or 1
    T_s, n_real, sec = 1, 0, 0.0
    while n_real == 0 or (sec < min_seconds and n_real < R):
        blk = min(cores, R - n_real)
        t = time.perf_counter()
        O.simulate(O.SIR, g.row_ptr, g.col_idx, seeds, beta=BETA, gamma=GAMMA, R=R, T=T_s,
                   rng_seed=RNG_SEED, r_lo=n_real, n_real=blk, nthreads=cores, outputs=("counts",))
        sec += time.perf_counter() - t
        n_real += blk
    return {"value": float(g.nnz) * n_real * T_s / sec, "unit": "edge-realization-steps/s",
            "cores": cores, "kind": "oracle",
            "sample": f"SIR, {n_real} realizations x {T_s} steps on the full graph, "
                      f"{sec:.1f} s of CPU work"}


# ---------------------------------------------------------------- batched requests

def run_batch_bench(args):
    """Batched requests: 64 BA/ER graphs with n log-uniform in 1k..2M, 4,096 requests
    (model uniform over SIR/SIS/IC/LT, R in 32..1024, seed sets of 1..500 nodes, beta in
    [0.005, 0.2], gamma 0.1, T = 100, IC/LT to quiescence), per-graph autotuning and
    CUDA-graph capture.  One bench step = the whole batch.  Units are the
    edge-realization-steps actually computed (IC/LT stop early)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2603_14895_gb300 import fsgp
    torch.cuda.set_device(0)
    t0 = time.time()
    graphs, reqs = W.batch_pool(n_graphs=args.batch_graphs, n_requests=args.batch_requests)
    log(f"[bench] batch pool: {len(graphs)} graphs, {sum(g.nnz for g in graphs)} arcs, "
        f"{len(reqs)} requests in {time.time() - t0:.1f}s")
    gobjs = [fsgp.Graph(g.row_ptr, g.col_idx) for g in graphs]
    spec = [dict(graph=gobjs[q.graph_index], model=q.model, seeds=q.seeds, R=q.R, T=q.T,
                 rng_seed=q.rng_seed, beta=q.beta, gamma=q.gamma, freq=True) for q in reqs]
    outs = None
    t0 = time.time()
    outs = fsgp.batch_run(spec, autotune=1)          # first run: tuning + allocation
    torch.cuda.synchronize()
    log(f"[bench] first batch (autotune) {time.time() - t0:.1f}s")
    for _ in range(max(0, args.warmup - 1)):
        fsgp.batch_run(spec)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(gpu_selector(torch))
    sampler.start()
    ev0.record()
    for _ in range(args.steps):
        outs = fsgp.batch_run(spec)
    ev1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    steps = [int(o["steps_run"][0].item()) for o in outs]
    units = sum(float(graphs[q.graph_index].nnz) * q.R * st for q, st in zip(reqs, steps))
    nominal = sum(float(graphs[q.graph_index].nnz) * q.R * q.T for q in reqs)
    return {"metric": "edge-realization-steps/sec", "value": units / (ms / 1e3),
            "unit": "edge-realization-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"batch_{len(reqs)}req_{len(graphs)}graphs",
                       "graphs": "BA m=2..8 and ER, n log-uniform 1k..2M",
                       "requests": len(reqs), "models": "SIR/SIS/IC/LT", "R": "32..1024",
                       "T": 100, "l2": "working set above L2 for the large graphs; no flush"},
            "requests_per_s": len(reqs) / (ms / 1e3),
            "nominal_units_per_s": nominal / (ms / 1e3),
            "clocks": clocks}


# ------------------------------------------------------- the smaller workloads

def run_config_bench(args, which: str):
    """Throughput on the other benchmark configurations (one bench step = one full run of
    every model of the configuration; units are the edge-realization-steps computed,
    IC/LT stopping at quiescence):
      ba1m:  BA n=1,000,000 m=5 (both directions), IC weighted cascade and LT, 50 seeds,
             R=1024, T<=100 to quiescence.
      er10k: ER n=10,000 mean degree 10, SIR beta=0.05 gamma=0.1, 1% seeds, R=64, T=50;
             the step loop is captured in a CUDA graph (launch-bound size)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2603_14895_gb300 import fsgp
    torch.cuda.set_device(0)
    if which == "ba1m":
        g = W.ba1m_graph()
        wls = [W.ba1m(W.IC, g), W.ba1m(W.LT, g)]
        opts = {}
    else:
        wls = [W.er10k_sir()]
        g = wls[0].graph
        opts = {"capture_graph": 1}
    graph = fsgp.Graph(g.row_ptr, g.col_idx)
    stream = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(stream):
        for wl in wls:
            outs.append(fsgp.simulate(graph, wl.model, wl.seed_sets, wl.R, wl.T, wl.rng_seed,
                                      beta=wl.beta, gamma=wl.gamma, ic_mode=wl.ic_mode, ic_p=wl.ic_p,
                                      freq=True, options=dict(opts), stream=stream))

    def step():
        for wl, o in zip(wls, outs):
            fsgp.simulate(graph, wl.model, wl.seed_sets, wl.R, wl.T, wl.rng_seed, beta=wl.beta,
                          gamma=wl.gamma, ic_mode=wl.ic_mode, ic_p=wl.ic_p, freq=True,
                          options=dict(opts), stream=stream, out=o)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    # time at least about a second, so that the clock sampler sees the run
    t_one = time.perf_counter()
    with torch.cuda.stream(stream):
        step()
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t_one
    reps = max(1, args.steps, int(1.0 / max(t_one, 1e-4)) + 1)
    sampler = ClockSampler(gpu_selector(torch))
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(reps):
            step()
        ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / reps
    units = 0.0
    per_model = {}
    for wl, o in zip(wls, outs):
        st = int(o["steps_run"][0].item())
        u = float(g.nnz) * wl.R * st
        units += u
        per_model[wl.name] = {"steps_run": st, "edge_realization_steps": u}
    name = "ba1m_ic_lt_R1024" if which == "ba1m" else "er10k_sir_R64_T50"
    return {"metric": "edge-realization-steps/sec", "value": units / (ms / 1e3),
            "unit": "edge-realization-steps/s", "n_gpus": 1, "steps": reps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": name, "n": g.n, "nnz": g.nnz, "models": per_model,
                       "l2": "state and graph fit in L2 for er10k; ba1m exceeds it; no flush"},
            "realization_runs_per_s": sum(wl.R for wl in wls) / (ms / 1e3),
            "clocks": clocks}


def step_bytes(n: int, nnz: int, R: int, planes: int) -> float:
    """Algorithmic bytes of one dense propagation step (every node updated from all its
    in-arcs, Sec. 2 Eq. nodestate over Sec. 3.1 Eq. agg): column indices 4E, row pointers
    4(N+1), one 32-byte sector (or the node's whole word run, if larger) per gathered
    source, and the node's own P state planes read and written."""
    ws = 1
    while ws * 32 < R:
        ws *= 2
    w = 4 * ws
    return 4.0 * nnz + 4.0 * (n + 1) + float(nnz) * max(32, w) + 2.0 * planes * n * w


def run_step_bench(args):
    """One mid-run dense step of SIR and of SIS on the R-MAT graph of --scale (R = 256,
    beta = 0.01, gamma = 0.05, the benchmark's seeds): the state after --t-mid steps is
    exported, and one step from it is timed per kernel kind over --steps repetitions.
    Each model's step also runs once inside the NVTX range "fsgp_step_<model>", with no
    profiling events, for an ncu capture of exactly that step's launches."""
    import torch
    from paper_2603_14895_gb300 import fsgp
    torch.cuda.set_device(0)
    g, seeds = build_workload(args.scale)
    graph = fsgp.Graph(g.row_ptr, g.col_idx)
    kinds = fsgp.PROFILE_KINDS
    peak, peak_kind = measured_peaks()
    res = {}
    for m, nm in zip(MODELS, ("SIR", "SIS")):
        o = fsgp.simulate(graph, m, [seeds], R, args.t_mid, RNG_SEED, beta=BETA, gamma=GAMMA,
                          freq=False, final_planes=True)
        planes = o["final_planes"][0].contiguous()
        empty = seeds[:0]

        def one(profile=None):
            opts = fsgp.make_options(t0=args.t_mid, init_planes=planes)
            if profile is not None:
                opts.profile = fsgp.ctypes.pointer(profile)
            return fsgp.simulate(graph, m, [empty], R, 1, RNG_SEED, beta=BETA, gamma=GAMMA,
                                 freq=False, options=opts)

        for _ in range(args.warmup):
            one()
        torch.cuda.synchronize()
        try:
            torch.cuda.nvtx.range_push(f"fsgp_step_{nm}")
            pushed = True
        except Exception as e:   # no NVTX: the step still runs, only unmarked
            log(f"[bench] no NVTX range: {e}")
            pushed = False
        one()
        torch.cuda.synchronize()
        if pushed:
            torch.cuda.nvtx.range_pop()
        prof = fsgp.fsgp_profile()
        reps = max(1, args.steps)
        for _ in range(reps):
            out = one(prof)
        torch.cuda.synchronize()
        step_kinds = [i for i in range(len(kinds)) if kinds[i] not in ("init", "results")]
        ms = sum(prof.ms[i] for i in step_kinds) / reps
        b = step_bytes(g.n, g.nnz, R, 2 if m == 0 else 1)
        res[nm] = {"t": args.t_mid, "step_ms": ms,
                   "infected_lanes": int(out["counts"][0, -1, 1].item()),
                   "step_bytes_alg": b, "achieved_GBps": b / (ms / 1e3) / 1e9,
                   "frac": b / (ms / 1e3) / 1e9 / peak,
                   "kinds": {kinds[i]: {"launches": prof.launches[i] // reps,
                                        "ms": prof.ms[i] / reps,
                                        "alg_bytes": prof.alg_bytes[i] / reps}
                             for i in step_kinds if prof.launches[i]}}
        log(f"[bench] {nm} step at t={args.t_mid}: {ms:.3f} ms")
        del planes, o
    graph.close()
    return {"workload": f"rmat{args.scale}_mid_step_t{args.t_mid}", "n": g.n, "nnz": g.nnz,
            "R": R, "peak_GBps": peak, "peak_source": peak_kind, "models": res}


def run_weighted_bench(args):
    """Weighted graphs: full Monte Carlo SIR on the R-MAT graph of --scale (default 26),
    arc weights w_e ~ U[0, 2) (mean 1, seeded), beta = 0.01, gamma = 0.05, the benchmark's
    seeds, R = 256, T = 100; each infectious in-arc transmits with probability beta * w_e.
    One bench step = one full run.  The roofline unit is the dense step, whose bytes add
    the 4-byte weight of every arc to the unweighted step's."""
    import numpy as np
    import torch
    from paper_2603_14895_gb300 import fsgp
    torch.cuda.set_device(0)
    g, seeds = build_workload(args.scale)
    w = np.random.default_rng(12345 + 7).uniform(0.0, 2.0, size=g.nnz).astype(np.float32)
    graph = fsgp.Graph(g.row_ptr, g.col_idx)
    graph.set_arc_weights(w)
    stream = torch.cuda.current_stream()
    out = fsgp.simulate(graph, fsgp.SIR, [seeds], R, T, RNG_SEED, beta=BETA, gamma=GAMMA, weighted=True)
    for _ in range(args.warmup):
        fsgp.simulate(graph, fsgp.SIR, [seeds], R, T, RNG_SEED, beta=BETA, gamma=GAMMA, weighted=True, out=out)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_selector(torch))
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        fsgp.simulate(graph, fsgp.SIR, [seeds], R, T, RNG_SEED, beta=BETA, gamma=GAMMA, weighted=True, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    peak, peak_kind = measured_peaks()
    b = step_bytes(g.n, g.nnz, R, 2) + 4.0 * g.nnz
    achieved = T * b / (ms / 1e3) / 1e9
    final = out["counts"][0, -1].cpu().tolist()
    graph.close()
    return {"metric": "edge-realization-steps/sec", "value": float(g.nnz) * R * T / (ms / 1e3),
            "unit": "edge-realization-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale}_sir_weighted_R{R}_T{T}", "n": g.n, "nnz": g.nnz,
                       "weights": "U[0, 2) per arc, seed 12352", "beta": BETA, "gamma": GAMMA,
                       "seeds": int(len(seeds)), "final_SIR": final,
                       "l2": "inputs larger than L2; no flush"},
            "roofline": {"bound": "hbm", "kernel": "dense propagation step (all row launches of a step)",
                         "achieved": achieved, "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "alg_bytes_per_step": b},
            "clocks": clocks}


def run_hk_bench(args):
    """Hegselmann-Krause opinion dynamics (Appendix A.2): BA n = 1,000,000, m = 5 (both
    arc directions, about 10M arcs), R = 64 opinion vectors U[-1, 1] (seeded), eps = 0.25,
    T = 30 steps.  One bench step = one full run from the same start opinions (device
    buffers).  Units are arcs x realizations x steps.  The roofline unit is one step:
    every arc's 32-lane source segments (4 B per realization), its column index once
    per 32-lane group, the node's own opinions read and written."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2603_14895_gb300 import fsgp
    torch.cuda.set_device(0)
    g = W.ba1m_graph()
    R_hk, T_hk, eps = 64, 30, 0.25
    h0 = torch.from_numpy(np.random.default_rng(12345 + 8).uniform(-1.0, 1.0, size=(R_hk, g.n))
                          .astype(np.float32)).cuda()
    graph = fsgp.Graph(g.row_ptr, g.col_idx)
    for _ in range(args.warmup):
        h, ch = fsgp.hk(graph, h0, T_hk, eps)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_selector(torch))
    sampler.start()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps)     # (--steps 100 times about 1.5 s)
    ev0.record(stream)
    for _ in range(reps):
        h, ch = fsgp.hk(graph, h0, T_hk, eps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / reps
    groups = (R_hk + 31) // 32
    b = 4.0 * g.nnz * groups * 32 + 4.0 * g.nnz * groups + 8.0 * g.n * groups * 32 + 4.0 * (g.n + 1)
    peak, peak_kind = measured_peaks()
    achieved = T_hk * b / (ms / 1e3) / 1e9
    return {"metric": "edge-realization-steps/sec", "value": float(g.nnz) * R_hk * T_hk / (ms / 1e3),
            "unit": "edge-realization-steps/s", "n_gpus": 1, "steps": reps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ba1m_hk_R64_T30_eps0.25", "n": g.n, "nnz": g.nnz,
                       "changes_last_step": int(ch[-1].item()), "changes_first_step": int(ch[1].item()),
                       "l2": "opinions 256 MB per buffer, above L2; no flush"},
            "roofline": {"bound": "hbm", "kernel": "k_hk_step (one step)", "achieved": achieved, "peak": peak,
                         "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "alg_bytes_per_step": b},
            "clocks": clocks}


# -------------------------------------------------------------- learned surrogate

SG_R, SG_T, SG_GAMMA, SG_K = 1024, 100, 0.1, 20


def _sg_forward_bytes(n: int, nnz: int, keep_h3: bool = False) -> float:
    """Compulsory bytes of one surrogate forward: every array read or written once
    (row pointers 4 B/node, column indices 4 B/arc, bfloat16 activations 2 B/value):
    layer 1 aggregate 36 n + 4 nnz, layer 1 dense 160 n, layers 2-3 aggregate
    260 n + 4 nnz each, layer 2 dense 384 n, layer 3 dense with the output head 256 n
    (+ 128 n when h3 is kept for training)."""
    return (1356.0 + (128.0 if keep_h3 else 0.0)) * n + 12.0 * nnz


def run_screen_bench(args):
    """Screening throughput of the surrogate alone: one BA graph (n = --screen-n, m = 4),
    a network with its initial weights (the timing does not depend on them), --sg-cands
    candidate 20-node seed sets screened per step.  One step = one fsgp_surrogate_screen
    call; launches replay one captured forward per candidate."""
    import torch
    import workloads as W
    from paper_2603_14895_gb300 import fsgp
    torch.cuda.set_device(0)
    g = W.ba(args.screen_n, 4, seed=11)
    graph = fsgp.Graph(g.row_ptr, g.col_idx)
    sg = fsgp.Surrogate(3)
    cands = W.surrogate_candidates(g, args.sg_cands, SG_K, seed=5)
    beta = args.sg_beta_screen
    for _ in range(args.warmup):
        sg.screen(graph, cands[:64], beta, SG_GAMMA)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_selector(torch))
    sampler.start()
    t = time.perf_counter()
    for _ in range(max(1, args.steps)):
        sg.screen(graph, cands, beta, SG_GAMMA)      # synchronises
    sec = (time.perf_counter() - t) / max(1, args.steps)
    clocks = sampler.stop()
    per = sec / len(cands)
    peak, peak_src = measured_peaks()
    b = _sg_forward_bytes(g.n, g.nnz)
    return {"metric": "surrogate-screened seed sets/sec", "value": len(cands) / sec,
            "unit": "seed sets/s", "n_gpus": 1, "steps": max(1, args.steps), "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"screen_ba{g.n}_m4_k{SG_K}", "n": g.n, "nnz": g.nnz,
                       "candidates": len(cands), "beta": beta, "gamma": SG_GAMMA,
                       "l2": "one candidate's activations (64 MB per layer at n = 500k) stay "
                             "partly L2-resident between the kernels of its forward; no flush"},
            "ms_per_candidate": per * 1e3,
            "roofline": {"bound": "hbm", "kernel": "screening forward (all launches of one candidate)",
                         "achieved": b / per / 1e9, "peak": peak, "peak_source": peak_src,
                         "unit": "GB/s", "frac": b / per / 1e9 / peak, "traffic": None,
                         "alg_bytes_per_candidate": b},
            "clocks": clocks}


def run_surrogate_bench(args):
    """Learned surrogate, end to end: graphs, Monte Carlo targets, training, held-out
    error, screening, Monte Carlo re-scoring.

    Graphs: args.sg_graphs synthetic BA / R-MAT graphs with n = 100k .. 1M; the first 80%
    train, the rest are held out.  Targets: per node, the fraction of R = 1024 SIR
    realizations (T = 100, gamma = 0.1) in which it was ever infected, for 8 random
    20-node seed sets per graph with beta ~ U[0.01, 0.1].  Error: mean absolute error of
    the predicted probabilities against those frequencies on the held-out graphs.
    Screening: 10,000 candidate 20-node sets per screened graph; the surrogate's top 100
    and 100 random candidates are re-scored by Monte Carlo (R = 1024, T = 100)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2603_14895_gb300 import fsgp
    torch.cuda.set_device(0)
    NG = args.sg_graphs
    n_train = max(1, int(round(0.8 * NG)))
    t0 = time.time()
    graphs = W.surrogate_pool(NG)
    log(f"[surrogate] {NG} graphs, {sum(g.n for g in graphs)} nodes, "
        f"{sum(g.nnz for g in graphs)} arcs in {time.time() - t0:.1f}s")
    gobjs = [fsgp.Graph(g.row_ptr, g.col_idx) for g in graphs]
    sets = [W.surrogate_sets(g, i) for i, g in enumerate(graphs)]

    # Monte Carlo targets, batched over requests, a slice of graphs at a time
    t0 = time.time()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    targets = [[None] * len(sets[i]) for i in range(NG)]
    mc_ms = 0.0
    for c0 in range(0, NG, 20):
        spec, where = [], []
        for gi in range(c0, min(NG, c0 + 20)):
            for j, (sd, beta) in enumerate(sets[gi]):
                spec.append(dict(graph=gobjs[gi], model=0, seeds=sd, R=SG_R, T=SG_T,
                                 rng_seed=1000 * gi + j + 1, beta=beta, gamma=SG_GAMMA, freq=True))
                where.append((gi, j))
        ev0.record()
        outs = fsgp.batch_run(spec, capture_graph=1)
        ev1.record()
        torch.cuda.synchronize()
        mc_ms += ev0.elapsed_time(ev1)
        for (gi, j), o in zip(where, outs):
            fr = o["freq"][0]
            targets[gi][j] = ((fr[1] + fr[2]).float() / SG_R).contiguous()
        del outs
        for gi in range(c0, min(NG, c0 + 20)):
            gobjs[gi].trim()
    mc_units = sum(float(graphs[gi].nnz) * SG_R * SG_T * len(sets[gi]) for gi in range(NG))
    log(f"[surrogate] targets: {sum(len(s) for s in sets)} runs, {mc_ms / 1e3:.1f}s on device, "
        f"{time.time() - t0:.1f}s wall")

    # training
    sg = fsgp.Surrogate(args.sg_seed)
    samples = [(gi, j) for gi in range(n_train) for j in range(len(sets[gi]))]
    rng = np.random.default_rng(args.sg_seed)
    E = args.sg_epochs
    total = E * len(samples)
    it = 0
    t0 = time.time()
    ev0.record()
    for ep in range(E):
        for idx in rng.permutation(len(samples)):
            gi, j = samples[idx]
            lr = args.sg_lr * (0.05 + 0.95 * 0.5 * (1 + np.cos(np.pi * it / total)))
            sd, beta = sets[gi][j]
            sg.train_step(gobjs[gi], sd, beta, SG_GAMMA, targets[gi][j], lr=float(lr), want_loss=False)
            it += 1
    ev1.record()
    torch.cuda.synchronize()
    train_ms = ev0.elapsed_time(ev1)
    train_nodes = sum(graphs[gi].n for gi, _ in samples) * E
    log(f"[surrogate] {E} epochs x {len(samples)} samples in {train_ms / 1e3:.1f}s")

    def mae_over(gis):
        err = nodes = 0.0
        const_err = 0.0
        rel = []
        ybar = float(np.mean([float(targets[g][j].mean()) for g in range(n_train) for j in range(len(sets[g]))]))
        for gi in gis:
            for j, (sd, beta) in enumerate(sets[gi]):
                p = sg.forward(gobjs[gi], sd, beta, SG_GAMMA)
                y = targets[gi][j]
                err += float((p - y).abs().sum())
                const_err += float((y - ybar).abs().sum())
                nodes += y.numel()
                ys, ps = float(y.sum()), float(p.sum())
                rel.append(abs(ps - ys) / max(ys, 1.0))
        return err / nodes, const_err / nodes, float(np.median(rel)), float(np.mean(rel))

    held = list(range(n_train, NG))
    mae_train, _, _, _ = mae_over(range(min(n_train, 8)))
    mae, mae_const, spread_rel_med, spread_rel_mean = mae_over(held)
    log(f"[surrogate] held-out MAE {mae:.4f} (constant predictor {mae_const:.4f}); "
        f"train MAE {mae_train:.4f}; spread rel. error median {spread_rel_med:.3f}")

    # screening on held-out graphs
    sampler = ClockSampler(gpu_selector(torch))
    sampler.start()
    screen = []
    scr_ms = mc_cand_ms = 0.0
    scr_bytes = 0.0
    n_scr = 0
    for gi in held[:args.sg_screen_graphs]:
        g = graphs[gi]
        beta = args.sg_beta_screen
        cands = W.surrogate_candidates(g, args.sg_cands, SG_K, seed=7000 + gi)
        sg.screen(gobjs[gi], cands[:64], beta, SG_GAMMA)     # warm-up (graph capture, buffers)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        scores = sg.screen(gobjs[gi], cands, beta, SG_GAMMA)
        dt = (time.perf_counter() - t1) * 1e3
        scr_ms += dt
        scr_bytes += _sg_forward_bytes(g.n, g.nnz) * len(cands)
        n_scr += len(cands)
        top = np.argsort(-scores)[:100]
        rnd = np.random.default_rng(gi).choice(len(cands), 100, replace=False)
        pick = np.concatenate([top, rnd])
        ev0.record()
        out = fsgp.simulate(gobjs[gi], 0, [cands[c] for c in pick], SG_R, SG_T, 77 + gi,
                            beta=beta, gamma=SG_GAMMA, freq=False, steps_run=False)
        ev1.record()
        torch.cuda.synchronize()
        gobjs[gi].trim()
        mc_cand_ms += ev0.elapsed_time(ev1)
        cnt = out["counts"].cpu().numpy()
        spread = (cnt[:, SG_T, 1] + cnt[:, SG_T, 2]) / SG_R
        st, sr = spread[:100], spread[100:]
        rs = np.argsort(np.argsort(scores[rnd]))
        rm = np.argsort(np.argsort(sr))
        screen.append({"graph": gi, "n": g.n, "nnz": g.nnz,
                       "top100_mc_mean": float(st.mean()), "random100_mc_mean": float(sr.mean()),
                       "top100_mc_best": float(st.max()), "random100_mc_best": float(sr.max()),
                       "spearman_random100": float(np.corrcoef(rs, rm)[0, 1]),
                       "screen_ms": dt})
        log(f"[surrogate] graph {gi} n={g.n}: screen {len(cands)} in {dt:.0f} ms; top-100 MC "
            f"{st.mean():.1f} vs random-100 {sr.mean():.1f}; spearman {screen[-1]['spearman_random100']:.2f}")
    clocks = sampler.stop()
    mc_per_cand_ms = mc_cand_ms / (200.0 * len(screen))
    sg_per_cand_ms = scr_ms / n_scr
    achieved = scr_bytes / (scr_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    return {"metric": "surrogate-screened seed sets/sec", "value": n_scr / (scr_ms / 1e3),
            "unit": "seed sets/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": scr_ms / max(1, len(screen)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"surrogate_{NG}graphs_{args.sg_cands}cands",
                       "graphs": "BA m=2..6 n=100k..1M and R-MAT scale 17..19 ef 8",
                       "train_graphs": n_train, "held_out_graphs": NG - n_train,
                       "sets_per_graph": 8, "seed_set_size": SG_K, "R": SG_R, "T": SG_T,
                       "beta_train": "U[0.01,0.1]", "beta_screen": args.sg_beta_screen, "gamma": SG_GAMMA,
                       "epochs": E, "lr": args.sg_lr,
                       "l2": "graphs of this size keep activations partly L2-resident"},
            "mae_vs_mc_R1024": mae, "mae_constant_predictor": mae_const, "mae_train_subset": mae_train,
            "spread_rel_err_median": spread_rel_med, "spread_rel_err_mean": spread_rel_mean,
            "mc_ms_per_candidate": mc_per_cand_ms, "surrogate_ms_per_candidate": sg_per_cand_ms,
            "screening_speedup": mc_per_cand_ms / sg_per_cand_ms,
            "screen": screen,
            "targets_mc": {"runs": sum(len(s) for s in sets), "device_s": mc_ms / 1e3,
                           "edge_realization_steps_per_s": mc_units / (mc_ms / 1e3)},
            "train": {"steps": total, "device_s": train_ms / 1e3,
                      "node_samples_per_s": train_nodes / (train_ms / 1e3)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if peak else None, "traffic": None,
                         "note": "whole screening forward, compulsory bytes; peak " + peak_src},
            "clocks": clocks}


# ----------------------------------------------------------------- multi-rank launch

def _free_port() -> int:
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def launch_ranks(n: int, argv) -> int:
    """Start n ranks of this script under torch.distributed.run on this node (rendezvous
    on 127.0.0.1) and return their exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.abspath(__file__), *argv]
    log(f"[bench] starting {n} ranks: {' '.join(cmd[1:6])} ...")
    return subprocess.call(cmd, cwd=ROOT)


def dry_run(args, world: int, rank: int, local: int) -> dict | None:
    """Join the process group, take this rank's realization shard, gather the shards on
    rank 0.  No simulation."""
    import torch
    import torch.distributed as dist
    from paper_2603_14895_gb300.shard import lane_shard
    use_nccl = torch.cuda.is_available() and torch.cuda.device_count() > local
    if world > 1:
        if use_nccl:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    r0, rl = lane_shard(R * world, world, rank)
    mine = {"rank": rank, "local_rank": local, "r_offset": r0, "R": rl}
    shards = [mine]
    if world > 1:
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        dist.destroy_process_group()
    if rank != 0:
        return None
    return {"dry_run": True, "n_gpus": world, "backend": ("nccl" if use_nccl else "gloo") if world > 1 else None,
            "lanes_per_rank": R, "ranks": shards}


# ------------------------------------------------------------------------- main

def main():
    global SCALE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fsgp", choices=["fsgp", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="rmat26",
                    choices=["rmat26", "batch", "surrogate", "ba1m", "er10k", "step", "screen", "weighted",
                             "hk"])
    ap.add_argument("--screen-n", type=int, default=500_000)
    ap.add_argument("--t-mid", type=int, default=50)
    ap.add_argument("--sg-graphs", type=int, default=200)
    ap.add_argument("--sg-epochs", type=int, default=6)
    ap.add_argument("--sg-lr", type=float, default=2e-3)
    ap.add_argument("--sg-seed", type=int, default=1)
    ap.add_argument("--sg-cands", type=int, default=10_000)
    ap.add_argument("--sg-screen-graphs", type=int, default=4)
    ap.add_argument("--sg-beta-screen", type=float, default=0.01)
    ap.add_argument("--single-reps", type=int, default=2)
    ap.add_argument("--batch-graphs", type=int, default=64)
    ap.add_argument("--batch-requests", type=int, default=4096)
    ap.add_argument("--dry-run", action="store_true")
    args = ap.parse_args()
    SCALE = args.scale

    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args.gpus, sys.argv[1:]))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.dry_run:
        out = dry_run(args, world, rank, local)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    if args.workload == "batch" and args.impl == "fsgp":
        print(json.dumps(run_batch_bench(args)), flush=True)
        return
    if args.workload == "surrogate" and args.impl == "fsgp":
        print(json.dumps(run_surrogate_bench(args)), flush=True)
        return
    if args.workload == "hk" and args.impl == "fsgp":
        print(json.dumps(run_hk_bench(args)), flush=True)
        return
    if args.workload == "weighted" and args.impl == "fsgp":
        print(json.dumps(run_weighted_bench(args)), flush=True)
        return
    if args.workload == "screen" and args.impl == "fsgp":
        print(json.dumps(run_screen_bench(args)), flush=True)
        return
    if args.workload == "step" and args.impl == "fsgp":
        print(json.dumps(run_step_bench(args)), flush=True)
        return
    if args.workload in ("ba1m", "er10k") and args.impl == "fsgp":
        print(json.dumps(run_config_bench(args, args.workload)), flush=True)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        g, seeds = build_workload(SCALE)
        out = run_reference(args, g, seeds, rank)
        print(json.dumps(out), flush=True)
        return

    import numpy as np
    import torch
    from paper_2603_14895_gb300 import fsgp

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    g, seeds = build_workload(SCALE)
    t0 = time.time()
    graph = fsgp.Graph(g.row_ptr, g.col_idx)
    torch.cuda.synchronize()
    log(f"[bench] graph on device in {time.time() - t0:.1f}s: {graph.info()}")
    from paper_2603_14895_gb300.shard import lane_shard
    r_offset, _ = lane_shard(R * world, world, rank)     # weak scaling: R lanes per rank
    shards = [{"rank": rank, "r_offset": r_offset, "R": R}]
    if dist is not None:
        shards = [None] * world
        dist.all_gather_object(shards, {"rank": rank, "r_offset": r_offset, "R": R})
    stream = torch.cuda.current_stream()
    outs = {m: fsgp.simulate(graph, m, [seeds], R, T, RNG_SEED, beta=BETA, gamma=GAMMA,
                             freq=True, device=True,
                             options=dict(r_offset=r_offset)) for m in MODELS}

    def step(profile=None):
        for m in MODELS:
            opts = fsgp.make_options(r_offset=r_offset)
            if profile is not None:
                opts.profile = fsgp.ctypes.pointer(profile[m])
            fsgp.simulate(graph, m, [seeds], R, T, RNG_SEED, beta=BETA, gamma=GAMMA,
                          device=True, options=opts, out=outs[m])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    profiles = {m: fsgp.fsgp_profile() for m in MODELS}
    sampler = ClockSampler(gpu_selector(torch))
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(profiles)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms_total = ev0.elapsed_time(ev1)
    if dist is not None:
        tt = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_total = float(tt.item())
    ms_per_step = ms_total / args.steps
    units_per_step = float(g.nnz) * R * T * len(MODELS)
    value = units_per_step * world / (ms_per_step / 1e3)

    # per-kernel roofline from the profiled timed region
    kinds = fsgp.PROFILE_KINDS
    NK = len(kinds)
    agg_ms = [sum(profiles[m].ms[i] for m in MODELS) for i in range(NK)]
    agg_b = [sum(profiles[m].alg_bytes[i] for m in MODELS) for i in range(NK)]
    agg_n = [sum(profiles[m].launches[i] for m in MODELS) for i in range(NK)]
    dom = max(range(NK), key=lambda i: agg_ms[i])
    peak, peak_kind = measured_peaks()
    dom_achieved = (agg_b[dom] / agg_n[dom]) / (agg_ms[dom] / agg_n[dom] / 1e3) / 1e9 if agg_n[dom] else 0.0
    # The roofline unit is the dense propagation step (its degree-class launches together):
    # algorithmic bytes per step x steps of both models over the whole timed run time
    # (initialisation and result kernels included).
    b_step = {"SIR": step_bytes(g.n, g.nnz, R, 2), "SIS": step_bytes(g.n, g.nnz, R, 1)}
    alg_run = T * (b_step["SIR"] + b_step["SIS"])
    achieved = alg_run / (ms_per_step / 1e3) / 1e9
    # DRAM traffic per step: each kind's measured DRAM / algorithmic ratio (small capture)
    # times the algorithmic bytes its launches processed here, averaged over the steps
    # (a step kind without a measured ratio for its model, e.g. SIR hub chunks, which
    # process arcs only in the first steps, counts its algorithmic bytes in full)
    ratios = ncu_traffic_ratios()
    traffic = None
    if ratios is not None:
        tot = 0.0
        for m, nm in zip(MODELS, ("SIR", "SIS")):
            for i in range(NK):
                b = profiles[m].alg_bytes[i]
                if b == 0 or kinds[i] in ("init", "results"):
                    continue
                tot += ratios.get(nm, {}).get(kinds[i], 1.0) * b
        traffic = tot / (args.steps * T * len(MODELS))
    launches = sum(profiles[m].kernel_launches for m in MODELS)
    per_kernel = {kinds[i]: {"launches": agg_n[i] // args.steps,
                             "ms_per_step": agg_ms[i] / args.steps,
                             "alg_GBps": (agg_b[i] / (agg_ms[i] / 1e3) / 1e9) if agg_ms[i] else 0.0}
                  for i in range(NK) if agg_n[i]}
    wall = {}
    for m, nm in zip(MODELS, ("SIR", "SIS")):
        wall[nm] = sum(profiles[m].ms) / args.steps / 1e3

    # the plain single-instance path (one realization, one byte per node) on the same
    # graph: a few realizations timed, the full R-realization run extrapolated
    single = None
    if args.single_reps > 0:
        ms_single = {}
        for m, nm in zip(MODELS, ("SIR", "SIS")):
            fsgp.simulate_single(graph, m, seeds, r_offset, T, RNG_SEED, beta=BETA, gamma=GAMMA,
                                 final_state=False)          # warm-up (workspace)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(args.single_reps):
                fsgp.simulate_single(graph, m, seeds, r_offset + i, T, RNG_SEED, beta=BETA,
                                     gamma=GAMMA, final_state=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_single[nm] = e0.elapsed_time(e1) / args.single_reps
        extrap_s = sum(ms_single.values()) * R / 1e3
        single = {"realizations_timed_per_model": args.single_reps,
                  "ms_per_realization": ms_single,
                  "full_mc_s_extrapolated": extrap_s,
                  "packed_full_mc_s": ms_per_step / 1e3,
                  "packed_speedup": extrap_s / (ms_per_step / 1e3),
                  "note": "single-instance time x R (extrapolated); same draws as packed lanes"}
        log(f"[bench] single-instance: {ms_single} ms/realization; full MC extrapolated "
            f"{extrap_s:.1f}s vs packed {ms_per_step / 1e3:.2f}s")

    # end to end through the public API with host buffers (graph upload included)
    e2e = None
    if not args.no_e2e:
        rp = torch.from_numpy(g.row_ptr).pin_memory()
        ci = torch.from_numpy(g.col_idx).pin_memory()
        sd = torch.from_numpy(seeds.astype(np.int32)).pin_memory()
        # result buffers in pinned host memory (what a caller streaming results would use)
        def pinned(shape, dt_torch):
            return torch.zeros(shape, dtype=dt_torch).pin_memory().numpy()
        host_out = {m: {"counts": pinned((1, T + 1, 3), torch.int64).view(np.uint64),
                        "freq": pinned((1, 3, g.n), torch.int32).view(np.uint32)} for m in MODELS}
        n_e2e = max(1, args.steps)
        graph.close()
        torch.cuda.synchronize()
        barrier()
        t = time.perf_counter()
        for _ in range(n_e2e):
            gh = fsgp.Graph(rp, ci)
            for m in MODELS:
                fsgp.simulate(gh, m, [sd.numpy()], R, T, RNG_SEED, beta=BETA, gamma=GAMMA,
                              device=False, options=dict(r_offset=r_offset), out=host_out[m])
            gh.close()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t) / n_e2e
        if dist is not None:
            tt = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_s = float(tt.item())
        h2d = g.row_ptr.nbytes + g.col_idx.nbytes + seeds.nbytes * len(MODELS)
        d2h = sum(v.nbytes for m in MODELS for v in host_out[m].values())
        e2e = {"value": units_per_step * world / e2e_s, "unit": "edge-realization-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "seconds_per_step": e2e_s}
        # the host results must equal the device results
        for m in MODELS:
            assert np.array_equal(host_out[m]["counts"][0],
                                  outs[m]["counts"][0].cpu().numpy().astype(np.uint64))
    else:
        graph.close()

    result = {
        "metric": "edge-realization-steps/sec", "value": value,
        "unit": "edge-realization-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(g, seeds),
        "full_mc_wall_s": wall,
        "roofline": {"bound": "hbm", "kernel": "dense propagation step (all row launches of a step)",
                     "achieved": achieved, "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "alg_bytes_per_step": (b_step["SIR"] + b_step["SIS"]) / 2,
                     "per_model_frac": {nm: T * b_step[nm] / wall[nm] / 1e9 / peak for nm in wall},
                     "dominant_kernel": {"kind": kinds[dom], "achieved": dom_achieved,
                                         "frac": dom_achieved / peak if peak else None,
                                         "alg_bytes": "rows and arcs the launches processed"}},
        "kernels": per_kernel,
        "dense_steps": sum(profiles[m].dense_steps for m in MODELS) // args.steps,
        "sparse_steps": sum(profiles[m].sparse_steps for m in MODELS) // args.steps,
        "clocks": clocks,
        "e2e": e2e,
        "single_instance": single,
        "gpu_launches": int(launches),
        "ranks": shards,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(g, seeds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
