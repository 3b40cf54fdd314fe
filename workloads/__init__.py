"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark.

This package only generates inputs (graphs in int32 in-CSR form, seed-node sets,
parameter draws).  It holds none of the propagation method's arithmetic and imports
neither the oracle nor the GPU library.  Graph generation is C (``gen.c``) driven by
a SplitMix64 counter hash, so every graph is a pure function of its seed.

The named workloads stand in for the paper's datasets (Sec. 5.1 dataset table):
ER n=10k ~ Cora/PubMed, BA n=1M ~ Yelp/Pokec, R-MAT scale 26 ~ Webbase.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfsgp_gen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           _SRC, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.gen_rmat.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_int, P, P]
            lib.gen_rmat.restype = ctypes.c_int
            lib.gen_ba_arcs.argtypes = [ctypes.c_int32, ctypes.c_int32]
            lib.gen_ba_arcs.restype = ctypes.c_int64
            lib.gen_ba.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P, P]
            lib.gen_ba.restype = ctypes.c_int
            lib.gen_er.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P, P, P]
            lib.gen_er.restype = ctypes.c_int
            lib.gen_seed_set.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P]
            lib.gen_seed_set.restype = ctypes.c_int
            lib.gen_hash.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.gen_hash.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Graph:
    """int32 in-CSR: row v lists the sources u of arcs u -> v."""
    row_ptr: np.ndarray
    col_idx: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def in_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


def rmat(scale: int, edge_factor: int = 16, a=0.57, b=0.19, c=0.19, seed: int = 0,
         nthreads: int | None = None) -> Graph:
    n = 1 << scale
    e = edge_factor * n
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col_idx = np.zeros(e, dtype=np.int32)
    rc = _load().gen_rmat(scale, e, a, b, c, seed, nthreads or os.cpu_count() or 1,
                          _p(row_ptr), _p(col_idx))
    if rc != 0:
        raise ValueError(f"gen_rmat failed ({rc})")
    return Graph(row_ptr, col_idx, f"rmat{scale}_ef{edge_factor}")


def ba(n: int, m: int, seed: int = 0) -> Graph:
    lib = _load()
    na = lib.gen_ba_arcs(n, m)
    if na < 0:
        raise ValueError("bad BA size")
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col_idx = np.zeros(na, dtype=np.int32)
    rc = lib.gen_ba(n, m, seed, _p(row_ptr), _p(col_idx))
    if rc != 0:
        raise ValueError(f"gen_ba failed ({rc})")
    return Graph(row_ptr, col_idx, f"ba{n}_m{m}")


def er(n: int, mean_deg: float, seed: int = 0) -> Graph:
    lib = _load()
    na = ctypes.c_int64(0)
    rc = lib.gen_er(n, mean_deg, seed, ctypes.byref(na), None, None)
    if rc != 0:
        raise ValueError(f"gen_er failed ({rc})")
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col_idx = np.zeros(max(na.value, 1), dtype=np.int32)
    rc = lib.gen_er(n, mean_deg, seed, ctypes.byref(na), _p(row_ptr), _p(col_idx))
    if rc != 0:
        raise ValueError(f"gen_er failed ({rc})")
    return Graph(row_ptr, col_idx[:na.value].copy(), f"er{n}_d{mean_deg:g}")


def seed_set(n: int, k: int, seed: int) -> np.ndarray:
    out = np.zeros(max(k, 1), dtype=np.int32)
    rc = _load().gen_seed_set(n, k, seed, _p(out))
    if rc != 0:
        raise ValueError("gen_seed_set failed")
    return out[:k].copy()


def hash64(seed: int, stream: int, i: int) -> int:
    return int(_load().gen_hash(seed, stream, i))


def uniform01(seed: int, stream: int, i: int) -> float:
    return (hash64(seed, stream, i) >> 11) * (1.0 / (1 << 53))


def from_arcs(n: int, src, dst, name: str = "custom") -> Graph:
    """In-CSR from an explicit arc list (for hand-built test graphs)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    order = np.lexsort((src, dst))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, dst + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return Graph(row_ptr, src.astype(np.int32), name)


# --------------------------------------------------------------------------- configs

SIR, SIS, IC, LT = 0, 1, 2, 3


@dataclass
class Workload:
    """One simulation input: graph, model, parameters, seed sets, R, T, rng seed."""
    name: str
    graph: Graph
    model: int
    beta: float = 0.0
    gamma: float = 0.0
    ic_mode: int = 0          # 0 weighted cascade (p = 1/d_in), 1 constant ic_p
    ic_p: float = 0.0
    seed_sets: list = field(default_factory=list)
    R: int = 1
    T: int = 0
    rng_seed: int = 1


def er10k_sir() -> Workload:
    """Undirected ER G(n=10,000, mean degree 10); SIR beta=0.05 gamma=0.1; 1% random
    seeds; R=64; T=50; rng_seed=1."""
    g = er(10_000, 10.0, seed=12345 + 1)
    seeds = seed_set(g.n, g.n // 100, seed=22345 + 1)
    return Workload("er10k_sir_R64_T50", g, SIR, beta=0.05, gamma=0.1, seed_sets=[seeds],
                    R=64, T=50, rng_seed=1)


def ba1m_graph() -> Graph:
    return ba(1_000_000, 5, seed=12345 + 2)


def ba1m(model: int, g: Graph | None = None) -> Workload:
    """BA n=1,000,000 m=5 (both arc directions); IC weighted cascade or LT (weights
    1/d_in, Philox thresholds); 50 random seeds; R=1024; T<=100 to quiescence."""
    g = g or ba1m_graph()
    seeds = seed_set(g.n, 50, seed=22345 + 2)
    nm = "ic" if model == IC else "lt"
    return Workload(f"ba1m_{nm}_R1024", g, model, ic_mode=0, seed_sets=[seeds], R=1024,
                    T=100, rng_seed=2)


def rmat26_graph(scale: int = 26) -> Graph:
    return rmat(scale, 16, 0.57, 0.19, 0.19, seed=12345 + 3)


def rmat26(model: int, g: Graph | None = None, scale: int = 26) -> Workload:
    """R-MAT scale 26, edge factor 16 (2^30 arcs, duplicates and self-loops kept);
    SIR or SIS beta=0.01 gamma=0.05; 0.01% random seeds; R=256; T=100."""
    g = g or rmat26_graph(scale)
    k = max(1, (g.n * 1) // 10_000)
    seeds = seed_set(g.n, k, seed=22345 + 3)
    nm = "sir" if model == SIR else "sis"
    return Workload(f"rmat{scale}_{nm}_R256_T100", g, model, beta=0.01, gamma=0.05,
                    seed_sets=[seeds], R=256, T=100, rng_seed=3)


# ------------------------------------------------------------- batched requests

@dataclass
class BatchRequest:
    graph_index: int
    model: int
    seeds: np.ndarray
    R: int
    T: int
    beta: float
    gamma: float
    rng_seed: int


def batch_pool(n_graphs: int = 64, n_requests: int = 4096, n_min: int = 1_000,
               n_max: int = 2_000_000, seed: int = 12345 + 4, T: int = 100):
    """Pool of power-law (BA, m in 2..8) and ER graphs with n log-uniform in
    [n_min, n_max], and requests with model uniform over SIR/SIS/IC/LT, R in
    {32, ..., 1024}, seed-set size uniform in 1..500, beta ~ U[0.005, 0.2], gamma = 0.1,
    IC weighted cascade, T steps (IC/LT stop earlier at quiescence)."""
    graphs = []
    lo, hi = np.log(n_min), np.log(n_max)
    for i in range(n_graphs):
        n = int(round(np.exp(lo + (hi - lo) * uniform01(seed, 1, i))))
        if hash64(seed, 2, i) % 4 == 0:
            deg = 4 + int(hash64(seed, 3, i) % 13)
            graphs.append(er(n, float(deg), seed=seed * 1000 + i))
        else:
            m = 2 + int(hash64(seed, 4, i) % 7)
            graphs.append(ba(max(n, m + 2), m, seed=seed * 1000 + i))
    Rs = [32, 64, 128, 256, 512, 1024]
    reqs = []
    for j in range(n_requests):
        gi = int(hash64(seed, 5, j) % n_graphs)
        g = graphs[gi]
        k = 1 + int(hash64(seed, 6, j) % 500)
        reqs.append(BatchRequest(
            graph_index=gi, model=int(hash64(seed, 7, j) % 4),
            seeds=seed_set(g.n, min(k, g.n), seed=seed * 100000 + j),
            R=Rs[int(hash64(seed, 8, j) % len(Rs))], T=T,
            beta=0.005 + 0.195 * uniform01(seed, 9, j), gamma=0.1, rng_seed=1 + j))
    return graphs, reqs


# ------------------------------------------------------------ surrogate training pool

def surrogate_pool(n_graphs: int = 200, n_min: int = 100_000, n_max: int = 1_000_000,
                   seed: int = 12345 + 5, threads: int | None = None):
    """Synthetic graphs for training and judging the seed-set surrogate: even indices
    are BA graphs (both arc directions, m in 2..6, n log-uniform in [n_min, n_max]),
    odd indices directed R-MAT graphs (a, b, c = 0.57, 0.19, 0.19, edge factor 8,
    scale in 17..19, i.e. n = 131,072 .. 524,288).  Generated in parallel threads."""
    from concurrent.futures import ThreadPoolExecutor
    lo, hi = np.log(n_min), np.log(n_max)

    def make(i):
        if i % 2 == 0:
            n = int(round(np.exp(lo + (hi - lo) * uniform01(seed, 1, i))))
            m = 2 + int(hash64(seed, 2, i) % 5)
            return ba(n, m, seed=seed * 1000 + i)
        scale = 17 + int(hash64(seed, 3, i) % 3)
        return rmat(scale, 8, 0.57, 0.19, 0.19, seed=seed * 1000 + i, nthreads=1)

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        return list(ex.map(make, range(n_graphs)))


def surrogate_sets(g: Graph, gi: int, n_sets: int = 8, k: int = 20, seed: int = 12345 + 6):
    """Training seed sets for graph gi: n_sets uniform random k-node sets, each with
    beta ~ U[0.01, 0.1] (gamma = 0.1 is fixed by the caller)."""
    out = []
    for j in range(n_sets):
        s = seed_set(g.n, k, seed=seed * 1_000_000 + gi * 1000 + j)
        out.append((s, 0.01 + 0.09 * uniform01(seed, gi, j)))
    return out


def surrogate_candidates(g: Graph, n_cand: int = 10_000, k: int = 20, seed: int = 0):
    """Candidate k-node seed sets for screening: candidate c takes round(k f_c) of its
    nodes by sampling arcs uniformly (a node with probability proportional to its
    out-degree) and the rest uniformly, f_c ~ U[0, 1], so candidates range from random
    sets to hub-heavy ones.  Nodes may repeat within a candidate."""
    rng = np.random.default_rng(seed)
    f = rng.random(n_cand)
    nb = np.rint(k * f).astype(np.int64)
    biased = g.col_idx[rng.integers(0, g.nnz, size=(n_cand, k))]
    uniform = rng.integers(0, g.n, size=(n_cand, k), dtype=np.int64)
    take = np.arange(k)[None, :] < nb[:, None]
    return np.where(take, biased, uniform).astype(np.int32)
