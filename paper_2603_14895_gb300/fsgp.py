"""Thin Python binding of libfsgp.so (C ABI declared in include/fsgp.h).

Argument marshalling only: every step of the simulation runs in the library's CUDA
kernels.  PyTorch provides device memory (result tensors) and the CUDA stream.  The
library is loaded from this package directory; if it is missing it is built with nvcc,
and if that fails the import fails -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

FSGP_OK = 0
FSGP_EINVAL, FSGP_ENOMEM, FSGP_ECUDA, FSGP_ETIMEOUT, FSGP_EUNSUPPORTED = -1, -2, -3, -4, -5
SIR, SIS, IC, LT = 0, 1, 2, 3
SI, SEIR, SEIS, SWIR = 4, 5, 6, 7
PTR_HOST, PTR_DEVICE = 0, 1
IC_WEIGHTED_CASCADE, IC_CONSTANT = 0, 1


class FsgpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fsgp error {code}: {msg}")
        self.code = code


class fsgp_params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("ic_mode", ctypes.c_int32), ("ic_p", ctypes.c_double),
                ("alpha", ctypes.c_double), ("mu", ctypes.c_double), ("nu", ctypes.c_double),
                ("weighted", ctypes.c_int32)]


PROF_KINDS = 10


class fsgp_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * PROF_KINDS), ("ms", ctypes.c_double * PROF_KINDS),
                ("alg_bytes", ctypes.c_double * PROF_KINDS), ("dense_steps", ctypes.c_int64),
                ("sparse_steps", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]


PROFILE_KINDS = ["init", "step_control", "frontier_mark", "hub_chunks", "hub_finalize",
                 "rows_warp", "rows_team", "results", "rows_team4", "rows_lane"]


class fsgp_options(ctypes.Structure):
    _fields_ = [("vector_words", ctypes.c_int32), ("small_max_deg", ctypes.c_int32),
                ("hub_min_deg", ctypes.c_int32), ("hub_chunk", ctypes.c_int32),
                ("sparse_frac", ctypes.c_double), ("r_offset", ctypes.c_int32),
                ("t0", ctypes.c_int32), ("init_planes", ctypes.c_void_p),
                ("profile", ctypes.POINTER(fsgp_profile)), ("capture_graph", ctypes.c_int32),
                ("lane_words", ctypes.c_int32), ("fuse_rows", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class fsgp_result(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("counts", ctypes.c_void_p),
                ("freq", ctypes.c_void_p), ("per_real", ctypes.c_void_p),
                ("final_planes", ctypes.c_void_p), ("steps_run", ctypes.c_void_p)]


class fsgp_request(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("model", ctypes.c_int32), ("params", fsgp_params),
                ("seed_nodes", ctypes.c_void_p), ("n_seeds", ctypes.c_int64),
                ("R", ctypes.c_int32), ("T", ctypes.c_int32), ("rng_seed", ctypes.c_uint64),
                ("result", fsgp_result)]


class fsgp_batch_options(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("capture_graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("reserved", ctypes.c_int32 * 8)]


def lib_path() -> str:
    return os.path.join(_HERE, "libfsgp.so")


def load():
    """Load libfsgp.so (building it first if absent).  Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.fsgp_graph_create.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                          P, ctypes.POINTER(P)]
        lib.fsgp_graph_create.restype = ctypes.c_int
        lib.fsgp_graph_destroy.argtypes = [P]
        lib.fsgp_graph_destroy.restype = ctypes.c_int
        lib.fsgp_graph_info.argtypes = [P, P, P, P, P]
        lib.fsgp_graph_info.restype = ctypes.c_int
        lib.fsgp_simulate_single.argtypes = [P, ctypes.c_int32, ctypes.POINTER(fsgp_params), P,
                                             ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_uint64, P, P, P, ctypes.c_uint32, P]
        lib.fsgp_simulate_single.restype = ctypes.c_int
        lib.fsgp_graph_trim.argtypes = [P]
        lib.fsgp_graph_trim.restype = ctypes.c_int
        lib.fsgp_model_planes.argtypes = [ctypes.c_int32]
        lib.fsgp_model_planes.restype = ctypes.c_int
        lib.fsgp_model_compartments.argtypes = [ctypes.c_int32]
        lib.fsgp_model_compartments.restype = ctypes.c_int
        lib.fsgp_simulate.argtypes = [P, ctypes.c_int32, ctypes.POINTER(fsgp_params), P, P,
                                      ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.POINTER(fsgp_options), ctypes.POINTER(fsgp_result), P]
        lib.fsgp_simulate.restype = ctypes.c_int
        lib.fsgp_step_noalloc.argtypes = [ctypes.c_int32, ctypes.POINTER(fsgp_params), P, P,
                                          ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_uint32, ctypes.c_uint64, P, P, P, P]
        lib.fsgp_step_noalloc.restype = ctypes.c_int
        lib.fsgp_batch_run.argtypes = [ctypes.POINTER(fsgp_request), ctypes.c_int32,
                                       ctypes.POINTER(fsgp_batch_options), P]
        lib.fsgp_batch_run.restype = ctypes.c_int
        lib.fsgp_autotune.argtypes = [P, ctypes.c_int32, ctypes.POINTER(fsgp_params), P,
                                      ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.POINTER(fsgp_options), P]
        lib.fsgp_autotune.restype = ctypes.c_int
        lib.fsgp_surrogate_num_params.argtypes = []
        lib.fsgp_surrogate_num_params.restype = ctypes.c_int
        lib.fsgp_surrogate_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(P)]
        lib.fsgp_surrogate_create.restype = ctypes.c_int
        lib.fsgp_surrogate_destroy.argtypes = [P]
        lib.fsgp_surrogate_destroy.restype = ctypes.c_int
        lib.fsgp_surrogate_params.argtypes = [P, P, P]
        lib.fsgp_surrogate_params.restype = ctypes.c_int
        lib.fsgp_surrogate_forward.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_double,
                                               ctypes.c_double, P, P]
        lib.fsgp_surrogate_forward.restype = ctypes.c_int
        lib.fsgp_surrogate_grad.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_double,
                                            ctypes.c_double, P, P, P, P]
        lib.fsgp_surrogate_grad.restype = ctypes.c_int
        lib.fsgp_surrogate_train_step.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_double,
                                                  ctypes.c_double, P, ctypes.c_float, P, P]
        lib.fsgp_surrogate_train_step.restype = ctypes.c_int
        lib.fsgp_surrogate_screen.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_double, P, P]
        lib.fsgp_surrogate_screen.restype = ctypes.c_int
        lib.fsgp_hk.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, P, P,
                                ctypes.c_uint32, P]
        lib.fsgp_hk.restype = ctypes.c_int
        lib.fsgp_graph_set_arc_weights.argtypes = [P, P, ctypes.c_uint32, P]
        lib.fsgp_graph_set_arc_weights.restype = ctypes.c_int
        lib.fsgp_selftest_barrier.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P]
        lib.fsgp_selftest_barrier.restype = ctypes.c_int
        lib.fsgp_last_error.argtypes = []
        lib.fsgp_last_error.restype = ctypes.c_char_p
        lib.fsgp_version.argtypes = []
        lib.fsgp_version.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc):
    if rc != FSGP_OK:
        raise FsgpError(rc, load().fsgp_last_error().decode())


def _ptr(x):
    """Raw address of a torch tensor, numpy array or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- C-ABI mirrors

def fsgp_last_error() -> str:
    return load().fsgp_last_error().decode()


def fsgp_version() -> int:
    return load().fsgp_version()


def fsgp_model_compartments(model: int) -> int:
    c = load().fsgp_model_compartments(model)
    if c < 0:
        raise FsgpError(c, load().fsgp_last_error().decode())
    return c


def fsgp_model_planes(model: int) -> int:
    rc = load().fsgp_model_planes(model)
    if rc < 0:
        _check(rc)
    return rc


def fsgp_graph_create(row_ptr, col_idx, n: int, nnz: int, flags: int, stream=None):
    h = ctypes.c_void_p()
    _check(load().fsgp_graph_create(_ptr(row_ptr), _ptr(col_idx), n, nnz, flags,
                                    _stream_handle(stream), ctypes.byref(h)))
    return h


def fsgp_graph_destroy(h) -> None:
    _check(load().fsgp_graph_destroy(h))


def fsgp_graph_trim(h) -> None:
    _check(load().fsgp_graph_trim(h))


def fsgp_graph_info(h) -> dict:
    n = ctypes.c_int32()
    nnz = ctypes.c_int64()
    md = ctypes.c_int32()
    b = ctypes.c_int64()
    _check(load().fsgp_graph_info(h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(md),
                                  ctypes.byref(b)))
    return {"n": n.value, "nnz": nnz.value, "max_in_degree": md.value, "device_bytes": b.value}


def fsgp_simulate(h, model, params: fsgp_params, seed_nodes, seed_offsets, n_sets, seed_flags,
                  R, T, rng_seed, options: fsgp_options | None, result: fsgp_result,
                  stream=None) -> None:
    opt = ctypes.byref(options) if options is not None else None
    _check(load().fsgp_simulate(h, model, ctypes.byref(params), _ptr(seed_nodes),
                                _ptr(seed_offsets), n_sets, seed_flags, R, T,
                                ctypes.c_uint64(rng_seed), opt, ctypes.byref(result),
                                _stream_handle(stream)))


def fsgp_step_noalloc(model, params: fsgp_params, row_ptr, col_idx, n, nnz, R, t, rng_seed,
                      cur_planes, next_planes, plane_counts, stream=None) -> None:
    """One synchronous step with no device allocation (see include/fsgp.h): for callers
    that cannot call cudaMalloc.  All array arguments are device tensors."""
    _check(load().fsgp_step_noalloc(model, ctypes.byref(params), _ptr(row_ptr), _ptr(col_idx),
                                    n, nnz, R, t, ctypes.c_uint64(rng_seed), _ptr(cur_planes),
                                    _ptr(next_planes), _ptr(plane_counts),
                                    _stream_handle(stream)))


def hk(graph: Graph, h0, T: int, eps: float, stream=None):
    """Hegselmann-Krause opinion dynamics (fsgp_hk): h0 [R][n] float32 (numpy: host
    buffers, numpy results; torch CUDA tensor: device results).  Returns (h_T [R][n],
    changes [T+1] u64)."""
    import torch
    if isinstance(h0, np.ndarray):
        h0 = np.ascontiguousarray(np.atleast_2d(h0), dtype=np.float32)
        out = np.zeros_like(h0)
        changes = np.zeros(T + 1, dtype=np.uint64)
        flags = PTR_HOST
    else:
        if h0.dtype != torch.float32 or not h0.is_cuda:
            raise TypeError("h0 must be a float32 numpy array or a float32 CUDA tensor")
        h0 = h0.contiguous()
        if h0.dim() == 1:
            h0 = h0[None]
        out = torch.empty_like(h0)
        changes = torch.zeros(T + 1, dtype=torch.int64, device=h0.device)
        flags = PTR_DEVICE
    R, n = h0.shape
    if n != graph.n:
        raise ValueError(f"h0 has {n} columns, the graph {graph.n} nodes")
    _check(load().fsgp_hk(graph.handle, _ptr(h0), R, T, float(eps), _ptr(out), _ptr(changes), flags,
                          _stream_handle(stream)))
    return out, changes


def fsgp_graph_set_arc_weights(h, w, stream=None) -> None:
    if w is None:
        _check(load().fsgp_graph_set_arc_weights(h, None, PTR_HOST, _stream_handle(stream)))
        return
    if isinstance(w, np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32)
        flags = PTR_HOST
    else:
        import torch
        if w.dtype != torch.float32:
            raise TypeError("arc weights must be float32")
        w = w.contiguous()
        flags = PTR_DEVICE if w.is_cuda else PTR_HOST
    _check(load().fsgp_graph_set_arc_weights(h, _ptr(w), flags, _stream_handle(stream)))


def fsgp_selftest_barrier(ctas: int, missing: int, rounds: int, spin_cycles: int, stream=None) -> int:
    """Status of the grid-barrier self-test (FSGP_OK or FSGP_ETIMEOUT; other codes raise)."""
    rc = load().fsgp_selftest_barrier(ctas, missing, rounds, ctypes.c_int64(spin_cycles),
                                      _stream_handle(stream))
    if rc not in (FSGP_OK, FSGP_ETIMEOUT):
        _check(rc)
    return rc


def fsgp_batch_run(reqs, n, options: fsgp_batch_options | None = None, stream=None) -> None:
    opt = ctypes.byref(options) if options is not None else None
    _check(load().fsgp_batch_run(reqs, n, opt, _stream_handle(stream)))


def fsgp_autotune(h, model, params: fsgp_params, seed_nodes, n_seeds, R, T_probe, rng_seed,
                  options: fsgp_options, stream=None) -> None:
    _check(load().fsgp_autotune(h, model, ctypes.byref(params), _ptr(seed_nodes), n_seeds, R,
                                T_probe, ctypes.c_uint64(rng_seed), ctypes.byref(options),
                                _stream_handle(stream)))


# ----------------------------------------------------------- convenience layer

class Graph:
    """Owns an fsgp_graph handle built from an int32 in-CSR (numpy or torch)."""

    def __init__(self, row_ptr, col_idx, stream=None):
        import torch
        if isinstance(row_ptr, np.ndarray):
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
            col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
            flags = PTR_HOST
        else:
            if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
                raise TypeError("row_ptr and col_idx must be int32")
            row_ptr = row_ptr.contiguous()
            col_idx = col_idx.contiguous()
            flags = PTR_DEVICE if row_ptr.is_cuda else PTR_HOST
        self.n = int(row_ptr.shape[0] - 1)
        self.nnz = int(col_idx.shape[0])
        self.handle = fsgp_graph_create(row_ptr, col_idx if self.nnz else None, self.n, self.nnz,
                                        flags, stream)

    def info(self) -> dict:
        return fsgp_graph_info(self.handle)

    def trim(self) -> None:
        """Free the cached simulation workspace (fsgp_graph_trim)."""
        fsgp_graph_trim(self.handle)

    def set_arc_weights(self, w, stream=None) -> None:
        """Per-arc weights (float32, the caller's arc order) for weighted runs; None
        detaches them (fsgp_graph_set_arc_weights)."""
        fsgp_graph_set_arc_weights(self.handle, w, stream)

    def close(self):
        if getattr(self, "handle", None) is not None:
            fsgp_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_options(**kw) -> fsgp_options:
    o = fsgp_options()
    for k, v in kw.items():
        if k == "init_planes":
            o.init_planes = _ptr(v)
        elif k == "profile":
            o.profile = ctypes.pointer(v)
        else:
            setattr(o, k, v)
    return o


def simulate(graph: Graph, model: int, seed_sets, R: int, T: int, rng_seed: int, *, beta=0.0,
             gamma=0.0, ic_mode=IC_WEIGHTED_CASCADE, ic_p=0.0, alpha=0.0, mu=0.0, nu=0.0,
             weighted=False, freq=True, per_real=False, final_planes=False, steps_run=True, device=True,
             options=None, stream=None, out=None):
    """Run fsgp_simulate; results are torch tensors on the current CUDA device
    (device=True) or numpy arrays (device=False).  weighted: SIR/SIS/SI on the graph's
    arc weights (Graph.set_arc_weights)."""
    import torch
    n = graph.n
    if isinstance(seed_sets, np.ndarray) and seed_sets.ndim == 1:
        seed_sets = [seed_sets]
    n_sets = len(seed_sets)
    offs = np.zeros(n_sets + 1, dtype=np.int64)
    for i, s in enumerate(seed_sets):
        offs[i + 1] = offs[i] + len(s)
    seeds = np.concatenate([np.asarray(s, dtype=np.int32) for s in seed_sets]) if offs[-1] \
        else np.zeros(1, dtype=np.int32)
    P = fsgp_model_planes(model)
    C = fsgp_model_compartments(model)
    W = (R + 31) // 32
    T1 = T + 1
    if out is None:
        out = {}
        if device:
            dev = torch.device("cuda", torch.cuda.current_device())
            mk = lambda shape, dt: torch.zeros(shape, dtype=dt, device=dev)  # noqa: E731
            out["counts"] = mk((n_sets, T1, C), torch.int64)
            if freq:
                out["freq"] = mk((n_sets, C, n), torch.int32)
            if per_real:
                out["per_real"] = mk((n_sets, R, T1, C), torch.int32)
            if final_planes:
                out["final_planes"] = mk((n_sets, P, n, W), torch.int32)
            if steps_run:
                out["steps_run"] = mk((n_sets,), torch.int32)
        else:
            out["counts"] = np.zeros((n_sets, T1, C), dtype=np.uint64)
            if freq:
                out["freq"] = np.zeros((n_sets, C, n), dtype=np.uint32)
            if per_real:
                out["per_real"] = np.zeros((n_sets, R, T1, C), dtype=np.uint32)
            if final_planes:
                out["final_planes"] = np.zeros((n_sets, P, n, W), dtype=np.uint32)
            if steps_run:
                out["steps_run"] = np.zeros((n_sets,), dtype=np.int32)
    res = fsgp_result()
    res.flags = PTR_DEVICE if device else PTR_HOST
    res.counts = _ptr(out.get("counts"))
    res.freq = _ptr(out.get("freq"))
    res.per_real = _ptr(out.get("per_real"))
    res.final_planes = _ptr(out.get("final_planes"))
    res.steps_run = _ptr(out.get("steps_run"))
    prm = fsgp_params(beta=beta, gamma=gamma, ic_mode=ic_mode, ic_p=ic_p, alpha=alpha, mu=mu, nu=nu,
                      weighted=1 if weighted else 0)
    if isinstance(options, dict):
        options = make_options(**options)
    fsgp_simulate(graph.handle, model, prm, seeds, offs, n_sets, PTR_HOST, R, T, rng_seed,
                  options, res, stream)
    return out


def simulate_single(graph: Graph, model: int, seeds, r: int, T: int, rng_seed: int, *, beta=0.0,
                    gamma=0.0, ic_mode=IC_WEIGHTED_CASCADE, ic_p=0.0, weighted=False, final_state=True,
                    stream=None):
    """The plain single-instance path (fsgp_simulate_single) for realization r; returns
    device tensors counts [T+1][3] (int64), final_state [n] (uint8) and steps_run.
    (weighted=True is rejected: the path has no weighted graphs.)"""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    counts = torch.zeros((T + 1, 3), dtype=torch.int64, device=dev)
    fs = torch.zeros(graph.n, dtype=torch.uint8, device=dev) if final_state else None
    sr = torch.zeros(1, dtype=torch.int32, device=dev)
    prm = fsgp_params(beta=beta, gamma=gamma, ic_mode=ic_mode, ic_p=ic_p, weighted=1 if weighted else 0)
    _check(load().fsgp_simulate_single(graph.handle, model, ctypes.byref(prm),
                                       seeds.ctypes.data if seeds.size else None, seeds.size, PTR_HOST,
                                       r, T, rng_seed, _ptr(counts), _ptr(fs), _ptr(sr), PTR_DEVICE,
                                       _stream_handle(stream)))
    out = {"counts": counts, "steps_run": sr}
    if fs is not None:
        out["final_state"] = fs
    return out


def batch_run(requests, *, n_streams=0, capture_graph=0, autotune=0, stream=None):
    """Run a list of request dicts {graph: Graph, model, seeds, R, T, rng_seed, beta,
    gamma, ic_mode, ic_p, freq: bool, per_real: bool} as one batch.  Returns one dict of
    device result tensors per request."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    n = len(requests)
    arr = (fsgp_request * max(n, 1))()
    outs, keep = [], []
    for i, rq in enumerate(requests):
        g = rq["graph"]
        seeds = np.ascontiguousarray(rq.get("seeds", np.zeros(0, np.int32)), dtype=np.int32)
        keep.append(seeds)
        R, T, model = int(rq["R"]), int(rq["T"]), int(rq["model"])
        C = fsgp_model_compartments(model)
        o = {"counts": torch.zeros((1, T + 1, C), dtype=torch.int64, device=dev),
             "steps_run": torch.zeros((1,), dtype=torch.int32, device=dev)}
        if rq.get("freq", True):
            o["freq"] = torch.zeros((1, C, g.n), dtype=torch.int32, device=dev)
        if rq.get("per_real", False):
            o["per_real"] = torch.zeros((1, R, T + 1, C), dtype=torch.int32, device=dev)
        outs.append(o)
        q = arr[i]
        q.graph = g.handle
        q.model = model
        q.params = fsgp_params(beta=rq.get("beta", 0.0), gamma=rq.get("gamma", 0.0),
                               ic_mode=rq.get("ic_mode", IC_WEIGHTED_CASCADE), ic_p=rq.get("ic_p", 0.0),
                               alpha=rq.get("alpha", 0.0), mu=rq.get("mu", 0.0), nu=rq.get("nu", 0.0),
                               weighted=1 if rq.get("weighted", False) else 0)
        q.seed_nodes = seeds.ctypes.data if seeds.size else None
        q.n_seeds = int(seeds.size)
        q.R, q.T, q.rng_seed = R, T, int(rq["rng_seed"])
        q.result.flags = PTR_DEVICE
        q.result.counts = _ptr(o["counts"])
        q.result.freq = _ptr(o.get("freq"))
        q.result.per_real = _ptr(o.get("per_real"))
        q.result.steps_run = _ptr(o["steps_run"])
    bo = fsgp_batch_options(n_streams=n_streams, capture_graph=capture_graph, autotune=autotune)
    fsgp_batch_run(arr, n, bo, stream)
    return outs


class Surrogate:
    """Owns an fsgp_surrogate handle (thin wrapper over the fsgp_surrogate_* calls)."""

    def __init__(self, init_seed: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.fsgp_surrogate_create(ctypes.c_uint64(init_seed), ctypes.byref(h)))
        self.handle = h
        self.n_params = lib.fsgp_surrogate_num_params()

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().fsgp_surrogate_params(self.handle, out.ctypes.data, None))
        return out

    def set_params(self, theta) -> None:
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {t.size}")
        _check(load().fsgp_surrogate_params(self.handle, None, t.ctypes.data))

    def forward(self, graph, seeds, beta, gamma, stream=None):
        import torch
        seeds = np.ascontiguousarray(seeds, dtype=np.int32)
        p = torch.empty(graph.n, dtype=torch.float32, device="cuda")
        _check(load().fsgp_surrogate_forward(self.handle, graph.handle,
                                             seeds.ctypes.data if seeds.size else None,
                                             seeds.size, beta, gamma, _ptr(p),
                                             _stream_handle(stream)))
        return p

    def grad(self, graph, seeds, beta, gamma, y, stream=None):
        seeds = np.ascontiguousarray(seeds, dtype=np.int32)
        loss = ctypes.c_double(0.0)
        g = np.zeros(self.n_params, dtype=np.float32)
        _check(load().fsgp_surrogate_grad(self.handle, graph.handle,
                                          seeds.ctypes.data if seeds.size else None, seeds.size,
                                          beta, gamma, _ptr(y), ctypes.byref(loss), g.ctypes.data,
                                          _stream_handle(stream)))
        return loss.value, g

    def train_step(self, graph, seeds, beta, gamma, y, lr=1e-3, stream=None, want_loss=True):
        """One Adam step; returns the loss before the step (synchronising the stream), or
        None without a synchronisation when want_loss is False."""
        seeds = np.ascontiguousarray(seeds, dtype=np.int32)
        loss = ctypes.c_double(0.0)
        _check(load().fsgp_surrogate_train_step(self.handle, graph.handle,
                                                seeds.ctypes.data if seeds.size else None,
                                                seeds.size, beta, gamma, _ptr(y),
                                                ctypes.c_float(lr),
                                                ctypes.byref(loss) if want_loss else None,
                                                _stream_handle(stream)))
        return loss.value if want_loss else None

    def screen(self, graph, candidates, beta, gamma, stream=None) -> np.ndarray:
        c = np.ascontiguousarray(candidates, dtype=np.int32)
        n_cand, k = c.shape
        out = np.zeros(n_cand, dtype=np.float32)
        _check(load().fsgp_surrogate_screen(self.handle, graph.handle, c.ctypes.data, k, n_cand,
                                            beta, gamma, out.ctypes.data, _stream_handle(stream)))
        return out

    def close(self):
        if getattr(self, "handle", None) is not None:
            load().fsgp_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
