"""CPU oracle for batched Monte Carlo propagation (SIR, SIS, IC, LT, SI, SEIR, SEIS, SWIR).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path never imports
this package, and this package never imports the product package.

The arithmetic lives in ``fsgp_oracle.c`` (plain loops, threads over realizations);
this module compiles it with gcc and marshals numpy arrays through ctypes.

Paper anchors: Algorithm 1 (traditional propagation loop) gives the loop nest;
Sec. 3.1, Eqs. (all)/(ms)/(agg)/(updata) give the node-synchronous update; Appendix
A.1 gives the SIR rule; Eq. (batch) gives independent randomness per realization.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsgp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfsgp_oracle.so")
_lock = threading.Lock()
_lib = None

SIR, SIS, IC, LT = 0, 1, 2, 3
SI, SEIR, SEIS, SWIR = 4, 5, 6, 7
TAG_INFECT, TAG_RECOVER, TAG_IC_EDGE, TAG_LT_THRESH, TAG_LATENT, TAG_WEAKEN = 1, 2, 3, 4, 5, 6
IC_WEIGHTED_CASCADE, IC_CONSTANT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, pthreads)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32]
            lib.orc_uniform.restype = ctypes.c_uint32
            lib.orc_survival_table.argtypes = [ctypes.c_double, ctypes.c_int64, P]
            lib.orc_survival_table.restype = None
            lib.orc_prob_threshold.argtypes = [ctypes.c_double]
            lib.orc_prob_threshold.restype = ctypes.c_uint64
            lib.orc_simulate.argtypes = [
                ctypes.c_int, ctypes.c_int32, P, P, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, ctypes.c_double, P, ctypes.c_int64, ctypes.c_int32,
                ctypes.c_uint64, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                ctypes.c_int, P, P, P, P, P]
            lib.orc_simulate.restype = ctypes.c_int
            lib.orc_simulate_ext.argtypes = [
                ctypes.c_int, ctypes.c_int32, P, P, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                P, ctypes.c_int64, ctypes.c_int32,
                ctypes.c_uint64, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                ctypes.c_int, P, P, P, P, P]
            lib.orc_simulate_ext.restype = ctypes.c_int
            lib.orc_simulate_w.argtypes = [
                ctypes.c_int, ctypes.c_int32, P, P, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                P, P, ctypes.c_int64, ctypes.c_int32,
                ctypes.c_uint64, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                ctypes.c_int, P, P, P, P, P]
            lib.orc_simulate_w.restype = ctypes.c_int
            lib.orc_hk.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                   P, P, ctypes.c_int]
            lib.orc_hk.restype = ctypes.c_int
            lib.orc_compartments.argtypes = [ctypes.c_int]
            lib.orc_compartments.restype = ctypes.c_int
            lib.orc_node_step.argtypes = [
                ctypes.c_int, P, P, ctypes.c_int32, P, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32,
                ctypes.c_uint64]
            lib.orc_node_step.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Raw Philox4x32-10 block (Salmon et al., SC'11): 4 u32 counter words, 2 key words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(rng_seed: int, tag: int, a: int, t: int, r: int) -> int:
    """The 32-bit uniform of realization r for (tag, subject a, step t)."""
    return int(_load().orc_uniform(rng_seed, tag, a, t, r))


def survival_table(beta: float, kmax: int) -> np.ndarray:
    """surv[k] for k = 0..kmax (u64), surv[0] = 2^32."""
    out = np.zeros(kmax + 1, dtype=np.uint64)
    _load().orc_survival_table(float(beta), int(kmax), _ptr(out))
    return out


def prob_threshold(p: float) -> int:
    return int(_load().orc_prob_threshold(float(p)))


def compartments(model: int) -> int:
    """Compartments reported for a model: 4 for SEIR and SWIR, 3 otherwise."""
    return int(_load().orc_compartments(int(model)))


@dataclass
class OracleResult:
    counts: np.ndarray        # [T+1, C] u64 over the realizations run
    per_real: np.ndarray      # [n_real, T+1, C] u32
    freq: np.ndarray          # [C, n] u32
    final_state: np.ndarray   # [n_real, n] u8 (0/1/2)
    quiet_step: np.ndarray    # [n_real] i32 (IC/LT: first step with empty frontier)


def simulate(model: int, row_ptr, col_idx, seeds, *, beta=0.0, gamma=0.0,
             ic_mode=IC_WEIGHTED_CASCADE, ic_p=0.0, alpha=0.0, mu=0.0, nu=0.0, R=1, T=0,
             rng_seed=0, r_lo=0, n_real=None, init_state=None, t0=0, nthreads=None,
             outputs=("counts", "per_real", "freq", "final_state"), arc_weights=None) -> OracleResult:
    """Run realizations r_lo .. r_lo+n_real-1 of one seed set on the in-CSR graph.
    `outputs` limits which result arrays are produced (counts always are).  alpha is the
    SEIR/SEIS latent rate (E -> I); SWIR takes kappa = beta, mu and nu.  arc_weights
    (float32 per arc of col_idx, SIR/SIS/SI only): arc e infects with probability
    beta * w_e per step (weighted graphs)."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    n = int(row_ptr.shape[0] - 1)
    if n_real is None:
        n_real = R - r_lo
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    C = compartments(model)
    counts = np.zeros((T + 1, C), dtype=np.uint64)
    per_real = np.zeros((n_real, T + 1, C), dtype=np.uint32) if "per_real" in outputs else None
    freq = np.zeros((C, n), dtype=np.uint32) if "freq" in outputs else None
    final_state = np.zeros((n_real, n), dtype=np.uint8) if "final_state" in outputs else None
    quiet = np.zeros(n_real, dtype=np.int32)
    if init_state is not None:
        init_state = np.ascontiguousarray(init_state, dtype=np.uint8)
        assert init_state.shape == (n_real, n)
    w = None
    if arc_weights is not None:
        w = np.ascontiguousarray(arc_weights, dtype=np.float32)
        assert w.shape == (col_idx.shape[0],)
    rc = lib.orc_simulate_w(int(model), n, _ptr(row_ptr), _ptr(col_idx), float(beta),
                              float(gamma), int(ic_mode), float(ic_p), float(alpha), float(mu),
                              float(nu), _ptr(w), _ptr(seeds), int(seeds.shape[0]), int(T), int(rng_seed),
                              _ptr(init_state), int(t0), int(r_lo), int(n_real), int(nthreads),
                              _ptr(counts), _ptr(per_real), _ptr(freq), _ptr(final_state),
                              _ptr(quiet))
    if rc != 0:
        raise ValueError(f"orc_simulate failed with code {rc}")
    return OracleResult(counts, per_real, freq, final_state, quiet)


def node_step(model: int, row_ptr, col_idx, v: int, X, *, beta=0.0, gamma=0.0,
              ic_mode=IC_WEIGHTED_CASCADE, ic_p=0.0, t: int, r: int, rng_seed: int) -> int:
    """State of node v at absolute step t in realization r, given step-(t-1) states X."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    s = _load().orc_node_step(int(model), _ptr(row_ptr), _ptr(col_idx), int(v), _ptr(X),
                              float(beta), float(gamma), int(ic_mode), float(ic_p),
                              int(t), int(r), int(rng_seed))
    if s < 0:
        raise ValueError("orc_node_step failed")
    return s


def hk(row_ptr, col_idx, h0, T: int, eps: float, nthreads=None):
    """Hegselmann-Krause opinion dynamics (Appendix A.2) on the in-CSR graph: h0 is
    [R][n] (float32, one opinion vector per realization); returns (h_T [R][n] float32,
    changes [T+1] u64: (node, realization) pairs whose opinion changed at each step)."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    h0 = np.ascontiguousarray(np.atleast_2d(h0), dtype=np.float32)
    R, n = h0.shape
    assert n == row_ptr.shape[0] - 1
    out = np.zeros_like(h0)
    changes = np.zeros(T + 1, dtype=np.uint64)
    rc = lib.orc_hk(n, _ptr(row_ptr), _ptr(col_idx), _ptr(h0), R, int(T), float(np.float32(eps)), _ptr(out),
                    _ptr(changes), int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError(f"orc_hk failed with code {rc}")
    return out, changes

