/*
 * fsgp.h -- C ABI of the GB300 batched Monte Carlo graph propagation library.
 *
 * One library, libfsgp.so, hand-written CUDA for sm_103a.  It runs the synchronous,
 * batched Monte Carlo propagation step of FS_GPlib (arXiv 2603.14895) for the SIR,
 * SIS, Independent Cascade (IC) and Linear Threshold (LT) models:
 *   - node-synchronous update, every node reads the step-(k-1) states of itself and of
 *     its in-neighbours and writes its step-k state (Sec. 2, Eq. nodestate; Sec. 3.1,
 *     Eqs. all / ms / agg / updata);
 *   - R independent realizations batched along a lane axis (Sec. 3.1, Eq. batch), here
 *     bit-packed: lane r of a node lives in bit (r & 31) of 32-bit word (r >> 5);
 *   - the SIR rule of Appendix A.1 (two indicator vectors h, r -> two bit-planes).
 *
 * Conventions for every entry point
 *   - Return value: FSGP_OK (0) or a negative FSGP_E* code.  A human-readable message
 *     for the last failure of the calling thread is available from fsgp_last_error().
 *     No C++ exception crosses this boundary.
 *   - Pointers are plain host or device pointers as the flags say; no framework types.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).  Work
 *     is enqueued on that stream.  Calls that return results in host memory synchronise
 *     the stream before returning; calls that return results in device memory do not.
 *   - Thread safety: distinct graph handles may be used concurrently.  Calls that use
 *     the same graph handle must not overlap (the handle owns the simulation
 *     workspace).
 *
 * Integer randomness contract (shared by every path; identical results for every
 * tuning choice and for any split of realizations across GPUs):
 *   key = (lo32(rng_seed), hi32(rng_seed));  for tag tau, subject a, step t, lane r:
 *   P_j = Philox4x32-10(key, ctr = (a, t, r >> 5, (tau << 8) | (j >> 2)))[j & 3],
 *   j = 0..31, and bit (31 - j) of the 32-bit uniform u is bit (r & 31) of P_j.
 *   Tags: 1 infection (a = node), 2 recovery (a = node), 3 IC arc trial (a = position
 *   of the arc in the in-CSR column array), 4 LT threshold (a = node, t = 0).
 *   Philox4x32-10: Salmon, Moraes, Dror, Shaw, SC'11.
 *
 * Decision rules (integer readings of the paper; thresholds are built on the host):
 *   SIR/SIS infection of a susceptible lane with k >= 1 infected in-arcs:
 *     u >= surv[k], surv[0] = 2^32, surv[k] = floor(surv[k-1] * q / 2^32),
 *     q = 2^32 - llrint(beta * 2^32)  (probability 1-(1-beta)^k up to k * 2^-32).
 *   Recovery of an infected lane: u < llrint(gamma * 2^32).
 *   IC arc (w -> v) tried at the step after w activates, if v is inactive:
 *     weighted cascade: u * d_in(v) < 2^32; constant: u < llrint(p * 2^32).
 *   LT: theta = u(tag 4, v, t = 0); an inactive lane with k >= 1 active in-arcs
 *     activates iff k * 2^32 >= theta * d_in(v).
 *   In-arcs count with multiplicity (duplicate arcs and self-loops are kept).
 */
#ifndef FSGP_H
#define FSGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define FSGP_OK 0
#define FSGP_EINVAL (-1)          /* an argument is out of range or inconsistent */
#define FSGP_ENOMEM (-2)          /* device or host allocation failed */
#define FSGP_ECUDA (-3)           /* a CUDA runtime call failed (message has details) */
#define FSGP_ETIMEOUT (-4)        /* a bounded device-side wait ran out (a grid barrier of the
                                     persistent step loop, or the surrogate's tensor-core
                                     completion wait) */
#define FSGP_EUNSUPPORTED (-5)    /* a valid request this library version does not implement */

/* ------------------------------------------------------------------------ models */
#define FSGP_SIR 0   /* planes: 0 = I (infected), 1 = R (recovered) */
#define FSGP_SIS 1   /* planes: 0 = I */
#define FSGP_IC 2    /* planes: 0 = A (active), 1 = F (activated at the last step) */
#define FSGP_LT 3    /* planes: 0 = A, 1 = F */
/* The discrete-time epidemic rows of Table 1 (named there; the rules are this library's
 * reading, k = in-arcs whose source is infectious, counted with multiplicity):
 *   SI: SIR without recovery.
 *   SEIR(DT): S -> E iff u >= surv_beta[k]; E -> I iff u(tag 5) < llrint(alpha * 2^32);
 *     I -> R iff u(tag 2) < llrint(gamma * 2^32).  SEIS(DT): the same with I -> S.
 *   SWIR: S -> I iff u >= surv_kappa[k] (kappa = beta), else S -> W iff u(tag 6) >=
 *     surv_mu[k]; W -> I iff u >= surv_nu[k]; I -> R after one step.
 *   One change per node, lane and step, from the state of the previous step. */
#define FSGP_SI 4    /* planes: 0 = I */
#define FSGP_SEIR 5  /* planes: 0 = I, 1 = R, 2 = E (exposed) */
#define FSGP_SEIS 6  /* planes: 0 = I, 1 = E */
#define FSGP_SWIR 7  /* planes: 0 = I, 1 = R, 2 = W (weakened) */

/* Compartments reported in counts / freq / per-realization counts (C per model, see
 * fsgp_model_compartments), in this order:
 *   SIR: S, I, R.  SIS and SI: S, I, 0.  IC and LT: inactive, newly active (F), active
 *   before the last step (A and not F).  SEIR: S, E, I, R.  SEIS: S, E, I.
 *   SWIR: S, W, I, R. */

/* ------------------------------------------------------------------------- flags */
#define FSGP_PTR_HOST 0u
#define FSGP_PTR_DEVICE 1u

#define FSGP_IC_WEIGHTED_CASCADE 0   /* arc probability 1 / d_in(target) */
#define FSGP_IC_CONSTANT 1           /* arc probability ic_p */

/* Opaque graph handle: owns a device copy of the in-CSR, its out-CSR, the degree
 * classes used to schedule rows, and the simulation workspace. */
typedef struct fsgp_graph fsgp_graph;

typedef struct {
    double beta;      /* per-arc infection probability (SWIR: kappa), [0, 1] */
    double gamma;     /* recovery probability, [0, 1] */
    int32_t ic_mode;  /* FSGP_IC_WEIGHTED_CASCADE or FSGP_IC_CONSTANT */
    double ic_p;      /* IC constant arc probability, [0, 1] */
    double alpha;     /* SEIR/SEIS: exposed -> infectious probability per step, [0, 1] */
    double mu;        /* SWIR: per-arc weakening probability, [0, 1] */
    double nu;        /* SWIR: per-arc infection probability of a weakened node, [0, 1] */
    int32_t weighted; /* SIR, SIS, SI: 1 = weighted graph (Table 1's edge weights): each
                         infectious in-arc e transmits independently with probability
                         beta * w_e per step (w from fsgp_graph_set_arc_weights), drawn per
                         arc (tag 7, keyed by e's position in col_idx, the step and the
                         realization): u < thr_e with p = (float)beta * w_e in single
                         precision, thr_e = 0 if p <= 0, 2^32 if p >= 1, else
                         round(p * 2^32).  0 = the unweighted rule.  Not supported by
                         fsgp_simulate_single and fsgp_step_noalloc (EUNSUPPORTED). */
} fsgp_params;

/* Optional per-kernel profile of one fsgp_simulate call (host struct).  Device times
 * come from CUDA events recorded around every launch on the call's stream; the call
 * synchronises that stream before returning when a profile is requested.  Algorithmic
 * bytes are the bytes each launch is required to move by the method's definition for
 * the rows it processed: 8 B of row pointers, the node's own state words read and
 * written (planes x 4 B x words), and per gathered in-arc 4 B of column index plus one
 * 32-byte sector (or more, for R > 256) of the source's state words. */
#define FSGP_PROF_KINDS 10
/* kinds: 0 init, 1 step control, 2 frontier marking, 3 hub chunks, 4 hub finalize,
 *        5 warp-per-row rows, 6 team-per-row rows (16..255 in-arcs, and every small row
 *        of a frontier step), 7 results, 8 team-per-row rows (4..15 in-arcs),
 *        9 thread-per-row rows (0..3 in-arcs) */
typedef struct {
    int64_t launches[FSGP_PROF_KINDS];
    double ms[FSGP_PROF_KINDS];
    double alg_bytes[FSGP_PROF_KINDS];
    int64_t dense_steps;
    int64_t sparse_steps;
    int64_t kernel_launches;   /* every kernel this library launched for the call */
} fsgp_profile;

/* Tuning and run options.  Zero-initialised = defaults.  No tuning field changes any
 * result bit; fsgp_autotune() picks the tuning fields. */
typedef struct {
    int32_t vector_words;   /* 32-bit state words per thread: 1, 2 or 4 (0 = auto: 2) */
    int32_t small_max_deg;  /* rows with in-degree <= this: one thread team per row;
                               rounded down to 2^k - 1 (0 = auto) */
    int32_t hub_min_deg;    /* rows with in-degree >= this: split over CTAs; rounded down
                               to a power of two (0 = auto) */
    int32_t hub_chunk;      /* arcs per CTA for split rows (0 = auto) */
    double sparse_frac;     /* take the frontier path when the out-arcs of the rows that
                               push are at most sparse_frac * nnz (0 = auto, <0 = never) */
    int32_t r_offset;       /* global realization index of lane 0 (multiple of 32) */
    int32_t t0;             /* absolute index of the starting step (resume) */
    const uint32_t *init_planes; /* optional start state instead of seeds,
                               [n_sets][planes][n][ceil(R/32)] u32, same memory kind
                               as the result buffers (fsgp_result.flags) */
    fsgp_profile *profile;  /* optional host struct, accumulated (not cleared) */
    int32_t capture_graph;  /* 1: capture the step loop of each launch wave into a CUDA
                               graph and launch it at once (ignored when profiling) */
    int32_t lane_words;     /* words per thread of the one-thread-per-row kernel (rows with
                               1..3 in-arcs): 1, 2, 4 or 8 (0 = auto) */
    int32_t fuse_rows;      /* 1: every row in one kernel per step (team per row when every
                               in-degree is <= 255, else warp per row), dense steps only,
                               for small graphs whose steps are bound by launch latency;
                               needs in-degree < 65536; -1: never; 0: auto (graphs of at
                               most 2^20 state words per plane, when no degree-class or
                               frontier field is set) */
    int32_t persistent;     /* fused team-per-row mode: 0 (auto) or 1 runs all T steps in one
                               cooperative launch, steps separated by grid barriers, when
                               per-realization counts and profiling are off and each thread
                               takes one word; every barrier wait is bounded (about a second)
                               and one that runs out ends the run: steps_run = -1 (device
                               results) or FSGP_ETIMEOUT (host results); -1: never */
    int32_t reserved[4];
} fsgp_options;

/* Caller-owned result buffers, all host or all device (flags).  NULL = not wanted,
 * except counts.  W = ceil(R / 32). */
typedef struct {
    uint32_t flags;          /* FSGP_PTR_HOST or FSGP_PTR_DEVICE */
    uint64_t *counts;        /* [n_sets][T+1][C]: compartment totals over all lanes */
    uint32_t *freq;          /* [n_sets][C][n]: per-node final compartment frequency */
    uint32_t *per_real;      /* [n_sets][R][T+1][C]: per-realization compartment counts */
    uint32_t *final_planes;  /* [n_sets][planes][n][W]: final state bit-planes */
    int32_t *steps_run;      /* [n_sets]: transitions computed (IC/LT stop at the first
                                step that activates nothing; later rows repeat); -1: a
                                bounded wait of the persistent step loop ran out and the
                                other results are not valid */
} fsgp_result;

/* Create a graph from an int32 in-CSR: row v lists the sources u of arcs u -> v
 * (pulling from in-neighbours, Sec. 2 paradigm definition; CSR definition of Sec. 2).
 *   row_ptr: n+1 entries, row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *   col_idx: nnz entries in [0, n).  The column order is kept: IC draws are keyed by
 *            the position of an arc in this array.
 *   flags:   FSGP_PTR_HOST or FSGP_PTR_DEVICE for both arrays (copied; the caller
 *            keeps ownership of its arrays).
 *   1 <= n < 2^31 - 1, 0 <= nnz < 2^31.
 * On success *out receives a handle released by fsgp_graph_destroy.  Errors: EINVAL for
 * a malformed CSR (checked on the device), ENOMEM, ECUDA.  Synchronises the stream. */
int fsgp_graph_create(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                      int64_t nnz, uint32_t flags, void *stream, fsgp_graph **out);

/* Release a graph and its workspace (NULL is accepted).  Synchronises the device. */
int fsgp_graph_destroy(fsgp_graph *g);

/* Free the graph's cached simulation workspace (state planes, lists, counters), which
 * fsgp_simulate / fsgp_batch_run keep between calls and grow to the largest run seen;
 * the next run allocates it again.  Useful when many graphs stay alive.  Synchronises
 * the device.  Errors: EINVAL (NULL), ECUDA. */
int fsgp_graph_trim(fsgp_graph *g);

/* Attach per-arc weights to graph g for weighted runs (fsgp_params.weighted): w[e] is
 * the weight of arc e of the col_idx given to fsgp_graph_create (the caller's arc
 * order), finite and >= 0; flags says whether w is host or device memory.  The graph
 * keeps a device copy (4 bytes per arc) until it is destroyed or w is NULL (detach).
 * Synchronises `stream`.  Errors: EINVAL (a weight negative, NaN or infinite: nothing
 * changes), ENOMEM, ECUDA. */
int fsgp_graph_set_arc_weights(fsgp_graph *g, const float *w, uint32_t flags, void *stream);

/* Query sizes: any output pointer may be NULL. */
int fsgp_graph_info(const fsgp_graph *g, int32_t *n, int64_t *nnz, int32_t *max_in_degree,
                    int64_t *device_bytes);

/* Number of state bit-planes of a model (1 for SIS and SI; 2 for SIR, IC, LT, SEIS;
 * 3 for SEIR and SWIR), or EINVAL. */
int fsgp_model_planes(int32_t model);

/* Number of compartments C a model reports (4 for SEIR and SWIR, 3 otherwise), or EINVAL. */
int fsgp_model_compartments(int32_t model);

/* Run R realizations of `model` for T synchronous steps from each of n_sets seed sets
 * (paper API: run_epochs(epochs = R, times = T), Sec. 4.2.1).
 *   seed_nodes/seed_offsets: set s is seed_nodes[seed_offsets[s] .. seed_offsets[s+1]);
 *     seed_offsets has n_sets+1 entries and is always a HOST array; seed_nodes is host
 *     or device per seed_flags.  Duplicate seeds are allowed.  All R lanes of a set
 *     start from the same seeds (I for SIR/SIS, A = F for IC/LT).  Ignored when
 *     opt->init_planes is set.
 *   1 <= R <= 4096, 0 <= T, n_sets >= 1, probabilities in [0, 1].
 *   opt may be NULL (defaults).  out->counts must be non-NULL.
 * Errors: EINVAL, ENOMEM, ECUDA.  Results land in caller buffers; see fsgp_result. */
int fsgp_simulate(const fsgp_graph *g, int32_t model, const fsgp_params *params,
                  const int32_t *seed_nodes, const int64_t *seed_offsets, int32_t n_sets,
                  uint32_t seed_flags, int32_t R, int32_t T, uint64_t rng_seed,
                  const fsgp_options *opt, fsgp_result *out, void *stream);

/* The plain single-instance path: ONE realization (global index r, any r >= 0) with one
 * byte of state per node and no bit packing, the per-node update of Sec. 2 (Eq.
 * nodestate) run as it is written.  Its draws are those of lane r of fsgp_simulate, so
 * its states and counts equal that lane's exactly; it exists as the baseline the packed
 * path is measured against.
 *   seed_nodes: n_seeds nodes, host or device per seed_flags.
 *   counts:      [T+1][3] u64 compartment counts (required).
 *   final_state: [n] u8 state after the run, 0/1/2 as in the compartment table (optional).
 *   steps_run:   transitions computed (IC/LT stop at the first step that activates
 *                nothing; later rows repeat), optional.
 *   All outputs host or all device per out_flags.  Synchronises the stream.
 * Errors: EINVAL (bad arguments, seed out of range), ENOMEM, ECUDA. */
int fsgp_simulate_single(const fsgp_graph *g, int32_t model, const fsgp_params *params,
                         const int32_t *seed_nodes, int64_t n_seeds, uint32_t seed_flags,
                         int32_t r, int32_t T, uint64_t rng_seed, uint64_t *counts,
                         uint8_t *final_state, int32_t *steps_run, uint32_t out_flags,
                         void *stream);

/* One request of a batch (fsgp_batch_run). */
typedef struct {
    const fsgp_graph *graph;
    int32_t model;
    fsgp_params params;
    const int32_t *seed_nodes;   /* host array of n_seeds nodes (all R lanes start there) */
    int64_t n_seeds;
    int32_t R;                   /* 1..4096 realizations (lanes 0..R-1) */
    int32_t T;
    uint64_t rng_seed;
    fsgp_result result;          /* device buffers only: result.flags = FSGP_PTR_DEVICE;
                                    one set, layouts as in fsgp_result */
} fsgp_request;

typedef struct {
    int32_t n_streams;      /* concurrent CUDA streams, one host thread each (0 = 4) */
    int32_t capture_graph;  /* 0 (default) or 1: capture each launch wave's step loop into
                               a CUDA graph; -1: launch kernels one by one */
    int32_t autotune;       /* 1: run fsgp_autotune once per graph before its requests and
                               keep its choice on the graph; 0: use the choice an earlier
                               call kept, if any, else the automatic defaults */
    int32_t reserved[8];
} fsgp_batch_options;

/* Run many requests over a pool of graphs (batched Monte Carlo, Sec. 3.1, Eq. batch,
 * across requests).  Requests on the same graph with the same model, IC mode and T run
 * side by side in one launch sequence; each request keeps its own key, thresholds and
 * lanes, so its results equal those of an fsgp_simulate call for it alone.  Graphs are
 * spread over n_streams streams (longest first onto the least loaded), each issued by
 * its own host thread.  Work is ordered after prior work on `stream`, and `stream`
 * waits for all of it; the call returns once everything is enqueued.  A graph may
 * appear in several requests but must not be used by other calls meanwhile.  Small
 * graphs run the launched step loop, never the persistent one (the streams share the
 * GPU's SMs, which a cooperative grid would have to wait for).
 * Errors: EINVAL (any bad request: nothing is run), ENOMEM, ECUDA. */
int fsgp_batch_run(const fsgp_request *reqs, int32_t n, const fsgp_batch_options *opt,
                   void *stream);

/* Pick the tuning fields of *inout (vector_words, small_max_deg, hub_min_deg,
 * hub_chunk) for graph g by timing short probe runs (T_probe steps from the given host
 * seed set) of *inout as given (its automatic choices, such as the fused small-graph
 * mode, which explicit bounds turn off) and of every candidate: words per thread
 * {1, 2, 4}, team-row bound {63, 255}, split-row bound {4096, 8192, 16384}.  *inout is
 * left unchanged when it is fastest.  Every candidate gives identical results; only
 * speed differs.  Synchronises `stream`.  Errors: EINVAL, ENOMEM, ECUDA. */
int fsgp_autotune(const fsgp_graph *g, int32_t model, const fsgp_params *params,
                  const int32_t *seed_nodes, int64_t n_seeds, int32_t R, int32_t T_probe,
                  uint64_t rng_seed, fsgp_options *inout, void *stream);

/* ------------------------------------------------------------ learned surrogate
 * The paper has no learned component.  This 3-layer message-passing network predicts
 * each node's probability of being infected by the end of a run from the seed set and
 * (beta, gamma), to screen many candidate seed sets before Monte Carlo re-scores the
 * best; plain Monte Carlo (fsgp_simulate) makes the final decision.
 *   x_v = [seed_v, beta, gamma, log(1+d_in), log(1+d_out), log(1+k_v), 0, 0], k_v = in-arcs
 *         of v from seeds (a seed listed twice counts twice)
 *   h'_v = ReLU(h_v Ws_l + mean_{u->v} h_u Wn_l + b_l), l = 1..3, width 64
 *   p_v = sigmoid(h3_v . w_o + b_o);  loss = mean_v (p_v - y_v)^2
 * Dense products run on the tensor cores with bfloat16 operands and float32 accumulation;
 * training keeps float32 master weights and Adam state.  Parameters are one float32
 * vector: Ws1[8x64] Wn1[8x64] b1[64] Ws2[64x64] Wn2[64x64] b2 Ws3 Wn3 b3 wo[64] bo[1]
 * (row-major, rows = input features). */
typedef struct fsgp_surrogate fsgp_surrogate;

int fsgp_surrogate_num_params(void);
/* He-normal weights from a SplitMix64 stream seeded by init_seed, zero biases. */
int fsgp_surrogate_create(uint64_t init_seed, fsgp_surrogate **out);
int fsgp_surrogate_destroy(fsgp_surrogate *s);
/* Copy the float32 parameters out (get_host) and/or in (set_host; resets Adam). */
int fsgp_surrogate_params(fsgp_surrogate *s, float *get_host, const float *set_host);
/* Per-node probabilities p_out (device, n floats) for one seed set (host array). */
int fsgp_surrogate_forward(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *seeds_host,
                           int64_t n_seeds, double beta, double gamma, float *p_out, void *stream);
/* Loss and gradient for targets y (device, n floats); outputs are host pointers (either
 * may be NULL).  Synchronises the stream. */
int fsgp_surrogate_grad(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *seeds_host,
                        int64_t n_seeds, double beta, double gamma, const float *y,
                        double *loss_out, float *grad_out, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on one sample;
 * loss_out (host, may be NULL) receives the loss before the step. */
int fsgp_surrogate_train_step(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *seeds_host,
                              int64_t n_seeds, double beta, double gamma, const float *y,
                              float lr, double *loss_out, void *stream);
/* Scores (sum over nodes of p) of n_cand candidate seed sets of k nodes each
 * (cand_host[n_cand][k]) into scores_out (host, n_cand floats).  One CUDA graph per call
 * is replayed once per candidate.  Synchronises the stream. */
int fsgp_surrogate_screen(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *cand_host,
                          int32_t k, int32_t n_cand, double beta, double gamma, float *scores_out,
                          void *stream);

/* One synchronous step (Eq. nodestate) of `model` that allocates no device memory.
 * The paper has no counterpart.  It serves callers that cannot call cudaMalloc: a
 * process that has handed its free device memory to its own pool up front (a serving
 * process with a fixed memory budget), or an embedding runtime that forbids device
 * allocation on its hot path.  It needs no graph handle.
 *   row_ptr, col_idx: device in-CSR as for fsgp_graph_create (not validated here).
 *   cur_planes: device input state, next_planes: device output state (must not alias),
 *     both [planes][n][Ws] u32 with Ws = the smallest power of two >= ceil(R/32);
 *     padding words and lanes >= R must be zero in cur_planes.
 *   t: absolute index of the step computed (the Philox counter; IC/LT apply no stop
 *     rule to a single step).  Lanes are realizations 0..R-1.
 *   plane_counts: device u64[2], set lanes of each plane of next_planes.
 *   Results equal those of fsgp_simulate run for one step from the same planes.
 * Every row takes the CTA-split path: per-lane partial counts of each row meet in a
 * scratch array that is a fixed 32 MiB device array inside the library, held by every
 * GPU that loads the library until the process exits.  Limits, checked before any
 * work (EINVAL with a message): n * 128 * Ws bytes plus about 1.1 MB of tables must fit
 * the 32 MiB; for SIR/SIS the in-degree may not exceed 65536 unless the survival table
 * reaches zero earlier (beta not tiny).  The first call on a device, with that device
 * current, looks up the array's device address (cudaGetSymbolAddress) and keeps it for
 * the process: make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) invalidates the kept address, so do not call this entry point after
 * one.  Every call shares the array and clears the part it uses; calls that overlap on
 * the GPU race, so order them (one stream, or events).  The call reads the chunk count
 * back to the host and therefore synchronises `stream` once.  Errors: EINVAL, ECUDA. */
int fsgp_step_noalloc(int32_t model, const fsgp_params *params, const int32_t *row_ptr,
                      const int32_t *col_idx, int32_t n, int64_t nnz, int32_t R, uint32_t t,
                      uint64_t rng_seed, const uint32_t *cur_planes, uint32_t *next_planes,
                      uint64_t *plane_counts, void *stream);

/* Hegselmann-Krause opinion dynamics (Appendix A.2; Table 1's continuous HK row): R
 * independent opinion vectors (realizations), updated synchronously for T steps.  At
 * each step node i takes the mean of the opinions h_j of its in-neighbours j (Sec. 2's
 * N^-(i); arcs with multiplicity; i itself only through a self-loop) with
 * |h_i - h_j| < eps (strict, as in the appendix's message definition); with no such
 * neighbour it keeps its opinion (the appendix's NaN case).  Single precision: eps is
 * rounded to float, the sum is taken in col_idx order and divided once, so results are
 * exactly those of that sequential loop.  No randomness.
 *   h0: [R][n] float32 start opinions (finite), h_out: [R][n] float32 opinions after T
 *     steps, changes: optional [T+1] u64, (node, realization) pairs whose opinion
 *     changed at step k (changes[0] = 0); all three host or all device (flags).
 * Uses the graph's workspace (4 * n * ceil(R/32) * 32 bytes, twice): the graph must not
 * be used by another call meanwhile.  Host buffers: synchronises `stream`.
 * Errors: EINVAL (eps negative or not finite, an opinion not finite, R outside
 * [1, 4096], T < 0), ENOMEM, ECUDA. */
int fsgp_hk(const fsgp_graph *g, const float *h0, int32_t R, int32_t T, double eps, float *h_out,
            uint64_t *changes, uint32_t flags, void *stream);

/* Self-test of the bounded grid barrier that separates the steps of the persistent step
 * loop (fsgp_options.persistent; a systems pattern, not in the paper).  Launches `ctas`
 * co-resident CTAs (cooperative launch) that pass the barrier `rounds` times; the barrier
 * expects ctas + missing CTAs, so with missing > 0 no round completes and every wait runs
 * out after spin_cycles SM clock cycles.  Returns FSGP_OK if every round completed,
 * FSGP_ETIMEOUT if a wait ran out (the device stays usable), FSGP_EINVAL for sizes out of
 * range (ctas beyond the CTAs that fit at once included).  Allocates 16 bytes of device
 * memory for the call; synchronises `stream`. */
int fsgp_selftest_barrier(int32_t ctas, int32_t missing, int32_t rounds, int64_t spin_cycles, void *stream);

/* Message for the last failure on the calling thread ("" if none).  The pointer stays
 * valid until the next fsgp_* call on this thread. */
const char *fsgp_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int fsgp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FSGP_H */
