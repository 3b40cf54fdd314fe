// step.cuh -- device side of one synchronous propagation step.
//
// Paper anchors: node-synchronous update (Sec. 3.1, Eqs. ms / agg / updata): the
// message of an in-arc is the source's step-(k-1) state, aggregation counts infected
// (SIR/SIS) or active (LT) in-arcs per realization, or ORs the live arcs (IC), and the
// update draws the uniforms of Appendix A.1.  Batched Monte Carlo (Eq. batch): 32
// realizations per 32-bit word, one bit per lane, one plane per indicator vector.
//
// Work decomposition (GB300-specific, not from the paper):
//   * several seed sets (or batched requests) can run side by side: set s owns words
//     [s*Ws, (s+1)*Ws) of every node, with its own randomness key, thresholds and
//     valid-lane mask, so each set's result equals a run of that set alone;
//   * a "team" of TEAM threads covers a slice of TEAM*V words of one node, V words per
//     thread (64-bit loads when V = 2, 128-bit when V = 4); a node of Wn = S*Ws words
//     has Wn / (TEAM*V) slices, each an independent work item;
//   * small rows: one team per row (a warp holds 32/TEAM rows of similar degree, the
//     rows come bucketed by degree);
//   * mid rows: one warp per row, arcs interleaved over the warp's teams, counters
//     merged with xor-shuffles;
//   * hub rows: arcs cut into chunks, one CTA per chunk; per-lane counts meet in a
//     scratch array and a finalize pass makes the decisions.
//   In-arc counts are bit-sliced: counter bit b of 32 lanes is one word, so one
//   LOP3-style full adder adds 32 lanes at once.
#pragma once

#include "fsgp_internal.cuh"

#include <vector>

namespace fsgp {

// Control block in device memory, one per simulation.
struct Ctl {
    int32_t stop;          // IC/LT: an earlier step activated nothing
    int32_t steps_done;    // transitions computed so far (relative to t0)
    int32_t sparse;        // the current step runs on the frontier lists
    int32_t err;           // a bounded wait of the persistent step loop ran out
    uint32_t list_n[2];    // rows listed for the next step (by step parity)
    uint64_t push_outdeg[2];
    uint32_t cand_n[2];    // sparse candidates: 0 = small rows, 1 = mid rows
    int32_t dense_steps;   // steps run on the full row lists
    int32_t sparse_steps;  // steps run on the frontier lists
    int32_t build_list;    // the current step lists its rows for the next step
    int32_t list_valid[2]; // the list of that parity was built
    uint32_t d0_n;         // rows without in-arcs listed by the step-0 scan (d0_list)
    uint32_t bar_count;    // persistent step loop: CTAs arrived at the grid barrier
    uint32_t bar_gen;      // persistent step loop: barrier generation
};

// The persistent step loop of a small graph (one launch for all T steps): the per-step
// fields of StepArgs, and the bound on each grid-barrier wait.
struct PersistArgs {
    uint32_t *buf0, *buf1;         // state buffers (step k reads buf[(k-1)&1], writes buf[k&1])
    unsigned long long *pc;        // [T+1][S][kPC]; rows 1..T are zero on entry and receive
                                   // each step's changes (running totals formed afterwards)
    int32_t T;
    uint32_t t0;
    long long spin_limit;          // SM clock cycles one barrier wait may last
};

// Per-set parameters (device array, one entry per set of the launch).
struct SetParams {
    uint32_t key0, key1;            // rng seed
    const uint64_t *surv;           // survival table (SIR/SIS)
    int32_t ksat;                   // first k with surv[k] = 0, or INT32_MAX
    int32_t W;                      // words holding valid lanes, ceil(R/32)
    uint32_t last_mask;             // valid lanes of word W-1
    int32_t R;
    uint64_t g_rec;                 // recovery threshold
    uint64_t p_const;               // IC constant threshold
    uint64_t a_lat;                 // SEIR/SEIS: exposed -> infectious threshold
    const uint64_t *surv_mu;        // SWIR: weakening survival table, and its K_sat
    int32_t ksat_mu;
    const uint64_t *surv_nu;        // SWIR: survival table of weakened lanes, and its K_sat
    int32_t ksat_nu;
    float beta_f;                   // weighted graphs: beta in single precision
};

// Running plane popcounts are kept for up to three planes per set.
constexpr int kPC = 3;

// Row ids are "new ids": the graph's rows relabelled in degree-bucket order (row i of
// the state planes is node orig[i]).  Random draws are keyed by the node (Philox subject)
// and, for IC, by the arc's position in the caller's column array, so relabelling changes
// no result bit.  A null orig / pos means the identity (callers without a graph handle).
struct StepArgs {
    // graph, new ids
    const int32_t *__restrict__ rp;      // [n+1] in-CSR row pointers
    const int32_t *__restrict__ col;     // [nnz] sources
    const int32_t *__restrict__ orig;    // [n] node of new row i, or null
    const int32_t *__restrict__ pos;     // [n] new id of node v, or null
    const int32_t *__restrict__ arc0;    // [n] caller's position of new row i's first arc
    const int32_t *__restrict__ out_ptr; // caller's out-CSR (nodes), frontier marking
    const int32_t *__restrict__ out_dst;
    int32_t n;
    int32_t Ws;            // words per set (power of two)
    int32_t ws_shift;      // log2(Ws)
    int32_t S;             // sets in this launch
    int32_t Wn;            // words per node = S * Ws
    int32_t nslices;       // work items per row = Wn / (TEAM * V)
    uint32_t gbase;        // global word index of word 0 of a set (realization offset / 32)
    int32_t small_max_deg; // 2^k - 1
    int32_t hub_min_deg;   // power of two
    // state: [planes][n][Wn] per buffer
    const uint32_t *__restrict__ cur;
    uint32_t *__restrict__ nxt;
    size_t plane_words;    // n * Wn
    // model parameters
    const SetParams *__restrict__ sp;   // [S]
    int32_t ic_mode;
    uint32_t t;            // absolute step index of the step being computed
    int32_t k;             // relative step index (1..T)
    // control and accumulators
    Ctl *ctl;
    unsigned long long *pc;        // [S][kPC] plane popcounts of this step (running totals)
    int32_t *lane_cnt;             // [planes][Wn*32] running per-lane plane counts, or null
    int32_t np;                    // planes of the model
    // dense steps: row classes as new-id ranges: small rows by in-degree class (16..,
    // 4..15, 1..3), mid rows; rows without in-arcs only through d0_list
    int32_t r_small, n_small, r_small4, n_small4, r_lane, n_lane, r_mid, n_mid;
    int32_t r_d0;                              // first row without in-arcs
    const int4 *__restrict__ lane_tab;         // aligned with [r_lane, r_lane + n_lane)
    int32_t *d0_list;                          // rows without in-arcs whose state can
                                               // change (listed at step 0), ctl->d0_n
    int32_t *cand_small;
    int32_t *cand_mid;
    uint32_t *bitmap;
    const int32_t *__restrict__ list_in;   // rows listed by the previous step
    int32_t *list_out;                     // rows listed for the next step
    // hubs: new ids 0 .. n_hubs-1
    const int64_t *__restrict__ hub_chunk_base;
    int32_t n_hubs;
    int64_t n_hub_chunks;
    int32_t hub_chunk;
    uint32_t *hub_scratch;          // [n_hubs][Wn*32] per-lane counts (IC: [n_hubs][Wn] masks)
    uint32_t *hub_sat;              // SIR/SIS: [n_hubs][nslices] the slice's susceptible lanes
                                    // all reached K_sat within the row's first chunk, or null
    unsigned long long *prof_bytes; // [FSGP_PROF_KINDS] algorithmic bytes per kind, or null
    const float *__restrict__ arc_w; // weighted graphs: [nnz] weights in the caller's arc order
};

// Weighted graphs: transmission threshold of the arc at caller position epos for a lane
// of set s.  p = beta * w_e in single precision; 0 if p <= 0, 2^32 (certain) if p >= 1,
// else round(p * 2^32) (the scaling by 2^32 is exact).
__device__ __forceinline__ uint64_t arc_threshold(const StepArgs &A, int s, int64_t epos) {
    const float p = __fmul_rn(__ldg(&A.sp[s].beta_f), __ldg(A.arc_w + epos));
    if (!(p > 0.0f)) return 0ull;
    if (p >= 1.0f) return TWO32;
    return (uint64_t)__float2ull_rn(__fmul_rn(p, 4294967296.0f));
}

// Node (Philox subject) of new row i, and new row of node v.
__device__ __forceinline__ uint32_t node_of(const StepArgs &A, int32_t i) {
    return A.orig ? (uint32_t)__ldg(A.orig + i) : (uint32_t)i;
}
__device__ __forceinline__ int32_t row_of(const StepArgs &A, int32_t v) {
    return A.pos ? __ldg(A.pos + v) : v;
}

// profile kinds (fsgp_profile)
enum { PK_INIT = 0, PK_BEGIN = 1, PK_MARK = 2, PK_HUB = 3, PK_HUBFIN = 4, PK_MID = 5,
       PK_SMALL = 6, PK_RESULTS = 7, PK_SMALL4 = 8, PK_LANE = 9 };

// Algorithmic bytes of one work item (a slice of `words` words of one row): row pointers,
// own state read + written, and per gathered in-arc the column index plus the source's
// words of the slice (at least one 32-byte sector).
__device__ __forceinline__ unsigned long long row_bytes(int words, int planes, bool gathered,
                                                        int64_t deg) {
    const unsigned long long own = 2ull * planes * 4ull * (unsigned long long)words;
    const unsigned long long src = words * 4 > 32 ? (unsigned long long)words * 4ull : 32ull;
    return 8ull + own + (gathered ? (unsigned long long)deg * (4ull + src) : 0ull);
}

// Everything one state word needs: its set, Philox word index, valid lanes, key.
struct WordCtx {
    int s;
    uint32_t g, vm, k0, k1;
};

__device__ __forceinline__ WordCtx word_ctx(const StepArgs &A, int w) {
    WordCtx c;
    c.s = w >> A.ws_shift;
    const int wl = w & (A.Ws - 1);
    const SetParams &p = A.sp[c.s];
    const int W = __ldg(&p.W);
    c.vm = wl < W - 1 ? 0xffffffffu : (wl == W - 1 ? __ldg(&p.last_mask) : 0u);
    c.g = A.gbase + (uint32_t)wl;
    c.k0 = __ldg(&p.key0);
    c.k1 = __ldg(&p.key1);
    return c;
}

// ------------------------------------------------------------ bit-sliced counters

// c += x0 + x1 + x2 + x3 (bit-sliced, 32 lanes per word).  Carry-save compression of
// the four inputs to three bit-planes, then a ripple that stops at the first zero carry.
template <int B>
__device__ __forceinline__ void add4(uint32_t (&c)[B], uint32_t x0, uint32_t x1, uint32_t x2,
                                     uint32_t x3) {
    const uint32_t sA = x0 ^ x1 ^ x2;
    const uint32_t cA = (x0 & x1) | (x2 & (x0 ^ x1));
    const uint32_t s0 = sA ^ x3;
    const uint32_t cB = sA & x3;
    const uint32_t s1 = cA ^ cB;
    const uint32_t s2 = cA & cB;
    uint32_t carry = c[0] & s0;
    c[0] ^= s0;
    uint32_t t = c[1];
    c[1] = t ^ s1 ^ carry;
    if constexpr (B == 2) return;   // counts below 4 (rows with at most 3 in-arcs)
    carry = (t & s1) | (carry & (t ^ s1));
    t = c[B > 2 ? 2 : 1];
    c[B > 2 ? 2 : 1] = t ^ s2 ^ carry;
    carry = (t & s2) | (carry & (t ^ s2));
#pragma unroll
    for (int b = 3; b < B; ++b) {
        if (!carry) break;
        const uint32_t nc = c[b] & carry;
        c[b] ^= carry;
        carry = nc;
    }
}

// c += d (both bit-sliced, no overflow by construction)
template <int B>
__device__ __forceinline__ void add_sliced(uint32_t (&c)[B], const uint32_t (&d)[B]) {
    uint32_t carry = 0;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const uint32_t a = c[b], e = d[b];
        c[b] = a ^ e ^ carry;
        carry = (a & e) | (carry & (a ^ e));
    }
}

// lanes whose count >= K (K < 2^B)
template <int B>
__device__ __forceinline__ uint32_t ge_const(const uint32_t (&c)[B], uint32_t K) {
    uint32_t gt = 0u, eq = 0xffffffffu;
#pragma unroll
    for (int b = B - 1; b >= 0; --b) {
        if ((K >> b) & 1u) {
            eq &= c[b];
        } else {
            gt |= eq & c[b];
            eq &= ~c[b];
        }
    }
    return gt | eq;
}

template <int B>
__device__ __forceinline__ uint32_t any_count(const uint32_t (&c)[B]) {
    uint32_t a = 0u;
#pragma unroll
    for (int b = 0; b < B; ++b) a |= c[b];
    return a;
}

// Count of one lane, and the lanes of `rem` whose count equals k.
template <int B>
__device__ __forceinline__ uint32_t lane_count(const uint32_t (&c)[B], int lane) {
    uint32_t k = 0u;
#pragma unroll
    for (int b = 0; b < B; ++b) k |= ((c[b] >> lane) & 1u) << b;
    return k;
}

template <int B>
__device__ __forceinline__ uint32_t lanes_with_count(const uint32_t (&c)[B], uint32_t rem,
                                                     uint32_t k) {
#pragma unroll
    for (int b = 0; b < B; ++b) rem &= ((k >> b) & 1u) ? c[b] : ~c[b];
    return rem;
}

// Largest / smallest count among the lanes of M (M != 0), MSB first.
template <int B>
__device__ __forceinline__ uint32_t max_count(const uint32_t (&c)[B], uint32_t M) {
    uint32_t k = 0u;
#pragma unroll
    for (int b = B - 1; b >= 0; --b) {
        const uint32_t t = M & c[b];
        if (t) {
            k |= 1u << b;
            M = t;
        }
    }
    return k;
}

template <int B>
__device__ __forceinline__ uint32_t min_count(const uint32_t (&c)[B], uint32_t M) {
    uint32_t k = 0u;
#pragma unroll
    for (int b = B - 1; b >= 0; --b) {
        const uint32_t t = M & ~c[b];
        if (t) M = t;
        else k |= 1u << b;
    }
    return k;
}

// One MSB-first step of "u < threshold": plane p holds bit (31-j) of u for every lane,
// tb is bit (31-j) of the threshold.  Lanes leave `eq` at their first differing bit.
#define FSGP_BIT_STEP(p, tb, lt, eq)  \
    do {                              \
        if (tb) {                     \
            (lt) |= (eq) & ~(p);      \
            (eq) &= (p);              \
        } else {                      \
            (eq) &= ~(p);             \
        }                             \
    } while (0)

// Highest counter plane set in any lane of M (-1 if none), branch-free.
template <int B>
__device__ __forceinline__ int top_plane(const uint32_t (&c)[B], uint32_t M) {
    int hb = -1;
#pragma unroll
    for (int b = 0; b < B; ++b) hb = (M & c[b]) ? b : hb;
    return hb;
}

// Lanes of `rem` whose uniform u(tag, a, t, lane) is below thr(k_lane), k_lane the
// lane's count, 1 <= k_lane <= kcap.  thr is monotone in k, so every threshold lies
// between thr(1) and thr(khi), khi = min(kcap, 2^(hb+1) - 1) with hb the highest counter
// plane in use, and shares their common binary prefix of L bits: all lanes are first
// compared with that prefix together, and only lanes still tied after it are resolved
// group by group (equal k, counts read from the hb+1 planes in use) from bit L on.
// Planes come in Philox blocks of four; the first two blocks are kept in registers once
// generated, deeper blocks are generated where needed.  The loops run over blocks and
// are not unrolled, to keep the kernels' instruction footprint small.
template <int B, class ThrFn>
__device__ __forceinline__ uint32_t grouped_u_less(const uint32_t (&c)[B], uint32_t rem,
                                                   ThrFn thr_of, uint32_t kcap, uint32_t a,
                                                   uint32_t t, uint32_t g, uint32_t tag,
                                                   uint32_t k0, uint32_t k1) {
    uint4 P0 = make_uint4(0u, 0u, 0u, 0u), P1 = P0;
    bool have0 = false, have1 = false;
    auto block = [&](uint32_t m) -> uint4 {
        if (m == 0u) {
            if (!have0) {
                P0 = philox4x32_10(make_uint4(a, t, g, tag << 8), k0, k1);
                have0 = true;
            }
            return P0;
        }
        if (m == 1u) {
            if (!have1) {
                P1 = philox4x32_10(make_uint4(a, t, g, (tag << 8) | 1u), k0, k1);
                have1 = true;
            }
            return P1;
        }
        return philox4x32_10(make_uint4(a, t, g, (tag << 8) | m), k0, k1);
    };
    const int nb = top_plane<B>(c, rem) + 1;    // rem lanes have k >= 1, so nb >= 1
    uint32_t khi = nb >= 32 ? 0xffffffffu : (1u << nb) - 1u;
    if (khi > kcap) khi = kcap;
    uint32_t res = 0u;
    int L = 0;
    uint32_t eq = rem;
    {
        const uint64_t ta = thr_of(1u);
        const uint64_t tb = thr_of(khi);
        if (ta > 0ull && ta < TWO32 && tb > 0ull && tb < TWO32) {
            const uint32_t x = (uint32_t)ta ^ (uint32_t)tb;
            L = x ? __clz(x) : 32;
            const uint32_t th = (uint32_t)ta;
            uint32_t lt = 0u;
#pragma unroll 1
            for (int m = 0; m * 4 < L && eq; ++m) {
                const uint4 Q = block((uint32_t)m);
                const uint32_t q[4] = {Q.x, Q.y, Q.z, Q.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j = m * 4 + i;
                    if (j < L) FSGP_BIT_STEP(q[i], (th >> (31 - j)) & 1u, lt, eq);
                }
            }
            res = lt;
            if (L == 32) return res;   // equal thresholds: lanes still tied have u == thr
        }
    }
#pragma unroll 1
    while (eq) {
        const int l0 = __ffs(eq) - 1;
        uint32_t k = 0u, M = eq;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (b < nb) {
                const uint32_t bit = (c[b] >> l0) & 1u;
                k |= bit << b;
                M &= bit ? c[b] : ~c[b];
            }
        }
        eq &= ~M;
        const uint64_t thr = thr_of(k);
        if (thr == 0ull) continue;
        if (thr >= TWO32) {
            res |= M;
            continue;
        }
        const uint32_t th = (uint32_t)thr;
        uint32_t lt = 0u, e2 = M;
#pragma unroll 1
        for (int m = L >> 2; m < 8 && e2; ++m) {
            const uint4 Q = block((uint32_t)m);
            const uint32_t q[4] = {Q.x, Q.y, Q.z, Q.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int j = m * 4 + i;
                if (j >= L) FSGP_BIT_STEP(q[i], (th >> (31 - j)) & 1u, lt, e2);
            }
        }
        res |= lt;
    }
    return res;
}

// ------------------------------------------------------- per-word update (Eq. updata)

struct WordOut {
    uint32_t n0, n1, n2;
};

// SIR / SIS word update from counts of infected in-arcs (Appendix A.1 rules).
template <int MODEL, int B>
__device__ __forceinline__ WordOut update_sir_word(const StepArgs &A, uint32_t v, const WordCtx &x,
                                                   uint32_t s0, uint32_t s1, int32_t d,
                                                   const uint32_t (&c)[B]) {
    const SetParams &p = A.sp[x.s];
    const uint32_t S = x.vm & ~s0 & ~s1;
    const uint32_t cand = S & any_count<B>(c);
    uint32_t infect = 0u;
    if (cand) {
        const int32_t ksat = __ldg(&p.ksat);
        uint32_t sat = 0u;
        if ((uint64_t)ksat < (1ull << B)) sat = ge_const<B>(c, (uint32_t)ksat) & cand;
        const uint32_t rem = cand & ~sat;
        uint32_t below = 0u;
        if (rem) {
            const uint64_t *surv = p.surv;
            // counts of rem lanes are at most d and below K_sat (the surv table covers both)
            const uint32_t kcap = (uint32_t)min(d, ksat - 1);
            below = grouped_u_less<B>(c, rem, [surv](uint32_t k) { return __ldg(surv + k); }, kcap,
                                      v, A.t, x.g, TAG_INFECT, x.k0, x.k1);
        }
        infect = sat | (rem & ~below);   // infected iff u >= surv[k]
    }
    const uint32_t I = s0 & x.vm;
    const uint32_t rec = lanes_u_less(I, __ldg(&p.g_rec), v, A.t, x.g, TAG_RECOVER, x.k0, x.k1);
    WordOut o;
    o.n0 = (s0 & ~rec) | infect;
    o.n1 = MODEL == FSGP_SIR ? (s1 | rec) : 0u;
    o.n2 = 0u;
    return o;
}

// Lanes of `cand` (susceptible lanes with k >= 1) whose uniform u(tag) reaches the
// survival threshold surv[k] of a table with first zero at K_sat (d: in-degree).
template <int B>
__device__ __forceinline__ uint32_t surv_reached(const StepArgs &A, uint32_t v, const WordCtx &x, uint32_t cand,
                                                 int32_t d, const uint32_t (&c)[B], const uint64_t *surv,
                                                 int32_t ksat, uint32_t tag) {
    if (!cand) return 0u;
    uint32_t sat = 0u;
    if ((uint64_t)ksat < (1ull << B)) sat = ge_const<B>(c, (uint32_t)ksat) & cand;
    const uint32_t rem = cand & ~sat;
    uint32_t below = 0u;
    if (rem) {
        const uint32_t kcap = (uint32_t)min(d, ksat - 1);
        below = grouped_u_less<B>(c, rem, [surv](uint32_t k) { return __ldg(surv + k); }, kcap, v, A.t, x.g,
                                  tag, x.k0, x.k1);
    }
    return sat | (rem & ~below);
}

// SEIR / SEIS word update (the discrete-time rows of Table 1): planes I (s0) and, SEIR:
// R (s1), E (s2); SEIS: E (s1).  S -> E with the infection rule, E -> I with alpha
// (tag 5), I -> R (SEIS: S) with gamma; one change per lane and step.
template <int MODEL, int B>
__device__ __forceinline__ WordOut update_seir_word(const StepArgs &A, uint32_t v, const WordCtx &x,
                                                    uint32_t s0, uint32_t s1, uint32_t s2, int32_t d,
                                                    const uint32_t (&c)[B]) {
    const SetParams &p = A.sp[x.s];
    const uint32_t I = s0 & x.vm;
    const uint32_t E = (MODEL == FSGP_SEIR ? s2 : s1) & x.vm;
    const uint32_t Rm = MODEL == FSGP_SEIR ? (s1 & x.vm) : 0u;
    const uint32_t S = x.vm & ~I & ~E & ~Rm;
    const uint32_t expose = surv_reached<B>(A, v, x, S & any_count<B>(c), d, c, p.surv, __ldg(&p.ksat), TAG_INFECT);
    const uint32_t lat = lanes_u_less(E, __ldg(&p.a_lat), v, A.t, x.g, TAG_LATENT, x.k0, x.k1);
    const uint32_t rec = lanes_u_less(I, __ldg(&p.g_rec), v, A.t, x.g, TAG_RECOVER, x.k0, x.k1);
    const uint32_t nI = (I & ~rec) | lat;
    const uint32_t nE = (E & ~lat) | expose;
    WordOut o;
    o.n0 = nI;
    if (MODEL == FSGP_SEIR) {
        o.n1 = Rm | rec;
        o.n2 = nE;
    } else {
        o.n1 = nE;
        o.n2 = 0u;
    }
    return o;
}

// SWIR word update: planes I (s0), R (s1), W (s2).  A susceptible lane with k >= 1 is
// infected with the kappa table (tag 1), otherwise weakened with the mu table (tag 6); a
// weakened lane with k >= 1 is infected with the nu table (tag 1); I -> R after a step.
template <int B>
__device__ __forceinline__ WordOut update_swir_word(const StepArgs &A, uint32_t v, const WordCtx &x,
                                                    uint32_t s0, uint32_t s1, uint32_t s2, int32_t d,
                                                    const uint32_t (&c)[B]) {
    const SetParams &p = A.sp[x.s];
    const uint32_t I = s0 & x.vm, Rm = s1 & x.vm, Wk = s2 & x.vm;
    const uint32_t S = x.vm & ~I & ~Rm & ~Wk;
    const uint32_t pressed = any_count<B>(c);
    const uint32_t infS = surv_reached<B>(A, v, x, S & pressed, d, c, p.surv, __ldg(&p.ksat), TAG_INFECT);
    const uint32_t weak = surv_reached<B>(A, v, x, S & pressed & ~infS, d, c, p.surv_mu, __ldg(&p.ksat_mu),
                                          TAG_WEAKEN);
    const uint32_t infW = surv_reached<B>(A, v, x, Wk & pressed, d, c, p.surv_nu, __ldg(&p.ksat_nu), TAG_INFECT);
    WordOut o;
    o.n0 = infS | infW;
    o.n1 = Rm | I;
    o.n2 = (Wk & ~infW) | weak;
    return o;
}

// LT word update from counts of active in-arcs: activate iff k*2^32 >= theta*d.
template <int B>
__device__ __forceinline__ WordOut update_lt_word(const StepArgs &A, uint32_t v, const WordCtx &x,
                                                  uint32_t s0, int32_t d, const uint32_t (&c)[B]) {
    const uint32_t cand = x.vm & ~s0 & any_count<B>(c);
    uint32_t act = 0u;
    if (cand) {
        uint32_t sat = 0u;
        if ((uint64_t)d < (1ull << B)) sat = ge_const<B>(c, (uint32_t)d) & cand;
        const uint32_t rem = cand & ~sat;
        if (rem) {
            const uint64_t dd = (uint64_t)d;
            act = grouped_u_less<B>(c, rem,
                                    [dd](uint32_t k) { return ((uint64_t)k << 32) / dd + 1ull; },
                                    (uint32_t)(d - 1), v, 0u, x.g, TAG_LT_THRESH, x.k0, x.k1);
        }
        act |= sat;
    }
    WordOut o;
    o.n0 = s0 | act;
    o.n1 = act;
    o.n2 = 0u;
    return o;
}

// ----------------------------------------------------------------- step epilogue

// Per-thread running sums, flushed once per CTA.
struct Accum {
    unsigned long long push_deg = 0;
    unsigned long long bytes = 0;
};

// Per-set plane-popcount changes of one CTA live in shared memory (kMaxSets x 2).
constexpr int kMaxSets = 128;

__device__ __forceinline__ void set_acc_zero(unsigned long long *s_pc, int S) {
    for (int i = threadIdx.x; i < kPC * S; i += blockDim.x) s_pc[i] = 0ull;
    __syncthreads();
}

__device__ __forceinline__ void set_acc_add(unsigned long long *s_pc, int s, long long d0, long long d1,
                                            long long d2 = 0) {
    if (d0) atomicAdd(&s_pc[kPC * s], (unsigned long long)d0);
    if (d1) atomicAdd(&s_pc[kPC * s + 1], (unsigned long long)d1);
    if (d2) atomicAdd(&s_pc[kPC * s + 2], (unsigned long long)d2);
}

// after a __syncthreads of the caller
__device__ __forceinline__ void set_acc_flush(const StepArgs &A, const unsigned long long *s_pc) {
    for (int i = threadIdx.x; i < kPC * A.S; i += blockDim.x)
        if (s_pc[i]) atomicAdd(&A.pc[i], s_pc[i]);
}

// Grid barrier of the persistent step loop (its CTAs are co-resident: cooperative
// launch) for `expected` CTAs.  Arrival is one atomic per CTA; the last CTA to arrive
// resets the count and advances the generation.  A wait lasts at most `limit` SM clock cycles: past that the
// CTA records the time-out in *err and goes on.  Returns, uniformly over the CTA,
// whether no time-out has been recorded so far.
__device__ __forceinline__ bool grid_barrier(uint32_t *count, uint32_t *gen, uint32_t expected, int32_t *err,
                                             long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *vgen = gen;
        const uint32_t g = *vgen;   // read before arriving: it cannot advance until we have
        __threadfence();            // this CTA's state writes and counter flushes first
        if (atomicAdd(count, 1u) == expected - 1u) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (clock64() - t0 > limit) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = *(volatile int32_t *)err == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// per-lane count changes of one word of one plane (s_plane: that plane's counters)
__device__ __forceinline__ void lane_deltas(int32_t *s_plane, int w, uint32_t olds, uint32_t news) {
    uint32_t ch = olds ^ news;
    while (ch) {
        const int l = __ffs(ch) - 1;
        ch &= ch - 1;
        atomicAdd(&s_plane[w * 32 + l], ((news >> l) & 1u) ? 1 : -1);
    }
}

__device__ __forceinline__ void flush_accum(const StepArgs &A, Accum acc, int list_slot, int kind) {
    __shared__ long long s_red[4][kBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.push_deg += __shfl_xor_sync(0xffffffffu, acc.push_deg, o);
        acc.bytes += __shfl_xor_sync(0xffffffffu, acc.bytes, o);
    }
    if (lane == 0) {
        s_red[0][wid] = 0;
        s_red[1][wid] = 0;
        s_red[2][wid] = (long long)acc.push_deg;
        s_red[3][wid] = (long long)acc.bytes;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, b = 0, c = 0, d = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += s_red[0][i];
            b += s_red[1][i];
            c += s_red[2][i];
            d += s_red[3][i];
        }
        (void)a;
        (void)b;
        if (A.prof_bytes && d) atomicAdd(&A.prof_bytes[kind], (unsigned long long)d);
        if (c) atomicAdd((unsigned long long *)&A.ctl->push_outdeg[list_slot], (unsigned long long)c);
    }
}

// per-CTA lane counters (shared memory) -> global running lane counts
__device__ __forceinline__ void flush_lanes(const StepArgs &A, int32_t *s_lane, int nl) {
    __syncthreads();
    for (int i = threadIdx.x; i < A.np * nl; i += blockDim.x) {
        const int32_t x = s_lane[i];
        if (x) atomicAdd(&A.lane_cnt[i], x);
    }
}

// Whether this step lists its rows for the next one (set by the step control kernel
// before the row kernels; read once per kernel).
__device__ __forceinline__ bool list_wanted(const StepArgs &A) {
    return *(volatile const int32_t *)&A.ctl->build_list != 0;
}

// Warp-aggregated append of flagged rows to the next step's list (build = list_wanted).
__device__ __forceinline__ void list_append(const StepArgs &A, bool build, bool want, int32_t entry,
                                            int list_slot) {
    if (!build) return;   // uniform per launch
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&A.ctl->list_n[list_slot], (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) A.list_out[base + __popc(m & ((1u << lane) - 1u))] = entry;
}

// Launch shape of the row kernels of one step (host side).
struct StepLaunch {
    int V, TEAM;           // words per thread, threads per slice team
    int grid_small, grid_mid, grid_hub, grid_fin, grid_small4, grid_lane;
    int swl;               // words per thread of the one-thread-per-row kernel
    size_t smem_lanes;     // dynamic shared memory for per-lane counters (0 = off)
    bool have_small, have_mid, have_hub, have_small4, have_lane;
    struct Prof *prof;     // host-side event recorder, or null
};

// Host-side recorder of CUDA events around launches (fsgp_profile).
struct Prof {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;   // kind of the interval that starts at ev[i]
    void start(int k, cudaStream_t s) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev.push_back(e);
        kind.push_back(k);
    }
    void stop(cudaStream_t s) { start(-1, s); }
};

// One seed set (or one batched request) of a run: parameters, inputs and caller-owned
// outputs (memory kind out_flags; NULL = not wanted, except counts).
struct SetSpec {
    double beta, gamma, ic_p, alpha, mu, nu;
    uint64_t rng_seed;
    int32_t R;
    const int32_t *seeds;          // seed nodes (memory kind seed_flags)
    int64_t n_seeds;
    uint32_t seed_flags;
    const uint32_t *init_planes;   // optional start planes [P][n][ceil(R/32)]
    uint64_t *counts;              // [T+1][C]
    uint32_t *freq;                // [C][n]
    uint32_t *per_real;            // [R][T+1][C]
    uint32_t *final_planes;        // [P][n][ceil(R/32)]
    int32_t *steps_run;            // [1]
    uint32_t out_flags;
};

// Runs every set for T steps on graph g (simulate.cu).  Sets with the same words per
// set run side by side in one launch sequence (up to kMaxSets at a time).
// weighted: SIR / SIS on the graph's arc weights (per-arc transmission draws).
int run_sets(fsgp_graph *g, int model, int ic_mode, int weighted, const SetSpec *sets, int n_sets, int T,
             const fsgp_options &opt, cudaStream_t s);

template <int MODEL>
int launch_persist(const StepArgs &A, const PersistArgs &Q, int TEAM, int grid, size_t smem, int sm_count,
                   cudaStream_t s, int *grid_out);

// Defined in rows.cuh, instantiated once per model (model_*.cu).
template <int MODEL>
int launch_rows(const StepArgs &A, const StepLaunch &L, cudaStream_t s);
struct RowOccupancy {
    int small, small4, lane, mid, hub;   // resident CTAs per SM of each row kernel
    int swl;                             // in: slice width of the lane kernel
};
template <int MODEL>
int occupancy_rows(int V, int TEAM, size_t smem, RowOccupancy *o);
template <int MODEL>
int launch_split_rows(const StepArgs &A, int V, int TEAM, int grid_chunks, int grid_fin,
                      cudaStream_t s);

}  // namespace fsgp
