// fsgp_internal.cuh -- device helpers and host-side structures shared by the library's
// translation units.  Nothing here is part of the C ABI (include/fsgp.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fsgp.h"

namespace fsgp {

// ----------------------------------------------------------------------- constants
constexpr uint32_t TAG_INFECT = 1u;
constexpr uint32_t TAG_RECOVER = 2u;
constexpr uint32_t TAG_IC_EDGE = 3u;
constexpr uint32_t TAG_LT_THRESH = 4u;
constexpr uint32_t TAG_LATENT = 5u;
constexpr uint32_t TAG_WEAKEN = 6u;
constexpr uint32_t TAG_ARC_INFECT = 7u;

// Row-kernel models of weighted graphs (not public model numbers: a run of FSGP_SIR or
// FSGP_SIS with fsgp_params.weighted set takes these kernels): an infectious in-arc e
// transmits with probability beta * w_e, drawn per arc like an IC arc.
constexpr int kSirW = 8;
constexpr int kSisW = 9;
constexpr uint64_t TWO32 = 4294967296ull;

constexpr int kBlock = 256;          // threads per CTA for the row kernels
constexpr int kSmallBits = 8;        // bit-sliced counter width, team-per-row rows (d <= 255)
constexpr int kWideBits = 16;        // warp-per-row rows and hub chunks (d <= 65535)
constexpr int kMaxR = 4096;

// list entry flag: the row's source lanes push to its out-neighbours next step
constexpr uint32_t kPushBit = 0x80000000u;

// ----------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11.
// Ten rounds of two 32x32->64 multiplies; the high halves are xored with the other
// counter words and the key; the key advances by the Weyl increments between rounds.
// Not inlined: one copy per kernel keeps the instruction footprint small.
static __device__ __noinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Lanes of M whose uniform u(tag, a, t, lane) is below thr (thr may be 2^32 or more =
// every lane).  The comparison runs MSB first over the bit-planes of u and stops as
// soon as every lane of M is decided, so most calls need one or two Philox blocks.
__device__ __forceinline__ uint32_t lanes_u_less(uint32_t M, uint64_t thr, uint32_t a,
                                                 uint32_t t, uint32_t g, uint32_t tag,
                                                 uint32_t k0, uint32_t k1) {
    if (M == 0u || thr == 0ull) return 0u;
    if (thr >= TWO32) return M;
    const uint32_t th = (uint32_t)thr;
    uint32_t lt = 0u, eq = M;
#pragma unroll 1
    for (uint32_t m = 0; m < 8u && eq; ++m) {
        const uint4 P = philox4x32_10(make_uint4(a, t, g, (tag << 8) | m), k0, k1);
        const uint32_t p[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = (int)m * 4 + i;
            if ((th >> (31 - j)) & 1u) {
                lt |= eq & ~p[i];
                eq &= p[i];
            } else {
                eq &= ~p[i];
            }
        }
    }
    return lt;
}

// ------------------------------------------------------------------ host structures
struct ClassInfo {
    int32_t bucket_count[33];   // rows per degree bucket (0: d=0, b>=1: 2^(b-1)<=d<2^b)
    int32_t bucket_start[34];   // start of each bucket in rows_sorted (descending order)
};

struct HubTable {
    int32_t min_deg = -1;       // table built for this hub threshold and chunk size
    int32_t chunk = -1;
    int32_t n_hubs = 0;
    int64_t n_chunks = 0;
    int64_t *d_chunk_base = nullptr;  // [n_hubs + 1] (hub rows are new ids 0 .. n_hubs-1)
};

struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// An instantiated CUDA graph of one run's step loop, kept for the next run whose launch
// sequence is the same byte for byte (kernel arguments, grids, output pointers).
struct ExecCache {
    std::vector<uint8_t> sig;
    cudaGraphExec_t exec = nullptr;
};
constexpr int kExecCacheSize = 4;

// Per-graph tables of the learned surrogate's aggregation, built on first use: rows with
// at least kSgLong arcs are split into chunks of kSgChunk arcs whose partial sums meet
// in a float32 accumulator (zero between uses).
constexpr int32_t kSgLong = 256;
constexpr int32_t kSgChunk = 256;
struct SgCache {
    int built = 0;
    float *inv_din = nullptr;     // [n] 1 / d_in (0 when d_in = 0)
    int4 *in_items = nullptr;     // chunks of long in-CSR rows: {row, begin, end, slot}
    int32_t n_in_items = 0;
    int32_t *in_long = nullptr;   // [n_in_long] the long in-CSR rows, by slot
    int32_t n_in_long = 0;
    int4 *out_items = nullptr;    // chunks of long out-CSR rows
    int32_t n_out_items = 0;
    int32_t *out_long = nullptr;
    int32_t n_out_long = 0;
    float *acc = nullptr;         // [max(n_in_long, n_out_long)][64]
};

}  // namespace fsgp

struct fsgp_graph {
    int device = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t max_deg = 0;
    int32_t max_out_deg = 0;
    int32_t *row_ptr = nullptr;     // [n+1] in-CSR
    int32_t *col = nullptr;         // [nnz]
    int32_t *out_ptr = nullptr;     // [n+1] out-CSR
    int32_t *out_dst = nullptr;     // [nnz]
    int32_t *rows_sorted = nullptr; // [n] rows by degree bucket, high buckets first
    // The propagation kernels work on the rows relabelled in rows_sorted order: row i of
    // the state planes is node rows_sorted[i] ("new id" i), so the rows of one degree
    // class are one contiguous range and the most-read sources (high-degree nodes) sit
    // together at the front of every plane.
    int32_t *pos = nullptr;         // [n] new id of each node (inverse of rows_sorted)
    int32_t *rp2 = nullptr;         // [n+1] in-CSR row pointers in new-id order
    int32_t *col2 = nullptr;        // [nnz] sources as new ids, rows in new-id order (each
                                    // row's arcs in their original order)
    int32_t *arc0 = nullptr;        // [n] position in col of the first arc of new row i
                                    // (IC draws are keyed by the original arc position)
    int4 *lane_tab = nullptr;       // new rows with 1..3 in-arcs (from bucket 2 to the
                                    // start of bucket 0): {node, src0, src1, src2}, sources
                                    // as new ids, -1 = none
    int32_t lane_start = 0;         // new id of lane_tab[0]
    int32_t d0_start = 0;           // new id of the first row without in-arcs
    fsgp::ClassInfo cls{};
    fsgp::HubTable hub{};
    fsgp::Workspace ws{};
    std::vector<fsgp::ExecCache> execs;   // most recent last (they point into ws)
    float *arc_w = nullptr;         // [nnz] arc weights in the caller's arc order, or null
    fsgp::SgCache sgc{};
    int tuned = 0;                  // fsgp_batch_run: tuning chosen by an autotuned call
    fsgp_options tuned_opt{};
    int sm_count = 0;
    size_t device_bytes = 0;
};

namespace fsgp {
// thread-local error message
// Host helpers shared by the simulation entry points (simulate.cu).
// Grow the graph's cached workspace to at least `bytes` (contents undefined).
int ensure_workspace(fsgp_graph *g, size_t bytes);
// Destroy the graph's cached step-loop executables (they refer to its workspace).
void drop_exec_cache(fsgp_graph *g);
// Exact integer survival table surv[k] ~ 2^32 (1 - beta)^k for k = 0 .. min(K_sat,
// max_deg), where surv[K_sat] = 0 (every lane with k >= K_sat is infected); ksat =
// INT32_MAX when the table never reaches 0 within max_deg.
void survival_table(double beta, int32_t max_deg, std::vector<uint64_t> &out, int32_t *ksat);

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
}  // namespace fsgp

#define FSGP_CUDA(call)                                              \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return ::fsgp::cuda_fail(_e, #call);  \
    } while (0)
