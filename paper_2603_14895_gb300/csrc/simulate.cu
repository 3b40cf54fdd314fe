// simulate.cu -- fsgp_simulate: initial state (Algorithm 1, "initialize states"), the
// step loop (one synchronous step per iteration, X^{k+1} <- X^k double buffer of
// Algorithm 1), the frontier path ("decide whether x needs to update", Algorithm 1),
// and the reductions of the results (per-step compartment counts, per-node final
// frequencies, per-realization counts; the 0/1/2 state conversion of Appendix A.1).
//
// Seed sets (and batched requests) with the same number of words per set run side by
// side: set s owns words [s*Ws, (s+1)*Ws) of every node (Eq. batch, independent
// randomness per realization; each set keeps its own key, so its result equals a run of
// that set alone).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "step.cuh"

namespace fsgp {

// Device-side output pointers of one set.
struct SetOut {
    unsigned long long *counts;   // [T+1][C]
    uint32_t *freq;               // [C][n]
    uint32_t *per_real;           // [R][T+1][C]
    uint32_t *planes;             // [P][n][W]
    int32_t *steps;               // [1] transitions computed (staging in the workspace)
};

// ------------------------------------------------------------------------ kernels

// Seed nodes of one set: all valid lanes of its source planes, in both buffers (rows are
// new ids: node v is row pos[v]).
__global__ void k_seed(uint32_t *buf0, uint32_t *buf1, size_t plane_words, int both_planes,
                       const int32_t *__restrict__ seeds, int64_t ns, const int32_t *__restrict__ pos,
                       int Wn, int ws0, int Ws, int W, uint32_t last_mask) {
    const int64_t total = ns * Ws;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t si = i / Ws;
        const int w = (int)(i % Ws);
        const int32_t v = pos[seeds[si]];
        const uint32_t m = w < W - 1 ? 0xffffffffu : (w == W - 1 ? last_mask : 0u);
        const size_t off = (size_t)v * Wn + ws0 + w;
        buf0[off] = m;
        buf1[off] = m;
        if (both_planes) {
            buf0[plane_words + off] = m;
            buf1[plane_words + off] = m;
        }
    }
}

// Caller-supplied start planes of one set [planes][n][W] (node order) -> both buffers
// (row order).
__global__ void k_import(const uint32_t *__restrict__ in, int planes, int32_t n, int W, int Ws,
                         int Wn, int ws0, uint32_t last_mask, const int32_t *__restrict__ pos,
                         uint32_t *buf0, uint32_t *buf1) {
    const int64_t total = (int64_t)planes * n * Ws;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % Ws);
        const int64_t pv = i / Ws;   // plane * n + node
        const int64_t p = pv / n, v = pv - p * n;
        uint32_t x = 0u;
        if (w < W) {
            x = in[pv * W + w];
            if (w == W - 1) x &= last_mask;
        }
        const size_t o = ((size_t)p * n + (size_t)pos[v]) * Wn + ws0 + w;
        buf0[o] = x;
        buf1[o] = x;
    }
}

// Step-0 totals per set, per-lane counts, the rows whose source lanes push at step 1, and
// the rows without in-arcs whose state can change (those that push: an infected lane can
// recover, a newly active lane stops being new), which dense steps visit through d0_list.
__global__ void __launch_bounds__(kBlock) k_init_scan(StepArgs A, int model) {
    extern __shared__ int32_t s_lane[];
    __shared__ unsigned long long s_pc[kPC * kMaxSets];
    const int nl = A.Wn * 32;
    const bool lanes_on = A.lane_cnt != nullptr;
    if (lanes_on)
        for (int i = threadIdx.x; i < A.np * nl; i += blockDim.x) s_lane[i] = 0;
    set_acc_zero(s_pc, A.S);
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    Accum acc;
    const int np = A.np;
    const bool cascade = model == FSGP_IC || model == FSGP_LT;
    const int e_plane = model == FSGP_SEIR ? 2 : (model == FSGP_SEIS ? 1 : -1);   // exposed lanes
    const bool build = list_wanted(A);
    for (int64_t base = gwarp * 32; base < A.n; base += nwarps * 32) {
        const int64_t v = base + lane;
        const bool has = v < A.n;
        bool push = false, self = false;
        if (has) {
            for (int w = 0; w < A.Wn; ++w) {
                const size_t off = (size_t)v * A.Wn + w;
                const uint32_t s0 = A.cur[off];
                const uint32_t s1 = np >= 2 ? A.cur[A.plane_words + off] : 0u;
                const uint32_t s2 = np >= 3 ? A.cur[2 * A.plane_words + off] : 0u;
                set_acc_add(s_pc, w >> A.ws_shift, __popc(s0), __popc(s1), __popc(s2));
                if (lanes_on) {
                    lane_deltas(s_lane, w, 0u, s0);
                    if (np >= 2) lane_deltas(s_lane + nl, w, 0u, s1);
                    if (np >= 3) lane_deltas(s_lane + 2 * nl, w, 0u, s2);
                }
                push |= cascade ? (s1 != 0u) : (s0 != 0u);
                if (e_plane >= 0) self |= (e_plane == 2 ? s2 : s1) != 0u;
            }
        }
        if (push) {
            const uint32_t node = node_of(A, (int32_t)v);
            acc.push_deg += (unsigned long long)(A.out_ptr[node + 1] - A.out_ptr[node]);
        }
        if (has && A.prof_bytes) acc.bytes += (unsigned long long)np * 4ull * (unsigned long long)A.Wn;
        // rows that push, or whose exposed lanes change on their own, are visited at step 1
        list_append(A, build, has && (push || self), (int32_t)((uint32_t)v | (push ? kPushBit : 0u)), 0);
        {
            const bool d0 = has && (push || self) && v >= A.r_d0;
            const unsigned m = __ballot_sync(0xffffffffu, d0);
            if (m) {
                const int leader = __ffs(m) - 1;
                uint32_t b = 0;
                if (lane == leader) b = atomicAdd(&A.ctl->d0_n, (uint32_t)__popc(m));
                b = __shfl_sync(0xffffffffu, b, leader);
                if (d0) A.d0_list[b + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
            }
        }
    }
    flush_accum(A, acc, 0, PK_INIT);
    set_acc_flush(A, s_pc);
    if (lanes_on) flush_lanes(A, s_lane, nl);
}

// Compartments (C = 3 or 4) from the popcounts p0, p1, p2 of the planes.
__host__ __device__ __forceinline__ int n_compartments(int model) {
    return (model == FSGP_SEIR || model == FSGP_SWIR) ? 4 : 3;
}

__device__ __forceinline__ void compartments(int model, int64_t total, int64_t p0, int64_t p1, int64_t p2,
                                             int64_t out[4]) {
    out[3] = 0;
    if (model == FSGP_SIR) {
        out[0] = total - p0 - p1; out[1] = p0; out[2] = p1;
    } else if (model == FSGP_SIS) {
        out[0] = total - p0; out[1] = p0; out[2] = 0;
    } else if (model == FSGP_SEIR) {          // planes I, R, E -> S, E, I, R
        out[0] = total - p0 - p1 - p2; out[1] = p2; out[2] = p0; out[3] = p1;
    } else if (model == FSGP_SEIS) {          // planes I, E -> S, E, I
        out[0] = total - p0 - p1; out[1] = p1; out[2] = p0;
    } else if (model == FSGP_SWIR) {          // planes I, R, W -> S, W, I, R
        out[0] = total - p0 - p1 - p2; out[1] = p2; out[2] = p0; out[3] = p1;
    } else {                                  // IC / LT: planes A, F
        out[0] = total - p0; out[1] = p1; out[2] = p0 - p1;
    }
}

// Per-realization snapshot of the running lane counts into per_real[r][kk][C] of every
// set that asked for it.
__device__ void snapshot_lanes(const StepArgs &A, int model, const SetOut *outs, int T1, int kk) {
    const int nl = A.Wn * 32;
    const int per_set = A.Ws * 32;
    const int C = n_compartments(model);
    for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < nl; i += blockDim.x * gridDim.x) {
        const int s = i / per_set, r = i - s * per_set;
        uint32_t *pr = outs[s].per_real;
        if (!pr || r >= A.sp[s].R) continue;
        int64_t o[4];
        compartments(model, A.n, A.lane_cnt[i], A.np >= 2 ? A.lane_cnt[nl + i] : 0,
                     A.np >= 3 ? A.lane_cnt[2 * nl + i] : 0, o);
        uint32_t *dst = pr + ((size_t)r * T1 + kk) * C;
        for (int c = 0; c < C; ++c) dst[c] = (uint32_t)o[c];
    }
}

// Start of step k: quiescence test (IC/LT, all sets), running totals, dense/sparse
// choice, and the per-realization snapshot of step k-1.
__global__ void k_begin(StepArgs A, int model, unsigned long long sparse_limit, int force_dense,
                        const SetOut *outs, int T1) {
    if (A.lane_cnt) snapshot_lanes(A, model, outs, T1, A.k - 1);
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    Ctl *C = A.ctl;
    const unsigned long long *prev = A.pc - kPC * A.S;
    bool quiet = true;   // IC / LT: no newly active lane (plane 1) in any set
    for (int i = 0; i < kPC * A.S; ++i) {
        A.pc[i] = prev[i];
        if ((i % kPC) == 1 && prev[i]) quiet = false;
    }
    if (C->stop) return;
    if ((model == FSGP_IC || model == FSGP_LT) && quiet) {
        C->stop = 1;
        return;
    }
    C->steps_done = A.k;
    const int slot = A.k & 1, pslot = (A.k - 1) & 1;
    C->sparse = (!force_dense && C->list_valid[pslot] && C->push_outdeg[pslot] <= sparse_limit) ? 1 : 0;
    // The list built now feeds step k+1; when the rows pushing at step k-1 were far
    // above the frontier limit the next step runs dense anyway, so skip building it.
    C->build_list = (sparse_limit > 0ull && C->push_outdeg[pslot] <= 4ull * sparse_limit) ? 1 : 0;
    C->list_valid[slot] = C->build_list;
    C->list_n[slot] = 0u;
    C->push_outdeg[slot] = 0ull;
    C->cand_n[0] = 0u;
    C->cand_n[1] = 0u;
    if (C->sparse) C->sparse_steps++; else C->dense_steps++;
}

// Frontier path: mark the rows listed by the previous step and, for rows whose source
// lanes push, their out-neighbours; newly marked rows go to the candidate lists (hub
// rows stay marked in the bitmap only).
__device__ __forceinline__ void mark_round(const StepArgs &A, int32_t x) {
    int cls = -1;
    if (x >= 0) {
        const uint32_t bit = 1u << (x & 31);
        const uint32_t old = atomicOr(&A.bitmap[x >> 5], bit);
        if (!(old & bit)) {
            const int32_t d = __ldg(A.rp + x + 1) - __ldg(A.rp + x);
            if (d < A.hub_min_deg) cls = d > A.small_max_deg ? 1 : 0;
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const unsigned m = __ballot_sync(0xffffffffu, cls == c);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&A.ctl->cand_n[c], (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (cls == c) (c ? A.cand_mid : A.cand_small)[base + __popc(m & ((1u << lane) - 1u))] = x;
    }
}

__global__ void __launch_bounds__(kBlock) k_mark(StepArgs A) {
    const Ctl *C = A.ctl;
    if (*(volatile const int32_t *)&C->stop || !*(volatile const int32_t *)&C->sparse) return;
    const uint32_t n_in = ((volatile const uint32_t *)C->list_n)[(A.k - 1) & 1];
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gwarp; i < n_in; i += nwarps) {
        const uint32_t entry = (uint32_t)__ldg(A.list_in + i);
        const int32_t v = (int32_t)(entry & ~kPushBit);
        mark_round(A, lane == 0 ? v : -1);
        if (entry & kPushBit) {
            const uint32_t node = node_of(A, v);   // out-arcs are listed by node
            const int32_t b = __ldg(A.out_ptr + node), e = __ldg(A.out_ptr + node + 1);
            for (int32_t j = b; j < e; j += 32) {
                const int32_t x = j + lane < e ? row_of(A, __ldg(A.out_dst + j + lane)) : -1;
                mark_round(A, x);
            }
        }
    }
}

// Results per set: compartment totals per step and the last per-realization snapshot.
__global__ void k_finalize(StepArgs A, int model, int T, const unsigned long long *pc_all,
                           const SetOut *outs) {
    const int S = A.S;
    const int C = n_compartments(model);
    for (int64_t i = threadIdx.x + (int64_t)blockIdx.x * blockDim.x; i < (int64_t)(T + 1) * S;
         i += (int64_t)blockDim.x * gridDim.x) {
        const int k = (int)(i / S), s = (int)(i % S);
        int64_t o[4];
        const int64_t NR = (int64_t)A.n * A.sp[s].R;
        const unsigned long long *p = pc_all + ((size_t)k * S + s) * kPC;
        compartments(model, NR, (int64_t)p[0], (int64_t)p[1], (int64_t)p[2], o);
        unsigned long long *c = outs[s].counts + (size_t)C * k;
        for (int j = 0; j < C; ++j) c[j] = (unsigned long long)o[j];
    }
    if (A.lane_cnt) snapshot_lanes(A, model, outs, T + 1, T);
    // IC/LT: the first step whose frontier is empty (later rows repeat); otherwise T
    for (int s = threadIdx.x + blockIdx.x * blockDim.x; s < S; s += blockDim.x * gridDim.x) {
        int st = T;
        if (*(volatile const int32_t *)&A.ctl->err) {   // the persistent loop timed out
            outs[s].steps[0] = -1;
            continue;
        }
        if (model == FSGP_IC || model == FSGP_LT)
            for (int k = 0; k <= T; ++k)
                if (pc_all[((size_t)k * S + s) * kPC + 1] == 0ull) {
                    st = k;
                    break;
                }
        outs[s].steps[0] = st;
    }
}

// Persistent step loop: rows 1..T of pc hold each step's changes; make them running
// totals (a stopped cascade's later rows repeat its last row).
__global__ void k_pc_prefix(unsigned long long *pc, int T, int width) {
    for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < width; i += blockDim.x * gridDim.x)
        for (int k = 1; k <= T; ++k) pc[(size_t)k * width + i] += pc[(size_t)(k - 1) * width + i];
}

// Self-test of the bounded grid barrier: every CTA arrives `rounds` times at a barrier
// that expects gridDim.x + missing CTAs; with missing > 0 no generation completes and
// every wait runs out after `limit` cycles.
__global__ void k_barrier_selftest(uint32_t *bar, int32_t *err, int rounds, int missing, long long limit) {
    for (int r = 0; r < rounds; ++r)
        if (!grid_barrier(bar, bar + 1, gridDim.x + (uint32_t)missing, err, limit)) break;
}

// Per-node final compartment frequencies of every set that asked for them.
__global__ void k_freq(StepArgs A, int model, const uint32_t *buf0, const uint32_t *buf1,
                       const SetOut *outs) {
    const uint32_t *st = (A.ctl->steps_done & 1) ? buf1 : buf0;
    const int np = A.np, C = n_compartments(model);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = node_of(A, (int32_t)i);   // row i holds node v
        for (int s = 0; s < A.S; ++s) {
            uint32_t *fr = outs[s].freq;
            if (!fr) continue;
            const int W = A.sp[s].W;
            int64_t p0 = 0, p1 = 0, p2 = 0;
            for (int w = 0; w < W; ++w) {
                const size_t off = (size_t)i * A.Wn + (size_t)s * A.Ws + w;
                p0 += __popc(st[off]);
                if (np >= 2) p1 += __popc(st[A.plane_words + off]);
                if (np >= 3) p2 += __popc(st[2 * A.plane_words + off]);
            }
            int64_t o[4];
            compartments(model, A.sp[s].R, p0, p1, p2, o);
            for (int c = 0; c < C; ++c) fr[(size_t)c * A.n + v] = (uint32_t)o[c];
        }
    }
}

// Final planes of one set -> caller layout [planes][n][W] in node order.
__global__ void k_export(StepArgs A, int planes, int ws0, int W, const uint32_t *buf0,
                         const uint32_t *buf1, uint32_t *out) {
    const uint32_t *st = (A.ctl->steps_done & 1) ? buf1 : buf0;
    const int64_t total = (int64_t)planes * A.n * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % W);
        const int64_t pv = i / W;   // plane * n + node
        const int64_t p = pv / A.n, v = pv - p * A.n;
        out[i] = st[((size_t)p * A.n + (size_t)row_of(A, (int32_t)v)) * A.Wn + ws0 + w];
    }
}

// ------------------------------------------------------------------------- host

static int grid_cap(int64_t work, int threads, int sm_count, int per_sm = 8) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

static int bitlen(int64_t x) {
    int b = 0;
    while (x > 0) {
        ++b;
        x >>= 1;
    }
    return b;
}

__global__ void k_row_degrees(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ rows,
                              int32_t nr, int32_t *deg) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += blockDim.x * gridDim.x) {
        const int32_t v = rows[i];
        deg[i] = row_ptr[v + 1] - row_ptr[v];
    }
}

// Hub chunk table for (hub bucket, chunk): hub rows are rows_sorted[0 .. n_hubs).
static int ensure_hub_table(fsgp_graph *g, int hub_min_deg, int chunk, cudaStream_t s) {
    HubTable &H = g->hub;
    if (H.min_deg == hub_min_deg && H.chunk == chunk) return FSGP_OK;
    const int bh = bitlen(hub_min_deg);   // bucket of hub_min_deg (a power of two)
    const int32_t n_hubs = bh >= 1 ? g->cls.bucket_start[bh - 1] : g->n;
    cudaFree(H.d_chunk_base);
    H.d_chunk_base = nullptr;
    H.n_hubs = n_hubs;
    H.n_chunks = 0;
    H.min_deg = hub_min_deg;
    H.chunk = chunk;
    if (n_hubs == 0) return FSGP_OK;
    int32_t *d_deg = nullptr;
    FSGP_CUDA(cudaMalloc(&d_deg, sizeof(int32_t) * (size_t)n_hubs));
    k_row_degrees<<<grid_cap(n_hubs, 256, g->sm_count), 256, 0, s>>>(g->row_ptr, g->rows_sorted, n_hubs, d_deg);
    std::vector<int32_t> deg((size_t)n_hubs);
    cudaError_t e = cudaMemcpyAsync(deg.data(), d_deg, sizeof(int32_t) * (size_t)n_hubs,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_deg);
    if (e != cudaSuccess) return cuda_fail(e, "hub degrees");
    std::vector<int64_t> base((size_t)n_hubs + 1);
    base[0] = 0;
    for (int32_t i = 0; i < n_hubs; ++i) base[i + 1] = base[i] + (deg[i] + chunk - 1) / chunk;
    FSGP_CUDA(cudaMalloc(&H.d_chunk_base, sizeof(int64_t) * base.size()));
    FSGP_CUDA(cudaMemcpyAsync(H.d_chunk_base, base.data(), sizeof(int64_t) * base.size(),
                              cudaMemcpyHostToDevice, s));
    FSGP_CUDA(cudaStreamSynchronize(s));
    H.n_chunks = base[n_hubs];
    return FSGP_OK;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

void drop_exec_cache(fsgp_graph *g) {
    for (ExecCache &c : g->execs)
        if (c.exec) cudaGraphExecDestroy(c.exec);
    g->execs.clear();
}

int ensure_workspace(fsgp_graph *g, size_t bytes) {
    if (g->ws.bytes >= bytes) return FSGP_OK;
    drop_exec_cache(g);
    cudaFree(g->ws.ptr);
    g->ws.ptr = nullptr;
    g->ws.bytes = 0;
    cudaError_t e = cudaMalloc(&g->ws.ptr, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (workspace)");
    g->ws.bytes = bytes;
    return FSGP_OK;
}

static int launch_rows_model(int model, const StepArgs &A, const StepLaunch &L, cudaStream_t s) {
    switch (model) {
        case FSGP_SIR: return launch_rows<FSGP_SIR>(A, L, s);
        case FSGP_SIS: return launch_rows<FSGP_SIS>(A, L, s);
        case FSGP_IC: return launch_rows<FSGP_IC>(A, L, s);
        case FSGP_LT: return launch_rows<FSGP_LT>(A, L, s);
        case FSGP_SEIR: return launch_rows<FSGP_SEIR>(A, L, s);
        case FSGP_SEIS: return launch_rows<FSGP_SEIS>(A, L, s);
        case FSGP_SWIR: return launch_rows<FSGP_SWIR>(A, L, s);
        case kSirW: return launch_rows<kSirW>(A, L, s);
        case kSisW: return launch_rows<kSisW>(A, L, s);
        default: return fail(FSGP_EINVAL, "model without row kernels");
    }
}

static int occupancy_model(int model, int V, int TEAM, size_t smem, RowOccupancy *o) {
    switch (model) {
        case FSGP_SIR: return occupancy_rows<FSGP_SIR>(V, TEAM, smem, o);
        case FSGP_SIS: return occupancy_rows<FSGP_SIS>(V, TEAM, smem, o);
        case FSGP_IC: return occupancy_rows<FSGP_IC>(V, TEAM, smem, o);
        case FSGP_LT: return occupancy_rows<FSGP_LT>(V, TEAM, smem, o);
        case FSGP_SEIR: return occupancy_rows<FSGP_SEIR>(V, TEAM, smem, o);
        case FSGP_SEIS: return occupancy_rows<FSGP_SEIS>(V, TEAM, smem, o);
        case FSGP_SWIR: return occupancy_rows<FSGP_SWIR>(V, TEAM, smem, o);
        case kSirW: return occupancy_rows<kSirW>(V, TEAM, smem, o);
        case kSisW: return occupancy_rows<kSisW>(V, TEAM, smem, o);
        default: return fail(FSGP_EINVAL, "model without row kernels");
    }
}

static int launch_persist_model(int model, const StepArgs &A, const PersistArgs &Q, int TEAM, int grid,
                                size_t smem, int sm_count, cudaStream_t s, int *grid_out) {
    switch (model) {
        case FSGP_SIR: return launch_persist<FSGP_SIR>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        case FSGP_SIS: return launch_persist<FSGP_SIS>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        case FSGP_IC: return launch_persist<FSGP_IC>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        case FSGP_LT: return launch_persist<FSGP_LT>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        case FSGP_SEIR: return launch_persist<FSGP_SEIR>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        case FSGP_SEIS: return launch_persist<FSGP_SEIS>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        case FSGP_SWIR: return launch_persist<FSGP_SWIR>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        case kSirW: return launch_persist<kSirW>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        case kSisW: return launch_persist<kSisW>(A, Q, TEAM, grid, smem, sm_count, s, grid_out);
        default: return fail(FSGP_EINVAL, "model without row kernels");
    }
}

// A grid-barrier wait of the persistent step loop lasts at most this many SM cycles
// (about one second at the GB300's clock): a step of a graph small enough for the loop
// takes microseconds.
constexpr long long kPersistSpinCycles = 2000000000ll;

constexpr int32_t kSmallMaxFused = 255;   // in-degree bound of the 8-bit team kernel

static int words_per_set(int R) {
    const int W = (R + 31) / 32;
    int Ws = 1;
    while (Ws < W) Ws <<= 1;
    return Ws;
}

// Survival table for one beta, up to min(K_sat, max in-degree); ksat = INT32_MAX if the
// table never reaches zero.
void survival_table(double beta, int32_t max_deg, std::vector<uint64_t> &out, int32_t *ksat) {
    const uint64_t b = (uint64_t)llrint(beta * 4294967296.0);
    const uint64_t q = TWO32 - b;
    out.push_back(TWO32);
    *ksat = INT32_MAX;
    uint64_t prev = TWO32;
    for (int64_t k = 1; k <= max_deg; ++k) {
        const uint64_t cur = (q == TWO32) ? prev : (prev * q) >> 32;
        out.push_back(cur);
        prev = cur;
        if (cur == 0) {
            *ksat = (int32_t)k;
            break;
        }
    }
}

// One launch sequence over S sets that share Ws.
static int run_wave(fsgp_graph *g, int model, int ic_mode, int weighted, const SetSpec *const *sets, int S,
                    int Ws, int T, const fsgp_options &opt, cudaStream_t s) {
    const int32_t n = g->n;
    // the row kernels' model: weighted graphs draw per arc (SIR and SIS only)
    const int kmodel = weighted ? (model == FSGP_SIR ? kSirW : kSisW) : model;
    const int P = fsgp_model_planes(model);
    const int C = n_compartments(model);
    const int Wn = S * Ws;
    const int pd = Ws << __builtin_ctz((unsigned)S);   // largest power of two dividing Wn
    // Small graphs: every row in one launch (team or warp per row), dense steps
    // only, so that a step is two launches; their steps are bound by launch latency.
    // (automatic only when no degree-class or frontier option is given)
    const bool auto_classes = opt.small_max_deg == 0 && opt.hub_min_deg == 0 && opt.hub_chunk == 0 &&
                              opt.sparse_frac == 0.0;
    const bool fuse = g->max_deg < 65536 &&
                      (opt.fuse_rows > 0 ||
                       (opt.fuse_rows == 0 && auto_classes && (int64_t)n * Wn <= ((int64_t)1 << 20)));
    // Words per thread: 2 measured best on GB300 for large graphs; small graphs, bound by
    // the longest per-thread chain of dependent instructions, take one word per thread.
    int V = opt.vector_words ? opt.vector_words : (fuse ? 1 : 2);
    if (V != 1 && V != 2 && V != 4) return fail(FSGP_EINVAL, "vector_words must be 1, 2 or 4");
    if (V > pd) V = pd;
    const int SW = std::min(32 * V, pd);
    const int TEAM = SW / V;
    const int nslices = Wn / SW;
    // words per thread of the one-thread-per-row kernel
    if (opt.lane_words != 0 && opt.lane_words != 1 && opt.lane_words != 2 && opt.lane_words != 4 &&
        opt.lane_words != 8)
        return fail(FSGP_EINVAL, "lane_words must be 1, 2, 4 or 8");
    // (three-plane models stage at most 4 words per thread)
    const int lane_swl = std::min(std::min(opt.lane_words > 0 ? opt.lane_words : 8, P >= 3 ? 4 : 8), pd);
    const bool host_out = sets[0]->out_flags == FSGP_PTR_HOST;
    bool want_lanes = false, want_freq = false, any_init = false, want_steps = false;
    for (int i = 0; i < S; ++i) {
        want_lanes |= sets[i]->per_real != nullptr;
        want_freq |= sets[i]->freq != nullptr;
        any_init |= sets[i]->init_planes != nullptr;
        want_steps |= sets[i]->steps_run != nullptr;
    }
    // degree classes
    int small_max = opt.small_max_deg > 0 ? opt.small_max_deg : 255;
    int hub_min = fuse ? 65536 : (opt.hub_min_deg > 0 ? opt.hub_min_deg : 8192);
    int bs = bitlen(small_max + 1) - 1;              // small: d <= 2^bs - 1
    if (bs < 0) bs = 0;
    if (bs > kSmallBits) bs = kSmallBits;             // small rows count on 8-bit slices
    int bh = bitlen(hub_min);                         // hub: d >= 2^(bh-1)
    if (bh > 17) bh = 17;                             // mid rows count on 16-bit slices
    if (bh <= bs + 1) bh = bs + 2;
    if (bh > 32) bh = 32;
    small_max = (1 << bs) - 1;
    hub_min = 1 << (bh - 1);
    const int chunk = opt.hub_chunk > 0 ? std::min(opt.hub_chunk, 65535) : 8192;
    const double sparse_frac = fuse ? -1.0 : (opt.sparse_frac == 0.0 ? 0.05 : opt.sparse_frac);
    const unsigned long long sparse_limit =
        sparse_frac < 0.0 ? 0ull : (unsigned long long)(sparse_frac * (double)g->nnz);
    const bool allow_sparse = sparse_frac >= 0.0;

    int rc = ensure_hub_table(g, hub_min, chunk, s);
    if (rc) return rc;
    const int32_t n_hubs = g->hub.n_hubs;
    const int32_t start_mid = bh >= 1 ? g->cls.bucket_start[bh - 1] : n;
    const int32_t start_small = g->cls.bucket_start[bs];
    const int32_t n_mid = start_small - start_mid;
    // small rows by in-degree class; new ids follow the buckets in descending order
    // (bucket b: 2^(b-1) <= d < 2^b, bucket 0: d = 0), so each class is one range; rows
    // without in-arcs (from d0_start on) are only visited through the d0 list
    const int32_t start_lane = std::max(bs >= 2 ? g->cls.bucket_start[2] : start_small, start_small);  // d 1..3
    const int32_t start_small4 = bs >= 4 ? g->cls.bucket_start[4] : start_small;   // d 4..15
    const int32_t d0_start = g->d0_start;
    const int32_t n_lane = std::max(0, d0_start - start_lane);
    const int32_t n_d0 = n - d0_start;
    const int32_t n_small4 = start_lane - std::max(start_small4, start_small);
    const int32_t n_small = std::max(start_small4, start_small) - start_small;        // d 16..small_max
    const int32_t n_small_all = n - start_small;

    // per-set parameters and survival tables
    std::vector<uint64_t> surv_all;
    std::vector<size_t> surv_off((size_t)S), survmu_off((size_t)S), survnu_off((size_t)S);
    std::vector<SetParams> hp((size_t)S);
    int64_t seeds_total = 0, preal_total = 0, planes_total = 0;
    std::vector<int64_t> seed_off((size_t)S), preal_off((size_t)S), planes_off((size_t)S);
    const bool infection_table = model == FSGP_SIR || model == FSGP_SIS || model == FSGP_SEIR ||
                                 model == FSGP_SEIS || model == FSGP_SWIR;
    for (int i = 0; i < S; ++i) {
        const SetSpec &x = *sets[i];
        SetParams &p = hp[i];
        p = SetParams{};
        surv_off[i] = surv_all.size();
        int32_t ksat = INT32_MAX;
        if (infection_table) survival_table(x.beta, g->max_deg, surv_all, &ksat);
        else surv_all.push_back(TWO32);
        survmu_off[i] = survnu_off[i] = surv_off[i];
        p.ksat_mu = p.ksat_nu = ksat;
        if (model == FSGP_SWIR) {
            survmu_off[i] = surv_all.size();
            survival_table(x.mu, g->max_deg, surv_all, &p.ksat_mu);
            survnu_off[i] = surv_all.size();
            survival_table(x.nu, g->max_deg, surv_all, &p.ksat_nu);
        }
        p.a_lat = (uint64_t)llrint(x.alpha * 4294967296.0);
        p.key0 = (uint32_t)(x.rng_seed & 0xffffffffu);
        p.key1 = (uint32_t)(x.rng_seed >> 32);
        p.ksat = ksat;
        p.W = (x.R + 31) / 32;
        p.last_mask = (x.R & 31) ? ((1u << (x.R & 31)) - 1u) : 0xffffffffu;
        p.R = x.R;
        p.g_rec = (uint64_t)llrint(x.gamma * 4294967296.0);
        p.beta_f = (float)x.beta;
        p.p_const = (uint64_t)llrint(x.ic_p * 4294967296.0);
        seed_off[i] = seeds_total;
        if (!x.init_planes && x.seed_flags == FSGP_PTR_HOST) seeds_total += x.n_seeds;
        preal_off[i] = preal_total;
        if (x.per_real) preal_total += (int64_t)x.R * (T + 1) * C;
        planes_off[i] = planes_total;
        if (x.final_planes || x.init_planes) planes_total += (int64_t)P * n * p.W;
    }

    // ---------------------------------------------------------------- workspace
    const size_t T1 = (size_t)T + 1;
    const size_t state_words = (size_t)P * n * Wn;
    enum { O_STATE, O_PC, O_CTL, O_LIST0, O_LIST1, O_CSMALL, O_CMID, O_BITMAP, O_LANES,
           O_HUB, O_SURV, O_SEEDS, O_COUNTS, O_FREQ, O_PREAL, O_PLANES, O_PROF, O_SP, O_OUT,
           O_STEPS, O_D0, O_HUBSAT, O_END };
    size_t sz[O_END] = {0};
    sz[O_STATE] = 2 * state_words * sizeof(uint32_t);
    sz[O_PC] = T1 * S * kPC * sizeof(unsigned long long);
    sz[O_CTL] = sizeof(Ctl);
    // a row is listed once per work item: slices of the team kernels or of the lane kernel
    sz[O_LIST0] = sz[O_LIST1] = (size_t)n * std::max(nslices, Wn / lane_swl) * sizeof(int32_t);
    sz[O_CSMALL] = sz[O_CMID] = (size_t)n * sizeof(int32_t);
    sz[O_BITMAP] = ((size_t)n + 31) / 32 * sizeof(uint32_t);
    sz[O_LANES] = want_lanes ? (size_t)P * Wn * 32 * sizeof(int32_t) : 0;
    sz[O_HUB] = (size_t)n_hubs * Wn * 32 * sizeof(uint32_t);
    sz[O_SURV] = surv_all.size() * sizeof(uint64_t);
    sz[O_SEEDS] = (size_t)seeds_total * sizeof(int32_t);
    sz[O_COUNTS] = host_out ? T1 * C * S * sizeof(uint64_t) : 0;
    sz[O_FREQ] = (host_out && want_freq) ? (size_t)C * n * S * sizeof(uint32_t) : 0;
    sz[O_PREAL] = host_out ? (size_t)preal_total * sizeof(uint32_t) : 0;
    sz[O_PLANES] = (host_out || any_init) ? (size_t)planes_total * sizeof(uint32_t) : 0;
    sz[O_PROF] = FSGP_PROF_KINDS * sizeof(unsigned long long);
    sz[O_SP] = (size_t)S * sizeof(SetParams);
    sz[O_OUT] = (size_t)S * sizeof(SetOut);
    sz[O_STEPS] = (size_t)S * sizeof(int32_t);
    sz[O_D0] = (size_t)n_d0 * sizeof(int32_t);
    const bool hub_sat = !weighted && (model == FSGP_SIR || model == FSGP_SIS || model == FSGP_SEIR || model == FSGP_SEIS);
    sz[O_HUBSAT] = hub_sat ? (size_t)n_hubs * nslices * sizeof(uint32_t) : 0;
    size_t off[O_END], total = 0;
    for (int i = 0; i < O_END; ++i) {
        off[i] = total;
        total += align_up(sz[i]);
    }
    rc = ensure_workspace(g, total);
    if (rc) return rc;
    char *ws = (char *)g->ws.ptr;
    uint32_t *buf0 = (uint32_t *)(ws + off[O_STATE]);
    uint32_t *buf1 = buf0 + state_words;
    unsigned long long *pc = (unsigned long long *)(ws + off[O_PC]);
    Ctl *ctl = (Ctl *)(ws + off[O_CTL]);
    int32_t *list[2] = {(int32_t *)(ws + off[O_LIST0]), (int32_t *)(ws + off[O_LIST1])};
    uint32_t *hub_scratch = (uint32_t *)(ws + off[O_HUB]);
    uint64_t *d_surv = (uint64_t *)(ws + off[O_SURV]);
    unsigned long long *d_prof = (unsigned long long *)(ws + off[O_PROF]);
    SetParams *d_sp = (SetParams *)(ws + off[O_SP]);
    SetOut *d_out = (SetOut *)(ws + off[O_OUT]);
    int32_t *d_steps = (int32_t *)(ws + off[O_STEPS]);
    for (int i = 0; i < S; ++i) {
        hp[i].surv = d_surv + surv_off[i];
        hp[i].surv_mu = d_surv + survmu_off[i];
        hp[i].surv_nu = d_surv + survnu_off[i];
    }
    FSGP_CUDA(cudaMemcpyAsync(d_surv, surv_all.data(), sz[O_SURV], cudaMemcpyHostToDevice, s));
    FSGP_CUDA(cudaMemcpyAsync(d_sp, hp.data(), sz[O_SP], cudaMemcpyHostToDevice, s));
    // device output pointers of each set (caller memory, or staging for host results)
    std::vector<SetOut> ho((size_t)S);
    for (int i = 0; i < S; ++i) {
        const SetSpec &x = *sets[i];
        SetOut &o = ho[i];
        if (host_out) {
            o.counts = (unsigned long long *)(ws + off[O_COUNTS]) + (size_t)i * T1 * C;
            o.freq = x.freq ? (uint32_t *)(ws + off[O_FREQ]) + (size_t)i * C * n : nullptr;
            o.per_real = x.per_real ? (uint32_t *)(ws + off[O_PREAL]) + preal_off[i] : nullptr;
            o.planes = x.final_planes ? (uint32_t *)(ws + off[O_PLANES]) + planes_off[i] : nullptr;
        } else {
            o.counts = (unsigned long long *)x.counts;
            o.freq = x.freq;
            o.per_real = x.per_real;
            o.planes = x.final_planes;
        }
        o.steps = d_steps + i;
    }
    FSGP_CUDA(cudaMemcpyAsync(d_out, ho.data(), sz[O_OUT], cudaMemcpyHostToDevice, s));

    // ---------------------------------------------------------------- launch shape
    const size_t smem_lanes = want_lanes ? (size_t)P * Wn * 32 * sizeof(int32_t) : 0;
    if (smem_lanes > 32 * 1024) return fail(FSGP_EINVAL, "per-lane counters exceed shared memory");
    RowOccupancy occ{};
    occ.swl = lane_swl;
    rc = occupancy_model(kmodel, V, TEAM, smem_lanes, &occ);
    if (rc) return rc;
    Prof prof;
    const bool profiling = opt.profile != nullptr;
    int64_t launches = 0;
    StepLaunch L;
    memset(&L, 0, sizeof L);   // padding too: the bytes form the graph-cache signature
    L.V = V;
    L.TEAM = TEAM;
    L.smem_lanes = smem_lanes;
    // the 16..small_max kernel also takes every small row of a frontier step
    // fused rows: the team-per-row kernel (8-bit counters) when every in-degree is below
    // 256, else the warp-per-row kernel (16-bit counters)
    const bool fuse_team = fuse && g->max_deg <= kSmallMaxFused;
    // all T steps in one cooperative launch (fused team rows, no per-lane counts)
    const bool persist = fuse_team && opt.persistent >= 0 && !want_lanes && !profiling && V == 1 && T >= 1 &&
                         n > 0;
    L.have_small = fuse ? (fuse_team && n > 0) : n_small_all > 0;
    L.have_small4 = n_small4 > 0 && !fuse;
    L.have_lane = (n_lane > 0 || n_d0 > 0) && !fuse;
    L.swl = occ.swl;
    L.have_mid = fuse ? (!fuse_team && n > 0) : n_mid > 0;
    L.have_hub = n_hubs > 0;
    L.prof = profiling ? &prof : nullptr;
    const int64_t items_small = (int64_t)(fuse_team ? n : n_small_all) * nslices;
    const int64_t items_mid = (int64_t)(fuse ? n : n_mid) * nslices;
    const int64_t items_lane = (int64_t)(n_lane + n_d0) * (Wn / occ.swl);
    const int per_block_small = (kBlock / 32) * (32 / TEAM);
    auto grid_for_items = [&](int per_sm, int64_t items) {
        return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * per_sm,
                                                           (items + per_block_small - 1) / per_block_small));
    };
    L.grid_small = grid_for_items(occ.small, items_small);
    L.grid_small4 = grid_for_items(occ.small4, (int64_t)n_small4 * nslices);
    L.grid_lane = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * occ.lane,
                                                              (items_lane + kBlock - 1) / kBlock));
    L.grid_mid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * occ.mid,
                                                             (items_mid + (kBlock / 32) - 1) / (kBlock / 32)));
    L.grid_hub = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * occ.hub,
                                                             g->hub.n_chunks * nslices));
    L.grid_fin = (int)std::max<int64_t>(1, ((int64_t)n_hubs + (kBlock / 32) - 1) / (kBlock / 32));

    const int grid_mark = g->sm_count * 8;
    const int grid_scan = grid_cap((int64_t)n, kBlock, g->sm_count, 8);

    StepArgs A;
    memset(&A, 0, sizeof A);
    A.rp = g->rp2;
    A.col = g->col2;
    A.orig = g->rows_sorted;
    A.pos = g->pos;
    A.arc0 = g->arc0;
    A.out_ptr = g->out_ptr;
    A.out_dst = g->out_dst;
    A.n = n;
    A.Ws = Ws;
    A.ws_shift = __builtin_ctz((unsigned)Ws);
    A.S = S;
    A.Wn = Wn;
    A.nslices = nslices;
    A.gbase = (uint32_t)(opt.r_offset >> 5);
    A.small_max_deg = small_max;
    A.hub_min_deg = hub_min;
    A.plane_words = (size_t)n * Wn;
    A.sp = d_sp;
    A.ic_mode = ic_mode;
    A.ctl = ctl;
    A.lane_cnt = want_lanes ? (int32_t *)(ws + off[O_LANES]) : nullptr;
    A.np = P;
    A.r_small = fuse_team ? 0 : start_small;
    A.n_small = fuse_team ? n : n_small;
    A.r_small4 = std::max(start_small4, start_small);
    A.n_small4 = n_small4;
    A.r_lane = start_lane;
    A.n_lane = n_lane;
    A.r_mid = fuse ? 0 : start_mid;
    A.n_mid = fuse ? n : n_mid;
    A.r_d0 = d0_start;
    A.lane_tab = (g->lane_tab && n_lane > 0) ? g->lane_tab + (start_lane - g->lane_start) : nullptr;
    A.d0_list = (int32_t *)(ws + off[O_D0]);
    A.cand_small = (int32_t *)(ws + off[O_CSMALL]);
    A.cand_mid = (int32_t *)(ws + off[O_CMID]);
    A.bitmap = (uint32_t *)(ws + off[O_BITMAP]);
    A.hub_chunk_base = g->hub.d_chunk_base;
    A.n_hubs = n_hubs;
    A.n_hub_chunks = g->hub.n_chunks;
    A.hub_chunk = chunk;
    A.hub_scratch = hub_scratch;
    A.hub_sat = (hub_sat && n_hubs > 0) ? (uint32_t *)(ws + off[O_HUBSAT]) : nullptr;
    A.prof_bytes = profiling ? d_prof : nullptr;
    A.arc_w = weighted ? g->arc_w : nullptr;

    FSGP_CUDA(cudaMemsetAsync(ws + off[O_STATE], 0, sz[O_STATE], s));
    FSGP_CUDA(cudaMemsetAsync(pc, 0, sz[O_PC], s));
    FSGP_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    {
        // the step-0 scan always lists the pushing rows for step 1
        static const int32_t one[3] = {1, 1, 0};
        FSGP_CUDA(cudaMemcpyAsync(&ctl->build_list, one, sizeof one, cudaMemcpyHostToDevice, s));
    }
    FSGP_CUDA(cudaMemsetAsync(A.bitmap, 0, sz[O_BITMAP], s));
    if (A.lane_cnt) FSGP_CUDA(cudaMemsetAsync(A.lane_cnt, 0, sz[O_LANES], s));
    if (sz[O_HUB]) FSGP_CUDA(cudaMemsetAsync(hub_scratch, 0, sz[O_HUB], s));
    if (sz[O_HUBSAT]) FSGP_CUDA(cudaMemsetAsync(A.hub_sat, 0, sz[O_HUBSAT], s));
    if (profiling) {
        FSGP_CUDA(cudaMemsetAsync(d_prof, 0, sz[O_PROF], s));
        prof.start(PK_INIT, s);
    }
    for (int i = 0; i < S; ++i) {
        const SetSpec &x = *sets[i];
        const int ws0 = i * Ws;
        if (x.init_planes) {
            const uint32_t *src = x.init_planes;
            if (host_out) {
                uint32_t *stage = (uint32_t *)(ws + off[O_PLANES]) + planes_off[i];
                FSGP_CUDA(cudaMemcpyAsync(stage, src, sizeof(uint32_t) * (size_t)P * n * hp[i].W,
                                          cudaMemcpyHostToDevice, s));
                src = stage;
            }
            k_import<<<grid_cap((int64_t)P * n * Ws, 256, g->sm_count, 16), 256, 0, s>>>(
                src, P, n, hp[i].W, Ws, Wn, ws0, hp[i].last_mask, g->pos, buf0, buf1);
            ++launches;
        } else if (x.n_seeds > 0) {
            const int32_t *sd = x.seeds;
            if (x.seed_flags == FSGP_PTR_HOST) {
                int32_t *stage = (int32_t *)(ws + off[O_SEEDS]) + seed_off[i];
                FSGP_CUDA(cudaMemcpyAsync(stage, sd, sizeof(int32_t) * (size_t)x.n_seeds,
                                          cudaMemcpyHostToDevice, s));
                sd = stage;
            }
            k_seed<<<grid_cap(x.n_seeds * Ws, 256, g->sm_count, 16), 256, 0, s>>>(
                buf0, buf1, A.plane_words, model == FSGP_IC || model == FSGP_LT, sd, x.n_seeds,
                g->pos, Wn, ws0, Ws, hp[i].W, hp[i].last_mask);
            ++launches;
        }
    }
    // The launch sequence from here to the results is free of host synchronisation and
    // host-memory copies, so it can be captured into one CUDA graph and launched at once.
    // (the legacy default stream cannot be captured; such callers launch directly)
    const bool capture = opt.capture_graph != 0 && !profiling && !persist && s != nullptr &&
                         s != cudaStreamLegacy && s != cudaStreamPerThread;
    // step 0
    A.cur = buf0;
    A.nxt = buf1;
    A.pc = pc;
    A.k = 0;
    A.t = (uint32_t)opt.t0;
    A.list_in = list[1];
    A.list_out = list[0];
    // The step loop's kernels and their arguments follow from these values (the
    // workspace and output pointers included): a run with the same signature reuses the
    // executable graph captured by an earlier run instead of capturing a new one.
    std::vector<uint8_t> sig;
    int cached = -1;
    if (capture) {
        auto put = [&sig](const void *p, size_t b) {
            sig.insert(sig.end(), (const uint8_t *)p, (const uint8_t *)p + b);
        };
        const int flags[6] = {kmodel, T, allow_sparse ? 1 : 0, any_init ? 1 : 0, want_lanes ? 1 : 0,
                              want_freq ? 1 : 0};
        put(flags, sizeof flags);
        put(&sparse_limit, sizeof sparse_limit);
        put(&A, sizeof A);
        put(&L, sizeof L);
        put(&d_out, sizeof d_out);
        for (int i = 0; i < S; ++i) {
            put(&ho[i].planes, sizeof ho[i].planes);
            put(&hp[i].W, sizeof hp[i].W);
        }
        for (size_t c = 0; c < g->execs.size(); ++c)
            if (g->execs[c].sig == sig) cached = (int)c;
    }
    if (cached >= 0) {
        FSGP_CUDA(cudaGraphLaunch(g->execs[(size_t)cached].exec, s));
    } else {
    if (capture) FSGP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    k_init_scan<<<grid_scan, kBlock, smem_lanes, s>>>(A, model);
    ++launches;
    if (profiling) prof.stop(s);
    FSGP_CUDA(cudaGetLastError());
    bool persisted = false;
    if (persist) {
        // no row lists: the loop runs dense steps only
        FSGP_CUDA(cudaMemsetAsync(&ctl->build_list, 0, sizeof(int32_t), s));
        PersistArgs Q;
        Q.buf0 = buf0;
        Q.buf1 = buf1;
        Q.pc = pc;
        Q.T = (int32_t)T;
        Q.t0 = (uint32_t)opt.t0;
        Q.spin_limit = kPersistSpinCycles;
        int grid_used = 0;
        rc = launch_persist_model(kmodel, A, Q, TEAM, L.grid_small, L.smem_lanes, g->sm_count, s, &grid_used);
        if (rc == FSGP_OK) {
            const int width = S * kPC;
            k_pc_prefix<<<(width + 255) / 256, 256, 0, s>>>(pc, (int)T, width);
            launches += 2;
            persisted = true;
        } else if (rc != FSGP_EUNSUPPORTED) {
            return rc;
        }
    }
    for (int k = 1; k <= T && !persisted; ++k) {
        A.k = k;
        A.t = (uint32_t)(opt.t0 + k);
        A.cur = (k & 1) ? buf0 : buf1;
        A.nxt = (k & 1) ? buf1 : buf0;
        A.pc = pc + (size_t)k * S * kPC;
        A.list_in = list[(k - 1) & 1];
        A.list_out = list[k & 1];
        const int force_dense = !allow_sparse || (k == 1 && any_init && model == FSGP_LT);
        if (profiling) prof.start(PK_BEGIN, s);
        k_begin<<<want_lanes ? std::max(1, (Wn * 32 + 255) / 256) : 1, 256, 0, s>>>(
            A, model, sparse_limit, force_dense, d_out, (int)T1);
        if (profiling) prof.stop(s);
        if (allow_sparse) {
            if (profiling) prof.start(PK_MARK, s);
            k_mark<<<grid_mark, kBlock, 0, s>>>(A);
            if (profiling) prof.stop(s);
        }
        rc = launch_rows_model(kmodel, A, L, s);
        if (rc) return rc;
        launches += 1 + (allow_sparse ? 1 : 0) + (L.have_hub ? (A.hub_sat ? 3 : 2) : 0) + (L.have_mid ? 1 : 0) +
                    (L.have_small ? 1 : 0) + (L.have_small4 ? 1 : 0) + (L.have_lane ? 1 : 0);
    }
    FSGP_CUDA(cudaGetLastError());
    if (profiling) prof.start(PK_RESULTS, s);
    const int64_t fin_work = std::max<int64_t>((int64_t)T1 * S, (int64_t)Wn * 32);
    k_finalize<<<(int)std::max<int64_t>(1, std::min<int64_t>(1024, (fin_work + 255) / 256)), 256, 0, s>>>(
        A, model, T, pc, d_out);
    ++launches;
    if (want_freq) {
        k_freq<<<grid_cap(n, 256, g->sm_count, 16), 256, 0, s>>>(A, model, buf0, buf1, d_out);
        ++launches;
    }
    for (int i = 0; i < S; ++i) {
        if (!ho[i].planes) continue;
        k_export<<<grid_cap((int64_t)P * n * hp[i].W, 256, g->sm_count, 16), 256, 0, s>>>(
            A, P, i * Ws, hp[i].W, buf0, buf1, ho[i].planes);
        ++launches;
    }
    if (profiling) prof.stop(s);
    if (capture) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return cuda_fail(e, "cudaGraphLaunch");
        }
        if ((int)g->execs.size() >= kExecCacheSize) {
            cudaGraphExecDestroy(g->execs.front().exec);   // released once its launches complete
            g->execs.erase(g->execs.begin());
        }
        g->execs.push_back(ExecCache{std::move(sig), exec});
    }
    }
    FSGP_CUDA(cudaGetLastError());

    if (want_steps && !host_out)
        for (int i = 0; i < S; ++i)
            if (sets[i]->steps_run)
                FSGP_CUDA(cudaMemcpyAsync(sets[i]->steps_run, d_steps + i, sizeof(int32_t),
                                          cudaMemcpyDeviceToDevice, s));
    std::vector<int32_t> hsteps;
    if (want_steps && host_out) {
        hsteps.resize((size_t)S);
        FSGP_CUDA(cudaMemcpyAsync(hsteps.data(), d_steps, sz[O_STEPS], cudaMemcpyDeviceToHost, s));
    }
    if (host_out) {
        for (int i = 0; i < S; ++i) {
            const SetSpec &x = *sets[i];
            FSGP_CUDA(cudaMemcpyAsync(x.counts, ho[i].counts, T1 * C * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
            if (x.freq)
                FSGP_CUDA(cudaMemcpyAsync(x.freq, ho[i].freq, (size_t)C * n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            if (x.per_real)
                FSGP_CUDA(cudaMemcpyAsync(x.per_real, ho[i].per_real, (size_t)x.R * T1 * C * sizeof(uint32_t),
                                          cudaMemcpyDeviceToHost, s));
            if (x.final_planes)
                FSGP_CUDA(cudaMemcpyAsync(x.final_planes, ho[i].planes, (size_t)P * n * hp[i].W * sizeof(uint32_t),
                                          cudaMemcpyDeviceToHost, s));
        }
    }
    int32_t timed_out = 0;
    if (persist && host_out) FSGP_CUDA(cudaMemcpyAsync(&timed_out, &ctl->err, sizeof timed_out, cudaMemcpyDeviceToHost, s));
    if (host_out || profiling) FSGP_CUDA(cudaStreamSynchronize(s));
    if (timed_out) return fail(FSGP_ETIMEOUT, "a grid barrier of the persistent step loop timed out");
    if (want_steps && host_out)
        for (int i = 0; i < S; ++i)
            if (sets[i]->steps_run) *sets[i]->steps_run = hsteps[i];
    if (profiling) {
        unsigned long long hb[FSGP_PROF_KINDS];
        Ctl hc;
        FSGP_CUDA(cudaMemcpyAsync(hb, d_prof, sizeof hb, cudaMemcpyDeviceToHost, s));
        FSGP_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, s));
        FSGP_CUDA(cudaStreamSynchronize(s));
        fsgp_profile *pf = opt.profile;
        for (size_t i = 0; i + 1 < prof.ev.size(); i += 2) {
            float ms = 0.f;
            FSGP_CUDA(cudaEventElapsedTime(&ms, prof.ev[i], prof.ev[i + 1]));
            const int kd = prof.kind[i];
            pf->ms[kd] += ms;
            pf->launches[kd] += 1;
        }
        for (cudaEvent_t e : prof.ev) cudaEventDestroy(e);
        for (int i = 0; i < FSGP_PROF_KINDS; ++i) pf->alg_bytes[i] += (double)hb[i];
        pf->dense_steps += hc.dense_steps;
        pf->sparse_steps += hc.sparse_steps;
        pf->kernel_launches += launches;
    }
    return FSGP_OK;
}

int run_sets(fsgp_graph *g, int model, int ic_mode, int weighted, const SetSpec *sets, int n_sets, int T,
             const fsgp_options &opt, cudaStream_t s) {
    if (n_sets < 1) return FSGP_OK;
    if (weighted) {
        if (model != FSGP_SIR && model != FSGP_SIS)
            return fail(FSGP_EINVAL, "weighted graphs: SIR, SIS or SI only");
        if (!g->arc_w) return fail(FSGP_EINVAL, "weighted run on a graph without arc weights");
    }
    const uint32_t of = sets[0].out_flags;
    for (int i = 0; i < n_sets; ++i) {
        const SetSpec &x = sets[i];
        if (x.R < 1 || x.R > kMaxR) return fail(FSGP_EINVAL, "R must be in [1, 4096]");
        if (!x.counts) return fail(FSGP_EINVAL, "result counts buffer is NULL");
        if (x.out_flags != of) return fail(FSGP_EINVAL, "all result buffers of one call must be host or all device");
        auto bad_p = [](double p) { return !(p >= 0.0 && p <= 1.0); };
        if (bad_p(x.beta) || bad_p(x.gamma) || bad_p(x.ic_p) || bad_p(x.alpha) || bad_p(x.mu) || bad_p(x.nu))
            return fail(FSGP_EINVAL, "probabilities must lie in [0, 1]");
        if (!x.init_planes && x.n_seeds > 0) {
            if (!x.seeds) return fail(FSGP_EINVAL, "seed_nodes is NULL");
            std::vector<int32_t> host_copy;
            const int32_t *hs = x.seeds;
            if (x.seed_flags == FSGP_PTR_DEVICE) {
                host_copy.resize((size_t)x.n_seeds);
                FSGP_CUDA(cudaMemcpy(host_copy.data(), x.seeds, sizeof(int32_t) * (size_t)x.n_seeds,
                                     cudaMemcpyDeviceToHost));
                hs = host_copy.data();
            }
            for (int64_t j = 0; j < x.n_seeds; ++j)
                if (hs[j] < 0 || hs[j] >= g->n) return fail(FSGP_EINVAL, "seed node out of range");
        }
    }
    // group by words per set, then waves of at most kMaxSets sets that fit the state
    // budget and, when per-realization counts are wanted, the shared-memory lane counters
    std::vector<int> order((size_t)n_sets);
    for (int i = 0; i < n_sets; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return words_per_set(sets[a].R) < words_per_set(sets[b].R);
    });
    const int P = fsgp_model_planes(model);
    const size_t budget = (size_t)48 << 30;   // bytes of double-buffered state per wave
    size_t i = 0;
    while (i < order.size()) {
        const int Ws = words_per_set(sets[order[i]].R);
        const size_t per_set_state = 2ull * P * (size_t)g->n * Ws * sizeof(uint32_t);
        const int smax = (int)std::max<size_t>(
            1, std::min<size_t>(kMaxSets, budget / std::max<size_t>(per_set_state, 1)));
        std::vector<const SetSpec *> wave;
        bool lanes = false;
        while (i < order.size() && words_per_set(sets[order[i]].R) == Ws && (int)wave.size() < smax) {
            const SetSpec *x = &sets[order[i]];
            const bool l2 = lanes || x->per_real;
            // 32 KB of lane counters: planes x words x 32 lanes x 4 B
            if (l2 && !wave.empty() && (int)(wave.size() + 1) * Ws * P > 256) break;
            lanes = l2;
            wave.push_back(x);
            ++i;
        }
        const int rc = run_wave(g, model, ic_mode, weighted, wave.data(), (int)wave.size(), Ws, T, opt, s);
        if (rc) return rc;
    }
    return FSGP_OK;
}

}  // namespace fsgp

using namespace fsgp;

extern "C" int fsgp_simulate(const fsgp_graph *gc, int32_t model, const fsgp_params *params,
                             const int32_t *seed_nodes, const int64_t *seed_offsets,
                             int32_t n_sets, uint32_t seed_flags, int32_t R, int32_t T,
                             uint64_t rng_seed, const fsgp_options *opt_in, fsgp_result *out,
                             void *stream) {
    set_error("");
    fsgp_graph *g = const_cast<fsgp_graph *>(gc);
    if (!g) return fail(FSGP_EINVAL, "graph is NULL");
    if (model < FSGP_SIR || model > FSGP_SWIR) return fail(FSGP_EINVAL, "unknown model");
    if (!params) return fail(FSGP_EINVAL, "params is NULL");
    if (!out || !out->counts) return fail(FSGP_EINVAL, "result counts buffer is NULL");
    if (out->flags != FSGP_PTR_HOST && out->flags != FSGP_PTR_DEVICE)
        return fail(FSGP_EINVAL, "bad result flags");
    if (R < 1 || R > kMaxR) return fail(FSGP_EINVAL, "R must be in [1, 4096]");
    if (T < 0) return fail(FSGP_EINVAL, "T must be >= 0");
    if (n_sets < 1) return fail(FSGP_EINVAL, "n_sets must be >= 1");
    if (params->ic_mode != FSGP_IC_WEIGHTED_CASCADE && params->ic_mode != FSGP_IC_CONSTANT)
        return fail(FSGP_EINVAL, "bad ic_mode");
    fsgp_options opt{};
    if (opt_in) opt = *opt_in;
    if (opt.r_offset < 0 || (opt.r_offset & 31)) return fail(FSGP_EINVAL, "r_offset must be a non-negative multiple of 32");
    if (opt.t0 < 0) return fail(FSGP_EINVAL, "t0 must be >= 0");
    if ((int64_t)opt.t0 + T > (int64_t)UINT32_MAX) return fail(FSGP_EINVAL, "t0 + T too large");
    const bool use_init = opt.init_planes != nullptr;
    if (!use_init) {
        if (!seed_offsets) return fail(FSGP_EINVAL, "seed_offsets is NULL");
        if (seed_flags != FSGP_PTR_HOST && seed_flags != FSGP_PTR_DEVICE) return fail(FSGP_EINVAL, "bad seed flags");
        if (seed_offsets[0] != 0) return fail(FSGP_EINVAL, "seed_offsets[0] must be 0");
        for (int s = 0; s < n_sets; ++s)
            if (seed_offsets[s + 1] < seed_offsets[s]) return fail(FSGP_EINVAL, "seed_offsets must be non-decreasing");
        if (seed_offsets[n_sets] > 0 && !seed_nodes) return fail(FSGP_EINVAL, "seed_nodes is NULL");
    }
    int dev = 0;
    FSGP_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(FSGP_EINVAL, "current device differs from the graph's device");
    const int P = fsgp_model_planes(model);
    const int C = n_compartments(model);
    const int W = (R + 31) / 32;
    const size_t T1 = (size_t)T + 1;
    // SI is SIS without recovery: the same planes, draws and compartments
    const bool si = model == FSGP_SI;
    const int run_model = si ? FSGP_SIS : model;
    std::vector<SetSpec> sets((size_t)n_sets);
    for (int i = 0; i < n_sets; ++i) {
        SetSpec &x = sets[i];
        x = SetSpec{};
        x.beta = params->beta;
        x.gamma = si ? 0.0 : params->gamma;
        x.ic_p = params->ic_p;
        x.alpha = params->alpha;
        x.mu = params->mu;
        x.nu = params->nu;
        x.rng_seed = rng_seed;
        x.R = R;
        if (use_init) {
            x.init_planes = opt.init_planes + (size_t)i * P * g->n * W;
        } else {
            x.seeds = seed_nodes ? seed_nodes + seed_offsets[i] : nullptr;
            x.n_seeds = seed_offsets[i + 1] - seed_offsets[i];
            x.seed_flags = seed_flags;
        }
        x.counts = out->counts + (size_t)i * T1 * C;
        x.freq = out->freq ? out->freq + (size_t)i * C * g->n : nullptr;
        x.per_real = out->per_real ? out->per_real + (size_t)i * R * T1 * C : nullptr;
        x.final_planes = out->final_planes ? out->final_planes + (size_t)i * P * g->n * W : nullptr;
        x.steps_run = out->steps_run ? out->steps_run + i : nullptr;
        x.out_flags = out->flags;
    }
    return run_sets(g, run_model, params->ic_mode, params->weighted ? 1 : 0, sets.data(), n_sets, T, opt,
                    (cudaStream_t)stream);
}

extern "C" int fsgp_selftest_barrier(int32_t ctas, int32_t missing, int32_t rounds, int64_t spin_cycles,
                                     void *stream) {
    set_error("");
    if (ctas < 1 || ctas > 4096 || missing < 0 || missing > 4096 || rounds < 1 || rounds > 1000000 ||
        spin_cycles < 1 || spin_cycles > ((int64_t)1 << 34))
        return fail(FSGP_EINVAL, "selftest_barrier: ctas in [1, 4096], missing in [0, 4096], rounds >= 1, "
                                 "spin_cycles in [1, 2^34]");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    FSGP_CUDA(cudaGetDevice(&dev));
    FSGP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FSGP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_selftest, 32, 0));
    if ((int64_t)ctas > (int64_t)per_sm * sms) return fail(FSGP_EINVAL, "selftest_barrier: more CTAs than fit at once");
    uint32_t *d = nullptr;
    FSGP_CUDA(cudaMalloc(&d, 4 * sizeof(uint32_t)));   // count, generation, error flag
    int rc = FSGP_OK;
    int32_t err = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, 4 * sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        uint32_t *bar = d;
        int32_t *errp = reinterpret_cast<int32_t *>(d + 2);
        int r = rounds, m = missing;
        long long lim = (long long)spin_cycles;
        void *args[] = {&bar, &errp, &r, &m, &lim};
        e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(ctas), dim3(32), args, 0, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d + 2, sizeof err, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "selftest_barrier");
    cudaFree(d);
    if (rc == FSGP_OK && err) rc = fail(FSGP_ETIMEOUT, "selftest_barrier: a barrier wait ran out");
    return rc;
}
