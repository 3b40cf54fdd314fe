// simulate.cu -- fsgp_simulate: initial state (Algorithm 1, "initialize states"), the
// step loop (one synchronous step per iteration, X^{k+1} <- X^k double buffer of
// Algorithm 1), the frontier path ("decide whether x needs to update", Algorithm 1),
// and the reductions of the results (per-step compartment counts, per-node final
// frequencies, per-realization counts; the 0/1/2 state conversion of Appendix A.1).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "step.cuh"

namespace fsgp {

// ------------------------------------------------------------------------ kernels

// Seed nodes: all valid lanes of the source planes set, in both buffers.
__global__ void k_seed(uint32_t *buf0, uint32_t *buf1, size_t plane_words, int both_planes,
                       const int32_t *__restrict__ seeds, int64_t ns, int Ws, int W,
                       uint32_t last_mask) {
    const int64_t total = ns * Ws;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t si = i / Ws;
        const int w = (int)(i % Ws);
        const int32_t v = seeds[si];
        const uint32_t m = w < W - 1 ? 0xffffffffu : (w == W - 1 ? last_mask : 0u);
        const size_t off = (size_t)v * Ws + w;
        buf0[off] = m;
        buf1[off] = m;
        if (both_planes) {
            buf0[plane_words + off] = m;
            buf1[plane_words + off] = m;
        }
    }
}

// Caller-supplied start planes [planes][n][W] -> both buffers [planes][n][Ws].
__global__ void k_import(const uint32_t *__restrict__ in, int planes, int32_t n, int W, int Ws,
                         uint32_t last_mask, uint32_t *buf0, uint32_t *buf1) {
    const int64_t total = (int64_t)planes * n * Ws;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % Ws);
        const int64_t pv = i / Ws;   // plane * n + v
        uint32_t x = 0u;
        if (w < W) {
            x = in[pv * W + w];
            if (w == W - 1) x &= last_mask;
        }
        buf0[i] = x;
        buf1[i] = x;
    }
}

// Step-0 totals, per-lane counts and the rows whose source lanes push at step 1.
__global__ void __launch_bounds__(kBlock) k_init_scan(StepArgs A, int model) {
    extern __shared__ int32_t s_lane[];
    const int nl = A.Ws * 32;
    const bool lanes_on = A.lane_cnt != nullptr;
    if (lanes_on) {
        for (int i = threadIdx.x; i < 2 * nl; i += blockDim.x) s_lane[i] = 0;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    Accum acc;
    const bool two = model != FSGP_SIS;
    for (int64_t base = gwarp * 32; base < A.n; base += nwarps * 32) {
        const int64_t v = base + lane;
        const bool has = v < A.n;
        bool push = false;
        if (has) {
            for (int w = 0; w < A.Ws; ++w) {
                const size_t off = (size_t)v * A.Ws + w;
                const uint32_t s0 = A.cur[off];
                const uint32_t s1 = two ? A.cur[A.plane_words + off] : 0u;
                acc.d0 += __popc(s0);
                acc.d1 += __popc(s1);
                if (lanes_on) {
                    lane_deltas(s_lane, w, 0u, s0);
                    if (two) lane_deltas(s_lane + nl, w, 0u, s1);
                }
                push |= (model == FSGP_SIR || model == FSGP_SIS) ? (s0 != 0u) : (s1 != 0u);
            }
        }
        if (push) acc.push_deg += (unsigned long long)(A.out_ptr[v + 1] - A.out_ptr[v]);
        if (has && A.prof_bytes) acc.bytes += (two ? 2ull : 1ull) * 4ull * (unsigned long long)A.Ws;
        list_append(A, has && push, (int32_t)((uint32_t)v | kPushBit), 0);
    }
    flush_accum(A, acc, 0, PK_INIT);
    if (lanes_on) flush_lanes(A, s_lane, nl);
}

__device__ __forceinline__ void compartments(int model, int64_t total, int64_t p0, int64_t p1,
                                             int64_t out[3]) {
    if (model == FSGP_SIR) {
        out[0] = total - p0 - p1; out[1] = p0; out[2] = p1;
    } else if (model == FSGP_SIS) {
        out[0] = total - p0; out[1] = p0; out[2] = 0;
    } else {
        out[0] = total - p0; out[1] = p1; out[2] = p0 - p1;
    }
}

// Per-realization snapshot of the running lane counts into per_real[r][kk][3].
__device__ void snapshot_lanes(const StepArgs &A, int model, uint32_t *per_real, int R, int T1,
                               int kk) {
    const int nl = A.Ws * 32;
    for (int r = threadIdx.x + blockIdx.x * blockDim.x; r < R; r += blockDim.x * gridDim.x) {
        int64_t o[3];
        compartments(model, A.n, A.lane_cnt[r], A.lane_cnt[nl + r], o);
        uint32_t *dst = per_real + ((size_t)r * T1 + kk) * 3;
        dst[0] = (uint32_t)o[0];
        dst[1] = (uint32_t)o[1];
        dst[2] = (uint32_t)o[2];
    }
}

// Start of step k: quiescence test (IC/LT), running totals, dense/sparse choice, and the
// per-realization snapshot of step k-1.
__global__ void k_begin(StepArgs A, int model, unsigned long long sparse_limit, int force_dense,
                        uint32_t *per_real, int R, int T1) {
    if (per_real) snapshot_lanes(A, model, per_real, R, T1, A.k - 1);
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    Ctl *C = A.ctl;
    unsigned long long *prev = A.pc - 2;
    A.pc[0] = prev[0];
    A.pc[1] = prev[1];
    if (C->stop) return;
    if ((model == FSGP_IC || model == FSGP_LT) && prev[1] == 0ull) {
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
            const int32_t d = __ldg(A.row_ptr + x + 1) - __ldg(A.row_ptr + x);
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
            const int32_t b = __ldg(A.out_ptr + v), e = __ldg(A.out_ptr + v + 1);
            for (int32_t j = b; j < e; j += 32) {
                const int32_t x = j + lane < e ? __ldg(A.out_dst + j + lane) : -1;
                mark_round(A, x);
            }
        }
    }
}

// Results: compartment totals per step, steps run, last per-realization snapshot.
__global__ void k_finalize(StepArgs A, int model, int T, unsigned long long NR,
                           const unsigned long long *pc_all, unsigned long long *counts,
                           int32_t *steps_run, uint32_t *per_real, int R) {
    for (int k = threadIdx.x + blockIdx.x * blockDim.x; k <= T; k += blockDim.x * gridDim.x) {
        int64_t o[3];
        compartments(model, (int64_t)NR, (int64_t)pc_all[2 * k], (int64_t)pc_all[2 * k + 1], o);
        counts[3 * k] = (unsigned long long)o[0];
        counts[3 * k + 1] = (unsigned long long)o[1];
        counts[3 * k + 2] = (unsigned long long)o[2];
    }
    if (per_real) snapshot_lanes(A, model, per_real, R, T + 1, T);
    if (steps_run && blockIdx.x == 0 && threadIdx.x == 0) *steps_run = A.ctl->steps_done;
}

// Per-node final compartment frequencies.
__global__ void k_freq(StepArgs A, int model, const uint32_t *buf0, const uint32_t *buf1, int R,
                       uint32_t *freq) {
    const uint32_t *st = (A.ctl->steps_done & 1) ? buf1 : buf0;
    const bool two = model != FSGP_SIS;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < A.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t p0 = 0, p1 = 0;
        for (int w = 0; w < A.W; ++w) {
            const size_t off = (size_t)v * A.Ws + w;
            p0 += __popc(st[off]);
            if (two) p1 += __popc(st[A.plane_words + off]);
        }
        int64_t o[3];
        compartments(model, R, p0, p1, o);
        freq[v] = (uint32_t)o[0];
        freq[(size_t)A.n + v] = (uint32_t)o[1];
        freq[2 * (size_t)A.n + v] = (uint32_t)o[2];
    }
}

// Final planes -> caller layout [planes][n][W].
__global__ void k_export(StepArgs A, int planes, const uint32_t *buf0, const uint32_t *buf1,
                         uint32_t *out) {
    const uint32_t *st = (A.ctl->steps_done & 1) ? buf1 : buf0;
    const int64_t total = (int64_t)planes * A.n * A.W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % A.W);
        const int64_t pv = i / A.W;
        out[i] = st[(size_t)pv * A.Ws + w];
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
    H.d_rows = nullptr;
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
    H.d_rows = g->rows_sorted;
    H.n_chunks = base[n_hubs];
    return FSGP_OK;
}

struct WsLayout {
    size_t off[16];
    size_t total;
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static int ensure_workspace(fsgp_graph *g, size_t bytes) {
    if (g->ws.bytes >= bytes) return FSGP_OK;
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
        default: return launch_rows<FSGP_LT>(A, L, s);
    }
}

static int occupancy_model(int model, int V, int TEAM, size_t smem, int *a, int *b) {
    switch (model) {
        case FSGP_SIR: return occupancy_rows<FSGP_SIR>(V, TEAM, smem, a, b);
        case FSGP_SIS: return occupancy_rows<FSGP_SIS>(V, TEAM, smem, a, b);
        case FSGP_IC: return occupancy_rows<FSGP_IC>(V, TEAM, smem, a, b);
        default: return occupancy_rows<FSGP_LT>(V, TEAM, smem, a, b);
    }
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
    if (model < FSGP_SIR || model > FSGP_LT) return fail(FSGP_EINVAL, "unknown model");
    if (!params) return fail(FSGP_EINVAL, "params is NULL");
    if (!out || !out->counts) return fail(FSGP_EINVAL, "result counts buffer is NULL");
    if (out->flags != FSGP_PTR_HOST && out->flags != FSGP_PTR_DEVICE)
        return fail(FSGP_EINVAL, "bad result flags");
    if (R < 1 || R > kMaxR) return fail(FSGP_EINVAL, "R must be in [1, 4096]");
    if (T < 0) return fail(FSGP_EINVAL, "T must be >= 0");
    if (n_sets < 1) return fail(FSGP_EINVAL, "n_sets must be >= 1");
    auto bad_p = [](double p) { return !(p >= 0.0 && p <= 1.0); };
    if (bad_p(params->beta) || bad_p(params->gamma) || bad_p(params->ic_p))
        return fail(FSGP_EINVAL, "probabilities must lie in [0, 1]");
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
        const int64_t ns_all = seed_offsets[n_sets];
        std::vector<int32_t> host_copy;
        const int32_t *hs = seed_nodes;
        if (seed_flags == FSGP_PTR_DEVICE && ns_all > 0) {
            host_copy.resize((size_t)ns_all);
            FSGP_CUDA(cudaMemcpy(host_copy.data(), seed_nodes, sizeof(int32_t) * (size_t)ns_all,
                                 cudaMemcpyDeviceToHost));
            hs = host_copy.data();
        }
        for (int64_t i = 0; i < ns_all; ++i)
            if (hs[i] < 0 || hs[i] >= g->n) return fail(FSGP_EINVAL, "seed node out of range");
    }
    int dev = 0;
    FSGP_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(FSGP_EINVAL, "current device differs from the graph's device");
    cudaStream_t s = (cudaStream_t)stream;

    // ---------------------------------------------------------------- shape
    const int32_t n = g->n;
    const int W = (R + 31) / 32;
    int Ws = 1;
    while (Ws < W) Ws <<= 1;
    const int P = fsgp_model_planes(model);
    const uint32_t last_mask = (R & 31) ? ((1u << (R & 31)) - 1u) : 0xffffffffu;
    int V = opt.vector_words ? opt.vector_words : std::min(2, Ws);   // measured best on GB300
    if (!opt.vector_words && Ws / V > 32) V = Ws / 32;                // R > 2048: 4 words/thread
    if (V != 1 && V != 2 && V != 4) return fail(FSGP_EINVAL, "vector_words must be 1, 2 or 4");
    if (V > Ws) V = Ws;
    const int TEAM = Ws / V;
    if (TEAM > 32) return fail(FSGP_EINVAL, "vector_words too small for R");
    // degree classes
    int small_max = opt.small_max_deg > 0 ? opt.small_max_deg : 255;
    int hub_min = opt.hub_min_deg > 0 ? opt.hub_min_deg : 8192;
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
    const double sparse_frac = opt.sparse_frac == 0.0 ? 0.05 : opt.sparse_frac;
    const unsigned long long sparse_limit =
        sparse_frac < 0.0 ? 0ull : (unsigned long long)(sparse_frac * (double)g->nnz);
    const bool allow_sparse = sparse_frac >= 0.0;

    int rc = ensure_hub_table(g, hub_min, chunk, s);
    if (rc) return rc;
    const int32_t n_hubs = g->hub.n_hubs;
    const int32_t start_mid = bh >= 1 ? g->cls.bucket_start[bh - 1] : n;
    const int32_t start_small = g->cls.bucket_start[bs];
    const int32_t n_mid = start_small - start_mid;
    const int32_t n_small = n - start_small;

    // -------------------------------------------------------- survival table
    std::vector<uint64_t> surv;
    int32_t ksat = INT32_MAX;
    if (model == FSGP_SIR || model == FSGP_SIS) {
        const uint64_t b = (uint64_t)llrint(params->beta * 4294967296.0);
        const uint64_t q = TWO32 - b;
        surv.push_back(TWO32);
        for (int64_t k = 1; k <= g->max_deg; ++k) {
            const uint64_t prev = surv.back();
            const uint64_t cur = (q == TWO32) ? prev : (prev * q) >> 32;
            surv.push_back(cur);
            if (cur == 0) {
                ksat = (int32_t)k;
                break;
            }
        }
    } else {
        surv.push_back(TWO32);
    }

    // ---------------------------------------------------------------- workspace
    const bool want_lanes = out->per_real != nullptr;
    const bool host_out = out->flags == FSGP_PTR_HOST;
    const size_t state_words = (size_t)P * n * Ws;
    const int64_t total_seeds = use_init ? 0 : seed_offsets[n_sets];
    enum { O_STATE, O_PC, O_CTL, O_LIST0, O_LIST1, O_CSMALL, O_CMID, O_BITMAP, O_LANES,
           O_HUB, O_SURV, O_SEEDS, O_COUNTS, O_FREQ, O_PREAL, O_PLANES, O_PROF, O_END };
    size_t sz[O_END] = {0};
    sz[O_STATE] = 2 * state_words * sizeof(uint32_t);
    sz[O_PC] = (size_t)(T + 1) * 2 * sizeof(unsigned long long);
    sz[O_CTL] = sizeof(Ctl);
    sz[O_LIST0] = sz[O_LIST1] = (size_t)n * sizeof(int32_t);
    sz[O_CSMALL] = sz[O_CMID] = (size_t)n * sizeof(int32_t);
    sz[O_BITMAP] = ((size_t)n + 31) / 32 * sizeof(uint32_t);
    sz[O_LANES] = want_lanes ? 2 * (size_t)Ws * 32 * sizeof(int32_t) : 0;
    sz[O_HUB] = (size_t)n_hubs * Ws * 32 * sizeof(uint32_t);
    sz[O_SURV] = surv.size() * sizeof(uint64_t);
    sz[O_SEEDS] = (!use_init && seed_flags == FSGP_PTR_HOST) ? (size_t)total_seeds * sizeof(int32_t) : 0;
    sz[O_COUNTS] = host_out ? (size_t)(T + 1) * 3 * sizeof(uint64_t) : 0;
    sz[O_FREQ] = (host_out && out->freq) ? 3 * (size_t)n * sizeof(uint32_t) : 0;
    sz[O_PREAL] = (host_out && out->per_real) ? (size_t)R * (T + 1) * 3 * sizeof(uint32_t) : 0;
    sz[O_PLANES] = ((host_out && out->final_planes) || use_init) ? (size_t)P * n * W * sizeof(uint32_t) : 0;
    sz[O_PROF] = FSGP_PROF_KINDS * sizeof(unsigned long long);
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
    int32_t *cand_small = (int32_t *)(ws + off[O_CSMALL]);
    int32_t *cand_mid = (int32_t *)(ws + off[O_CMID]);
    uint32_t *bitmap = (uint32_t *)(ws + off[O_BITMAP]);
    int32_t *lanes = want_lanes ? (int32_t *)(ws + off[O_LANES]) : nullptr;
    uint32_t *hub_scratch = (uint32_t *)(ws + off[O_HUB]);
    uint64_t *d_surv = (uint64_t *)(ws + off[O_SURV]);
    unsigned long long *d_prof = (unsigned long long *)(ws + off[O_PROF]);
    Prof prof;
    const bool profiling = opt.profile != nullptr;
    int64_t launches = 0;   // kernels launched by this call (profile only)
    FSGP_CUDA(cudaMemcpyAsync(d_surv, surv.data(), sz[O_SURV], cudaMemcpyHostToDevice, s));

    // ---------------------------------------------------------------- launch shape
    const size_t smem_lanes = want_lanes ? 2 * (size_t)Ws * 32 * sizeof(int32_t) : 0;
    if (smem_lanes > 48 * 1024) {
        // 2 planes x 4096 lanes x 4 B = 32 KB at most: always below the default limit
        return fail(FSGP_EINVAL, "per-lane counters exceed shared memory");
    }
    int bps_rows = 1, bps_hub = 1;
    rc = occupancy_model(model, V, TEAM, smem_lanes, &bps_rows, &bps_hub);
    if (rc) return rc;
    StepLaunch L{};
    L.V = V;
    L.TEAM = TEAM;
    L.smem_lanes = smem_lanes;
    L.have_small = n_small > 0;
    L.have_mid = n_mid > 0;
    L.have_hub = n_hubs > 0;
    L.prof = profiling ? &prof : nullptr;
    const int rows_per_block_small = (kBlock / 32) * (32 / TEAM);
    L.grid_small = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * bps_rows,
                                                               ((int64_t)n_small + rows_per_block_small - 1) / rows_per_block_small));
    L.grid_mid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * bps_rows,
                                                             ((int64_t)n_mid + (kBlock / 32) - 1) / (kBlock / 32)));
    L.grid_hub = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * bps_hub, g->hub.n_chunks));
    L.grid_fin = (int)std::max<int64_t>(1, ((int64_t)n_hubs + (kBlock / 32) - 1) / (kBlock / 32));
    const int grid_mark = g->sm_count * 8;
    const int grid_scan = grid_cap((int64_t)n, kBlock, g->sm_count, 8);

    StepArgs A{};
    A.row_ptr = g->row_ptr;
    A.col = g->col;
    A.out_ptr = g->out_ptr;
    A.out_dst = g->out_dst;
    A.n = n;
    A.Ws = Ws;
    A.W = W;
    A.last_mask = last_mask;
    A.gbase = (uint32_t)(opt.r_offset >> 5);
    A.small_max_deg = small_max;
    A.hub_min_deg = hub_min;
    A.plane_words = (size_t)n * Ws;
    A.surv = d_surv;
    A.surv_last = (int32_t)surv.size() - 1;
    A.ksat = ksat;
    A.g_rec = (uint64_t)llrint(params->gamma * 4294967296.0);
    A.p_const = (uint64_t)llrint(params->ic_p * 4294967296.0);
    A.ic_mode = params->ic_mode;
    A.key0 = (uint32_t)(rng_seed & 0xffffffffu);
    A.key1 = (uint32_t)(rng_seed >> 32);
    A.ctl = ctl;
    A.lane_cnt = lanes;
    A.rows_small = g->rows_sorted + start_small;
    A.rows_mid = g->rows_sorted + start_mid;
    A.n_small = n_small;
    A.n_mid = n_mid;
    A.cand_small = cand_small;
    A.cand_mid = cand_mid;
    A.bitmap = bitmap;
    A.hub_rows = g->hub.d_rows;
    A.hub_chunk_base = g->hub.d_chunk_base;
    A.n_hubs = n_hubs;
    A.n_hub_chunks = g->hub.n_chunks;
    A.hub_chunk = chunk;
    A.hub_scratch = hub_scratch;
    A.prof_bytes = profiling ? d_prof : nullptr;

    const size_t T1 = (size_t)T + 1;
    for (int set = 0; set < n_sets; ++set) {
        // outputs of this set (device pointers: caller's or staging)
        unsigned long long *counts_d = host_out ? (unsigned long long *)(ws + off[O_COUNTS])
                                                : (unsigned long long *)(out->counts + (size_t)set * T1 * 3);
        uint32_t *freq_d = !out->freq ? nullptr
                           : host_out ? (uint32_t *)(ws + off[O_FREQ]) : out->freq + (size_t)set * 3 * n;
        uint32_t *preal_d = !out->per_real ? nullptr
                            : host_out ? (uint32_t *)(ws + off[O_PREAL]) : out->per_real + (size_t)set * R * T1 * 3;
        uint32_t *planes_d = !out->final_planes ? nullptr
                             : host_out ? (uint32_t *)(ws + off[O_PLANES]) : out->final_planes + (size_t)set * P * n * W;
        int32_t *steps_d = (out->steps_run && !host_out) ? out->steps_run + set : nullptr;

        FSGP_CUDA(cudaMemsetAsync(ws + off[O_STATE], 0, sz[O_STATE], s));
        FSGP_CUDA(cudaMemsetAsync(pc, 0, sz[O_PC], s));
        FSGP_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
        {
            // the step-0 scan always lists the pushing rows for step 1
            const int32_t one[3] = {1, 1, 0};
            FSGP_CUDA(cudaMemcpyAsync(&ctl->build_list, one, sizeof one, cudaMemcpyHostToDevice, s));
        }
        FSGP_CUDA(cudaMemsetAsync(bitmap, 0, sz[O_BITMAP], s));
        if (lanes) FSGP_CUDA(cudaMemsetAsync(lanes, 0, sz[O_LANES], s));
        if (sz[O_HUB]) FSGP_CUDA(cudaMemsetAsync(hub_scratch, 0, sz[O_HUB], s));
        if (profiling) {
            FSGP_CUDA(cudaMemsetAsync(d_prof, 0, sz[O_PROF], s));
            prof.start(PK_INIT, s);
        }

        if (use_init) {
            const uint32_t *src = opt.init_planes + (size_t)set * P * n * W;
            if (host_out) {
                uint32_t *stage = (uint32_t *)(ws + off[O_PLANES]);
                FSGP_CUDA(cudaMemcpyAsync(stage, src, sz[O_PLANES], cudaMemcpyHostToDevice, s));
                src = stage;
            }
            k_import<<<grid_cap((int64_t)P * n * Ws, 256, g->sm_count, 16), 256, 0, s>>>(
                src, P, n, W, Ws, last_mask, buf0, buf1);
            ++launches;
        } else {
            const int64_t ns = seed_offsets[set + 1] - seed_offsets[set];
            const int32_t *sd = seed_nodes + seed_offsets[set];
            if (ns > 0) {
                if (seed_flags == FSGP_PTR_HOST) {
                    int32_t *stage = (int32_t *)(ws + off[O_SEEDS]) + seed_offsets[set];
                    FSGP_CUDA(cudaMemcpyAsync(stage, sd, sizeof(int32_t) * (size_t)ns, cudaMemcpyHostToDevice, s));
                    sd = stage;
                }
                k_seed<<<grid_cap(ns * Ws, 256, g->sm_count, 16), 256, 0, s>>>(
                    buf0, buf1, A.plane_words, model != FSGP_SIR && model != FSGP_SIS, sd, ns, Ws, W, last_mask);
                ++launches;
            }
        }
        // step 0
        A.cur = buf0;
        A.nxt = buf1;
        A.pc = pc;
        A.k = 0;
        A.t = (uint32_t)opt.t0;
        A.list_in = list[1];
        A.list_out = list[0];
        k_init_scan<<<grid_scan, kBlock, smem_lanes, s>>>(A, model);
        ++launches;
        if (profiling) prof.stop(s);
        FSGP_CUDA(cudaGetLastError());
        for (int k = 1; k <= T; ++k) {
            A.k = k;
            A.t = (uint32_t)(opt.t0 + k);
            A.cur = (k & 1) ? buf0 : buf1;
            A.nxt = (k & 1) ? buf1 : buf0;
            A.pc = pc + 2 * (size_t)k;
            A.list_in = list[(k - 1) & 1];
            A.list_out = list[k & 1];
            const int force_dense = !allow_sparse || (k == 1 && use_init && model == FSGP_LT);
            if (profiling) prof.start(PK_BEGIN, s);
            k_begin<<<preal_d ? std::max(1, (R + 255) / 256) : 1, 256, 0, s>>>(
                A, model, sparse_limit, force_dense, preal_d, R, (int)T1);
            if (profiling) prof.stop(s);
            if (allow_sparse) {
                if (profiling) prof.start(PK_MARK, s);
                k_mark<<<grid_mark, kBlock, 0, s>>>(A);
                if (profiling) prof.stop(s);
            }
            rc = launch_rows_model(model, A, L, s);
            if (rc) return rc;
            launches += 1 + (allow_sparse ? 1 : 0) + (L.have_hub ? 2 : 0) + (L.have_mid ? 1 : 0) +
                        (L.have_small ? 1 : 0);
        }
        FSGP_CUDA(cudaGetLastError());
        if (profiling) prof.start(PK_RESULTS, s);
        k_finalize<<<std::max(1, (int)((std::max<size_t>(T1, (size_t)R) + 255) / 256)), 256, 0, s>>>(
            A, model, T, (unsigned long long)n * (unsigned long long)R, pc, counts_d, steps_d, preal_d, R);
        if (freq_d)
            k_freq<<<grid_cap(n, 256, g->sm_count, 16), 256, 0, s>>>(A, model, buf0, buf1, R, freq_d);
        if (planes_d)
            k_export<<<grid_cap((int64_t)P * n * W, 256, g->sm_count, 16), 256, 0, s>>>(A, P, buf0, buf1, planes_d);
        if (profiling) prof.stop(s);
        launches += 1 + (freq_d ? 1 : 0) + (planes_d ? 1 : 0);
        FSGP_CUDA(cudaGetLastError());
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
            prof.ev.clear();
            prof.kind.clear();
            for (int i = 0; i < FSGP_PROF_KINDS; ++i) pf->alg_bytes[i] += (double)hb[i];
            pf->dense_steps += hc.dense_steps;
            pf->sparse_steps += hc.sparse_steps;
            pf->kernel_launches += launches;
            launches = 0;
        }
        if (host_out) {
            FSGP_CUDA(cudaMemcpyAsync(out->counts + (size_t)set * T1 * 3, counts_d, T1 * 3 * sizeof(uint64_t),
                                      cudaMemcpyDeviceToHost, s));
            if (freq_d)
                FSGP_CUDA(cudaMemcpyAsync(out->freq + (size_t)set * 3 * n, freq_d, 3 * (size_t)n * sizeof(uint32_t),
                                          cudaMemcpyDeviceToHost, s));
            if (preal_d)
                FSGP_CUDA(cudaMemcpyAsync(out->per_real + (size_t)set * R * T1 * 3, preal_d,
                                          (size_t)R * T1 * 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            if (planes_d)
                FSGP_CUDA(cudaMemcpyAsync(out->final_planes + (size_t)set * P * n * W, planes_d,
                                          (size_t)P * n * W * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            if (out->steps_run) {
                Ctl hc;
                FSGP_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
                FSGP_CUDA(cudaStreamSynchronize(s));
                out->steps_run[set] = hc.steps_done;
            }
            FSGP_CUDA(cudaStreamSynchronize(s));
        }
    }
    FSGP_CUDA(cudaGetLastError());
    return FSGP_OK;
}
