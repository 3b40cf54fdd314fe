// noalloc.cu -- fsgp_step_noalloc: one synchronous propagation step that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: code whose memory is fully budgeted up front (a
// serving process that has handed all free device memory to its own pool), or an
// embedding runtime that forbids allocation on its hot path.  For them this entry point
// computes one dense step
// of SIR, SIS, IC or LT over a graph and state planes that the caller already holds in
// device memory, with every row taking the CTA-split path of the hub rows: each row's
// in-arcs are cut into chunks, one CTA per chunk adds per-lane counts (IC: live lanes)
// into scratch, and a finalize pass decides every lane.  The scratch -- that per-lane
// merge area, the chunk table, the control block and the survival table -- is one
// file-scope device array of fixed size, so nothing is allocated per call.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "step.cuh"

namespace fsgp {
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;   // 32 MiB per GPU
constexpr int kNoAllocChunk = 4096;                   // arcs per CTA
constexpr int kSurvCap = 65536;                       // survival-table entries beyond k = 0

// The scratch of fsgp_step_noalloc.  Host code must not use this name as a device
// address: the address comes from cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocBytes / sizeof(uint32_t)];

constexpr size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Fixed head of the scratch (byte offsets).
constexpr size_t kOffCtl = 0;
constexpr size_t kOffPc = 256;            // kPC x u64 plane popcounts (2 used)
constexpr size_t kOffInfo = 512;          // u64 info[4]: max in-degree, chunks, k_sat
constexpr size_t kOffSet = 768;           // SetParams of the single set
constexpr size_t kOffSurv = 1024;         // (kSurvCap + 1) x u64
constexpr size_t kOffRows = kOffSurv + a256(sizeof(uint64_t) * (kSurvCap + 1));

std::mutex g_mu;
void *g_ptr[256] = {};

// Device address of the scratch on the current device, looked up once per device (the
// first call on a device, with it current) and kept for the process; a device reset
// invalidates it.
int noalloc_scratch(int dev, char **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 256) return fail(FSGP_EINVAL, "device ordinal out of range");
    if (!g_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_ptr[dev] = p;
    }
    *out = (char *)g_ptr[dev];
    return FSGP_OK;
}

// Row list (identity), chunk counts per row, max in-degree, and the popcounts of the
// current planes (the base that the step's deltas are added to).
__global__ void k_na_prep(const int32_t *__restrict__ row_ptr, int32_t n, int32_t *rows,
                          int64_t *nch, unsigned long long *info, const uint32_t *__restrict__ cur,
                          int planes, int Ws, unsigned long long *pc) {
    unsigned long long p0 = 0, p1 = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        rows[v] = (int32_t)v;
        const int32_t d = row_ptr[v + 1] - row_ptr[v];
        nch[v] = (d + kNoAllocChunk - 1) / kNoAllocChunk;
        atomicMax(&info[0], (unsigned long long)d);
        for (int w = 0; w < Ws; ++w) {
            p0 += __popc(cur[(size_t)v * Ws + w]);
            if (planes == 2) p1 += __popc(cur[(size_t)n * Ws + (size_t)v * Ws + w]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        p0 += __shfl_xor_sync(0xffffffffu, p0, o);
        p1 += __shfl_xor_sync(0xffffffffu, p1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (p0) atomicAdd(&pc[0], p0);
        if (p1) atomicAdd(&pc[1], p1);
    }
}

// In-place exclusive scan of the chunk counts (one CTA); base[n] and info[1] get the total.
__global__ void k_na_scan(int64_t *base, int32_t n, unsigned long long *info) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t b0 = 0; b0 < n; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t x = i < n ? base[i] : 0;
        int64_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int64_t s = lane < nw ? ws[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            if (lane < nw) ws[lane] = s;
        }
        __syncthreads();
        const int64_t off = (wid ? ws[wid - 1] : 0) + incl - x;
        const int64_t total = ws[nw - 1];
        if (i < n) base[i] = carry + off;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        base[n] = carry;
        info[1] = (unsigned long long)carry;
    }
}

// Survival table surv[0..min(max in-degree, kSurvCap)] (stops at the first zero) and the
// first k with surv[k] = 0 in info[2] (0 = none within the table).
__global__ void k_na_surv(double beta, unsigned long long *info, uint64_t *surv) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const uint64_t b = (uint64_t)llrint(beta * 4294967296.0);
    const uint64_t q = TWO32 - b;
    const uint64_t kmax = info[0] < (unsigned long long)kSurvCap ? info[0] : (unsigned long long)kSurvCap;
    surv[0] = TWO32;
    info[2] = 0;
    for (uint64_t k = 1; k <= kmax; ++k) {
        const uint64_t prev = surv[k - 1];
        const uint64_t cur = q == TWO32 ? prev : (prev * q) >> 32;
        surv[k] = cur;
        if (cur == 0) {
            info[2] = k;
            break;
        }
    }
}

int launch_split_model(int model, const StepArgs &A, int V, int TEAM, int gc, int gf, cudaStream_t s) {
    switch (model) {
        case FSGP_SIR: return launch_split_rows<FSGP_SIR>(A, V, TEAM, gc, gf, s);
        case FSGP_SIS: return launch_split_rows<FSGP_SIS>(A, V, TEAM, gc, gf, s);
        case FSGP_IC: return launch_split_rows<FSGP_IC>(A, V, TEAM, gc, gf, s);
        default: return launch_split_rows<FSGP_LT>(A, V, TEAM, gc, gf, s);
    }
}

}  // namespace
}  // namespace fsgp

using namespace fsgp;

extern "C" int fsgp_step_noalloc(int32_t model, const fsgp_params *params, const int32_t *row_ptr,
                                 const int32_t *col_idx, int32_t n, int64_t nnz, int32_t R,
                                 uint32_t t, uint64_t rng_seed, const uint32_t *cur_planes,
                                 uint32_t *next_planes, uint64_t *plane_counts, void *stream) {
    set_error("");
    if (model > FSGP_LT && model <= FSGP_SWIR)
        return fail(FSGP_EUNSUPPORTED, "this entry point covers the SIR, SIS, IC and LT models");
    if (model < FSGP_SIR || model > FSGP_LT) return fail(FSGP_EINVAL, "unknown model");
    if (!params || !row_ptr || !cur_planes || !next_planes || !plane_counts || (nnz > 0 && !col_idx))
        return fail(FSGP_EINVAL, "NULL argument");
    if (n < 1 || nnz < 0 || nnz >= (int64_t)INT32_MAX) return fail(FSGP_EINVAL, "n or nnz out of range");
    if (R < 1 || R > kMaxR) return fail(FSGP_EINVAL, "R must be in [1, 4096]");
    if (cur_planes == next_planes) return fail(FSGP_EINVAL, "cur_planes and next_planes must not alias");
    auto bad_p = [](double p) { return !(p >= 0.0 && p <= 1.0); };
    if (bad_p(params->beta) || bad_p(params->gamma) || bad_p(params->ic_p))
        return fail(FSGP_EINVAL, "probabilities must lie in [0, 1]");
    if (params->weighted) return fail(FSGP_EUNSUPPORTED, "the no-allocation step has no weighted graphs");
    if (params->ic_mode != FSGP_IC_WEIGHTED_CASCADE && params->ic_mode != FSGP_IC_CONSTANT)
        return fail(FSGP_EINVAL, "bad ic_mode");
    const int W = (R + 31) / 32;
    int Ws = 1;
    while (Ws < W) Ws <<= 1;
    const int P = model == FSGP_SIS ? 1 : 2;
    const int nl = Ws * 32;
    const size_t off_base = kOffRows + a256(sizeof(int32_t) * (size_t)n);
    const size_t off_slots = off_base + a256(sizeof(int64_t) * ((size_t)n + 1));
    const size_t need = off_slots + sizeof(uint32_t) * (size_t)n * nl;
    if (need > kNoAllocBytes)
        return fail(FSGP_EINVAL, "graph too large for fsgp_step_noalloc: n * 128 * ceil(R/32, pow2) bytes of "
                                 "scratch exceed its 32 MiB maximum");
    int dev = 0;
    FSGP_CUDA(cudaGetDevice(&dev));
    char *base = nullptr;
    int rc = noalloc_scratch(dev, &base);
    if (rc) return rc;
    int sm_count = 0;
    FSGP_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;

    Ctl *ctl = (Ctl *)(base + kOffCtl);
    unsigned long long *pc = (unsigned long long *)(base + kOffPc);
    unsigned long long *info = (unsigned long long *)(base + kOffInfo);
    uint64_t *surv = (uint64_t *)(base + kOffSurv);
    int32_t *rows = (int32_t *)(base + kOffRows);
    int64_t *chunk_base = (int64_t *)(base + off_base);
    uint32_t *slots = (uint32_t *)(base + off_slots);

    // the array keeps the last call's contents: clear what must start at zero
    FSGP_CUDA(cudaMemsetAsync(base, 0, kOffSet, s));
    FSGP_CUDA(cudaMemsetAsync(slots, 0, sizeof(uint32_t) * (size_t)n * nl, s));
    const int grid = (int)std::min<int64_t>((int64_t)sm_count * 8, ((int64_t)n + 255) / 256);
    k_na_prep<<<std::max(grid, 1), 256, 0, s>>>(row_ptr, n, rows, chunk_base, info, cur_planes, P, Ws, pc);
    k_na_scan<<<1, 1024, 0, s>>>(chunk_base, n, info);
    if (model == FSGP_SIR || model == FSGP_SIS) k_na_surv<<<1, 1, 0, s>>>(params->beta, info, surv);
    FSGP_CUDA(cudaGetLastError());
    unsigned long long h_info[3] = {0, 0, 0};
    FSGP_CUDA(cudaMemcpyAsync(h_info, info, sizeof h_info, cudaMemcpyDeviceToHost, s));
    FSGP_CUDA(cudaStreamSynchronize(s));
    const int64_t max_deg = (int64_t)h_info[0];
    const int64_t n_chunks = (int64_t)h_info[1];
    int32_t ksat = INT32_MAX;
    if (model == FSGP_SIR || model == FSGP_SIS) {
        if (h_info[2]) ksat = (int32_t)h_info[2];
        else if (max_deg > kSurvCap)
            return fail(FSGP_EINVAL, "in-degree beyond the 65536-entry survival table of fsgp_step_noalloc "
                                     "for this beta");
    }

    SetParams hp{};
    hp.key0 = (uint32_t)(rng_seed & 0xffffffffu);
    hp.key1 = (uint32_t)(rng_seed >> 32);
    hp.surv = surv;
    hp.ksat = ksat;
    hp.W = W;
    hp.last_mask = (R & 31) ? ((1u << (R & 31)) - 1u) : 0xffffffffu;
    hp.R = R;
    hp.g_rec = (uint64_t)llrint(params->gamma * 4294967296.0);
    hp.p_const = (uint64_t)llrint(params->ic_p * 4294967296.0);
    SetParams *d_sp = (SetParams *)(base + kOffSet);
    FSGP_CUDA(cudaMemcpyAsync(d_sp, &hp, sizeof hp, cudaMemcpyHostToDevice, s));
    const int V = std::min(2, Ws);
    const int SW = std::min(32 * V, Ws);
    const int TEAM = SW / V;

    StepArgs A{};
    A.rp = row_ptr;        // rows are the caller's nodes: no relabelling (orig, pos null)
    A.col = col_idx;
    A.arc0 = row_ptr;      // IC arc keys: the caller's arc positions
    A.out_ptr = row_ptr;   // read only for frontier bookkeeping, which this step discards
    A.out_dst = nullptr;
    A.n = n;
    A.Ws = Ws;
    A.ws_shift = __builtin_ctz((unsigned)Ws);
    A.S = 1;
    A.Wn = Ws;
    A.nslices = Ws / SW;
    A.gbase = 0;
    A.cur = cur_planes;
    A.nxt = next_planes;
    A.plane_words = (size_t)n * Ws;
    A.sp = d_sp;
    A.ic_mode = params->ic_mode;
    A.t = t;
    A.k = 1;
    A.ctl = ctl;
    A.pc = pc;
    A.hub_chunk_base = chunk_base;
    A.n_hubs = n;
    A.n_hub_chunks = n_chunks;
    A.hub_chunk = kNoAllocChunk;
    A.hub_scratch = slots;
    const int gc = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count * 4, n_chunks * A.nslices));
    const int gf = (int)std::max<int64_t>(1, ((int64_t)n + (kBlock / 32) - 1) / (kBlock / 32));
    rc = launch_split_model(model, A, V, TEAM, gc, gf, s);
    if (rc) return rc;
    FSGP_CUDA(cudaGetLastError());
    FSGP_CUDA(cudaMemcpyAsync(plane_counts, pc, 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    return FSGP_OK;
}
