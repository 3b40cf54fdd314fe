// single.cu -- the plain single-instance path: ONE realization, one byte of state per
// node (0 = S / inactive, 1 = I / newly active, 2 = R / active before the last step), no
// bit packing and no bit-sliced counting.  It applies the same synchronous update
// (Sec. 2, Eq. nodestate; SIR rule of Sec. 4.3) with the same counter-based uniforms as
// lane r of the packed path (Philox4x32-10 bit-planes, MSB first), so its states equal
// that lane's bit for bit.  It is the baseline the packed path is measured against.
//
// Per step: rows with in-degree below kBigDeg are handled by 8-lane teams, one row per
// team; rows at or above it by one CTA each.  A tally kernel counts the compartments
// and a one-thread kernel flips the double buffer and applies the IC/LT stop rule
// (the first step that leaves no newly active node), all without host round trips.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "fsgp_internal.cuh"

namespace fsgp {
namespace single {

constexpr int32_t kBigDeg = 4096;     // = 2^12: degree buckets 13 and up
constexpr int kTeam = 8;

struct Ctl {
    int32_t cur;          // buffer holding the state of the last completed step
    int32_t quiet;        // IC/LT: the stop rule fired
    int32_t steps_done;   // transitions computed
    int32_t pad;
};

struct Params {
    const uint64_t *surv;  // survival table (SIR/SIS)
    int32_t surv_last;     // last index of surv
    uint64_t g_rec;        // recovery threshold
    uint64_t p_const;      // IC constant arc threshold
    int32_t ic_mode;
    uint32_t k0, k1;       // Philox key (rng seed)
    uint32_t r;            // global realization index
};

__device__ __forceinline__ bool u_less(const Params &p, uint64_t thr, uint32_t tag, uint32_t a, uint32_t t) {
    return lanes_u_less(1u << (p.r & 31u), thr, a, t, p.r >> 5, tag, p.k0, p.k1) != 0u;
}

// The state of row v after step t, from the gathered in-arc facts (lane 0 of a team,
// or thread 0 of a CTA): k = number of in-arcs whose source is I (SIR/SIS) or active
// (LT); live = some in-arc from a newly active source drew live (IC).
template <int MODEL>
__device__ __forceinline__ uint8_t decide(const Params &p, uint8_t s, int32_t v, int64_t k, bool live,
                                          int32_t d, uint32_t t) {
    if (MODEL == FSGP_SIR || MODEL == FSGP_SIS) {
        if (s == 0) {
            if (k == 0) return 0;
            const uint64_t thr = p.surv[k < p.surv_last ? k : p.surv_last];
            return u_less(p, thr, TAG_INFECT, (uint32_t)v, t) ? 0 : 1;   // infected iff u >= surv[k]
        }
        if (s == 1) {
            if (u_less(p, p.g_rec, TAG_RECOVER, (uint32_t)v, t)) return MODEL == FSGP_SIR ? 2 : 0;
            return 1;
        }
        return 2;
    }
    if (s != 0) return 2;
    if (MODEL == FSGP_IC) return live ? 1 : 0;
    // LT: active iff k 2^32 >= theta d, theta drawn once (t = 0) per node and realization
    if (k == 0) return 0;
    const uint64_t thr = (((uint64_t)k << 32) / (uint64_t)d) + 1ull;   // theta < thr
    return u_less(p, thr, TAG_LT_THRESH, (uint32_t)v, 0u) ? 1 : 0;
}

// One in-arc's contribution: counted (SIR/SIS/LT) or drawn (IC).
template <int MODEL>
__device__ __forceinline__ void arc_fact(const Params &p, uint8_t src, int32_t e, int32_t d, uint32_t t,
                                         int64_t &k, bool &live) {
    if (MODEL == FSGP_SIR || MODEL == FSGP_SIS) {
        k += src == 1;
    } else if (MODEL == FSGP_LT) {
        k += src != 0;
    } else if (src == 1 && !live) {
        const uint64_t thr = p.ic_mode == FSGP_IC_WEIGHTED_CASCADE ? (TWO32 - 1ull) / (uint64_t)d + 1ull
                                                                    : p.p_const;
        live = u_less(p, thr, TAG_IC_EDGE, (uint32_t)e, t);   // live iff u d < 2^32 (or u < p)
    }
}

template <int MODEL>
__global__ void __launch_bounds__(256) k_rows(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                              int32_t n, const Ctl *ctl, uint8_t *buf0, uint8_t *buf1, Params p,
                                              uint32_t t) {
    if (ctl->quiet) return;
    const uint8_t *X = ctl->cur ? buf1 : buf0;
    uint8_t *Y = ctl->cur ? buf0 : buf1;
    const int lane = threadIdx.x & (kTeam - 1);
    const unsigned mask = 0xFFu << (threadIdx.x & 31 & ~(kTeam - 1));
    const int64_t team = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kTeam;
    const int64_t teams = ((int64_t)gridDim.x * blockDim.x) / kTeam;
    for (int64_t v = team; v < n; v += teams) {
        const int32_t b = row_ptr[v], e = row_ptr[v + 1], d = e - b;
        if (d >= kBigDeg) continue;                       // k_big_rows
        const uint8_t s = X[v];
        const bool gather = (s == 0);                     // S / inactive rows need their in-arcs
        int64_t k = 0;
        bool live = false;
        if (gather)
            for (int32_t a = b + lane; a < e; a += kTeam) arc_fact<MODEL>(p, X[__ldg(col + a)], a, d, t, k, live);
        // team reduction (k < 2^12 here)
        int kk = (int)k;
        int lv = live ? 1 : 0;
#pragma unroll
        for (int o = kTeam / 2; o > 0; o >>= 1) {
            kk += __shfl_xor_sync(mask, kk, o);
            lv |= __shfl_xor_sync(mask, lv, o);
        }
        if (lane == 0) Y[v] = decide<MODEL>(p, s, (int32_t)v, kk, lv != 0, d, t);
    }
}

template <int MODEL>
__global__ void __launch_bounds__(256) k_big_rows(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                                  const int32_t *__restrict__ big, int32_t n_big, const Ctl *ctl,
                                                  uint8_t *buf0, uint8_t *buf1, Params p, uint32_t t) {
    if (ctl->quiet) return;
    const uint8_t *X = ctl->cur ? buf1 : buf0;
    uint8_t *Y = ctl->cur ? buf0 : buf1;
    __shared__ unsigned long long s_k[8];
    __shared__ int s_live[8];
    for (int32_t i = blockIdx.x; i < n_big; i += gridDim.x) {
        const int32_t v = big[i];
        const int32_t b = row_ptr[v], e = row_ptr[v + 1], d = e - b;
        const uint8_t s = X[v];
        int64_t k = 0;
        bool live = false;
        if (s == 0)
            for (int32_t a = b + threadIdx.x; a < e; a += blockDim.x) arc_fact<MODEL>(p, X[__ldg(col + a)], a, d, t, k, live);
        unsigned long long kk = (unsigned long long)k;
        int lv = live ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kk += __shfl_xor_sync(0xffffffffu, kk, o);
            lv |= __shfl_xor_sync(0xffffffffu, lv, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_k[threadIdx.x >> 5] = kk;
            s_live[threadIdx.x >> 5] = lv;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long ks = 0;
            int ls = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                ks += s_k[w];
                ls |= s_live[w];
            }
            Y[v] = decide<MODEL>(p, s, v, (int64_t)ks, ls != 0, d, t);
        }
        __syncthreads();
    }
}

// counts[k][c] = number of nodes in compartment c after step k (repeat the last row once
// the stop rule fired).
__global__ void k_tally(const Ctl *ctl, const uint8_t *buf0, const uint8_t *buf1, int32_t n, int32_t k,
                        unsigned long long *counts, int after_step) {
    if (after_step && ctl->quiet) {
        if (blockIdx.x == 0 && threadIdx.x < 3) counts[(size_t)k * 3 + threadIdx.x] = counts[(size_t)(k - 1) * 3 + threadIdx.x];
        return;
    }
    // after a step the new state is in the other buffer; before the first step, in cur
    const int which = after_step ? (ctl->cur ^ 1) : ctl->cur;
    const uint8_t *X = which ? buf1 : buf0;
    unsigned c0 = 0, c1 = 0, c2 = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t s = X[v];
        c0 += s == 0;
        c1 += s == 1;
        c2 += s == 2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts + (size_t)k * 3 + 0, (unsigned long long)c0);
        atomicAdd(counts + (size_t)k * 3 + 1, (unsigned long long)c1);
        atomicAdd(counts + (size_t)k * 3 + 2, (unsigned long long)c2);
    }
}

// Flip the buffers after step k and apply the IC/LT stop rule.
__global__ void k_advance(Ctl *ctl, const unsigned long long *counts, int32_t k, int stop_rule) {
    if (ctl->quiet) return;
    if (k > 0) {
        ctl->cur ^= 1;
        ctl->steps_done = k;
    }
    if (stop_rule && counts[(size_t)k * 3 + 1] == 0ull) ctl->quiet = 1;
}

__global__ void k_seed_state(uint8_t *X, int32_t n, const int32_t *seeds, int64_t n_seeds, int *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_seeds; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = seeds[i];
        if (v < 0 || v >= n) atomicExch(bad, 1);
        else X[v] = 1;
    }
}

template <int MODEL>
void launch_step(const fsgp_graph *g, const int32_t *big, int32_t n_big, const Ctl *ctl, uint8_t *b0, uint8_t *b1,
                 const Params &p, uint32_t t, cudaStream_t st) {
    const int64_t teams_needed = (int64_t)g->n;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((teams_needed * kTeam + 255) / 256, (int64_t)g->sm_count * 16));
    k_rows<MODEL><<<grid, 256, 0, st>>>(g->row_ptr, g->col, g->n, ctl, b0, b1, p, t);
    if (n_big)
        k_big_rows<MODEL><<<std::min<int32_t>(n_big, g->sm_count * 4), 256, 0, st>>>(g->row_ptr, g->col, big, n_big,
                                                                                     ctl, b0, b1, p, t);
}

}  // namespace single
}  // namespace fsgp

using namespace fsgp;
using namespace fsgp::single;

extern "C" int fsgp_simulate_single(const fsgp_graph *gc, int32_t model, const fsgp_params *params,
                                    const int32_t *seed_nodes, int64_t n_seeds, uint32_t seed_flags,
                                    int32_t r, int32_t T, uint64_t rng_seed, uint64_t *counts,
                                    uint8_t *final_state, int32_t *steps_run, uint32_t out_flags,
                                    void *stream) {
    set_error("");
    fsgp_graph *g = const_cast<fsgp_graph *>(gc);   // the cached workspace is grown
    if (!g || !params || !counts) return fail(FSGP_EINVAL, "NULL argument");
    if (model > FSGP_LT && model <= FSGP_SWIR)
        return fail(FSGP_EUNSUPPORTED, "this entry point covers the SIR, SIS, IC and LT models");
    if (model < FSGP_SIR || model > FSGP_LT) return fail(FSGP_EINVAL, "unknown model");
    if (r < 0 || T < 0 || n_seeds < 0 || (n_seeds > 0 && !seed_nodes)) return fail(FSGP_EINVAL, "bad r, T or seeds");
    if (seed_flags > FSGP_PTR_DEVICE || out_flags > FSGP_PTR_DEVICE) return fail(FSGP_EINVAL, "bad flags");
    if (!(params->beta >= 0.0 && params->beta <= 1.0 && params->gamma >= 0.0 && params->gamma <= 1.0 &&
          params->ic_p >= 0.0 && params->ic_p <= 1.0))
        return fail(FSGP_EINVAL, "probability outside [0, 1]");
    if (params->weighted) return fail(FSGP_EUNSUPPORTED, "the single-instance path has no weighted graphs");
    if (params->ic_mode != FSGP_IC_WEIGHTED_CASCADE && params->ic_mode != FSGP_IC_CONSTANT)
        return fail(FSGP_EINVAL, "unknown ic_mode");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    FSGP_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(FSGP_EINVAL, "graph lives on another device");

    std::vector<uint64_t> surv;
    int32_t ksat_unused = INT32_MAX;
    if (model == FSGP_SIR || model == FSGP_SIS) survival_table(params->beta, g->max_deg, surv, &ksat_unused);
    else surv.push_back(0);
    const int32_t n = g->n;
    int32_t n_big = 0;
    for (int b = 13; b <= 32; ++b) n_big += g->cls.bucket_count[b];   // rows_sorted starts with them

    // workspace: [ctl 256 B][bad flag 256 B][counts (T+1)*3 u64][surv][seeds][buf0 n][buf1 n]
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_bad = 256, o_counts = 512;
    const size_t o_surv = o_counts + up(sizeof(uint64_t) * 3 * ((size_t)T + 1));
    const size_t o_seeds = o_surv + up(sizeof(uint64_t) * surv.size());
    const size_t o_b0 = o_seeds + up(sizeof(int32_t) * (size_t)std::max<int64_t>(n_seeds, 1));
    const size_t o_b1 = o_b0 + up((size_t)n);
    const size_t total = o_b1 + up((size_t)n);
    int rc = ensure_workspace(g, total);
    if (rc) return rc;
    char *ws = (char *)g->ws.ptr;
    Ctl *ctl = (Ctl *)ws;
    int *bad = (int *)(ws + o_bad);
    unsigned long long *d_counts = (unsigned long long *)(ws + o_counts);
    uint64_t *d_surv = (uint64_t *)(ws + o_surv);
    uint8_t *b0 = (uint8_t *)(ws + o_b0), *b1 = (uint8_t *)(ws + o_b1);
    const int32_t *d_seeds = seed_nodes;
    if (n_seeds > 0 && seed_flags == FSGP_PTR_HOST) {
        FSGP_CUDA(cudaMemcpyAsync(ws + o_seeds, seed_nodes, sizeof(int32_t) * (size_t)n_seeds, cudaMemcpyHostToDevice, st));
        d_seeds = (const int32_t *)(ws + o_seeds);
    }
    FSGP_CUDA(cudaMemsetAsync(ws, 0, o_surv, st));   // ctl, bad flag, counts
    FSGP_CUDA(cudaMemcpyAsync(d_surv, surv.data(), sizeof(uint64_t) * surv.size(), cudaMemcpyHostToDevice, st));
    FSGP_CUDA(cudaMemsetAsync(b0, 0, (size_t)n, st));
    if (n_seeds > 0) {
        const int gs = (int)std::min<int64_t>((n_seeds + 255) / 256, 1024);
        k_seed_state<<<gs, 256, 0, st>>>(b0, n, d_seeds, n_seeds, bad);
    }
    Params p{};
    p.surv = d_surv;
    p.surv_last = (int32_t)surv.size() - 1;
    p.g_rec = (uint64_t)llrint(params->gamma * 4294967296.0);
    p.p_const = (uint64_t)llrint(params->ic_p * 4294967296.0);
    p.ic_mode = params->ic_mode;
    p.k0 = (uint32_t)(rng_seed & 0xFFFFFFFFu);
    p.k1 = (uint32_t)(rng_seed >> 32);
    p.r = (uint32_t)r;
    const int stop_rule = (model == FSGP_IC || model == FSGP_LT) ? 1 : 0;
    const int gt = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)g->sm_count * 8));
    k_tally<<<gt, 256, 0, st>>>(ctl, b0, b1, n, 0, d_counts, 0);
    k_advance<<<1, 1, 0, st>>>(ctl, d_counts, 0, stop_rule);
    for (int32_t k = 1; k <= T; ++k) {
        switch (model) {
            case FSGP_SIR: launch_step<FSGP_SIR>(g, g->rows_sorted, n_big, ctl, b0, b1, p, (uint32_t)k, st); break;
            case FSGP_SIS: launch_step<FSGP_SIS>(g, g->rows_sorted, n_big, ctl, b0, b1, p, (uint32_t)k, st); break;
            case FSGP_IC: launch_step<FSGP_IC>(g, g->rows_sorted, n_big, ctl, b0, b1, p, (uint32_t)k, st); break;
            default: launch_step<FSGP_LT>(g, g->rows_sorted, n_big, ctl, b0, b1, p, (uint32_t)k, st); break;
        }
        k_tally<<<gt, 256, 0, st>>>(ctl, b0, b1, n, k, d_counts, 1);
        k_advance<<<1, 1, 0, st>>>(ctl, d_counts, k, stop_rule);
    }
    FSGP_CUDA(cudaGetLastError());
    // results
    Ctl h_ctl{};
    int h_bad = 0;
    FSGP_CUDA(cudaMemcpyAsync(&h_ctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    FSGP_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    FSGP_CUDA(cudaStreamSynchronize(st));
    if (h_bad) return fail(FSGP_EINVAL, "seed node out of range");
    const cudaMemcpyKind kind = out_flags == FSGP_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    FSGP_CUDA(cudaMemcpyAsync(counts, d_counts, sizeof(uint64_t) * 3 * ((size_t)T + 1), kind, st));
    if (final_state)
        FSGP_CUDA(cudaMemcpyAsync(final_state, h_ctl.cur ? b1 : b0, (size_t)n, kind, st));
    if (steps_run) {
        const int32_t sr = stop_rule ? h_ctl.steps_done : T;
        if (out_flags == FSGP_PTR_HOST) *steps_run = sr;
        else FSGP_CUDA(cudaMemcpyAsync(steps_run, &sr, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    FSGP_CUDA(cudaStreamSynchronize(st));
    return FSGP_OK;
}
