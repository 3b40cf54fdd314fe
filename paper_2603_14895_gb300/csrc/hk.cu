// hk.cu -- Hegselmann-Krause opinion dynamics (Appendix A.2): continuous opinions, R
// independent opinion vectors (realizations) updated synchronously.  At step k node i
// takes the mean of the opinions h_j of its in-neighbours j (arcs with multiplicity)
// with |h_i - h_j| < eps; with none it keeps its opinion (the NaN case of the appendix).
//
// GB300 layout: opinions are [n][Rp] float32 (Rp = R rounded up to 32), so that the 32
// lanes of a warp are 32 realizations of one node and every gathered in-neighbour is one
// 128-byte row segment.  One warp per node and up to two 32-realization groups, hub rows
// first (the degree-bucket order); the arcs of a row are visited in col_idx order and summed in
// single precision with one division, the order the definition's sum is taken in, so
// that the result is exactly the sequential one.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fsgp_internal.cuh"

namespace fsgp {
namespace {

// [R][n] (caller) -> [n][Rp] (lanes); padding lanes get 0.
__global__ void k_hk_in(const float *__restrict__ src, int32_t n, int32_t R, int32_t Rp, float *dst) {
    const int64_t total = (int64_t)n * Rp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / Rp;
        const int32_t r = (int32_t)(i - v * Rp);
        dst[i] = r < R ? src[(size_t)r * n + v] : 0.0f;
    }
}

// [n][Rp] -> [R][n]
__global__ void k_hk_out(const float *__restrict__ src, int32_t n, int32_t R, int32_t Rp, float *dst) {
    const int64_t total = (int64_t)R * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n;
        const int64_t v = i - r * n;
        dst[i] = src[(size_t)v * Rp + r];
    }
}

__global__ void k_hk_check(const float *__restrict__ h, int64_t m, int32_t *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = h[i];
        if (isnan(x) || isinf(x)) atomicExch(bad, 1);
    }
}

constexpr int kHkUnroll = 8;   // gathered rows in flight per lane and group
constexpr int kHkMaxVG = 2;    // 32-realization groups of one node per warp

// One synchronous step.  A warp takes VG consecutive 32-realization groups of one node
// (the column indices are loaded once for all of them, and VG x kHkUnroll gathered rows
// are in flight per lane).  changes: (node, realization) pairs whose opinion changed.
template <int VG>
__global__ void __launch_bounds__(256) k_hk_step(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                                 const int32_t *__restrict__ order, int32_t n, int32_t R, int32_t Rp,
                                                 float eps, const float *__restrict__ cur, float *__restrict__ nxt,
                                                 unsigned long long *changes) {
    const int lane = threadIdx.x & 31;
    const int G = Rp >> 5;
    const int GW = (G + VG - 1) / VG;   // warp items per node
    const int64_t items = (int64_t)n * GW;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long ch = 0ull;
    for (int64_t it = gwarp; it < items; it += nwarps) {
        const int64_t q = it / GW;
        const int32_t g0 = (int32_t)(it - q * GW) * VG;
        const int32_t i = __ldg(order + q);
        const float *base = cur + g0 * 32 + lane;
        float hi[VG], sum[VG];
        int32_t cnt[VG];
#pragma unroll
        for (int v = 0; v < VG; ++v) {
            hi[v] = g0 + v < G ? base[(size_t)i * Rp + v * 32] : 0.0f;
            sum[v] = 0.0f;
            cnt[v] = 0;
        }
        const int32_t beg = __ldg(row_ptr + i), end = __ldg(row_ptr + i + 1);
        for (int32_t e0 = beg; e0 < end; e0 += 32) {
            // 32 column indices at once, one per lane, handed out by shuffles
            const int32_t mine = e0 + lane < end ? __ldg(col + e0 + lane) : 0;
            const int m = min(32, end - e0);
            for (int a0 = 0; a0 < m; a0 += kHkUnroll) {
                float hj[kHkUnroll][VG];
#pragma unroll
                for (int u = 0; u < kHkUnroll; ++u) {
                    const int32_t j = __shfl_sync(0xffffffffu, mine, (a0 + u) & 31);
#pragma unroll
                    for (int v = 0; v < VG; ++v)
                        hj[u][v] = (a0 + u < m && g0 + v < G) ? base[(size_t)j * Rp + v * 32] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < kHkUnroll; ++u) {
#pragma unroll
                    for (int v = 0; v < VG; ++v) {
                        if (a0 + u < m && fabsf(__fsub_rn(hi[v], hj[u][v])) < eps) {
                            sum[v] = __fadd_rn(sum[v], hj[u][v]);
                            ++cnt[v];
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int v = 0; v < VG; ++v) {
            if (g0 + v >= G) break;   // uniform over the warp
            const int32_t r = (g0 + v) * 32 + lane;
            const float out = cnt[v] > 0 ? __fdiv_rn(sum[v], (float)cnt[v]) : hi[v];
            nxt[(size_t)i * Rp + r] = out;
            const unsigned chm = __ballot_sync(0xffffffffu, r < R && out != hi[v]);
            if (lane == 0) ch += (unsigned long long)__popc(chm);
        }
    }
    __shared__ unsigned long long s_ch;
    if (threadIdx.x == 0) s_ch = 0ull;
    __syncthreads();
    if (lane == 0 && ch) atomicAdd(&s_ch, ch);
    __syncthreads();
    if (threadIdx.x == 0 && s_ch) atomicAdd(changes, s_ch);
}

}  // namespace
}  // namespace fsgp

using namespace fsgp;

extern "C" int fsgp_hk(const fsgp_graph *gc, const float *h0, int32_t R, int32_t T, double eps, float *h_out,
                       uint64_t *changes, uint32_t flags, void *stream) {
    set_error("");
    fsgp_graph *g = const_cast<fsgp_graph *>(gc);
    if (!g || !h0 || !h_out) return fail(FSGP_EINVAL, "NULL argument");
    if (R < 1 || R > kMaxR) return fail(FSGP_EINVAL, "R must be in [1, 4096]");
    if (T < 0) return fail(FSGP_EINVAL, "T must be >= 0");
    if (!(eps >= 0.0) || std::isinf(eps)) return fail(FSGP_EINVAL, "eps must be finite and >= 0");
    if (flags != FSGP_PTR_HOST && flags != FSGP_PTR_DEVICE) return fail(FSGP_EINVAL, "bad flags");
    int dev = 0;
    FSGP_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(FSGP_EINVAL, "current device differs from the graph's device");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = g->n;
    const int32_t Rp = (R + 31) & ~31;
    const int64_t m = (int64_t)R * n;
    if (flags == FSGP_PTR_HOST)
        for (int64_t i = 0; i < m; ++i)
            if (std::isnan(h0[i]) || std::isinf(h0[i])) return fail(FSGP_EINVAL, "opinions must be finite");
    // workspace: two [n][Rp] buffers, the per-step change counts, a flag, and (host
    // buffers) a [R][n] staging area
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_state = al(sizeof(float) * (size_t)n * Rp);
    const size_t b_ch = al(sizeof(unsigned long long) * ((size_t)T + 1));
    const size_t b_flag = al(sizeof(int32_t));
    const size_t b_stage = flags == FSGP_PTR_HOST ? al(sizeof(float) * (size_t)std::max<int64_t>(m, 1)) : 0;
    int rc = ensure_workspace(g, 2 * b_state + b_ch + b_flag + b_stage);
    if (rc) return rc;
    uint8_t *ws = (uint8_t *)g->ws.ptr;
    float *buf0 = (float *)ws;
    float *buf1 = (float *)(ws + b_state);
    unsigned long long *d_ch = (unsigned long long *)(ws + 2 * b_state);
    int32_t *d_flag = (int32_t *)(ws + 2 * b_state + b_ch);
    float *stage = b_stage ? (float *)(ws + 2 * b_state + b_ch + b_flag) : nullptr;
    const int grid_el = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n * Rp + 255) / 256,
                                                                     (int64_t)g->sm_count * 16));
    const float *src = h0;
    if (flags == FSGP_PTR_HOST) {
        if (m > 0) FSGP_CUDA(cudaMemcpyAsync(stage, h0, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, s));
        src = stage;
    } else if (m > 0) {
        int32_t bad = 0;
        FSGP_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int32_t), s));
        k_hk_check<<<grid_el, 256, 0, s>>>(h0, m, d_flag);
        FSGP_CUDA(cudaMemcpyAsync(&bad, d_flag, sizeof bad, cudaMemcpyDeviceToHost, s));
        FSGP_CUDA(cudaStreamSynchronize(s));
        if (bad) return fail(FSGP_EINVAL, "opinions must be finite");
    }
    FSGP_CUDA(cudaMemsetAsync(d_ch, 0, sizeof(unsigned long long) * ((size_t)T + 1), s));
    if (n > 0) k_hk_in<<<grid_el, 256, 0, s>>>(src, n, R, Rp, buf0);
    const float eps_f = (float)eps;
    const int G = Rp / 32;
    const int VG = std::min(G, kHkMaxVG) >= 4 ? 4 : (std::min(G, kHkMaxVG) >= 2 ? 2 : 1);
    const int64_t warps = (int64_t)n * ((G + VG - 1) / VG);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)g->sm_count * 8));
    float *cur = buf0, *nxt = buf1;
    for (int32_t k = 1; k <= T && n > 0; ++k) {
        if (VG == 4)
            k_hk_step<4><<<grid, 256, 0, s>>>(g->row_ptr, g->col, g->rows_sorted, n, R, Rp, eps_f, cur, nxt, d_ch + k);
        else if (VG == 2)
            k_hk_step<2><<<grid, 256, 0, s>>>(g->row_ptr, g->col, g->rows_sorted, n, R, Rp, eps_f, cur, nxt, d_ch + k);
        else
            k_hk_step<1><<<grid, 256, 0, s>>>(g->row_ptr, g->col, g->rows_sorted, n, R, Rp, eps_f, cur, nxt, d_ch + k);
        std::swap(cur, nxt);
    }
    FSGP_CUDA(cudaGetLastError());
    float *dst = flags == FSGP_PTR_HOST ? stage : h_out;
    if (n > 0) k_hk_out<<<grid_el, 256, 0, s>>>(cur, n, R, Rp, dst);
    FSGP_CUDA(cudaGetLastError());
    if (flags == FSGP_PTR_HOST) {
        if (m > 0) FSGP_CUDA(cudaMemcpyAsync(h_out, stage, sizeof(float) * (size_t)m, cudaMemcpyDeviceToHost, s));
        if (changes)
            FSGP_CUDA(cudaMemcpyAsync(changes, d_ch, sizeof(uint64_t) * ((size_t)T + 1), cudaMemcpyDeviceToHost, s));
        FSGP_CUDA(cudaStreamSynchronize(s));
    } else if (changes) {
        FSGP_CUDA(cudaMemcpyAsync(changes, d_ch, sizeof(uint64_t) * ((size_t)T + 1), cudaMemcpyDeviceToDevice, s));
    }
    return FSGP_OK;
}
