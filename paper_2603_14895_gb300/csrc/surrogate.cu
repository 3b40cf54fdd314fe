// surrogate.cu -- learned seed-set surrogate: a 3-layer message-passing network that
// predicts each node's infection probability from the seed set and the model
// parameters, trained on the simulator's own per-node final frequencies, used to
// screen many candidate seed sets before Monte Carlo re-scores the best of them.
// The paper has no learned component; this is the project's screening surrogate.
//
//   x_v  = [seed_v, beta, gamma, log(1+d_in), log(1+d_out), log(1+k_v), 0, 0]
//          (k_v = in-arcs of v whose source is a seed, with multiplicity)
//   m_v  = mean over in-arcs u -> v of h_u          (message passing, Sec. 3.1 Eq. agg)
//   h'_v = ReLU(h_v Ws_l + m_v Wn_l + b_l), l = 1..3, width 64
//   p_v  = sigmoid(h3_v . w_o + b_o),  loss = mean_v (p_v - y_v)^2
//
// Dense products run on the tensor cores (mma.sync m16n8k16, bfloat16 operands, float32
// accumulation); activations are stored as bfloat16, gradients and the Adam state in
// float32.  Every kernel is this project's own.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "fsgp_internal.cuh"

namespace fsgp {
namespace sg {

constexpr int H = 64;          // hidden width
constexpr int F0 = 8;          // input features (5 used, zero padded)
// flat parameter layout (float32): Ws1 Wn1 b1 Ws2 Wn2 b2 Ws3 Wn3 b3 wo bo
constexpr int kW1 = F0 * H, kW = H * H;
constexpr int OFF_WS1 = 0, OFF_WN1 = OFF_WS1 + kW1, OFF_B1 = OFF_WN1 + kW1;
constexpr int OFF_WS2 = OFF_B1 + H, OFF_WN2 = OFF_WS2 + kW, OFF_B2 = OFF_WN2 + kW;
constexpr int OFF_WS3 = OFF_B2 + H, OFF_WN3 = OFF_WS3 + kW, OFF_B3 = OFF_WN3 + kW;
constexpr int OFF_WO = OFF_B3 + H, OFF_BO = OFF_WO + H;
constexpr int N_PARAMS = OFF_BO + 1;

__host__ __device__ constexpr int off_ws(int l) { return l == 1 ? OFF_WS1 : (l == 2 ? OFF_WS2 : OFF_WS3); }
__host__ __device__ constexpr int off_wn(int l) { return l == 1 ? OFF_WN1 : (l == 2 ? OFF_WN2 : OFF_WN3); }
__host__ __device__ constexpr int off_b(int l) { return l == 1 ? OFF_B1 : (l == 2 ? OFF_B2 : OFF_B3); }

typedef __nv_bfloat16 bf16;
typedef __nv_bfloat162 bf162;

// ------------------------------------------------------------------ forward kernels

// Input features; seed bits come from the (device) seed list of candidate *cur.
__global__ void k_features(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ out_ptr,
                           int32_t n, float beta, float gamma, bf16 *x) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const float din = (float)(row_ptr[v + 1] - row_ptr[v]);
        const float dout = (float)(out_ptr[v + 1] - out_ptr[v]);
        bf16 *r = x + (size_t)v * F0;
        r[0] = __float2bfloat16(0.f);
        r[1] = __float2bfloat16(beta);
        r[2] = __float2bfloat16(gamma);
        r[3] = __float2bfloat16(log1pf(din));
        r[4] = __float2bfloat16(log1pf(dout));
        r[5] = r[6] = r[7] = __float2bfloat16(0.f);
    }
}

// Seed in-arc counts: for every out-arc s -> v of the seeds of candidate *cur add `delta`
// to cnt[v] (one warp per seed).
__global__ void k_seed_count(const int32_t *__restrict__ cand, int32_t k, const int32_t *cur,
                             const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_dst,
                             int32_t delta, int32_t *cnt) {
    const int c = *cur;
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < k; i += (gridDim.x * blockDim.x) >> 5) {
        const int32_t sd = cand[(size_t)c * k + i];
        for (int32_t a = out_ptr[sd] + lane; a < out_ptr[sd + 1]; a += 32) atomicAdd(&cnt[out_dst[a]], delta);
    }
}

// Feature 5 = log(1 + cnt[v]) for the out-neighbours of the seeds of candidate *cur.
__global__ void k_seed_feat(const int32_t *__restrict__ cand, int32_t k, const int32_t *cur,
                            const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_dst,
                            const int32_t *__restrict__ cnt, bf16 *x) {
    const int c = *cur;
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < k; i += (gridDim.x * blockDim.x) >> 5) {
        const int32_t sd = cand[(size_t)c * k + i];
        for (int32_t a = out_ptr[sd] + lane; a < out_ptr[sd + 1]; a += 32) {
            const int32_t v = out_dst[a];
            x[(size_t)v * F0 + 5] = __float2bfloat16(log1pf((float)cnt[v]));
        }
    }
}

// Set (value 1) or clear (value 0) the seed bit of the seeds of candidate *cur; the
// clearing pass also advances *cur.
__global__ void k_seed_bits(const int32_t *__restrict__ cand, int32_t k, int32_t *cur, float value,
                            int advance, bf16 *x) {
    const int c = *cur;
    for (int i = threadIdx.x; i < k; i += blockDim.x) x[(size_t)cand[(size_t)c * k + i] * F0] = __float2bfloat16(value);
    __syncthreads();
    if (advance && threadIdx.x == 0) *cur = c + 1;
}

// m_v = mean over in-arcs of h_u (bfloat16 in and out, float32 sums).  F/2 threads per
// row, one bfloat16 pair each.
template <int F>
__global__ void k_agg(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                      const bf16 *__restrict__ h, bf16 *m) {
    constexpr int TPR = F / 2;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int j = (int)(t % TPR);
    for (int64_t v = t / TPR; v < n; v += nthreads / TPR) {
        const int32_t b = row_ptr[v], e = row_ptr[v + 1];
        float s0 = 0.f, s1 = 0.f;
        for (int32_t a = b; a < e; ++a) {
            const bf162 x = reinterpret_cast<const bf162 *>(h + (size_t)__ldg(col + a) * F)[j];
            s0 += __bfloat162float(x.x);
            s1 += __bfloat162float(x.y);
        }
        const float inv = e > b ? 1.f / (float)(e - b) : 0.f;
        reinterpret_cast<bf162 *>(m + (size_t)v * F)[j] = __floats2bfloat162_rn(s0 * inv, s1 * inv);
    }
}

__device__ __forceinline__ uint32_t ld_b32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// y = ReLU([h | m] W + b) for a row tile: one warp per 16 rows x 64 columns, K = 2F.
// W (K x 64, rows of Ws then Wn) is staged transposed in shared memory.
template <int F>
__global__ void __launch_bounds__(128) k_dense(const bf16 *__restrict__ h, const bf16 *__restrict__ m,
                                               const bf16 *__restrict__ Ws, const bf16 *__restrict__ Wn,
                                               const float *__restrict__ bias, int32_t n, bf16 *y) {
    constexpr int K = 2 * F;
    constexpr int KP = K + 8;   // padded row (bank spread)
    __shared__ __align__(16) bf16 Wt[H * KP];
    for (int i = threadIdx.x; i < K * H; i += blockDim.x) {
        const int k = i / H, c = i % H;
        Wt[c * KP + k] = k < F ? Ws[k * H + c] : Wn[(k - F) * H + c];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int64_t tiles = ((int64_t)n + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < K / 16; ++ks) {
            const int k0 = ks * 16;
            // A fragment: columns k0 + 2tg (+1) and k0 + 8 + 2tg (+1) of rows r0, r1
            uint32_t a[4];
            const int ca = k0 + 2 * tg, cb = k0 + 8 + 2 * tg;
            auto col_ptr = [&](int64_t r, int c) -> const bf16 * {
                return c < F ? h + (size_t)r * F + c : m + (size_t)r * F + (c - F);
            };
            a[0] = r0 < n ? ld_b32(col_ptr(r0, ca)) : 0u;
            a[1] = r1 < n ? ld_b32(col_ptr(r1, ca)) : 0u;
            a[2] = r0 < n ? ld_b32(col_ptr(r0, cb)) : 0u;
            a[3] = r1 < n ? ld_b32(col_ptr(r1, cb)) : 0u;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const bf16 *wr = Wt + (nt * 8 + g) * KP;
                const uint32_t b0 = ld_b32(wr + k0 + 2 * tg);
                const uint32_t b1 = ld_b32(wr + k0 + 8 + 2 * tg);
                mma_bf16(acc[nt], a, b0, b1);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * tg;
            const float bb0 = bias[c], bb1 = bias[c + 1];
            if (r0 < n)
                *reinterpret_cast<bf162 *>(y + (size_t)r0 * H + c) =
                    __floats2bfloat162_rn(fmaxf(acc[nt][0] + bb0, 0.f), fmaxf(acc[nt][1] + bb1, 0.f));
            if (r1 < n)
                *reinterpret_cast<bf162 *>(y + (size_t)r1 * H + c) =
                    __floats2bfloat162_rn(fmaxf(acc[nt][2] + bb0, 0.f), fmaxf(acc[nt][3] + bb1, 0.f));
        }
    }
}

// p_v = sigmoid(h3 . wo + bo); optional sum of p into *psum (screening score).
__global__ void k_head(const bf16 *__restrict__ h3, const bf16 *__restrict__ wo, const float *__restrict__ bo,
                       int32_t n, float *p, float *psum, const int32_t *cur) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bf162 w = reinterpret_cast<const bf162 *>(wo)[lane];
    float local = 0.f;
    for (int64_t v = warp; v < n; v += nw) {
        const bf162 x = reinterpret_cast<const bf162 *>(h3 + (size_t)v * H)[lane];
        float s = __bfloat162float(x.x) * __bfloat162float(w.x) + __bfloat162float(x.y) * __bfloat162float(w.y);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float pv = 1.f / (1.f + expf(-(s + bo[0])));
        if (lane == 0) {
            if (p) p[v] = pv;
            local += pv;
        }
    }
    if (psum && lane == 0 && local != 0.f) atomicAdd(psum + *cur, local);
}

// ----------------------------------------------------------------- backward kernels

// dlogit = 2 (p - y) / n * p (1 - p); dh3 = dlogit * wo; grad wo += sum h3 dlogit,
// grad bo += sum dlogit; loss += sum (p - y)^2 / n (double).
__global__ void k_head_bwd(const bf16 *__restrict__ h3, const bf16 *__restrict__ wo, const float *__restrict__ p,
                           const float *__restrict__ y, int32_t n, float *dh, float *grad, double *loss) {
    __shared__ float s_gwo[8][H];
    __shared__ float s_gbo[8];
    __shared__ double s_loss[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bf162 w = reinterpret_cast<const bf162 *>(wo)[lane];
    float g0 = 0.f, g1 = 0.f, gb = 0.f;
    double ls = 0.0;
    for (int64_t v = warp; v < n; v += nw) {
        const float pv = p[v], diff = pv - y[v];
        const float dl = 2.f * diff / (float)n * pv * (1.f - pv);
        const bf162 x = reinterpret_cast<const bf162 *>(h3 + (size_t)v * H)[lane];
        g0 += __bfloat162float(x.x) * dl;
        g1 += __bfloat162float(x.y) * dl;
        reinterpret_cast<float2 *>(dh + (size_t)v * H)[lane] =
            make_float2(dl * __bfloat162float(w.x), dl * __bfloat162float(w.y));
        if (lane == 0) {
            gb += dl;
            ls += (double)diff * diff;
        }
    }
    s_gwo[wid][2 * lane] = g0;
    s_gwo[wid][2 * lane + 1] = g1;
    if (lane == 0) {
        s_gbo[wid] = gb;
        s_loss[wid] = ls;
    }
    __syncthreads();
    if (threadIdx.x < H) {
        float s = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += s_gwo[i][threadIdx.x];
        atomicAdd(grad + OFF_WO + threadIdx.x, s);
    }
    if (threadIdx.x == 0) {
        float s = 0.f;
        double l = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            s += s_gbo[i];
            l += s_loss[i];
        }
        atomicAdd(grad + OFF_BO, s);
        atomicAdd(loss, l / (double)n);
    }
}

// One layer backward for a block of rows: dz = dy * (y > 0); grad Ws += h^T dz,
// grad Wn += m^T dz, grad b += sum dz; dah = dz Ws^T, dam = dz Wn^T (float32).
// 256 threads: thread (i, j4) accumulates grad rows i (of 2F) and 4 columns.
template <int F>
__global__ void __launch_bounds__(256) k_dense_bwd(const bf16 *__restrict__ h, const bf16 *__restrict__ m,
                                                   const bf16 *__restrict__ y, const float *__restrict__ dy,
                                                   const bf16 *__restrict__ Ws, const bf16 *__restrict__ Wn,
                                                   int32_t n, float *dah, float *dam, float *grad, int l) {
    constexpr int K = 2 * F;
    constexpr int ROWS = 16;   // 4 KB dz + 8 KB inputs + 32 KB weights of static shared memory
    __shared__ float s_dz[ROWS][H];
    __shared__ float s_a[ROWS][K];
    __shared__ float s_w[K][H];
    for (int i = threadIdx.x; i < K * H; i += blockDim.x) {
        const int k = i / H, c = i % H;
        s_w[k][c] = __bfloat162float(k < F ? Ws[k * H + c] : Wn[(k - F) * H + c]);
    }
    // gradient accumulators: K x H entries over 256 threads
    constexpr int PER = (K * H + 255) / 256;
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = 0.f;
    float accb = 0.f;   // bias column threadIdx.x (< H)
    __syncthreads();
    for (int64_t r0 = (int64_t)blockIdx.x * ROWS; r0 < n; r0 += (int64_t)gridDim.x * ROWS) {
        const int rows = (int)min((int64_t)ROWS, (int64_t)n - r0);
        for (int i = threadIdx.x; i < ROWS * H; i += blockDim.x) {
            const int rr = i / H, c = i % H;
            float dz = 0.f;
            if (rr < rows) {
                const size_t o = (size_t)(r0 + rr) * H + c;
                dz = __bfloat162float(y[o]) > 0.f ? dy[o] : 0.f;
            }
            s_dz[rr][c] = dz;
        }
        for (int i = threadIdx.x; i < ROWS * K; i += blockDim.x) {
            const int rr = i / K, k = i % K;
            float a = 0.f;
            if (rr < rows) a = __bfloat162float(k < F ? h[(size_t)(r0 + rr) * F + k] : m[(size_t)(r0 + rr) * F + (k - F)]);
            s_a[rr][k] = a;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = threadIdx.x + q * 256;
            if (e < K * H) {
                const int k = e / H, c = e % H;
                float s = 0.f;
                for (int rr = 0; rr < rows; ++rr) s += s_a[rr][k] * s_dz[rr][c];
                acc[q] += s;
            }
        }
        if (threadIdx.x < H)
            for (int rr = 0; rr < rows; ++rr) accb += s_dz[rr][threadIdx.x];
        // input gradients: thread -> (row, column of 2F)
        for (int i = threadIdx.x; i < rows * K; i += blockDim.x) {
            const int rr = i / K, k = i % K;
            float s = 0.f;
#pragma unroll 8
            for (int c = 0; c < H; ++c) s += s_dz[rr][c] * s_w[k][c];
            if (k < F) dah[(size_t)(r0 + rr) * F + k] = s;
            else dam[(size_t)(r0 + rr) * F + (k - F)] = s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = threadIdx.x + q * 256;
        if (e < K * H) {
            const int k = e / H, c = e % H;
            atomicAdd(grad + (k < F ? off_ws(l) + k * H + c : off_wn(l) + (k - F) * H + c), acc[q]);
        }
    }
    if (threadIdx.x < H) atomicAdd(grad + off_b(l) + threadIdx.x, accb);
}

// dh_u = dah_u + sum over out-arcs u -> v of dam_v / d_in(v)   (adjoint of the mean)
template <int F>
__global__ void k_agg_bwd(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ out_ptr,
                          const int32_t *__restrict__ out_dst, int32_t n, const float *__restrict__ dah,
                          const float *__restrict__ dam, float *dh) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t; i < (int64_t)n * F; i += nthreads) {
        const int64_t u = i / F;
        const int j = (int)(i % F);
        float s = dah[i];
        const int32_t b = out_ptr[u], e = out_ptr[u + 1];
        for (int32_t a = b; a < e; ++a) {
            const int32_t v = out_dst[a];
            s += dam[(size_t)v * F + j] / (float)(row_ptr[v + 1] - row_ptr[v]);
        }
        dh[i] = s;
    }
}

// Adam (Kingma and Ba, 2015) with bias correction, then the bfloat16 copies.
__global__ void k_adam(float *theta, float *m, float *v, const float *g, int np, float lr, float b1,
                       float b2, float eps, float c1, float c2, bf16 *wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += blockDim.x * gridDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        theta[i] = th;
        wb[i] = __float2bfloat16(th);
    }
}

__global__ void k_to_bf16(const float *theta, int np, bf16 *wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += blockDim.x * gridDim.x)
        wb[i] = __float2bfloat16(theta[i]);
}

}  // namespace sg
}  // namespace fsgp

using namespace fsgp;
using namespace fsgp::sg;

struct fsgp_surrogate {
    int device = 0;
    int sm_count = 0;
    float *theta = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
    bf16 *wb = nullptr;        // bfloat16 copy of theta (same layout)
    int64_t step = 0;
    // activations / gradients for graphs up to cap nodes
    int64_t cap = 0;
    bf16 *x = nullptr, *m1 = nullptr, *h1 = nullptr, *m2 = nullptr, *h2 = nullptr, *m3 = nullptr, *h3 = nullptr;
    float *p = nullptr, *y = nullptr, *dh = nullptr, *dah = nullptr, *dam = nullptr, *dh2 = nullptr;
    double *loss = nullptr;
    int32_t *cur = nullptr;
    int32_t *cnt = nullptr;     // seed in-arc counts per node (kept at zero between calls)
};

namespace {

void sg_free_acts(fsgp_surrogate *s) {
    void *ptrs[] = {s->x, s->m1, s->h1, s->m2, s->h2, s->m3, s->h3, s->p, s->y, s->dh, s->dah, s->dam, s->dh2, s->cnt};
    for (void *p : ptrs) cudaFree(p);
    s->cnt = nullptr;
    s->x = s->m1 = s->h1 = s->m2 = s->h2 = s->m3 = s->h3 = nullptr;
    s->p = s->y = s->dh = s->dah = s->dam = s->dh2 = nullptr;
    s->cap = 0;
}

int sg_ensure(fsgp_surrogate *s, int64_t n) {
    if (n <= s->cap) return FSGP_OK;
    sg_free_acts(s);
    const size_t nb = (size_t)n;
    cudaError_t e;
    if ((e = cudaMalloc(&s->x, nb * F0 * sizeof(bf16))) != cudaSuccess ||
        (e = cudaMalloc(&s->m1, nb * F0 * sizeof(bf16))) != cudaSuccess ||
        (e = cudaMalloc(&s->h1, nb * H * sizeof(bf16))) != cudaSuccess ||
        (e = cudaMalloc(&s->m2, nb * H * sizeof(bf16))) != cudaSuccess ||
        (e = cudaMalloc(&s->h2, nb * H * sizeof(bf16))) != cudaSuccess ||
        (e = cudaMalloc(&s->m3, nb * H * sizeof(bf16))) != cudaSuccess ||
        (e = cudaMalloc(&s->h3, nb * H * sizeof(bf16))) != cudaSuccess ||
        (e = cudaMalloc(&s->p, nb * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&s->y, nb * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&s->dh, nb * H * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&s->dah, nb * H * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&s->dam, nb * H * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&s->dh2, nb * H * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&s->cnt, nb * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemset(s->cnt, 0, nb * sizeof(int32_t))) != cudaSuccess) {
        sg_free_acts(s);
        return cuda_fail(e, "cudaMalloc (surrogate activations)");
    }
    s->cap = n;
    return FSGP_OK;
}

int grid_of(const fsgp_surrogate *s, int64_t work, int threads, int per_sm = 8) {
    int64_t g = (work + threads - 1) / threads;
    g = std::min<int64_t>(g, (int64_t)s->sm_count * per_sm);
    return (int)std::max<int64_t>(g, 1);
}

// Forward of the three layers and the head from features s->x (already seeded).
void sg_forward(fsgp_surrogate *s, const fsgp_graph *g, float *p, float *psum, cudaStream_t st) {
    const int32_t n = g->n;
    const bf16 *W = s->wb;
    const float *B = s->theta;
    k_agg<F0><<<grid_of(s, (int64_t)n * (F0 / 2), 256), 256, 0, st>>>(g->row_ptr, g->col, n, s->x, s->m1);
    k_dense<F0><<<grid_of(s, ((int64_t)n + 63) / 64 * 128, 128, 16), 128, 0, st>>>(
        s->x, s->m1, W + OFF_WS1, W + OFF_WN1, B + OFF_B1, n, s->h1);
    k_agg<H><<<grid_of(s, (int64_t)n * (H / 2), 256), 256, 0, st>>>(g->row_ptr, g->col, n, s->h1, s->m2);
    k_dense<H><<<grid_of(s, ((int64_t)n + 63) / 64 * 128, 128, 16), 128, 0, st>>>(
        s->h1, s->m2, W + OFF_WS2, W + OFF_WN2, B + OFF_B2, n, s->h2);
    k_agg<H><<<grid_of(s, (int64_t)n * (H / 2), 256), 256, 0, st>>>(g->row_ptr, g->col, n, s->h2, s->m3);
    k_dense<H><<<grid_of(s, ((int64_t)n + 63) / 64 * 128, 128, 16), 128, 0, st>>>(
        s->h2, s->m3, W + OFF_WS3, W + OFF_WN3, B + OFF_B3, n, s->h3);
    k_head<<<grid_of(s, (int64_t)n * 32, 256), 256, 0, st>>>(s->h3, W + OFF_WO, B + OFF_BO, n, p, psum, s->cur);
}

int sg_prepare_inputs(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *seeds_host, int64_t ns,
                      double beta, double gamma, cudaStream_t st) {
    for (int64_t i = 0; i < ns; ++i)
        if (seeds_host[i] < 0 || seeds_host[i] >= g->n) return fail(FSGP_EINVAL, "seed node out of range");
    int rc = sg_ensure(s, g->n);
    if (rc) return rc;
    k_features<<<grid_of(s, g->n, 256), 256, 0, st>>>(g->row_ptr, g->out_ptr, g->n, (float)beta, (float)gamma, s->x);
    if (ns > 0) {
        // seed bits: small host list staged through the activation buffer y (floats)
        int32_t *d_seeds = reinterpret_cast<int32_t *>(s->y);
        if (ns > s->cap) return fail(FSGP_EINVAL, "more seeds than nodes");
        FSGP_CUDA(cudaMemcpyAsync(d_seeds, seeds_host, sizeof(int32_t) * (size_t)ns, cudaMemcpyHostToDevice, st));
        FSGP_CUDA(cudaMemsetAsync(s->cur, 0, sizeof(int32_t), st));
        k_seed_bits<<<1, 256, 0, st>>>(d_seeds, (int32_t)ns, s->cur, 1.f, 0, s->x);
        const int gk = (int)std::min<int64_t>(((int64_t)ns * 32 + 255) / 256, 1024);
        k_seed_count<<<gk, 256, 0, st>>>(d_seeds, (int32_t)ns, s->cur, g->out_ptr, g->out_dst, 1, s->cnt);
        k_seed_feat<<<gk, 256, 0, st>>>(d_seeds, (int32_t)ns, s->cur, g->out_ptr, g->out_dst, s->cnt, s->x);
        k_seed_count<<<gk, 256, 0, st>>>(d_seeds, (int32_t)ns, s->cur, g->out_ptr, g->out_dst, -1, s->cnt);
    }
    FSGP_CUDA(cudaGetLastError());
    return FSGP_OK;
}

int sg_backward(fsgp_surrogate *s, const fsgp_graph *g, cudaStream_t st) {
    const int32_t n = g->n;
    const bf16 *W = s->wb;
    FSGP_CUDA(cudaMemsetAsync(s->grad, 0, sizeof(float) * N_PARAMS, st));
    FSGP_CUDA(cudaMemsetAsync(s->loss, 0, sizeof(double), st));
    k_head_bwd<<<grid_of(s, (int64_t)n * 32, 256), 256, 0, st>>>(s->h3, W + OFF_WO, s->p, s->y, n, s->dh, s->grad, s->loss);
    const int gb = grid_of(s, (int64_t)n, 16, 2);
    // layer 3: dy = dh (float), outputs dh2 = d h2
    k_dense_bwd<H><<<gb, 256, 0, st>>>(s->h2, s->m3, s->h3, s->dh, W + OFF_WS3, W + OFF_WN3, n, s->dah, s->dam, s->grad, 3);
    k_agg_bwd<H><<<grid_of(s, (int64_t)n * H, 256), 256, 0, st>>>(g->row_ptr, g->out_ptr, g->out_dst, n, s->dah, s->dam, s->dh2);
    // layer 2
    k_dense_bwd<H><<<gb, 256, 0, st>>>(s->h1, s->m2, s->h2, s->dh2, W + OFF_WS2, W + OFF_WN2, n, s->dah, s->dam, s->grad, 2);
    k_agg_bwd<H><<<grid_of(s, (int64_t)n * H, 256), 256, 0, st>>>(g->row_ptr, g->out_ptr, g->out_dst, n, s->dah, s->dam, s->dh);
    // layer 1 (input gradients not needed beyond the weights)
    k_dense_bwd<F0><<<gb, 256, 0, st>>>(s->x, s->m1, s->h1, s->dh, W + OFF_WS1, W + OFF_WN1, n, s->dah, s->dam, s->grad, 1);
    FSGP_CUDA(cudaGetLastError());
    return FSGP_OK;
}

// init: He normal weights from a SplitMix64 stream (Box-Muller), zero biases
uint64_t sm64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" int fsgp_surrogate_num_params(void) { return N_PARAMS; }

extern "C" int fsgp_surrogate_create(uint64_t init_seed, fsgp_surrogate **out) {
    set_error("");
    if (!out) return fail(FSGP_EINVAL, "out is NULL");
    *out = nullptr;
    fsgp_surrogate *s = new (std::nothrow) fsgp_surrogate();
    if (!s) return fail(FSGP_ENOMEM, "host allocation failed");
    cudaError_t e;
    if ((e = cudaGetDevice(&s->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device)) != cudaSuccess ||
        (e = cudaMalloc(&s->theta, sizeof(float) * N_PARAMS)) != cudaSuccess ||
        (e = cudaMalloc(&s->adam_m, sizeof(float) * N_PARAMS)) != cudaSuccess ||
        (e = cudaMalloc(&s->adam_v, sizeof(float) * N_PARAMS)) != cudaSuccess ||
        (e = cudaMalloc(&s->grad, sizeof(float) * N_PARAMS)) != cudaSuccess ||
        (e = cudaMalloc(&s->wb, sizeof(bf16) * N_PARAMS)) != cudaSuccess ||
        (e = cudaMalloc(&s->loss, sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&s->cur, sizeof(int32_t))) != cudaSuccess) {
        fsgp_surrogate_destroy(s);
        return cuda_fail(e, "cudaMalloc (surrogate)");
    }
    std::vector<float> th(N_PARAMS, 0.f);
    uint64_t st = init_seed;
    auto normal = [&]() {
        const double u1 = ((sm64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((sm64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    };
    auto fill = [&](int off, int count, double sd) {
        for (int i = 0; i < count; ++i) th[off + i] = (float)(sd * normal());
    };
    fill(OFF_WS1, kW1, sqrt(2.0 / (2 * F0)));
    fill(OFF_WN1, kW1, sqrt(2.0 / (2 * F0)));
    for (int l = 2; l <= 3; ++l) {
        fill(off_ws(l), kW, sqrt(2.0 / (2 * H)));
        fill(off_wn(l), kW, sqrt(2.0 / (2 * H)));
    }
    fill(OFF_WO, H, sqrt(1.0 / H));
    if ((e = cudaMemcpy(s->theta, th.data(), sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(s->adam_m, 0, sizeof(float) * N_PARAMS)) != cudaSuccess ||
        (e = cudaMemset(s->adam_v, 0, sizeof(float) * N_PARAMS)) != cudaSuccess) {
        fsgp_surrogate_destroy(s);
        return cuda_fail(e, "surrogate init");
    }
    k_to_bf16<<<32, 256>>>(s->theta, N_PARAMS, s->wb);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        fsgp_surrogate_destroy(s);
        return cuda_fail(e, "surrogate init");
    }
    *out = s;
    return FSGP_OK;
}

extern "C" int fsgp_surrogate_destroy(fsgp_surrogate *s) {
    set_error("");
    if (!s) return FSGP_OK;
    cudaDeviceSynchronize();
    sg_free_acts(s);
    cudaFree(s->theta);
    cudaFree(s->adam_m);
    cudaFree(s->adam_v);
    cudaFree(s->grad);
    cudaFree(s->wb);
    cudaFree(s->loss);
    cudaFree(s->cur);
    delete s;
    return FSGP_OK;
}

extern "C" int fsgp_surrogate_params(fsgp_surrogate *s, float *get_host, const float *set_host) {
    set_error("");
    if (!s) return fail(FSGP_EINVAL, "surrogate is NULL");
    if (set_host) {
        FSGP_CUDA(cudaMemcpy(s->theta, set_host, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice));
        FSGP_CUDA(cudaMemset(s->adam_m, 0, sizeof(float) * N_PARAMS));
        FSGP_CUDA(cudaMemset(s->adam_v, 0, sizeof(float) * N_PARAMS));
        s->step = 0;
        k_to_bf16<<<32, 256>>>(s->theta, N_PARAMS, s->wb);
        FSGP_CUDA(cudaDeviceSynchronize());
    }
    if (get_host) FSGP_CUDA(cudaMemcpy(get_host, s->theta, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost));
    return FSGP_OK;
}

extern "C" int fsgp_surrogate_forward(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *seeds_host,
                                      int64_t n_seeds, double beta, double gamma, float *p_out, void *stream) {
    set_error("");
    if (!s || !g || !p_out || (n_seeds > 0 && !seeds_host)) return fail(FSGP_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = sg_prepare_inputs(s, g, seeds_host, n_seeds, beta, gamma, st);
    if (rc) return rc;
    sg_forward(s, g, p_out, nullptr, st);
    FSGP_CUDA(cudaGetLastError());
    return FSGP_OK;
}

extern "C" int fsgp_surrogate_grad(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *seeds_host,
                                   int64_t n_seeds, double beta, double gamma, const float *y,
                                   double *loss_out, float *grad_out, void *stream) {
    set_error("");
    if (!s || !g || !y || (n_seeds > 0 && !seeds_host)) return fail(FSGP_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = sg_prepare_inputs(s, g, seeds_host, n_seeds, beta, gamma, st);
    if (rc) return rc;
    FSGP_CUDA(cudaMemcpyAsync(s->y, y, sizeof(float) * (size_t)g->n, cudaMemcpyDeviceToDevice, st));
    sg_forward(s, g, s->p, nullptr, st);
    rc = sg_backward(s, g, st);
    if (rc) return rc;
    if (loss_out) FSGP_CUDA(cudaMemcpyAsync(loss_out, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_out) FSGP_CUDA(cudaMemcpyAsync(grad_out, s->grad, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, st));
    FSGP_CUDA(cudaStreamSynchronize(st));
    return FSGP_OK;
}

extern "C" int fsgp_surrogate_train_step(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *seeds_host,
                                         int64_t n_seeds, double beta, double gamma, const float *y,
                                         float lr, double *loss_out, void *stream) {
    set_error("");
    if (!s || !g || !y || (n_seeds > 0 && !seeds_host)) return fail(FSGP_EINVAL, "NULL argument");
    if (!(lr > 0.f)) return fail(FSGP_EINVAL, "learning rate must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = sg_prepare_inputs(s, g, seeds_host, n_seeds, beta, gamma, st);
    if (rc) return rc;
    FSGP_CUDA(cudaMemcpyAsync(s->y, y, sizeof(float) * (size_t)g->n, cudaMemcpyDeviceToDevice, st));
    sg_forward(s, g, s->p, nullptr, st);
    rc = sg_backward(s, g, st);
    if (rc) return rc;
    s->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)s->step), c2 = 1.f - powf(b2, (float)s->step);
    k_adam<<<grid_of(s, N_PARAMS, 256), 256, 0, st>>>(s->theta, s->adam_m, s->adam_v, s->grad, N_PARAMS, lr,
                                                      b1, b2, 1e-8f, c1, c2, s->wb);
    FSGP_CUDA(cudaGetLastError());
    if (loss_out) {
        FSGP_CUDA(cudaMemcpyAsync(loss_out, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        FSGP_CUDA(cudaStreamSynchronize(st));
    }
    return FSGP_OK;
}

extern "C" int fsgp_surrogate_screen(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *cand_host,
                                     int32_t k, int32_t n_cand, double beta, double gamma, float *scores_out,
                                     void *stream) {
    set_error("");
    if (!s || !g || !cand_host || !scores_out || k < 1 || n_cand < 1) return fail(FSGP_EINVAL, "bad argument");
    for (int64_t i = 0; i < (int64_t)k * n_cand; ++i)
        if (cand_host[i] < 0 || cand_host[i] >= g->n) return fail(FSGP_EINVAL, "candidate node out of range");
    cudaStream_t caller = (cudaStream_t)stream;
    int rc = sg_ensure(s, g->n);
    if (rc) return rc;
    // captures are not allowed on the legacy default stream: work on a private stream
    // ordered after the caller's work
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    FSGP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    FSGP_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    FSGP_CUDA(cudaEventRecord(ev, caller));
    FSGP_CUDA(cudaStreamWaitEvent(st, ev, 0));
    int32_t *d_cand = nullptr;
    float *d_scores = nullptr;
    FSGP_CUDA(cudaMalloc(&d_cand, sizeof(int32_t) * (size_t)k * n_cand));
    cudaError_t e = cudaMalloc(&d_scores, sizeof(float) * (size_t)n_cand);
    if (e != cudaSuccess) {
        cudaFree(d_cand);
        return cuda_fail(e, "cudaMalloc (screen)");
    }
    rc = FSGP_OK;
    do {
        if ((e = cudaMemcpyAsync(d_cand, cand_host, sizeof(int32_t) * (size_t)k * n_cand, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_scores, 0, sizeof(float) * (size_t)n_cand, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(s->cur, 0, sizeof(int32_t), st)) != cudaSuccess) {
            rc = cuda_fail(e, "screen setup");
            break;
        }
        k_features<<<grid_of(s, g->n, 256), 256, 0, st>>>(g->row_ptr, g->out_ptr, g->n, (float)beta, (float)gamma, s->x);
        // one candidate = set its seed bits, forward, add sum(p) into its score, clear the
        // bits and advance the device-side candidate index; captured once, replayed n_cand times
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            rc = cuda_fail(e, "capture");
            break;
        }
        const int gk = (int)std::min<int64_t>(((int64_t)k * 32 + 255) / 256, 1024);
        k_seed_bits<<<1, 256, 0, st>>>(d_cand, k, s->cur, 1.f, 0, s->x);
        k_seed_count<<<gk, 256, 0, st>>>(d_cand, k, s->cur, g->out_ptr, g->out_dst, 1, s->cnt);
        k_seed_feat<<<gk, 256, 0, st>>>(d_cand, k, s->cur, g->out_ptr, g->out_dst, s->cnt, s->x);
        sg_forward(s, g, nullptr, d_scores, st);
        k_seed_count<<<gk, 256, 0, st>>>(d_cand, k, s->cur, g->out_ptr, g->out_dst, -1, s->cnt);
        k_seed_feat<<<gk, 256, 0, st>>>(d_cand, k, s->cur, g->out_ptr, g->out_dst, s->cnt, s->x);
        k_seed_bits<<<1, 256, 0, st>>>(d_cand, k, s->cur, 0.f, 1, s->x);
        e = cudaStreamEndCapture(st, &graph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "screen graph");
            break;
        }
        for (int32_t c = 0; c < n_cand && e == cudaSuccess; ++c) e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(scores_out, d_scores, sizeof(float) * (size_t)n_cand, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) rc = cuda_fail(e, "screen");
    } while (0);
    cudaFree(d_cand);
    cudaFree(d_scores);
    cudaEventDestroy(ev);
    cudaStreamDestroy(st);
    return rc;
}
