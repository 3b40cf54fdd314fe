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
// The forward dense layers run on the fifth-generation tensor cores (tcgen05.mma into
// tensor memory, bfloat16 operands, float32 accumulation; the last layer applies the
// output head in its epilogue); the backward products use mma.sync m16n8k16 on the same
// operand types.  Activations are stored as bfloat16, gradients and the Adam state in
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
// to cnt[v] (one CTA per seed, so hub seeds spread over the CTA's threads).
__global__ void k_seed_count(const int32_t *__restrict__ cand, int32_t k, const int32_t *cur,
                             const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_dst,
                             int32_t delta, int32_t *cnt) {
    const int c = *cur;
    for (int i = blockIdx.x; i < k; i += gridDim.x) {
        const int32_t sd = cand[(size_t)c * k + i];
        for (int32_t a = out_ptr[sd] + threadIdx.x; a < out_ptr[sd + 1]; a += blockDim.x)
            atomicAdd(&cnt[out_dst[a]], delta);
    }
}

// Feature 5 = log(1 + cnt[v]) for the out-neighbours of the seeds of candidate *cur.
__global__ void k_seed_feat(const int32_t *__restrict__ cand, int32_t k, const int32_t *cur,
                            const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_dst,
                            const int32_t *__restrict__ cnt, bf16 *x) {
    const int c = *cur;
    for (int i = blockIdx.x; i < k; i += gridDim.x) {
        const int32_t sd = cand[(size_t)c * k + i];
        for (int32_t a = out_ptr[sd] + threadIdx.x; a < out_ptr[sd + 1]; a += blockDim.x) {
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

// m_v = mean over in-arcs of h_u (bfloat16 in and out, float32 sums).  A group of
// G = agg_arcs<F>() * F/8 threads takes one work item: F/8 threads cover the F features
// of a source row (16 bytes each) and the subgroups take every agg_arcs-th arc, so each
// load instruction fetches several source rows; the subgroups' sums meet by shuffle.
// (Measured on GB300, BA n = 500k: two subgroups for F = 64, four for F = 8.)
// Items 0..n-1 are rows (rows with >= kSgLong arcs are skipped); items n.. are the chunks
// of those long rows, whose partial sums go to acc[slot] for k_agg_fin.
template <int F>
__host__ __device__ constexpr int agg_arcs() { return F == 8 ? 4 : 2; }
template <int F>
__global__ void k_agg(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                      const bf16 *__restrict__ h, bf16 *m, const int4 *__restrict__ items, int32_t n_items,
                      float *acc) {
    constexpr int TPR = F / 8;
    constexpr int kAggArcs = agg_arcs<F>();
    constexpr int G = TPR * kAggArcs;
    static_assert(G <= 32 && (32 % G) == 0, "a group lies within a warp");
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int j = (int)(t % TPR);                // 16-byte feature chunk
    const int sub = (int)((t / TPR) % kAggArcs); // arc subgroup
    const int64_t total = (int64_t)n + n_items;
    // whole warps iterate together (the shuffles below need every lane of the group)
    const int64_t v_end = (total + (nthreads / G) - 1) / (nthreads / G) * (nthreads / G);
    for (int64_t v = t / G; v < v_end; v += nthreads / G) {
        int32_t row = 0, b = 0, e = 0, slot = -1;
        bool skip = v >= total;
        if (!skip) {
            if (v < n) {
                row = (int32_t)v;
                b = row_ptr[v];
                e = row_ptr[v + 1];
                if (e - b >= kSgLong) skip = true;
            } else {
                const int4 it = items[v - n];
                row = it.x, b = it.y, e = it.z, slot = it.w;
            }
        }
        float sum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (!skip) {
#pragma unroll 2
            for (int32_t a = b + sub; a < e; a += kAggArcs) {
                const uint4 x = __ldg(reinterpret_cast<const uint4 *>(h + (size_t)__ldg(col + a) * F) + j);
                const bf162 *xp = reinterpret_cast<const bf162 *>(&x);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    sum[2 * i] += __bfloat162float(xp[i].x);
                    sum[2 * i + 1] += __bfloat162float(xp[i].y);
                }
            }
        }
#pragma unroll
        for (int o = TPR; o < G; o <<= 1)
#pragma unroll
            for (int i = 0; i < 8; ++i) sum[i] += __shfl_xor_sync(0xffffffffu, sum[i], o);
        if (skip || sub != 0) continue;
        if (slot < 0) {
            const float inv = e > b ? 1.f / (float)(e - b) : 0.f;
            uint4 o;
            bf162 *op = reinterpret_cast<bf162 *>(&o);
#pragma unroll
            for (int i = 0; i < 4; ++i) op[i] = __floats2bfloat162_rn(sum[2 * i] * inv, sum[2 * i + 1] * inv);
            reinterpret_cast<uint4 *>(m + (size_t)row * F)[j] = o;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) atomicAdd(acc + (size_t)slot * F + 8 * j + i, sum[i]);
        }
    }
}

// Long rows: m = acc / d_in, and acc back to zero.
template <int F>
__global__ void k_agg_fin(const int32_t *__restrict__ long_rows, int32_t n_long, const int32_t *__restrict__ row_ptr,
                          float *acc, bf16 *m) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n_long * (F / 2);
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = i / (F / 2);
        const int j = (int)(i % (F / 2));
        const int32_t row = long_rows[slot];
        const float inv = 1.f / (float)(row_ptr[row + 1] - row_ptr[row]);
        float *p = acc + slot * F + 2 * j;
        reinterpret_cast<bf162 *>(m + (size_t)row * F)[j] = __floats2bfloat162_rn(p[0] * inv, p[1] * inv);
        p[0] = p[1] = 0.f;
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

// ------------------------------------------------------- dense layer on tcgen05 / TMEM
//
// y = ReLU([h | m] W + b) for tiles of 128 rows, K = 2F (16 or 128), N = 64, on the
// fifth-generation tensor cores: both operands staged in shared memory in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices; the two K-neighbour core
// matrices of one instruction lie 128 B apart, 8-row groups K*16 B apart), one elected
// thread issues K/16 tcgen05.mma (kind::f16: bfloat16 in, float32 accumulate) into a
// 128-lane x 64-column tensor-memory accumulator, commits them to an mbarrier, and the
// four warps read their 32 lanes back (tcgen05.ld) for bias, ReLU and the bfloat16 store.
// Persistent CTAs loop over tiles; W^T is staged once per CTA.

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row group)
// byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Byte offset of the 16-byte chunk kc of row r in a K-major core-matrix tile of KC chunks.
__device__ __forceinline__ uint32_t core_off(int r, int kc, int KC) {
    return (uint32_t)(((r >> 3) * KC + kc) * 128 + (r & 7) * 16);
}

constexpr int kTcRows = 128;            // rows per tile (MMA M)
constexpr int kTcWaitLimit = 1 << 24;   // mbarrier polls before giving up

// Two A tiles (the next one is fetched with cp.async while the current one is multiplied)
// and W^T.
template <int F>
constexpr size_t tc_smem_bytes() { return (size_t)(2 * kTcRows + H) * (2 * F) * 2; }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    // a source size of 0 fills the 16 bytes with zeros (rows past the end)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0));
}

// HEAD: the epilogue also applies the output head, p = sigmoid(h . w_o + b_o) of the
// bfloat16 layer output, and writes p (when p_out is set) and / or adds the sum of p
// into psum[*cur] (screening); y (the layer output) may then be null.
template <int F, bool HEAD>
__global__ void __launch_bounds__(128) k_dense_tc(const bf16 *__restrict__ h, const bf16 *__restrict__ m,
                                                  const bf16 *__restrict__ Ws, const bf16 *__restrict__ Wn,
                                                  const float *__restrict__ bias, int32_t n, bf16 *y,
                                                  const bf16 *__restrict__ wo, const float *__restrict__ bo,
                                                  float *p_out, float *psum, const int32_t *cur, int32_t *err) {
    constexpr int K = 2 * F;
    constexpr int KC = K / 8;            // 16-byte chunks per row
    constexpr int TILE = kTcRows * K * 2;
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    uint8_t *sA0 = tc_smem;                         // 2 x (128 x K)
    uint8_t *sB = tc_smem + 2 * TILE;               // 64 x K (W transposed)
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tiles = ((int64_t)n + kTcRows - 1) / kTcRows;
    if ((int64_t)blockIdx.x >= tiles) return;
    auto stage = [&](int buf, int64_t tile) {
        const uint32_t base = smem_addr(sA0 + buf * TILE);
        const int64_t row0 = tile * kTcRows;
        for (int c = tid; c < kTcRows * KC; c += blockDim.x) {
            const int r = c / KC, kc = c % KC;
            const int64_t row = row0 + r;
            const bool valid = row < n;
            const int64_t rr = valid ? row : 0;
            const bf16 *src = kc < KC / 2 ? h + (size_t)rr * F + kc * 8 : m + (size_t)rr * F + (kc - KC / 2) * 8;
            cp_async16(base + core_off(r, kc, KC), src, valid);
        }
        asm volatile("cp.async.commit_group;");
    };
    stage(0, blockIdx.x);
    // B: output column c holds its K inputs, Ws rows then Wn rows (coalesced row reads,
    // element-wise transposed stores)
    for (int i = tid; i < K * H; i += blockDim.x) {
        const int k = i / H, col = i % H;
        const bf16 w = k < F ? Ws[k * H + col] : Wn[(k - F) * H + col];
        *reinterpret_cast<bf16 *>(sB + core_off(col, k >> 3, KC) + (k & 7) * 2) = w;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // kind::f16: D f32 (bit 4), A and B bf16 (bits 7, 10), K-major, N = 64, M = 128
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                               ((uint32_t)(kTcRows >> 4) << 24);
    float wo_f[HEAD ? H : 1];
    float bo_f = 0.f;
    if constexpr (HEAD) {
#pragma unroll
        for (int j = 0; j < H; ++j) wo_f[j] = __bfloat162float(wo[j]);
        bo_f = bo[0];
    }
    float psum_local = 0.f;
    uint32_t phase = 0;
    bool ok = true;
    int buf = 0;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, buf ^= 1) {
        const int64_t next = tile + gridDim.x;
        if (next < tiles) {
            stage(buf ^ 1, next);
            asm volatile("cp.async.wait_group 1;");   // this tile's copies are done
        } else {
            asm volatile("cp.async.wait_group 0;");
        }
        asm volatile("fence.proxy.async.shared::cta;");   // smem writes -> tensor-core reads
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t tbase = tmem_base;
        if (tid == 0) {
            const uint32_t a0 = smem_addr(sA0 + buf * TILE), b0 = smem_addr(sB);
#pragma unroll
            for (int k = 0; k < K / 16; ++k) {
                const uint64_t ad = umma_desc(a0 + k * 256, 128, KC * 128);
                const uint64_t bd = umma_desc(b0 + k * 256, 128, KC * 128);
                const uint32_t accum = k > 0 ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             ::"r"(tbase), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_addr(&mbar)));
        }
        uint32_t done = 0;
        for (int it = 0; it < kTcWaitLimit && !done; ++it)
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                         " selp.u32 %0, 1, 0, p;\n}"
                         : "=r"(done) : "r"(smem_addr(&mbar)), "r"(phase));
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!done) {
            ok = false;
            atomicExch(err, 1);
            // give the issued MMAs a second bounded wait before the TMEM is freed
            for (int it = 0; it < kTcWaitLimit && !done; ++it)
                asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                             " selp.u32 %0, 1, 0, p;\n}"
                             : "=r"(done) : "r"(smem_addr(&mbar)), "r"(phase ^ 1u));
        } else {
            const int64_t row = tile * kTcRows + 32 * warp + lane;   // this thread's lane
            float dot = 0.f;
#pragma unroll
            for (int c0 = 0; c0 < H; c0 += 16) {
                uint32_t r[16];
                const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                               "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                bf162 o[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    o[j] = __floats2bfloat162_rn(fmaxf(__uint_as_float(r[2 * j]) + bias[c0 + 2 * j], 0.f),
                                                 fmaxf(__uint_as_float(r[2 * j + 1]) + bias[c0 + 2 * j + 1], 0.f));
                if constexpr (HEAD) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        dot += __bfloat162float(o[j].x) * wo_f[c0 + 2 * j] + __bfloat162float(o[j].y) * wo_f[c0 + 2 * j + 1];
                }
                if (y && row < n) {
                    uint4 *dst = reinterpret_cast<uint4 *>(y + (size_t)row * H + c0);
                    dst[0] = *reinterpret_cast<const uint4 *>(&o[0]);
                    dst[1] = *reinterpret_cast<const uint4 *>(&o[4]);
                }
            }
            if constexpr (HEAD) {
                if (row < n) {
                    const float pv = 1.f / (1.f + expf(-(dot + bo_f)));
                    if (p_out) p_out[row] = pv;
                    psum_local += pv;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok) != 0;   // also orders this tile's reads before the next tile
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("cp.async.wait_group 0;");
    if constexpr (HEAD) {
        if (psum) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) psum_local += __shfl_xor_sync(0xffffffffu, psum_local, o);
            if (lane == 0 && psum_local != 0.f) atomicAdd(psum + *cur, psum_local);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem_base));
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

// One layer backward on the tensor cores.  dz = dy * (y > 0) is rounded to bfloat16 and
// both products take bfloat16 operands with float32 accumulation:
//   input gradients   [dah | dam] = dz W^T      (rows x 2F, float32 out; skipped for layer 1)
//   weight gradients  [gWs ; gWn] += [h | m]^T dz   (2F x 64, accumulated in registers)
//   bias gradient     gb += sum_rows dz          (float32, from the unrounded dz)
// A CTA of 8 warps walks 32-row tiles staged in shared memory: dz (row-major), the input
// tile A = [h | m] (row-major) and W = [Ws ; Wn] (2F x 64, row-major, staged once).
// Fragments for the transposed operands are packed from two bfloat16 half-words.
__device__ __forceinline__ uint32_t pack_bf16(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <int F>
__global__ void __launch_bounds__(256) k_dense_bwd(const bf16 *__restrict__ h, const bf16 *__restrict__ m,
                                                   const bf16 *__restrict__ y, const float *__restrict__ dy,
                                                   const bf16 *__restrict__ Ws, const bf16 *__restrict__ Wn,
                                                   int32_t n, float *dah, float *dam, float *grad, int l,
                                                   int input_grad) {
    constexpr int K = 2 * F;
    constexpr int RT = 32;            // rows per tile
    constexpr int WP = H + 8;         // padded row of W and dz (bank spread)
    constexpr int AP = K + 8;         // padded row of the input tile
    constexpr int WT = K / 16 * 8;    // weight-gradient (16 x 8) tiles
    constexpr int WPW = (WT + 7) / 8; // of them per warp
    __shared__ __align__(16) bf16 Wsm[K * WP];
    __shared__ __align__(16) bf16 Zs[RT * WP];
    __shared__ __align__(16) bf16 As[RT * AP];
    __shared__ float s_b[8][H];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    for (int i = threadIdx.x; i < K * H; i += blockDim.x) {
        const int k = i / H, c = i % H;
        Wsm[k * WP + c] = k < F ? Ws[k * H + c] : Wn[(k - F) * H + c];
    }
    float wacc[WPW][4];
#pragma unroll
    for (int j = 0; j < WPW; ++j) wacc[j][0] = wacc[j][1] = wacc[j][2] = wacc[j][3] = 0.f;
    float gb0 = 0.f, gb1 = 0.f;       // bias columns 2 lane, 2 lane + 1
    for (int64_t r0 = (int64_t)blockIdx.x * RT; r0 < n; r0 += (int64_t)gridDim.x * RT) {
        __syncthreads();              // previous tile's readers are done (and W is staged)
        // dz tile: each thread always handles column pair `lane`
        for (int rr = warp; rr < RT; rr += 8) {
            const int64_t r = r0 + rr;
            float2 d = make_float2(0.f, 0.f);
            if (r < n) {
                const float2 v = reinterpret_cast<const float2 *>(dy + (size_t)r * H)[lane];
                const bf162 yy = reinterpret_cast<const bf162 *>(y + (size_t)r * H)[lane];
                d.x = __bfloat162float(yy.x) > 0.f ? v.x : 0.f;
                d.y = __bfloat162float(yy.y) > 0.f ? v.y : 0.f;
            }
            gb0 += d.x;
            gb1 += d.y;
            *reinterpret_cast<bf162 *>(Zs + rr * WP + 2 * lane) = __floats2bfloat162_rn(d.x, d.y);
        }
        for (int i = threadIdx.x; i < RT * (K / 2); i += blockDim.x) {
            const int rr = i / (K / 2), k = 2 * (i % (K / 2));
            const int64_t r = r0 + rr;
            bf162 v = __floats2bfloat162_rn(0.f, 0.f);
            if (r < n)
                v = k < F ? reinterpret_cast<const bf162 *>(h + (size_t)r * F + k)[0]
                          : reinterpret_cast<const bf162 *>(m + (size_t)r * F + (k - F))[0];
            *reinterpret_cast<bf162 *>(As + rr * AP + k) = v;
        }
        __syncthreads();
        // input gradients: (16-row m-tile, 8-column n-tile) pairs over the warps
        if (input_grad) {
            for (int t = warp; t < 2 * (K / 8); t += 8) {
                const int mt = t & 1, nt = t >> 1;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int ks = 0; ks < H / 16; ++ks) {
                    const int c0 = ks * 16 + 2 * tg;
                    const bf16 *z0 = Zs + (mt * 16 + g) * WP, *z1 = z0 + 8 * WP;
                    uint32_t a[4];
                    a[0] = ld_b32(z0 + c0);
                    a[1] = ld_b32(z1 + c0);
                    a[2] = ld_b32(z0 + c0 + 8);
                    a[3] = ld_b32(z1 + c0 + 8);
                    const bf16 *w = Wsm + (nt * 8 + g) * WP;
                    mma_bf16(acc, a, ld_b32(w + c0), ld_b32(w + c0 + 8));
                }
                const int k = nt * 8 + 2 * tg;
                const int64_t ra = r0 + mt * 16 + g, rb = ra + 8;
                float *dst = k < F ? dah : dam;
                const int kk = k < F ? k : k - F;
                if (ra < n) *reinterpret_cast<float2 *>(dst + (size_t)ra * F + kk) = make_float2(acc[0], acc[1]);
                if (rb < n) *reinterpret_cast<float2 *>(dst + (size_t)rb * F + kk) = make_float2(acc[2], acc[3]);
            }
        }
        // weight gradients: A^T (K x RT) times dz (RT x 64), reduction over the tile's rows
#pragma unroll
        for (int j = 0; j < WPW; ++j) {
            const int t = warp + 8 * j;
            if (t < WT) {
                const int mt = t >> 3, nt = t & 7;
                const int ka = mt * 16 + g, cb = nt * 8 + g;
#pragma unroll
                for (int ks = 0; ks < RT / 16; ++ks) {
                    const int rA = ks * 16 + 2 * tg;
                    uint32_t a[4];
                    a[0] = pack_bf16(As[rA * AP + ka], As[(rA + 1) * AP + ka]);
                    a[1] = pack_bf16(As[rA * AP + ka + 8], As[(rA + 1) * AP + ka + 8]);
                    a[2] = pack_bf16(As[(rA + 8) * AP + ka], As[(rA + 9) * AP + ka]);
                    a[3] = pack_bf16(As[(rA + 8) * AP + ka + 8], As[(rA + 9) * AP + ka + 8]);
                    const uint32_t b0 = pack_bf16(Zs[rA * WP + cb], Zs[(rA + 1) * WP + cb]);
                    const uint32_t b1 = pack_bf16(Zs[(rA + 8) * WP + cb], Zs[(rA + 9) * WP + cb]);
                    mma_bf16(wacc[j], a, b0, b1);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < WPW; ++j) {
        const int t = warp + 8 * j;
        if (t < WT) {
            const int mt = t >> 3, nt = t & 7;
            const int c = nt * 8 + 2 * tg;
            const int ka = mt * 16 + g, kb = ka + 8;
            float *ga = grad + (ka < F ? off_ws(l) + ka * H : off_wn(l) + (ka - F) * H) + c;
            float *gbp = grad + (kb < F ? off_ws(l) + kb * H : off_wn(l) + (kb - F) * H) + c;
            atomicAdd(ga, wacc[j][0]);
            atomicAdd(ga + 1, wacc[j][1]);
            atomicAdd(gbp, wacc[j][2]);
            atomicAdd(gbp + 1, wacc[j][3]);
        }
    }
    s_b[warp][2 * lane] = gb0;
    s_b[warp][2 * lane + 1] = gb1;
    __syncthreads();
    if (threadIdx.x < H) {
        float sb = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) sb += s_b[w][threadIdx.x];
        atomicAdd(grad + off_b(l) + threadIdx.x, sb);
    }
}

// dh_u = dah_u + sum over out-arcs u -> v of dam_v / d_in(v)   (adjoint of the mean).
// One thread per (item, feature); items as in k_agg but over the out-CSR: long out-rows
// are skipped here and finished by k_agg_bwd_fin from the chunks' partial sums.
template <int F>
__global__ void k_agg_bwd(const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_dst,
                          const float *__restrict__ inv_din, int32_t n, const float *__restrict__ dah,
                          const float *__restrict__ dam, float *dh, const int4 *__restrict__ items,
                          int32_t n_items, float *acc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = ((int64_t)n + n_items) * F;
    for (int64_t i = t; i < total; i += nthreads) {
        const int64_t v = i / F;
        const int j = (int)(i % F);
        int32_t u, b, e, slot = -1;
        if (v < n) {
            u = (int32_t)v;
            b = out_ptr[v];
            e = out_ptr[v + 1];
            if (e - b >= kSgLong) continue;
        } else {
            const int4 it = items[v - n];
            u = it.x, b = it.y, e = it.z, slot = it.w;
        }
        float s = 0.f;
#pragma unroll 4
        for (int32_t a = b; a < e; ++a) {
            const int32_t w = __ldg(out_dst + a);
            s += dam[(size_t)w * F + j] * __ldg(inv_din + w);
        }
        if (slot < 0) dh[(size_t)u * F + j] = dah[(size_t)u * F + j] + s;
        else atomicAdd(acc + (size_t)slot * F + j, s);
    }
}

template <int F>
__global__ void k_agg_bwd_fin(const int32_t *__restrict__ long_rows, int32_t n_long, const float *__restrict__ dah,
                              float *acc, float *dh) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n_long * F;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = i / F;
        const int j = (int)(i % F);
        const size_t o = (size_t)long_rows[slot] * F + j;
        dh[o] = dah[o] + acc[i];
        acc[i] = 0.f;
    }
}

// Per-graph tables: 1 / d_in and the long rows of a CSR.
__global__ void k_inv_deg(const int32_t *__restrict__ row_ptr, int32_t n, float *inv) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = row_ptr[v + 1] - row_ptr[v];
        inv[v] = d > 0 ? 1.f / (float)d : 0.f;
    }
}

__global__ void k_long_rows(const int32_t *__restrict__ ptr, int32_t n, int32_t cap, int4 *out, int32_t *count) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = ptr[v], e = ptr[v + 1];
        if (e - b >= kSgLong) {
            const int32_t i = atomicAdd(count, 1);
            if (i < cap) out[i] = make_int4((int32_t)v, b, e, 0);
        }
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
    int32_t *tc_err = nullptr;  // set by a dense-layer CTA whose tensor-core wait ran out
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

// Persistent CTAs of the tensor-core dense layer: two per SM at most, one per tile at least.
int tc_grid(const fsgp_surrogate *s, int64_t n) {
    const int64_t tiles = (n + kTcRows - 1) / kTcRows;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)s->sm_count * 2));
}

// A tensor-core wait of an earlier launch ran out (the flag is sticky): FSGP_ETIMEOUT.
int sg_check_tc(fsgp_surrogate *s, cudaStream_t st) {
    int32_t h = 0;
    FSGP_CUDA(cudaMemcpyAsync(&h, s->tc_err, sizeof h, cudaMemcpyDeviceToHost, st));
    FSGP_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(FSGP_ETIMEOUT, "a tensor-core completion wait of the surrogate's dense layer ran out");
    return FSGP_OK;
}

int grid_of(const fsgp_surrogate *s, int64_t work, int threads, int per_sm = 8) {
    int64_t g = (work + threads - 1) / threads;
    g = std::min<int64_t>(g, (int64_t)s->sm_count * per_sm);
    return (int)std::max<int64_t>(g, 1);
}

// Long rows of one CSR (ptr) as chunk items and a slot -> row list (host build, once).
int sg_long_table(const int32_t *ptr, int32_t n, int64_t nnz, int sm_count, int4 **items, int32_t *n_items,
                  int32_t **long_rows, int32_t *n_long) {
    const int64_t cap = nnz / kSgLong + 1;
    int4 *d_tmp = nullptr;
    int32_t *d_cnt = nullptr;
    FSGP_CUDA(cudaMalloc(&d_tmp, sizeof(int4) * (size_t)cap));
    cudaError_t e = cudaMalloc(&d_cnt, sizeof(int32_t));
    int32_t cnt = 0;
    std::vector<int4> rows;
    if (e == cudaSuccess) e = cudaMemset(d_cnt, 0, sizeof(int32_t));
    if (e == cudaSuccess) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)sm_count * 8));
        k_long_rows<<<grid, 256>>>(ptr, n, (int32_t)cap, d_tmp, d_cnt);
        e = cudaMemcpy(&cnt, d_cnt, sizeof(int32_t), cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess && cnt > 0) {
        rows.resize((size_t)cnt);
        e = cudaMemcpy(rows.data(), d_tmp, sizeof(int4) * (size_t)cnt, cudaMemcpyDeviceToHost);
    }
    cudaFree(d_tmp);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate long rows");
    std::sort(rows.begin(), rows.end(), [](const int4 &x, const int4 &y) { return x.x < y.x; });
    std::vector<int4> it;
    std::vector<int32_t> lr;
    for (size_t sl = 0; sl < rows.size(); ++sl) {
        lr.push_back(rows[sl].x);
        for (int32_t b = rows[sl].y; b < rows[sl].z; b += kSgChunk)
            it.push_back(make_int4(rows[sl].x, b, std::min(b + kSgChunk, rows[sl].z), (int32_t)sl));
    }
    *n_items = (int32_t)it.size();
    *n_long = (int32_t)lr.size();
    if (!it.empty()) {
        FSGP_CUDA(cudaMalloc(items, sizeof(int4) * it.size()));
        FSGP_CUDA(cudaMemcpy(*items, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
        FSGP_CUDA(cudaMalloc(long_rows, sizeof(int32_t) * lr.size()));
        FSGP_CUDA(cudaMemcpy(*long_rows, lr.data(), sizeof(int32_t) * lr.size(), cudaMemcpyHostToDevice));
    }
    return FSGP_OK;
}

// Build the graph's aggregation tables on first use (synchronous; call outside captures).
int sg_cache(const fsgp_graph *gc, int sm_count) {
    fsgp_graph *g = const_cast<fsgp_graph *>(gc);   // lazily built cache of the handle
    SgCache &C = g->sgc;
    if (C.built) return FSGP_OK;
    FSGP_CUDA(cudaMalloc(&C.inv_din, sizeof(float) * (size_t)g->n));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, (int64_t)sm_count * 8));
    k_inv_deg<<<grid, 256>>>(g->row_ptr, g->n, C.inv_din);
    int rc = sg_long_table(g->row_ptr, g->n, g->nnz, sm_count, &C.in_items, &C.n_in_items, &C.in_long, &C.n_in_long);
    if (rc) return rc;
    rc = sg_long_table(g->out_ptr, g->n, g->nnz, sm_count, &C.out_items, &C.n_out_items, &C.out_long, &C.n_out_long);
    if (rc) return rc;
    const size_t nl = (size_t)std::max(C.n_in_long, C.n_out_long);
    if (nl) {
        FSGP_CUDA(cudaMalloc(&C.acc, sizeof(float) * nl * H));
        FSGP_CUDA(cudaMemset(C.acc, 0, sizeof(float) * nl * H));
    }
    FSGP_CUDA(cudaDeviceSynchronize());
    C.built = 1;
    return FSGP_OK;
}

// Forward of the three layers and the head from features s->x (already seeded).
void sg_forward(fsgp_surrogate *s, const fsgp_graph *g, float *p, float *psum, cudaStream_t st) {
    const int32_t n = g->n;
    const bf16 *W = s->wb;
    const float *B = s->theta;
    const SgCache &C = g->sgc;
    const int64_t items = (int64_t)n + C.n_in_items;
    k_agg<F0><<<grid_of(s, items * (F0 / 8) * agg_arcs<F0>(), 256), 256, 0, st>>>(g->row_ptr, g->col, n, s->x, s->m1, C.in_items,
                                                                 C.n_in_items, C.acc);
    if (C.n_in_long)
        k_agg_fin<F0><<<grid_of(s, (int64_t)C.n_in_long * (F0 / 2), 256), 256, 0, st>>>(C.in_long, C.n_in_long,
                                                                                     g->row_ptr, C.acc, s->m1);
    k_dense_tc<F0, false><<<tc_grid(s, n), 128, tc_smem_bytes<F0>(), st>>>(
        s->x, s->m1, W + OFF_WS1, W + OFF_WN1, B + OFF_B1, n, s->h1, nullptr, nullptr, nullptr, nullptr, nullptr,
        s->tc_err);
    k_agg<H><<<grid_of(s, items * (H / 8) * agg_arcs<H>(), 256), 256, 0, st>>>(g->row_ptr, g->col, n, s->h1, s->m2, C.in_items,
                                                              C.n_in_items, C.acc);
    if (C.n_in_long)
        k_agg_fin<H><<<grid_of(s, (int64_t)C.n_in_long * (H / 2), 256), 256, 0, st>>>(C.in_long, C.n_in_long,
                                                                                   g->row_ptr, C.acc, s->m2);
    k_dense_tc<H, false><<<tc_grid(s, n), 128, tc_smem_bytes<H>(), st>>>(
        s->h1, s->m2, W + OFF_WS2, W + OFF_WN2, B + OFF_B2, n, s->h2, nullptr, nullptr, nullptr, nullptr, nullptr,
        s->tc_err);
    k_agg<H><<<grid_of(s, items * (H / 8) * agg_arcs<H>(), 256), 256, 0, st>>>(g->row_ptr, g->col, n, s->h2, s->m3, C.in_items,
                                                              C.n_in_items, C.acc);
    if (C.n_in_long)
        k_agg_fin<H><<<grid_of(s, (int64_t)C.n_in_long * (H / 2), 256), 256, 0, st>>>(C.in_long, C.n_in_long,
                                                                                   g->row_ptr, C.acc, s->m3);
    // layer 3 with the head in its epilogue; h3 is kept only when p is (the backward
    // pass reads both)
    k_dense_tc<H, true><<<tc_grid(s, n), 128, tc_smem_bytes<H>(), st>>>(
        s->h2, s->m3, W + OFF_WS3, W + OFF_WN3, B + OFF_B3, n, p ? s->h3 : nullptr, W + OFF_WO, B + OFF_BO, p, psum,
        s->cur, s->tc_err);
}

int sg_prepare_inputs(fsgp_surrogate *s, const fsgp_graph *g, const int32_t *seeds_host, int64_t ns,
                      double beta, double gamma, cudaStream_t st) {
    for (int64_t i = 0; i < ns; ++i)
        if (seeds_host[i] < 0 || seeds_host[i] >= g->n) return fail(FSGP_EINVAL, "seed node out of range");
    int rc = sg_ensure(s, g->n);
    if (rc) return rc;
    rc = sg_cache(g, s->sm_count);
    if (rc) return rc;
    k_features<<<grid_of(s, g->n, 256), 256, 0, st>>>(g->row_ptr, g->out_ptr, g->n, (float)beta, (float)gamma, s->x);
    if (ns > 0) {
        // seed bits: small host list staged through the activation buffer y (floats)
        int32_t *d_seeds = reinterpret_cast<int32_t *>(s->y);
        if (ns > s->cap) return fail(FSGP_EINVAL, "more seeds than nodes");
        FSGP_CUDA(cudaMemcpyAsync(d_seeds, seeds_host, sizeof(int32_t) * (size_t)ns, cudaMemcpyHostToDevice, st));
        FSGP_CUDA(cudaMemsetAsync(s->cur, 0, sizeof(int32_t), st));
        k_seed_bits<<<1, 256, 0, st>>>(d_seeds, (int32_t)ns, s->cur, 1.f, 0, s->x);
        const int gk = (int)std::min<int64_t>(ns, 1024);
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
    const int gb = grid_of(s, ((int64_t)n + 31) / 32, 1, 2);
    // layer 3: dy = dh (float), outputs dh2 = d h2
    k_dense_bwd<H><<<gb, 256, 0, st>>>(s->h2, s->m3, s->h3, s->dh, W + OFF_WS3, W + OFF_WN3, n, s->dah, s->dam, s->grad, 3, 1);
    const SgCache &C = g->sgc;
    const int64_t items = (int64_t)n + C.n_out_items;
    k_agg_bwd<H><<<grid_of(s, items * H, 256), 256, 0, st>>>(g->out_ptr, g->out_dst, C.inv_din, n, s->dah, s->dam,
                                                            s->dh2, C.out_items, C.n_out_items, C.acc);
    if (C.n_out_long)
        k_agg_bwd_fin<H><<<grid_of(s, (int64_t)C.n_out_long * H, 256), 256, 0, st>>>(C.out_long, C.n_out_long,
                                                                                  s->dah, C.acc, s->dh2);
    // layer 2
    k_dense_bwd<H><<<gb, 256, 0, st>>>(s->h1, s->m2, s->h2, s->dh2, W + OFF_WS2, W + OFF_WN2, n, s->dah, s->dam, s->grad, 2, 1);
    k_agg_bwd<H><<<grid_of(s, items * H, 256), 256, 0, st>>>(g->out_ptr, g->out_dst, C.inv_din, n, s->dah, s->dam,
                                                            s->dh, C.out_items, C.n_out_items, C.acc);
    if (C.n_out_long)
        k_agg_bwd_fin<H><<<grid_of(s, (int64_t)C.n_out_long * H, 256), 256, 0, st>>>(C.out_long, C.n_out_long,
                                                                                  s->dah, C.acc, s->dh);
    // layer 1 (input gradients not needed beyond the weights)
    k_dense_bwd<F0><<<gb, 256, 0, st>>>(s->x, s->m1, s->h1, s->dh, W + OFF_WS1, W + OFF_WN1, n, s->dah, s->dam, s->grad, 1, 0);
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
        (e = cudaMalloc(&s->cur, sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc(&s->tc_err, sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemset(s->tc_err, 0, sizeof(int32_t))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_dense_tc<F0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem_bytes<F0>())) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_dense_tc<H, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem_bytes<H>())) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_dense_tc<H, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem_bytes<H>())) != cudaSuccess) {
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
    cudaFree(s->tc_err);
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
    return sg_check_tc(s, st);
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
    rc = sg_cache(g, s->sm_count);
    if (rc) return rc;
    // captures are not allowed on the legacy default stream: work on a private stream
    // ordered after the caller's work
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    int32_t *d_cand = nullptr;
    float *d_scores = nullptr;
    cudaError_t e;
    rc = FSGP_OK;
    do {
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventRecord(ev, caller)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, ev, 0)) != cudaSuccess ||
            (e = cudaMalloc(&d_cand, sizeof(int32_t) * (size_t)k * n_cand)) != cudaSuccess ||
            (e = cudaMalloc(&d_scores, sizeof(float) * (size_t)n_cand)) != cudaSuccess) {
            rc = cuda_fail(e, "screen setup");
            break;
        }
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
        const int gk = std::min<int32_t>(k, 1024);
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
        else rc = sg_check_tc(s, st);
    } while (0);
    cudaFree(d_cand);
    cudaFree(d_scores);
    if (ev) cudaEventDestroy(ev);
    if (st) cudaStreamDestroy(st);
    return rc;
}
