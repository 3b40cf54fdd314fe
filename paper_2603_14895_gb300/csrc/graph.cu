// graph.cu -- graph handle: device copy of the in-CSR (CSR definition, Sec. 2), input
// validation, the out-CSR used by the frontier path, and the degree buckets used to
// schedule rows.  Also the thread-local error plumbing of the C ABI.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fsgp_internal.cuh"

namespace fsgp {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) {
    g_last_error = msg;
    if (msg.empty()) (void)cudaGetLastError();   // entry of an API call: drop stale errors
}

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FSGP_ENOMEM : FSGP_ECUDA;
}

// ------------------------------------------------------------------------ kernels

__device__ __forceinline__ int degree_bucket(int32_t d) {
    return d <= 0 ? 0 : 32 - __clz(d);   // d in [2^(b-1), 2^b) -> b
}

// Checks row_ptr[0] = 0, monotone, row_ptr[n] = nnz; records the max in-degree and the
// degree-bucket histogram.
__global__ void k_check_rows(const int32_t *__restrict__ row_ptr, int32_t n, int64_t nnz,
                             int32_t *err, int32_t *max_deg, int32_t *bucket_hist) {
    __shared__ int32_t hist[33];
    for (int i = threadIdx.x; i < 33; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    int32_t local_max = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = row_ptr[v], e = row_ptr[v + 1];
        if (e < b) atomicOr(err, 1);
        const int32_t d = e - b;
        local_max = max(local_max, d);
        atomicAdd(&hist[degree_bucket(d)], 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (row_ptr[0] != 0) atomicOr(err, 2);
        if ((int64_t)row_ptr[n] != nnz) atomicOr(err, 4);
    }
    atomicMax(max_deg, local_max);
    __syncthreads();
    for (int i = threadIdx.x; i < 33; i += blockDim.x)
        if (hist[i]) atomicAdd(&bucket_hist[i], hist[i]);
}

// Column range check and out-degree histogram.
__global__ void k_check_cols(const int32_t *__restrict__ col, int64_t nnz, int32_t n,
                             int32_t *err, int32_t *out_cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = col[e];
        if (u < 0 || u >= n) {
            atomicOr(err, 8);
        } else {
            atomicAdd(&out_cnt[u], 1);
        }
    }
}

// Three-phase exclusive scan of int32 counts into int32 offsets (total < 2^31).
constexpr int kScanItems = 4;
constexpr int kScanThreads = 512;
constexpr int kScanTile = kScanItems * kScanThreads;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t *total) {
    __shared__ int64_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int64_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const int64_t warp_off = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + incl - x;
}

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int64_t n, int64_t *tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    int64_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int64_t *tile_sums, int64_t n_tiles) {
    // one CTA: sequential over chunks of blockDim.x
    int64_t carry = 0;
    for (int64_t b = 0; b < n_tiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int64_t x = i < n_tiles ? tile_sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(x, &total);
        if (i < n_tiles) tile_sums[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const int32_t *__restrict__ in, int64_t n,
                             const int64_t *__restrict__ tile_off, int32_t *out) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int64_t total;
    int64_t off = block_exclusive_scan(s, &total) + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = (int32_t)off;
        off += v[i];
    }
}

// Out-CSR scatter: one warp per target row.
__global__ void k_out_scatter(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                              int32_t n, const int32_t *__restrict__ out_ptr, int32_t *cursor,
                              int32_t *out_dst) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += n_warps) {
        const int32_t b = row_ptr[v], e = row_ptr[v + 1];
        for (int32_t k = b + lane; k < e; k += 32) {
            const int32_t u = col[k];
            const int32_t pos = atomicAdd(&cursor[u], 1);
            out_dst[out_ptr[u] + pos] = (int32_t)v;
        }
    }
}

__global__ void k_max_out(const int32_t *__restrict__ cnt, int32_t n, int32_t *mx) {
    int32_t m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        m = max(m, cnt[v]);
    atomicMax(mx, m);
}

// Rows grouped by degree bucket, highest bucket first, and in node order inside a bucket
// (stable counting sort; node order keeps the state words of a warp's rows close).
// Phase 1: one warp per chunk of kChunkRows rows counts its rows per bucket, written
// bucket-major (bucket 32 first) so that one exclusive scan gives every chunk's offsets.
constexpr int kChunkRows = 1024;

__global__ void k_bucket_chunk_hist(const int32_t *__restrict__ row_ptr, int32_t n,
                                    int64_t n_chunks, int32_t *hist /*[33][n_chunks]*/) {
    __shared__ int32_t cnt[8][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t chunk = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    for (int b = lane; b < 33; b += 32) cnt[wid][b] = 0;
    __syncwarp();
    if (chunk < n_chunks) {
        const int64_t v0 = chunk * kChunkRows;
        for (int64_t v = v0 + lane; v < min((int64_t)n, v0 + kChunkRows); v += 32)
            atomicAdd(&cnt[wid][degree_bucket(row_ptr[v + 1] - row_ptr[v])], 1);
    }
    __syncwarp();
    if (chunk < n_chunks)
        for (int b = lane; b < 33; b += 32) hist[(size_t)(32 - b) * n_chunks + chunk] = cnt[wid][b];
}

// Phase 2: the same warps place their rows in order at the scanned offsets.
__global__ void k_bucket_chunk_scatter(const int32_t *__restrict__ row_ptr, int32_t n,
                                       int64_t n_chunks, const int32_t *__restrict__ off,
                                       int32_t *rows_sorted) {
    __shared__ int32_t run[8][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t chunk = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (chunk >= n_chunks) return;
    for (int b = lane; b < 33; b += 32) run[wid][b] = off[(size_t)(32 - b) * n_chunks + chunk];
    __syncwarp();
    const int64_t v0 = chunk * kChunkRows;
    const int64_t v1 = min((int64_t)n, v0 + kChunkRows);
    for (int64_t base = v0; base < v1; base += 32) {
        const int64_t v = base + lane;
        const bool has = v < v1;
        const int b = has ? degree_bucket(row_ptr[v + 1] - row_ptr[v]) : 33 + lane;
        const unsigned same = __match_any_sync(0xffffffffu, b);
        const int rank = __popc(same & ((1u << lane) - 1u));
        int32_t pos = 0;
        if (has) pos = run[wid][b] + rank;
        __syncwarp();
        if (has && rank == 0) run[wid][b] += __popc(same);
        __syncwarp();
        if (has) rows_sorted[pos] = (int32_t)v;
    }
}

static int grid_for(int64_t work, int threads, int sm_count) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

int exclusive_scan_i32(const int32_t *in, int64_t n, int32_t *out, int64_t *tile_tmp,
                       cudaStream_t s) {
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) return FSGP_OK;
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, tile_tmp);
    k_scan_sums<<<1, 1024, 0, s>>>(tile_tmp, tiles);
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, tile_tmp, out);
    FSGP_CUDA(cudaGetLastError());
    return FSGP_OK;
}

// Relabelling (new id i = position of node rows_sorted[i]): inverse map, per-row in-degree
// in new order (scanned into rp2 afterwards) and the original position of each row's first
// arc.
__global__ void k_relabel_rows(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ rows,
                               int32_t n, int32_t *pos, int32_t *deg2, int32_t *arc0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = rows[i];
        pos[v] = (int32_t)i;
        const int32_t b = row_ptr[v];
        deg2[i] = row_ptr[v + 1] - b;
        arc0[i] = b;
    }
}

// Sources as new ids, rows in new order (one warp per row; rows of a warp's neighbourhood
// have similar degrees because new ids follow the degree buckets).
__global__ void k_relabel_cols(const int32_t *__restrict__ arc0, const int32_t *__restrict__ rp2,
                               const int32_t *__restrict__ col, const int32_t *__restrict__ pos,
                               int32_t n, int32_t *col2) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += n_warps) {
        const int32_t b = arc0[i], o = rp2[i], d = rp2[i + 1] - o;
        for (int32_t k = lane; k < d; k += 32) col2[o + k] = pos[col[b + k]];
    }
}

// New rows with 1..3 in-arcs: the node and its (up to 3) sources in one 16-byte entry.
__global__ void k_lane_tab(const int32_t *__restrict__ rp2, const int32_t *__restrict__ col2,
                           const int32_t *__restrict__ rows, int32_t first, int32_t count, int4 *tab) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = first + r;
        const int32_t b = rp2[i], d = rp2[i + 1] - b;
        tab[r] = make_int4(rows[i], d > 0 ? col2[b] : -1, d > 1 ? col2[b + 1] : -1, d > 2 ? col2[b + 2] : -1);
    }
}

static void release(fsgp_graph *g) {
    if (!g) return;
    drop_exec_cache(g);
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->out_ptr);
    cudaFree(g->out_dst);
    cudaFree(g->rows_sorted);
    cudaFree(g->pos);
    cudaFree(g->rp2);
    cudaFree(g->col2);
    cudaFree(g->arc0);
    cudaFree(g->lane_tab);
    cudaFree(g->arc_w);
    cudaFree(g->hub.d_chunk_base);
    cudaFree(g->ws.ptr);
    cudaFree(g->sgc.inv_din);
    cudaFree(g->sgc.in_items);
    cudaFree(g->sgc.in_long);
    cudaFree(g->sgc.out_items);
    cudaFree(g->sgc.out_long);
    cudaFree(g->sgc.acc);
    delete g;
}

}  // namespace fsgp

using namespace fsgp;

extern "C" const char *fsgp_last_error(void) { return g_last_error.c_str(); }

extern "C" int fsgp_version(void) { return 10000; }

extern "C" int fsgp_model_planes(int32_t model) {
    switch (model) {
        case FSGP_SIR: return 2;
        case FSGP_SIS: return 1;
        case FSGP_IC: return 2;
        case FSGP_LT: return 2;
        case FSGP_SI: return 1;
        case FSGP_SEIR: return 3;
        case FSGP_SEIS: return 2;
        case FSGP_SWIR: return 3;
        default: return fail(FSGP_EINVAL, "unknown model");
    }
}

extern "C" int fsgp_model_compartments(int32_t model) {
    if (model < FSGP_SIR || model > FSGP_SWIR) return fail(FSGP_EINVAL, "unknown model");
    return (model == FSGP_SEIR || model == FSGP_SWIR) ? 4 : 3;
}

extern "C" int fsgp_graph_create(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                                 int64_t nnz, uint32_t flags, void *stream, fsgp_graph **out) {
    set_error("");
    if (!out) return fail(FSGP_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n >= INT32_MAX) return fail(FSGP_EINVAL, "n out of range");
    if (nnz < 0 || nnz >= (int64_t)INT32_MAX) return fail(FSGP_EINVAL, "nnz out of range");
    if (!row_ptr || (nnz > 0 && !col_idx)) return fail(FSGP_EINVAL, "NULL CSR array");
    if (flags != FSGP_PTR_HOST && flags != FSGP_PTR_DEVICE) return fail(FSGP_EINVAL, "bad flags");
    cudaStream_t s = (cudaStream_t)stream;
    fsgp_graph *g = new (std::nothrow) fsgp_graph();
    if (!g) return fail(FSGP_ENOMEM, "host allocation failed");
    int rc = FSGP_OK;
    int32_t *d_tmp = nullptr;     // err, max_deg, max_out, bucket hist[33], cursor[33]
    int32_t *d_cnt = nullptr;     // out-degree counts / cursors
    int64_t *d_tiles = nullptr;
    do {
        cudaError_t e;
        if ((e = cudaGetDevice(&g->device)) != cudaSuccess) { rc = cuda_fail(e, "cudaGetDevice"); break; }
        if ((e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess) {
            rc = cuda_fail(e, "cudaDeviceGetAttribute");
            break;
        }
        g->n = n;
        g->nnz = nnz;
        const size_t rp_bytes = sizeof(int32_t) * ((size_t)n + 1);
        const size_t col_bytes = sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1);
        if ((e = cudaMalloc(&g->row_ptr, rp_bytes)) != cudaSuccess ||
            (e = cudaMalloc(&g->col, col_bytes)) != cudaSuccess ||
            (e = cudaMalloc(&g->out_ptr, rp_bytes)) != cudaSuccess ||
            (e = cudaMalloc(&g->out_dst, col_bytes)) != cudaSuccess ||
            (e = cudaMalloc(&g->rows_sorted, sizeof(int32_t) * (size_t)n)) != cudaSuccess ||
            (e = cudaMalloc(&d_tmp, sizeof(int32_t) * 72)) != cudaSuccess ||
            (e = cudaMalloc(&d_cnt, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMalloc (graph)");
            break;
        }
        g->device_bytes = 2 * rp_bytes + 2 * col_bytes + sizeof(int32_t) * (size_t)n;
        const int64_t tiles = ((int64_t)n + 1 + kScanTile - 1) / kScanTile;
        if ((e = cudaMalloc(&d_tiles, sizeof(int64_t) * (size_t)(tiles + 1))) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMalloc (scan)");
            break;
        }
        const cudaMemcpyKind kind = flags == FSGP_PTR_DEVICE ? cudaMemcpyDeviceToDevice
                                                             : cudaMemcpyHostToDevice;
        if ((e = cudaMemcpyAsync(g->row_ptr, row_ptr, rp_bytes, kind, s)) != cudaSuccess ||
            (nnz > 0 && (e = cudaMemcpyAsync(g->col, col_idx, sizeof(int32_t) * (size_t)nnz, kind, s)) != cudaSuccess) ||
            (e = cudaMemsetAsync(d_tmp, 0, sizeof(int32_t) * 72, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * ((size_t)n + 1), s)) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMemcpyAsync (graph)");
            break;
        }
        int32_t *d_err = d_tmp, *d_maxdeg = d_tmp + 1, *d_maxout = d_tmp + 2;
        int32_t *d_hist = d_tmp + 3;
        k_check_rows<<<grid_for(n, 256, g->sm_count), 256, 0, s>>>(g->row_ptr, n, nnz, d_err, d_maxdeg, d_hist);
        int32_t h_head[3];
        if ((e = cudaMemcpyAsync(h_head, d_tmp, sizeof h_head, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            rc = cuda_fail(e, "row check");
            break;
        }
        if (h_head[0]) {
            rc = fail(FSGP_EINVAL, "malformed row_ptr (must start at 0, be non-decreasing and end at nnz)");
            break;
        }
        if (nnz > 0)
            k_check_cols<<<grid_for(nnz, 256, g->sm_count), 256, 0, s>>>(g->col, nnz, n, d_err, d_cnt);
        if ((e = cudaMemcpyAsync(h_head, d_tmp, sizeof h_head, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            rc = cuda_fail(e, "column check");
            break;
        }
        if (h_head[0]) {
            rc = fail(FSGP_EINVAL, "column index out of range [0, n)");
            break;
        }
        g->max_deg = h_head[1];
        // out-CSR: counts -> offsets (n+1 entries; d_cnt[n] = 0 gives out_ptr[n] = nnz)
        if ((rc = exclusive_scan_i32(d_cnt, (int64_t)n + 1, g->out_ptr, d_tiles, s)) != FSGP_OK) break;
        k_max_out<<<grid_for(n, 256, g->sm_count), 256, 0, s>>>(d_cnt, n, d_maxout);
        if ((e = cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * ((size_t)n + 1), s)) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMemsetAsync");
            break;
        }
        if (nnz > 0)
            k_out_scatter<<<grid_for((int64_t)n * 32, 256, g->sm_count), 256, 0, s>>>(
                g->row_ptr, g->col, n, g->out_ptr, d_cnt, g->out_dst);
        // degree buckets, descending
        int32_t hist[33];
        if ((e = cudaMemcpyAsync(hist, d_hist, sizeof hist, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(h_head, d_tmp, sizeof h_head, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            rc = cuda_fail(e, "bucket histogram");
            break;
        }
        g->max_out_deg = h_head[2];
        int32_t start[34];
        int32_t acc = 0;
        for (int b = 32; b >= 0; --b) {
            start[b] = acc;
            acc += hist[b];
        }
        start[33] = 0;
        for (int b = 0; b < 33; ++b) {
            g->cls.bucket_count[b] = hist[b];
            g->cls.bucket_start[b] = start[b];
        }
        g->cls.bucket_start[33] = n;
        {
            // stable bucket order: per-chunk histograms, one scan, ordered placement
            const int64_t n_chunks = ((int64_t)n + kChunkRows - 1) / kChunkRows;
            const int64_t hn = 33 * n_chunks;
            int32_t *d_hist = nullptr, *d_off = nullptr;
            int64_t *d_t2 = nullptr;
            const int64_t t2 = (hn + kScanTile - 1) / kScanTile + 1;
            if ((e = cudaMalloc(&d_hist, sizeof(int32_t) * (size_t)hn)) != cudaSuccess ||
                (e = cudaMalloc(&d_off, sizeof(int32_t) * (size_t)hn)) != cudaSuccess ||
                (e = cudaMalloc(&d_t2, sizeof(int64_t) * (size_t)t2)) != cudaSuccess) {
                cudaFree(d_hist);
                cudaFree(d_off);
                rc = cuda_fail(e, "cudaMalloc (bucket sort)");
                break;
            }
            const unsigned blocks = (unsigned)((n_chunks + 7) / 8);
            k_bucket_chunk_hist<<<blocks, 256, 0, s>>>(g->row_ptr, n, n_chunks, d_hist);
            rc = exclusive_scan_i32(d_hist, hn, d_off, d_t2, s);
            if (rc == FSGP_OK)
                k_bucket_chunk_scatter<<<blocks, 256, 0, s>>>(g->row_ptr, n, n_chunks, d_off, g->rows_sorted);
            e = cudaStreamSynchronize(s);
            cudaFree(d_hist);
            cudaFree(d_off);
            cudaFree(d_t2);
            if (rc != FSGP_OK) break;
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "bucket sort");
                break;
            }
        }
        // relabelled in-CSR (new ids in rows_sorted order) and the table of rows with 1..3
        // in-arcs
        g->lane_start = g->cls.bucket_start[2];
        g->d0_start = g->cls.bucket_start[0];
        const int32_t n_lane = g->d0_start - g->lane_start;
        if ((e = cudaMalloc(&g->pos, sizeof(int32_t) * (size_t)n)) != cudaSuccess ||
            (e = cudaMalloc(&g->rp2, rp_bytes)) != cudaSuccess ||
            (e = cudaMalloc(&g->col2, col_bytes)) != cudaSuccess ||
            (e = cudaMalloc(&g->arc0, sizeof(int32_t) * (size_t)n)) != cudaSuccess ||
            (n_lane > 0 && (e = cudaMalloc(&g->lane_tab, sizeof(int4) * (size_t)n_lane)) != cudaSuccess)) {
            rc = cuda_fail(e, "cudaMalloc (relabelled graph)");
            break;
        }
        g->device_bytes += 2 * sizeof(int32_t) * (size_t)n + rp_bytes + col_bytes + sizeof(int4) * (size_t)n_lane;
        // d_cnt (n+1 entries) holds the degrees in new order; entry n = 0 ends the scan
        if ((e = cudaMemsetAsync(d_cnt + n, 0, sizeof(int32_t), s)) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMemsetAsync");
            break;
        }
        k_relabel_rows<<<grid_for(n, 256, g->sm_count), 256, 0, s>>>(g->row_ptr, g->rows_sorted, n, g->pos,
                                                                     d_cnt, g->arc0);
        if ((rc = exclusive_scan_i32(d_cnt, (int64_t)n + 1, g->rp2, d_tiles, s)) != FSGP_OK) break;
        if (nnz > 0)
            k_relabel_cols<<<grid_for((int64_t)n * 32, 256, g->sm_count), 256, 0, s>>>(g->arc0, g->rp2, g->col,
                                                                                      g->pos, n, g->col2);
        if (n_lane > 0)
            k_lane_tab<<<grid_for(n_lane, 256, g->sm_count), 256, 0, s>>>(g->rp2, g->col2, g->rows_sorted,
                                                                          g->lane_start, n_lane, g->lane_tab);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            rc = cuda_fail(e, "graph build kernels");
            break;
        }
    } while (0);
    cudaFree(d_tmp);
    cudaFree(d_cnt);
    cudaFree(d_tiles);
    if (rc != FSGP_OK) {
        release(g);
        return rc;
    }
    *out = g;
    return FSGP_OK;
}

extern "C" int fsgp_graph_destroy(fsgp_graph *g) {
    set_error("");
    if (!g) return FSGP_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    release(g);
    cudaSetDevice(dev);
    return FSGP_OK;
}

// Weights of a device array: flag a negative, NaN or infinite one.
__global__ void k_check_weights(const float *w, int64_t n, int32_t *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = w[i];
        if (!(x >= 0.0f) || isinf(x)) atomicExch(bad, 1);
    }
}

extern "C" int fsgp_graph_set_arc_weights(fsgp_graph *g, const float *w, uint32_t flags, void *stream) {
    set_error("");
    if (!g) return fail(FSGP_EINVAL, "graph is NULL");
    if (flags != FSGP_PTR_HOST && flags != FSGP_PTR_DEVICE) return fail(FSGP_EINVAL, "bad weight flags");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    FSGP_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(FSGP_EINVAL, "current device differs from the graph's device");
    if (!w) {   // detach
        FSGP_CUDA(cudaStreamSynchronize(s));
        drop_exec_cache(g);
        cudaFree(g->arc_w);
        g->arc_w = nullptr;
        return FSGP_OK;
    }
    const int64_t m = g->nnz;
    if (flags == FSGP_PTR_HOST) {
        for (int64_t i = 0; i < m; ++i)
            if (!(w[i] >= 0.0f) || std::isinf(w[i])) return fail(FSGP_EINVAL, "arc weights must be finite and >= 0");
    } else if (m > 0) {
        int32_t *d_bad = nullptr, bad = 0;
        FSGP_CUDA(cudaMalloc(&d_bad, sizeof(int32_t)));
        cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(int32_t), s);
        if (e == cudaSuccess) {
            const int grid = (int)std::min<int64_t>((m + 255) / 256, (int64_t)g->sm_count * 8);
            k_check_weights<<<grid, 256, 0, s>>>(w, m, d_bad);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_bad);
        if (e != cudaSuccess) return cuda_fail(e, "arc weight check");
        if (bad) return fail(FSGP_EINVAL, "arc weights must be finite and >= 0");
    }
    if (!g->arc_w) {
        float *d = nullptr;
        if (cudaMalloc(&d, sizeof(float) * (size_t)std::max<int64_t>(m, 1)) != cudaSuccess) {
            cudaGetLastError();
            return fail(FSGP_ENOMEM, "device allocation of the arc weights failed");
        }
        g->arc_w = d;
    }
    if (m > 0)
        FSGP_CUDA(cudaMemcpyAsync(g->arc_w, w, sizeof(float) * (size_t)m,
                                  flags == FSGP_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    FSGP_CUDA(cudaStreamSynchronize(s));
    return FSGP_OK;
}

extern "C" int fsgp_graph_trim(fsgp_graph *g) {
    set_error("");
    if (!g) return fail(FSGP_EINVAL, "graph is NULL");
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(g->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) drop_exec_cache(g);
    if (e == cudaSuccess && g->ws.ptr) e = cudaFree(g->ws.ptr);
    if (e == cudaSuccess) {
        g->ws.ptr = nullptr;
        g->ws.bytes = 0;
    }
    cudaSetDevice(dev);
    return e == cudaSuccess ? FSGP_OK : cuda_fail(e, "fsgp_graph_trim");
}

extern "C" int fsgp_graph_info(const fsgp_graph *g, int32_t *n, int64_t *nnz,
                               int32_t *max_in_degree, int64_t *device_bytes) {
    set_error("");
    if (!g) return fail(FSGP_EINVAL, "graph is NULL");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (max_in_degree) *max_in_degree = g->max_deg;
    if (device_bytes) *device_bytes = (int64_t)(g->device_bytes + g->ws.bytes);
    return FSGP_OK;
}
