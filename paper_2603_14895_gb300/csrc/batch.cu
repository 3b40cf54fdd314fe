// batch.cu -- batched requests and the autotuner.
//
// fsgp_batch_run takes many simulation requests over a pool of graphs (mixed models,
// R, parameters, seed sets; the batched Monte Carlo method of Sec. 3.1, Eq. batch,
// extended across requests).  Requests on the same graph with the same model and T run
// side by side in one launch sequence (each keeps its own key, thresholds and lanes, so
// its result equals an fsgp_simulate call for it alone).  Graphs are spread over a few
// CUDA streams by longest-processing-time order so that small graphs overlap, and each
// launch wave's step loop is captured into a CUDA graph.  One host thread issues the
// work of each stream, so that a wave that waits for its stream (host-to-device uploads
// of its small tables) does not hold up the others.
//
// fsgp_autotune times short probe runs of the tuning choices (words per thread, degree
// class bounds); every choice gives identical results, only the speed differs.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "step.cuh"

namespace fsgp {
namespace {

int ws_of(int R) {
    const int W = (R + 31) / 32;
    int Ws = 1;
    while (Ws < W) Ws <<= 1;
    return Ws;
}

struct StreamSet {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    ~StreamSet() {
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (cudaStream_t s : streams) cudaStreamDestroy(s);
    }
};

// One probe run of `opt` on the caller's stream; returns milliseconds (events).
int probe(fsgp_graph *g, int model, const fsgp_params *p, const int32_t *seeds, int64_t ns, int R,
          int T, uint64_t rng_seed, const fsgp_options &opt, uint64_t *d_counts, cudaStream_t s,
          float *ms) {
    SetSpec x{};
    x.beta = p->beta;
    x.gamma = model == FSGP_SI ? 0.0 : p->gamma;
    x.ic_p = p->ic_p;
    x.alpha = p->alpha;
    x.mu = p->mu;
    x.nu = p->nu;
    x.rng_seed = rng_seed;
    x.R = R;
    x.seeds = seeds;
    x.n_seeds = ns;
    x.seed_flags = FSGP_PTR_HOST;
    x.counts = d_counts;
    x.out_flags = FSGP_PTR_DEVICE;
    cudaEvent_t a, b;
    FSGP_CUDA(cudaEventCreate(&a));
    FSGP_CUDA(cudaEventCreate(&b));
    cudaEventRecord(a, s);
    int rc = run_sets(g, model == FSGP_SI ? FSGP_SIS : model, p->ic_mode, p->weighted ? 1 : 0, &x, 1, T, opt, s);
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    if (rc == FSGP_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    return FSGP_OK;
}

}  // namespace
}  // namespace fsgp

using namespace fsgp;

extern "C" int fsgp_autotune(const fsgp_graph *gc, int32_t model, const fsgp_params *params,
                             const int32_t *seed_nodes, int64_t n_seeds, int32_t R, int32_t T_probe,
                             uint64_t rng_seed, fsgp_options *inout, void *stream) {
    set_error("");
    fsgp_graph *g = const_cast<fsgp_graph *>(gc);
    if (!g || !params || !inout || (n_seeds > 0 && !seed_nodes)) return fail(FSGP_EINVAL, "NULL argument");
    if (model < FSGP_SIR || model > FSGP_SWIR) return fail(FSGP_EINVAL, "unknown model");
    if (R < 1 || R > kMaxR) return fail(FSGP_EINVAL, "R must be in [1, 4096]");
    if (T_probe < 1) return fail(FSGP_EINVAL, "T_probe must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *d_counts = nullptr;
    FSGP_CUDA(cudaMalloc(&d_counts, sizeof(uint64_t) * 3 * ((size_t)T_probe + 1)));
    const int Ws = ws_of(R);
    const int vws[3] = {1, 2, 4};
    const int smalls[2] = {63, 255};
    const int hubs[3] = {4096, 8192, 16384};
    fsgp_options best = *inout;
    float best_ms = 1e30f;
    int rc = FSGP_OK;
    {
        // the caller's own fields first (automatic choices: e.g. the fused small-graph
        // mode, which any explicit degree-class bound below turns off)
        fsgp_options o = *inout;
        o.profile = nullptr;
        o.init_planes = nullptr;
        float ms = 0.f, m2 = 0.f;
        rc = probe(g, model, params, seed_nodes, n_seeds, R, T_probe, rng_seed, o, d_counts, s, &ms);
        if (rc == FSGP_OK) rc = probe(g, model, params, seed_nodes, n_seeds, R, T_probe, rng_seed, o, d_counts, s, &m2);
        if (rc == FSGP_OK) best_ms = std::min(ms, m2);
    }
    for (int vi = 0; vi < 3 && rc == FSGP_OK; ++vi) {
        if (vws[vi] > Ws && vws[vi] > 1) continue;
        for (int si = 0; si < 2 && rc == FSGP_OK; ++si)
            for (int hi = 0; hi < 3 && rc == FSGP_OK; ++hi) {
                fsgp_options o = *inout;
                o.vector_words = vws[vi];
                o.small_max_deg = smalls[si];
                o.hub_min_deg = hubs[hi];
                o.hub_chunk = hubs[hi];
                o.profile = nullptr;
                o.init_planes = nullptr;
                float ms = 0.f, m2 = 0.f;
                rc = probe(g, model, params, seed_nodes, n_seeds, R, T_probe, rng_seed, o, d_counts, s, &ms);
                if (rc) break;
                rc = probe(g, model, params, seed_nodes, n_seeds, R, T_probe, rng_seed, o, d_counts, s, &m2);
                if (rc) break;
                ms = std::min(ms, m2);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = o;
                }
            }
    }
    cudaFree(d_counts);
    if (rc) return rc;
    inout->vector_words = best.vector_words;
    inout->small_max_deg = best.small_max_deg;
    inout->hub_min_deg = best.hub_min_deg;
    inout->hub_chunk = best.hub_chunk;
    return FSGP_OK;
}

extern "C" int fsgp_batch_run(const fsgp_request *reqs, int32_t n, const fsgp_batch_options *bo_in,
                              void *stream) {
    set_error("");
    if (n < 0 || (n > 0 && !reqs)) return fail(FSGP_EINVAL, "bad request array");
    fsgp_batch_options bo{};
    if (bo_in) bo = *bo_in;
    const int K = bo.n_streams > 0 ? std::min(bo.n_streams, 32) : 4;
    int dev = 0;
    FSGP_CUDA(cudaGetDevice(&dev));
    for (int i = 0; i < n; ++i) {
        const fsgp_request &q = reqs[i];
        if (!q.graph) return fail(FSGP_EINVAL, "request without a graph");
        if (q.graph->device != dev) return fail(FSGP_EINVAL, "request graph on another device");
        if (q.model < FSGP_SIR || q.model > FSGP_SWIR) return fail(FSGP_EINVAL, "unknown model");
        if (q.R < 1 || q.R > kMaxR) return fail(FSGP_EINVAL, "R must be in [1, 4096]");
        if (q.T < 0) return fail(FSGP_EINVAL, "T must be >= 0");
        if (q.n_seeds < 0 || (q.n_seeds > 0 && !q.seed_nodes)) return fail(FSGP_EINVAL, "bad seed set");
        if (!q.result.counts || q.result.flags != FSGP_PTR_DEVICE)
            return fail(FSGP_EINVAL, "batch results must be device buffers with counts");
        if (q.params.ic_mode != FSGP_IC_WEIGHTED_CASCADE && q.params.ic_mode != FSGP_IC_CONSTANT)
            return fail(FSGP_EINVAL, "bad ic_mode");
    }
    if (n == 0) return FSGP_OK;
    cudaStream_t caller = (cudaStream_t)stream;

    // groups: (graph, model, ic_mode, T, weighted) -> requests
    using Key = std::tuple<const fsgp_graph *, int, int, int, int>;
    std::map<Key, std::vector<int>> groups;
    std::map<const fsgp_graph *, double> cost;
    for (int i = 0; i < n; ++i) {
        const fsgp_request &q = reqs[i];
        // SI runs as SIS without recovery
        groups[Key(q.graph, q.model == FSGP_SI ? FSGP_SIS : q.model, q.params.ic_mode, q.T,
                   q.params.weighted ? 1 : 0)].push_back(i);
        cost[q.graph] += (double)(q.graph->nnz + q.graph->n) * q.R * std::max(q.T, 1);
    }
    // per-graph tuning (optional): one probe series on the graph's first request
    std::map<const fsgp_graph *, fsgp_options> tuned;
    for (auto &kv : groups) {
        const fsgp_graph *g = std::get<0>(kv.first);
        if (tuned.count(g)) continue;
        fsgp_options o{};
        fsgp_graph *gm = const_cast<fsgp_graph *>(g);
        if (bo.autotune) {
            const fsgp_request &q = reqs[kv.second[0]];
            const int rc = fsgp_autotune(g, q.model, &q.params, q.seed_nodes, q.n_seeds, q.R,
                                         std::max(1, std::min(q.T, 8)), q.rng_seed, &o, caller);
            if (rc) return rc;
            gm->tuned = 1;   // kept for later calls on this graph
            gm->tuned_opt = o;
        } else if (gm->tuned) {
            o = gm->tuned_opt;
        }
        o.capture_graph = bo.capture_graph >= 0 ? 1 : 0;
        // the graphs share the GPU through concurrent streams: no persistent step loop,
        // whose grid barrier would wait for CTAs that SMs busy with other streams hold
        o.persistent = -1;
        tuned[g] = o;
    }
    // graphs to streams, longest first onto the least loaded stream
    std::vector<std::pair<double, const fsgp_graph *>> order;
    for (auto &kv : cost) order.push_back({kv.second, kv.first});
    std::sort(order.begin(), order.end(), [](auto &a, auto &b) { return a.first > b.first; });
    std::map<const fsgp_graph *, int> stream_of;
    std::vector<double> load((size_t)K, 0.0);
    for (auto &pr : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        stream_of[pr.second] = k;
        load[k] += pr.first;
    }
    StreamSet ss;
    cudaEvent_t start;
    FSGP_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    ss.events.push_back(start);
    FSGP_CUDA(cudaEventRecord(start, caller));
    for (int k = 0; k < K; ++k) {
        cudaStream_t st;
        FSGP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        ss.streams.push_back(st);
        FSGP_CUDA(cudaStreamWaitEvent(st, start, 0));
    }
    // per graph, its groups from the largest state to the smallest (the graph's
    // workspace then grows at most once)
    std::map<const fsgp_graph *, std::vector<Key>> by_graph;
    for (auto &kv : groups) by_graph[std::get<0>(kv.first)].push_back(kv.first);
    std::vector<std::vector<const fsgp_graph *>> graphs_of((size_t)K);
    for (auto &pr : order) graphs_of[stream_of[pr.second]].push_back(pr.second);
    std::vector<int> rcs((size_t)K, FSGP_OK);
    std::vector<std::string> msgs((size_t)K);
    auto worker = [&](int k) {
        cudaSetDevice(dev);
        cudaStream_t st = ss.streams[k];
        for (const fsgp_graph *g : graphs_of[k]) {
            std::vector<Key> &keys = by_graph.at(g);
            auto state_words = [&](const Key &key) {
                size_t w = 0;
                for (int i : groups.at(key)) w += (size_t)ws_of(reqs[i].R);
                return w;
            };
            std::sort(keys.begin(), keys.end(), [&](const Key &a, const Key &b) {
                return state_words(a) > state_words(b);
            });
            for (const Key &key : keys) {
                const std::vector<int> &idx = groups.at(key);
                std::vector<SetSpec> specs(idx.size());
                for (size_t j = 0; j < idx.size(); ++j) {
                    const fsgp_request &q = reqs[idx[j]];
                    SetSpec &x = specs[j];
                    x = SetSpec{};
                    x.beta = q.params.beta;
                    x.gamma = q.model == FSGP_SI ? 0.0 : q.params.gamma;
                    x.ic_p = q.params.ic_p;
                    x.alpha = q.params.alpha;
                    x.mu = q.params.mu;
                    x.nu = q.params.nu;
                    x.rng_seed = q.rng_seed;
                    x.R = q.R;
                    x.seeds = q.seed_nodes;
                    x.n_seeds = q.n_seeds;
                    x.seed_flags = FSGP_PTR_HOST;
                    x.counts = q.result.counts;
                    x.freq = q.result.freq;
                    x.per_real = q.result.per_real;
                    x.final_planes = q.result.final_planes;
                    x.steps_run = q.result.steps_run;
                    x.out_flags = FSGP_PTR_DEVICE;
                }
                const int rc = run_sets(const_cast<fsgp_graph *>(g), std::get<1>(key), std::get<2>(key), std::get<4>(key),
                                        specs.data(), (int)specs.size(), std::get<3>(key), tuned.at(g), st);
                if (rc) {
                    rcs[k] = rc;
                    msgs[k] = fsgp_last_error();
                    return;
                }
            }
        }
    };
    {
        std::vector<std::thread> th;
        for (int k = 0; k < K; ++k) th.emplace_back(worker, k);
        for (auto &t : th) t.join();
    }
    for (int k = 0; k < K; ++k)
        if (rcs[k]) return fail(rcs[k], msgs[k]);
    // join back into the caller's stream
    for (int k = 0; k < K; ++k) {
        cudaEvent_t e;
        FSGP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ss.events.push_back(e);
        FSGP_CUDA(cudaEventRecord(e, ss.streams[k]));
        FSGP_CUDA(cudaStreamWaitEvent(caller, e, 0));
    }
    FSGP_CUDA(cudaGetLastError());
    return FSGP_OK;
}
