// rows.cuh -- the row kernels of one propagation step (gather + count + decide + write),
// templated on the model, the words per thread V and the team width TEAM.  Included by
// one translation unit per model so that the instantiations compile in parallel.
#pragma once

#include <algorithm>

#include "step.cuh"

namespace fsgp {

template <int V>
struct Vec {
    uint32_t w[V];
};

template <int V>
__device__ __forceinline__ Vec<V> ldg_vec(const uint32_t *p) {
    Vec<V> r;
    if constexpr (V == 4) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
        r.w[0] = q.x; r.w[1] = q.y; r.w[2] = q.z; r.w[3] = q.w;
    } else if constexpr (V == 2) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
        r.w[0] = q.x; r.w[1] = q.y;
    } else {
        r.w[0] = __ldg(p);
    }
    return r;
}

// State loads of a kernel that reads planes written earlier in the same launch (the
// persistent step loop): through L2 only (ld.global.cg), never the non-coherent path.
template <int V, bool CG>
__device__ __forceinline__ Vec<V> ld_vec(const uint32_t *p) {
    if constexpr (!CG) {
        return ldg_vec<V>(p);
    } else {
        Vec<V> r;
        if constexpr (V == 4) {
            const uint4 q = __ldcg(reinterpret_cast<const uint4 *>(p));
            r.w[0] = q.x; r.w[1] = q.y; r.w[2] = q.z; r.w[3] = q.w;
        } else if constexpr (V == 2) {
            const uint2 q = __ldcg(reinterpret_cast<const uint2 *>(p));
            r.w[0] = q.x; r.w[1] = q.y;
        } else {
            r.w[0] = __ldcg(p);
        }
        return r;
    }
}

template <bool CG>
__device__ __forceinline__ uint32_t ld_word(const uint32_t *p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}

template <int V>
__device__ __forceinline__ void st_vec(uint32_t *p, const uint32_t (&w)[V]) {
    if constexpr (V == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    } else {
        *p = w[0];
    }
}

template <int MODEL>
struct ModelTraits {
    // SIR: I, R.  SIS: I.  IC, LT: A, F.  SEIR: I, R, E.  SEIS: I, E.  SWIR: I, R, W.
    // Weighted SIR / SIS: as SIR / SIS.
    static constexpr int planes = (MODEL == FSGP_SIS || MODEL == kSisW)
                                      ? 1
                                      : ((MODEL == FSGP_SEIR || MODEL == FSGP_SWIR) ? 3 : 2);
    // plane gathered from in-neighbours: I (epidemic models), F (IC), A (LT)
    static constexpr int src_plane = MODEL == FSGP_IC ? 1 : 0;
    // per-arc draws (live-lane masks) instead of in-arc counts: IC and weighted graphs
    static constexpr bool weighted = MODEL == kSirW || MODEL == kSisW;
    static constexpr bool counts = MODEL != FSGP_IC && !weighted;
    // the state's source lanes are plane 1 (F) for IC / LT, plane 0 (I) otherwise
    static constexpr bool cascade = MODEL == FSGP_IC || MODEL == FSGP_LT;
    // hub rows may stop reading once every susceptible lane reaches K_sat
    static constexpr bool saturates = MODEL == FSGP_SIR || MODEL == FSGP_SIS || MODEL == FSGP_SEIR ||
                                      MODEL == FSGP_SEIS;
};

// Lanes that can change through their in-arcs: susceptible (SWIR: also weakened) or
// inactive lanes.
template <int MODEL>
__device__ __forceinline__ uint32_t need_of(uint32_t vm, uint32_t s0, uint32_t s1, uint32_t s2) {
    if constexpr (MODEL == FSGP_SIR || MODEL == kSirW || MODEL == FSGP_SEIS || MODEL == FSGP_SWIR)
        return vm & ~s0 & ~s1;
    else if constexpr (MODEL == FSGP_SEIR) return vm & ~s0 & ~s1 & ~s2;
    else return vm & ~s0;
}

// One word of the synchronous update (Eq. updata) from the in-arc counts c (IC: the
// lanes made active by a live arc, `newly`).
template <int MODEL, int B>
__device__ __forceinline__ WordOut update_word(const StepArgs &A, uint32_t node, const WordCtx &x, uint32_t s0,
                                               uint32_t s1, uint32_t s2, int32_t d, const uint32_t (&c)[B],
                                               uint32_t newly) {
    WordOut o;
    if constexpr (MODEL == FSGP_SIR || MODEL == FSGP_SIS) {
        o = update_sir_word<MODEL, B>(A, node, x, s0, s1, d, c);
    } else if constexpr (MODEL == FSGP_IC) {
        o.n0 = s0 | newly;
        o.n1 = newly;
        o.n2 = 0u;
    } else if constexpr (ModelTraits<MODEL>::weighted) {
        // infected: a susceptible lane some infectious in-arc transmitted to; recovery
        // as in SIR / SIS
        const uint32_t infect = newly & need_of<MODEL>(x.vm, s0, s1, 0u);
        const uint32_t rec = lanes_u_less(s0 & x.vm, __ldg(&A.sp[x.s].g_rec), node, A.t, x.g, TAG_RECOVER,
                                          x.k0, x.k1);
        o.n0 = (s0 & ~rec) | infect;
        o.n1 = MODEL == kSirW ? (s1 | rec) : 0u;
        o.n2 = 0u;
    } else if constexpr (MODEL == FSGP_LT) {
        o = update_lt_word<B>(A, node, x, s0, d, c);
    } else if constexpr (MODEL == FSGP_SWIR) {
        o = update_swir_word<B>(A, node, x, s0, s1, s2, d, c);
    } else {
        o = update_seir_word<MODEL, B>(A, node, x, s0, s1, s2, d, c);
    }
    return o;
}

// Row flags of a decided word: bit 0 the new state has source lanes (its out-neighbours
// are pressed next step), bit 1 the row changed or can change on its own next step
// (an exposed lane: SEIR / SEIS).
template <int MODEL>
__device__ __forceinline__ uint32_t word_flags(const WordOut &o, uint32_t s0, uint32_t s1, uint32_t s2) {
    uint32_t fl = 0u;
    if (o.n0 != s0 || o.n1 != s1 || o.n2 != s2) fl |= 2u;
    if (ModelTraits<MODEL>::cascade ? (o.n1 != 0u) : (o.n0 != 0u)) fl |= 1u;
    if constexpr (MODEL == FSGP_SEIR) if (o.n2) fl |= 2u;
    if constexpr (MODEL == FSGP_SEIS) if (o.n1) fl |= 2u;
    return fl;
}

// IC live-arc threshold of a word: weighted cascade (live iff u * d < 2^32, i.e.
// u < floor((2^32 - 1) / d) + 1) or the set's constant probability.
__device__ __forceinline__ uint64_t ic_threshold(const StepArgs &A, int s, int32_t d) {
    if (A.ic_mode == FSGP_IC_WEIGHTED_CASCADE) return d > 0 ? (TWO32 - 1ull) / (uint64_t)d + 1ull : 0ull;
    return __ldg(&A.sp[s].p_const);
}

// Gather the in-arcs [e_begin, e_end) with stride `step` (groups of 4 consecutive arcs)
// into bit-sliced counters (SIR/SIS/LT) or live-lane masks (IC).  Software pipelined:
// the column indices of the next group are loaded while the state words of the current
// group are in flight, so each group costs one memory latency instead of two.
// IC draws are keyed by the arc's position in the caller's column array: arc e of the
// relabelled array is caller arc e + arcb.
template <int MODEL, int V, int B, bool CG = false>
__device__ __forceinline__ void gather_arcs(const StepArgs &A, int64_t e_begin, int64_t e_end,
                                            int64_t step, int64_t arcb, int w0, const uint32_t (&need)[V],
                                            const uint64_t (&ic_thr)[V], const WordCtx (&x)[V],
                                            uint32_t (&c)[V][B], uint32_t (&newly)[V]) {
    const uint32_t *src = A.cur + (size_t)ModelTraits<MODEL>::src_plane * A.plane_words + w0;
    const size_t Wn = (size_t)A.Wn;
    int32_t u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = e_begin + j < e_end ? __ldg(A.col + e_begin + j) : -1;
    for (int64_t e = e_begin; e < e_end; e += step) {
        Vec<V> xs[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (u[j] >= 0) {
                xs[j] = ld_vec<V, CG>(src + (size_t)u[j] * Wn);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i) xs[j].w[i] = 0u;
            }
        }
        const int64_t en = e + step;
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = en + j < e_end ? __ldg(A.col + en + j) : -1;
        if constexpr (ModelTraits<MODEL>::counts) {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if (xs[0].w[i] | xs[1].w[i] | xs[2].w[i] | xs[3].w[i])
                    add4<B>(c[i], xs[0].w[i], xs[1].w[i], xs[2].w[i], xs[3].w[i]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const uint32_t m = xs[j].w[i] & need[i] & ~newly[i];
                    if (m) {
                        constexpr bool W = ModelTraits<MODEL>::weighted;
                        const int64_t ep = e + j + arcb;   // the caller's arc position
                        const uint64_t thr = W ? arc_threshold(A, x[i].s, ep) : ic_thr[i];
                        newly[i] |= lanes_u_less(m, thr, (uint32_t)ep, A.t, x[i].g, W ? TAG_ARC_INFECT : TAG_IC_EDGE,
                                                 x[i].k0, x[i].k1);
                    }
                }
            }
        }
    }
}

// Counter plane b of word i of a thread's V words, by selects (i is not a compile-time
// constant where this is used; indexing the array with it would move it to local memory).
template <int V, int B>
__device__ __forceinline__ uint32_t pick(const uint32_t (&c)[V][B], int i, int b) {
    uint32_t r = c[0][b];
#pragma unroll
    for (int q = 1; q < V; ++q) r = i == q ? c[q][b] : r;
    return r;
}

// Resident CTAs per SM the register allocation is bounded for: wider thread words hold
// more counters, narrower ones run more warps to keep more loads in flight.
template <int V, bool WIDE>
constexpr int min_ctas() { return V == 4 ? 2 : (V == 2 ? (WIDE ? 3 : 4) : 4); }

// Row kernel: one work item is one slice (TEAM*V words) of one row.
// WARP_ROW = false: one team per item; true: one warp per item.
// BT: counter bits of a team kernel, sized to its rows' in-degree bound (fewer planes =
// fewer registers and cheaper counting and grouping).
// which: 0 = small rows with 16..small_max in-arcs (and every small row of a frontier
// step), 1 = mid rows, 3 = rows with 4..15 in-arcs (dense steps only).
// CG: the state planes are read through L2 only (the persistent step loop, which reads
// in one launch the planes that other CTAs wrote at the previous step).
// AG (team rows only): each row is taken by AG teams that split its arcs (every AG-th
// group of 4 arcs) and merge their counts by shuffles; the first team decides.  Shorter
// per-thread chains for small graphs, whose steps are bound by the longest chain.
template <int MODEL, int V, int TEAM, bool WARP_ROW, int BT, bool CG, int AG = 1>
__device__ __forceinline__ void rows_body(const StepArgs &A, int which, int32_t *s_lane,
                                          unsigned long long *s_pc) {
    static_assert(AG == 1 || (!WARP_ROW && TEAM * AG <= 32), "arc groups: team rows within a warp");
    constexpr int B = WARP_ROW ? kWideBits : BT;
    constexpr int TPW = 32 / TEAM;
    constexpr int SW = TEAM * V;
    constexpr int P = ModelTraits<MODEL>::planes;
    const Ctl *C = A.ctl;
    if (*(volatile const int32_t *)&C->stop) return;
    const bool sparse = *(volatile const int32_t *)&C->sparse != 0;
    const int32_t *rows = nullptr;   // frontier steps: candidate rows; dense: a range
    int32_t r0 = 0;
    int64_t nrows;
    if (sparse) {
        if (which >= 2) return;
        rows = which ? A.cand_mid : A.cand_small;
        nrows = (int64_t)((volatile const uint32_t *)C->cand_n)[which];
    } else {
        r0 = which == 0 ? A.r_small : which == 1 ? A.r_mid : A.r_small4;
        nrows = which == 0 ? A.n_small : which == 1 ? A.n_mid : A.n_small4;
    }
    if (nrows == 0) return;
    const int nl = A.Wn * 32;
    const bool lanes_on = A.lane_cnt != nullptr;
    const bool build = list_wanted(A);
    if (lanes_on)
        for (int i = threadIdx.x; i < A.np * nl; i += blockDim.x) s_lane[i] = 0;
    set_acc_zero(s_pc, A.S);
    const int lane = threadIdx.x & 31;
    const int team = lane / TEAM;
    const int tl = lane % TEAM;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int RPI = WARP_ROW ? 1 : TPW / AG;
    const int grp = team % AG;          // arc group of the row (AG > 1)
    const int list_slot = A.k & 1;
    const int64_t nitems = nrows * A.nslices;
    Accum acc;
    // The word contexts and the plane popcount changes belong to the thread's current
    // slice: recomputed / flushed to shared memory only when the slice changes (never,
    // when a row is a single slice).
    int ctx_slice = -1;
    WordCtx x[V];
    int32_t d0[V], d1[V], d2[V];
#pragma unroll
    for (int i = 0; i < V; ++i) d0[i] = d1[i] = d2[i] = 0;

    for (int64_t base = gwarp * RPI; base < nitems; base += nwarps * RPI) {
        const int64_t item = WARP_ROW ? base : base + team / AG;
        const bool has_row = item < nitems;
        const int64_t ridx = has_row ? item / A.nslices : 0;
        const int slice = has_row ? (int)(item - ridx * A.nslices) : 0;
        const int32_t v = has_row ? (rows ? __ldg(rows + ridx) : r0 + (int32_t)ridx) : 0;   // new id
        const uint32_t node = has_row ? node_of(A, v) : 0u;                                  // Philox subject
        const int w0 = slice * SW + tl * V;
        const size_t off = (size_t)v * A.Wn + w0;
        if (slice != ctx_slice) {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if (ctx_slice >= 0) set_acc_add(s_pc, x[i].s, d0[i], d1[i], d2[i]);
                d0[i] = d1[i] = d2[i] = 0;
                x[i] = word_ctx(A, w0 + i);
            }
            ctx_slice = slice;
        }
        // lanes that can change through their in-arcs: S (SIR/SIS) or inactive (IC/LT)
        uint32_t need[V];
        {
            Vec<V> a = has_row ? ld_vec<V, CG>(A.cur + off) : Vec<V>{};
            Vec<V> b{}, e{};
            if (P >= 2 && MODEL != FSGP_IC && MODEL != FSGP_LT && has_row) b = ld_vec<V, CG>(A.cur + A.plane_words + off);
            if (MODEL == FSGP_SEIR && has_row) e = ld_vec<V, CG>(A.cur + 2 * A.plane_words + off);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const uint32_t vm = has_row ? x[i].vm : 0u;
                need[i] = need_of<MODEL>(vm, a.w[i], b.w[i], e.w[i]);
            }
        }
        uint32_t any_need = 0u;
#pragma unroll
        for (int i = 0; i < V; ++i) any_need |= need[i];
#pragma unroll
        for (int o = 1; o < TEAM; o <<= 1) any_need |= __shfl_xor_sync(0xffffffffu, any_need, o);

        uint32_t c[V][B];
        uint32_t newly[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            newly[i] = 0u;
#pragma unroll
            for (int b = 0; b < B; ++b) c[i][b] = 0u;
        }
        int32_t beg = 0, end = 0;
        if (has_row) {
            beg = __ldg(A.rp + v);
            end = __ldg(A.rp + v + 1);
        }
        if (any_need) {
            uint64_t ic_thr[V];
            int64_t arcb = 0;
            if constexpr (!ModelTraits<MODEL>::counts) arcb = (int64_t)__ldg(A.arc0 + v) - beg;
#pragma unroll
            for (int i = 0; i < V; ++i)
                ic_thr[i] = ModelTraits<MODEL>::counts ? 0ull : ic_threshold(A, x[i].s, end - beg);
            if (WARP_ROW)
                gather_arcs<MODEL, V, B, CG>(A, (int64_t)beg + 4 * team, end, 4 * TPW, arcb, w0, need, ic_thr, x, c, newly);
            else
                gather_arcs<MODEL, V, B, CG>(A, (int64_t)beg + 4 * grp, end, 4 * AG, arcb, w0, need, ic_thr, x, c,
                                             newly);
        }
        constexpr bool SPLIT = WARP_ROW && TPW >= V;   // enough teams to give each word one
        if constexpr (SPLIT && V == 2 && ModelTraits<MODEL>::counts) {
            // merge the teams' counters, reduce-scatter first: at the first butterfly level
            // the partners (teams 2j, 2j+1) swap halves and keep word (team & 1) each, so
            // the remaining levels add one word instead of two; team i < 2 ends up with
            // the warp total of word i, which it decides below
            const int par = team & 1;
            uint32_t d[B];
#pragma unroll
            for (int b = 0; b < B; ++b) d[b] = __shfl_xor_sync(0xffffffffu, par ? c[0][b] : c[1][b], TEAM);
#pragma unroll
            for (int b = 0; b < B; ++b) c[0][b] = par ? c[1][b] : c[0][b];
            add_sliced<B>(c[0], d);
#pragma unroll
            for (int o = 2 * TEAM; o < 32; o <<= 1) {
#pragma unroll
                for (int b = 0; b < B; ++b) d[b] = __shfl_xor_sync(0xffffffffu, c[0][b], o);
                add_sliced<B>(c[0], d);
            }
#pragma unroll
            for (int b = 0; b < B; ++b) c[1][b] = c[0][b];
        } else if (WARP_ROW || AG > 1) {
            // merge the teams' partial results (the warp is converged here)
#pragma unroll
            for (int o = TEAM; o < (WARP_ROW ? 32 : TEAM * AG); o <<= 1) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    if constexpr (ModelTraits<MODEL>::counts) {
                        uint32_t d[B];
#pragma unroll
                        for (int b = 0; b < B; ++b) d[b] = __shfl_xor_sync(0xffffffffu, c[i][b], o);
                        add_sliced<B>(c[i], d);
                    } else {
                        newly[i] |= __shfl_xor_sync(0xffffffffu, newly[i], o);
                    }
                }
            }
        }
        uint32_t fl = 0u;
        bool writer;
        if constexpr (SPLIT) {
            // every team holds the merged counts of the same words: team i < V decides the
            // i-th word of each thread's V words, so the decisions of a row run V-wide
            // instead of V-deep
            writer = has_row && team < V;
            if (writer) {
                const int i = team;
                uint32_t cw[B];
#pragma unroll
                for (int b = 0; b < B; ++b) cw[b] = pick<V, B>(c, i, b);
                WordCtx xw = x[0];
                uint32_t nw = newly[0];
#pragma unroll
                for (int q = 1; q < V; ++q) {
                    if (i == q) {
                        xw = x[q];
                        nw = newly[q];
                    }
                }
                const uint32_t s0 = ld_word<CG>(A.cur + off + i);
                const uint32_t s1 = P >= 2 ? ld_word<CG>(A.cur + A.plane_words + off + i) : 0u;
                const uint32_t s2 = P >= 3 ? ld_word<CG>(A.cur + 2 * A.plane_words + off + i) : 0u;
                const WordOut o = update_word<MODEL, B>(A, node, xw, s0, s1, s2, end - beg, cw, nw);
                A.nxt[off + i] = o.n0;
                if (P >= 2) A.nxt[A.plane_words + off + i] = o.n1;
                if (P >= 3) A.nxt[2 * A.plane_words + off + i] = o.n2;
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    if (i == q) {
                        d0[q] += __popc(o.n0) - __popc(s0);
                        d1[q] += __popc(o.n1) - __popc(s1);
                        d2[q] += __popc(o.n2) - __popc(s2);
                    }
                }
                if (lanes_on) {
                    lane_deltas(s_lane, w0 + i, s0, o.n0);
                    if (P >= 2) lane_deltas(s_lane + nl, w0 + i, s1, o.n1);
                    if (P >= 3) lane_deltas(s_lane + 2 * nl, w0 + i, s2, o.n2);
                }
                fl |= word_flags<MODEL>(o, s0, s1, s2);
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) fl |= __shfl_xor_sync(0xffffffffu, fl, o);
            writer = has_row && team == 0;
        } else {
        writer = has_row && (WARP_ROW ? team == 0 : grp == 0);
        if (writer) {
            // own state again (L1/L2-resident): not kept live across the gather
            uint32_t s0[V], s1[V], s2[V];
            {
                Vec<V> a = ld_vec<V, CG>(A.cur + off);
                Vec<V> b{}, e{};
                if (P >= 2) b = ld_vec<V, CG>(A.cur + A.plane_words + off);
                if (P >= 3) e = ld_vec<V, CG>(A.cur + 2 * A.plane_words + off);
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    s0[i] = a.w[i];
                    s1[i] = P >= 2 ? b.w[i] : 0u;
                    s2[i] = P >= 3 ? e.w[i] : 0u;
                }
            }
            uint32_t n0[V], n1[V], n2[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const WordOut o = update_word<MODEL, B>(A, node, x[i], s0[i], s1[i], s2[i], end - beg, c[i], newly[i]);
                n0[i] = o.n0;
                n1[i] = o.n1;
                n2[i] = o.n2;
                d0[i] += __popc(o.n0) - __popc(s0[i]);
                d1[i] += __popc(o.n1) - __popc(s1[i]);
                d2[i] += __popc(o.n2) - __popc(s2[i]);
                if (lanes_on) {
                    lane_deltas(s_lane, w0 + i, s0[i], o.n0);
                    if (P >= 2) lane_deltas(s_lane + nl, w0 + i, s1[i], o.n1);
                    if (P >= 3) lane_deltas(s_lane + 2 * nl, w0 + i, s2[i], o.n2);
                }
                fl |= word_flags<MODEL>(o, s0[i], s1[i], s2[i]);
            }
            st_vec<V>(A.nxt + off, n0);
            if (P >= 2) st_vec<V>(A.nxt + A.plane_words + off, n1);
            if (P >= 3) st_vec<V>(A.nxt + 2 * A.plane_words + off, n2);
        }
#pragma unroll
        for (int o = 1; o < TEAM; o <<= 1) fl |= __shfl_xor_sync(0xffffffffu, fl, o);
        }
        const bool leader = writer && tl == 0;
        const bool want = leader && fl != 0u;
        if (want && (fl & 1u)) acc.push_deg += (unsigned long long)(__ldg(A.out_ptr + node + 1) - __ldg(A.out_ptr + node));
        if (A.prof_bytes && leader) acc.bytes += row_bytes(SW, P, any_need != 0u, end - beg);
        list_append(A, build, want, (int32_t)((uint32_t)v | ((fl & 1u) ? kPushBit : 0u)), list_slot);
        if (sparse && leader) atomicAnd(&A.bitmap[v >> 5], ~(1u << (v & 31)));
    }
    if (ctx_slice >= 0) {
#pragma unroll
        for (int i = 0; i < V; ++i) set_acc_add(s_pc, x[i].s, d0[i], d1[i], d2[i]);
    }
    flush_accum(A, acc, list_slot, WARP_ROW ? PK_MID : (BT == 4 ? PK_SMALL4 : PK_SMALL));
    set_acc_flush(A, s_pc);
    if (lanes_on) flush_lanes(A, s_lane, nl);
}

template <int MODEL, int V, int TEAM, bool WARP_ROW, int BT = kSmallBits>
__global__ void __launch_bounds__(kBlock, min_ctas<V, WARP_ROW>()) k_rows(StepArgs A, int which) {
    extern __shared__ int32_t s_lane[];
    __shared__ unsigned long long s_pc[kPC * kMaxSets];
    rows_body<MODEL, V, TEAM, WARP_ROW, BT, false>(A, which, s_lane, s_pc);
}

// Persistent step loop of a small graph: all T dense steps in one launch, the row work of
// the fused mode (every row, one kernel) separated by grid barriers instead of kernel
// boundaries.  The step control of the launched loop is folded in: each step's plane
// popcount changes go to its own row of pc (running totals are formed after the loop),
// and the cascade models stop at the first step whose previous step activated nothing,
// a decision every CTA takes alike from the same counts.  State is read through L2
// (CG loads): a CTA reads at step k the words other CTAs wrote at step k-1.
// (bounded for 2 resident CTAs per SM: the loop is meant for graphs that fill a few CTAs
// per SM at most, and the body then keeps its state in registers)
template <int MODEL, int V, int TEAM, bool WARP_ROW, int BT = kSmallBits, int AG = 1>
__global__ void __launch_bounds__(kBlock, 2)
    k_rows_persist(const __grid_constant__ StepArgs A0, const __grid_constant__ PersistArgs Q) {
    extern __shared__ int32_t s_lane[];
    __shared__ unsigned long long s_pc[kPC * kMaxSets];
    __shared__ StepArgs sA;
    __shared__ unsigned long long s_new[kMaxSets];   // cascade: lanes newly active at the last step
    __shared__ int s_stop;
    constexpr bool cascade = ModelTraits<MODEL>::cascade;
    Ctl *C = A0.ctl;
    {
        const int32_t *src = reinterpret_cast<const int32_t *>(&A0);
        int32_t *dst = reinterpret_cast<int32_t *>(&sA);
        for (int i = threadIdx.x; i < (int)(sizeof(StepArgs) / sizeof(int32_t)); i += blockDim.x) dst[i] = src[i];
    }
    if (cascade)
        for (int s = threadIdx.x; s < A0.S; s += blockDim.x) s_new[s] = __ldcg(Q.pc + (size_t)s * kPC + 1);
    for (int k = 1; k <= Q.T; ++k) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int stop = 0;
            if (cascade) {
                stop = 1;
                for (int s = 0; s < A0.S; ++s)
                    if (s_new[s]) stop = 0;
            }
            s_stop = stop;
            sA.k = k;
            sA.t = Q.t0 + (uint32_t)k;
            sA.cur = (k & 1) ? Q.buf0 : Q.buf1;
            sA.nxt = (k & 1) ? Q.buf1 : Q.buf0;
            sA.pc = Q.pc + (size_t)k * A0.S * kPC;
        }
        __syncthreads();
        if (s_stop) {
            if (blockIdx.x == 0 && threadIdx.x == 0) C->stop = 1;
            break;
        }
        rows_body<MODEL, V, TEAM, WARP_ROW, BT, true, AG>(sA, WARP_ROW ? 1 : 0, s_lane, s_pc);
        if (!grid_barrier(&C->bar_count, &C->bar_gen, gridDim.x, &C->err, Q.spin_limit)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) C->steps_done = k;
        if (cascade)
            for (int s = threadIdx.x; s < A0.S; s += blockDim.x)
                s_new[s] += __ldcg(Q.pc + ((size_t)k * A0.S + s) * kPC + 1);
    }
}

// Hub rows, phase 1: one CTA per (chunk of in-arcs, word slice); per-lane partial counts
// (IC: live masks) are added into the hub's scratch slot.
//   pass 0: every chunk;
//   pass 1 (SIR/SIS): the first chunk of every hub row only; when every susceptible lane
//     of the slice already counts K_sat infected in-arcs there, the slice is flagged:
//     its lanes are infected whatever the rest of the row holds (every count from K_sat
//     on decides the same way), so its other chunks need not be read;
//   pass 2 (SIR/SIS): the other chunks of the slices not flagged.
template <int MODEL, int V, int TEAM>
__global__ void __launch_bounds__(kBlock, min_ctas<V, true>()) k_hub_chunks(StepArgs A, int pass) {
    __shared__ uint32_t s_cnt[kMaxR];
    constexpr int B = kWideBits;
    constexpr int TPB = kBlock / TEAM;
    constexpr int SW = TEAM * V;
    constexpr int P = ModelTraits<MODEL>::planes;
    const Ctl *C = A.ctl;
    if (*(volatile const int32_t *)&C->stop) return;
    const bool sparse = *(volatile const int32_t *)&C->sparse != 0;
    const int nl = A.Wn * 32;
    const int tl = threadIdx.x % TEAM;
    const int team = threadIdx.x / TEAM;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < SW * 32; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();
    const int64_t n_items = (pass == 1 ? (int64_t)A.n_hubs : A.n_hub_chunks) * A.nslices;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        int64_t item = it / A.nslices;      // chunk index (pass 1: hub index)
        const int slice = (int)(it - item * A.nslices);
        int h;
        if (pass == 1) {
            h = (int)item;
            item = __ldg(A.hub_chunk_base + h);
        } else {
            int lo = 0, hi = A.n_hubs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(A.hub_chunk_base + mid) <= item) lo = mid; else hi = mid - 1;
            }
            h = lo;
            if (pass == 2 && (item == __ldg(A.hub_chunk_base + h) ||
                              *(volatile const uint32_t *)&A.hub_sat[(int64_t)h * A.nslices + slice]))
                continue;   // the first chunk ran in pass 1, or the slice is saturated
        }
        const int32_t v = h;   // hub rows are new ids 0 .. n_hubs-1
        if (sparse && !((A.bitmap[v >> 5] >> (v & 31)) & 1u)) continue;
        const int ws0 = slice * SW;        // first word of the slice
        const int w0 = ws0 + tl * V;
        WordCtx x[V];
        uint32_t need[V];
        uint32_t any_need = 0u;
        {
            const size_t off = (size_t)v * A.Wn + w0;
            Vec<V> a = ldg_vec<V>(A.cur + off);
            Vec<V> b{}, e{};
            if (P >= 2) b = ldg_vec<V>(A.cur + A.plane_words + off);
            if (P >= 3) e = ldg_vec<V>(A.cur + 2 * A.plane_words + off);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                x[i] = word_ctx(A, w0 + i);
                need[i] = need_of<MODEL>(x[i].vm, a.w[i], b.w[i], e.w[i]);
                any_need |= need[i];
            }
        }
#pragma unroll
        for (int o = 1; o < TEAM; o <<= 1) any_need |= __shfl_xor_sync(0xffffffffu, any_need, o);
        if (!any_need) continue;   // identical in every team: they share the slice
        const int32_t rb = __ldg(A.rp + v), re = __ldg(A.rp + v + 1);
        int64_t arcb = 0;
        if constexpr (!ModelTraits<MODEL>::counts) arcb = (int64_t)__ldg(A.arc0 + v) - rb;
        const int64_t cidx = item - __ldg(A.hub_chunk_base + h);
        const int64_t beg = (int64_t)rb + cidx * A.hub_chunk;
        const int64_t end = min((int64_t)re, beg + A.hub_chunk);
        uint32_t c[V][B];
        uint32_t newly[V];
        uint64_t ic_thr[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            newly[i] = 0u;
            ic_thr[i] = ModelTraits<MODEL>::counts ? 0ull : ic_threshold(A, x[i].s, re - rb);
#pragma unroll
            for (int b = 0; b < B; ++b) c[i][b] = 0u;
        }
        gather_arcs<MODEL, V, B>(A, beg + 4 * team, end, 4 * TPB, arcb, w0, need, ic_thr, x, c, newly);
#pragma unroll
        for (int o = TEAM; o < 32; o <<= 1) {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if constexpr (ModelTraits<MODEL>::counts) {
                    uint32_t d[B];
#pragma unroll
                    for (int b = 0; b < B; ++b) d[b] = __shfl_xor_sync(0xffffffffu, c[i][b], o);
                    add_sliced<B>(c[i], d);
                } else {
                    newly[i] |= __shfl_xor_sync(0xffffffffu, newly[i], o);
                }
            }
        }
        if constexpr (ModelTraits<MODEL>::counts) {
            // every team holds the warp's merged counts: the lanes' counts are read out
            // by all teams, each taking every (32/TEAM)-th lane
            constexpr int TPW = 32 / TEAM;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int wsl = w0 + i - ws0;   // word within the slice
                for (int l = team % TPW; l < 32; l += TPW) {
                    const uint32_t k = lane_count<B>(c[i], l);
                    if (k) atomicAdd(&s_cnt[wsl * 32 + l], k);
                }
            }
        } else if (lane < TEAM) {   // team 0 of the warp holds the warp's live masks
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int wsl = w0 + i - ws0;
                if (newly[i]) atomicOr(&s_cnt[wsl], newly[i]);
            }
        }
        if (A.prof_bytes && threadIdx.x == 0)
            atomicAdd(&A.prof_bytes[PK_HUB], row_bytes(SW, P, true, end - beg));
        __syncthreads();
        if constexpr (ModelTraits<MODEL>::saturates) {
            if (pass == 1) {
                // team 0 holds the slice's susceptible lanes (need); all of them at K_sat?
                bool sat = true;
                if (team == 0) {
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        const int32_t ks = __ldg(&A.sp[x[i].s].ksat);
                        uint32_t m = need[i];
                        if (m && ks == INT32_MAX) sat = false;
                        const int wsl = w0 + i - ws0;
                        while (m && sat) {
                            const int l = __ffs(m) - 1;
                            m &= m - 1;
                            if (s_cnt[wsl * 32 + l] < (uint32_t)ks) sat = false;
                        }
                    }
                }
                if (__syncthreads_and(sat) && threadIdx.x == 0)
                    A.hub_sat[(int64_t)h * A.nslices + slice] = 1u;
            }
        }
        uint32_t *slot = A.hub_scratch + (size_t)h * nl;
        if constexpr (ModelTraits<MODEL>::counts) {
            for (int i = threadIdx.x; i < SW * 32; i += blockDim.x) {
                const uint32_t xv = s_cnt[i];
                if (xv) {
                    atomicAdd(slot + ws0 * 32 + i, xv);
                    s_cnt[i] = 0u;
                }
            }
        } else {
            for (int i = threadIdx.x; i < SW; i += blockDim.x) {
                const uint32_t xv = s_cnt[i];
                if (xv) {
                    atomicOr(slot + ws0 + i, xv);
                    s_cnt[i] = 0u;
                }
            }
        }
        __syncthreads();
    }
}

// Hub rows, phase 2: one warp per hub row; lane l decides word g0 + l.  The per-lane
// counts are re-sliced with ballots (32-bit counters), the scratch slot is cleared.
template <int MODEL>
__global__ void __launch_bounds__(kBlock) k_hub_finalize(StepArgs A) {
    extern __shared__ int32_t s_lane[];
    __shared__ unsigned long long s_pc[kPC * kMaxSets];
    constexpr int P = ModelTraits<MODEL>::planes;
    const Ctl *C = A.ctl;
    if (*(volatile const int32_t *)&C->stop) return;
    const bool sparse = *(volatile const int32_t *)&C->sparse != 0;
    const int nl = A.Wn * 32;
    const bool lanes_on = A.lane_cnt != nullptr;
    const bool build = list_wanted(A);
    if (lanes_on)
        for (int i = threadIdx.x; i < A.np * nl; i += blockDim.x) s_lane[i] = 0;
    set_acc_zero(s_pc, A.S);
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int list_slot = A.k & 1;
    Accum acc;
    for (int64_t h = gwarp; h < A.n_hubs; h += nwarps) {
        const int32_t v = (int32_t)h;
        const uint32_t node = node_of(A, v);
        const bool cand = !sparse || ((A.bitmap[v >> 5] >> (v & 31)) & 1u);
        uint32_t fl = 0u;
        if (cand) {
            const int32_t d = __ldg(A.rp + v + 1) - __ldg(A.rp + v);
            uint32_t *slot = A.hub_scratch + (size_t)h * nl;
            for (int g0 = 0; g0 < A.Wn; g0 += 32) {
                const int w = g0 + lane;
                const bool act = w < A.Wn;
                uint32_t c[32];
#pragma unroll
                for (int b = 0; b < 32; ++b) c[b] = 0u;
                uint32_t newly = 0u;
                if constexpr (ModelTraits<MODEL>::counts) {
                    const int nw = min(32, A.Wn - g0);
                    for (int ww = 0; ww < nw; ++ww) {
                        const uint32_t kv = slot[(g0 + ww) * 32 + lane];
                        if (kv) slot[(g0 + ww) * 32 + lane] = 0u;
#pragma unroll
                        for (int b = 0; b < 32; ++b) {
                            const uint32_t bb = __ballot_sync(0xffffffffu, (kv >> b) & 1u);
                            if (lane == ww) c[b] = bb;
                        }
                    }
                } else {
                    if (act) {
                        newly = slot[w];
                        if (newly) slot[w] = 0u;
                    }
                }
                if (act) {
                    const size_t off = (size_t)v * A.Wn + w;
                    const uint32_t s0 = __ldg(A.cur + off);
                    const uint32_t s1 = P >= 2 ? __ldg(A.cur + A.plane_words + off) : 0u;
                    const uint32_t s2 = P >= 3 ? __ldg(A.cur + 2 * A.plane_words + off) : 0u;
                    const WordCtx x = word_ctx(A, w);
                    const WordOut o = update_word<MODEL, 32>(A, node, x, s0, s1, s2, d, c, newly & x.vm & ~s0);
                    A.nxt[off] = o.n0;
                    if (P >= 2) A.nxt[A.plane_words + off] = o.n1;
                    if (P >= 3) A.nxt[2 * A.plane_words + off] = o.n2;
                    set_acc_add(s_pc, x.s, (long long)__popc(o.n0) - __popc(s0),
                                (long long)__popc(o.n1) - __popc(s1), (long long)__popc(o.n2) - __popc(s2));
                    if (lanes_on) {
                        lane_deltas(s_lane, w, s0, o.n0);
                        if (P >= 2) lane_deltas(s_lane + nl, w, s1, o.n1);
                        if (P >= 3) lane_deltas(s_lane + 2 * nl, w, s2, o.n2);
                    }
                    fl |= word_flags<MODEL>(o, s0, s1, s2);
                }
            }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) fl |= __shfl_xor_sync(0xffffffffu, fl, o);
        if (A.hub_sat)
            for (int sl = lane; sl < A.nslices; sl += 32) A.hub_sat[h * A.nslices + sl] = 0u;
        const bool want = cand && lane == 0 && fl != 0u;
        if (want && (fl & 1u)) acc.push_deg += (unsigned long long)(__ldg(A.out_ptr + node + 1) - __ldg(A.out_ptr + node));
        if (A.prof_bytes && cand && lane == 0)
            acc.bytes += row_bytes(A.Wn, P, false, 0) + 2ull * 4ull * 32ull * (unsigned long long)A.Wn;
        list_append(A, build, want, (int32_t)((uint32_t)v | ((fl & 1u) ? kPushBit : 0u)), list_slot);
        if (sparse && cand && lane == 0) atomicAnd(&A.bitmap[v >> 5], ~(1u << (v & 31)));
    }
    flush_accum(A, acc, list_slot, PK_HUBFIN);
    set_acc_flush(A, s_pc);
    if (lanes_on) flush_lanes(A, s_lane, nl);
}

// Rows with 1..3 in-arcs, and the rows without in-arcs whose state can change (listed by
// the step-0 scan: seeds, or imported rows with infected / newly active lanes; every
// other row without in-arcs keeps its state for the whole run and is never touched),
// dense steps only (on frontier steps such rows come through the candidate lists of
// k_rows).  Most rows of a power-law graph
// are of this kind and carry little gather work, so the cost is the chain of dependent
// loads per row: one THREAD per item (a slice of SWL <= 8 words of one row) keeps four
// to eight times as many rows in flight per SM as a team per row.  The thread loads its
// own words and the (at most three) sources' words at once, stages them in shared memory,
// and then decides its words one at a time through a single, non-unrolled copy of the
// per-word update (counts of at most 3 need 2-bit counters).
constexpr int kLaneMaxDeg = 3;
template <int SWL, int NP>
struct LaneStage {
    uint32_t v[NP + 3][SWL][kBlock];   // own planes, then the sources' words (x0, x1, x2)
};

// Lanes that change on their own (without in-arcs): infectious lanes that may recover,
// newly active lanes that stop being new (IC / LT), exposed lanes (SEIR / SEIS).
template <int MODEL>
__device__ __forceinline__ uint32_t self_lanes(uint32_t s0, uint32_t s1, uint32_t s2) {
    if constexpr (MODEL == FSGP_IC || MODEL == FSGP_LT) return s1;
    else if constexpr (MODEL == FSGP_SEIR) return s0 | s2;
    else if constexpr (MODEL == FSGP_SEIS) return s0 | s1;
    else return s0;
}

template <int MODEL, int SWL>
__global__ void __launch_bounds__(kBlock) k_rows_lane(StepArgs A) {
    extern __shared__ int32_t s_lane[];
    __shared__ unsigned long long s_pc[kPC * kMaxSets];
    constexpr int P = ModelTraits<MODEL>::planes;
    __shared__ LaneStage<SWL, P> st;
    const Ctl *C = A.ctl;
    if (*(volatile const int32_t *)&C->stop) return;
    if (*(volatile const int32_t *)&C->sparse) return;
    const int nsl = A.Wn / SWL;
    const int64_t n_rows = (int64_t)A.n_lane + *(volatile const uint32_t *)&C->d0_n;
    const int64_t nitems = n_rows * nsl;
    if (nitems == 0) return;
    const int nl = A.Wn * 32;
    const bool lanes_on = A.lane_cnt != nullptr;
    const bool build = list_wanted(A);
    if (lanes_on)
        for (int i = threadIdx.x; i < A.np * nl; i += blockDim.x) s_lane[i] = 0;
    set_acc_zero(s_pc, A.S);
    const int list_slot = A.k & 1;
    const int tid = threadIdx.x;
    const uint32_t *src_plane = A.cur + (size_t)ModelTraits<MODEL>::src_plane * A.plane_words;
    Accum acc;
    int cur_s = -1;           // set of the plane-count deltas not yet flushed
    int32_t dd0 = 0, dd1 = 0, dd2 = 0;
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + tid; item - tid < nitems;
         item += (int64_t)gridDim.x * blockDim.x) {
        const bool has = item < nitems;
        int32_t v = 0, beg = 0, d = 0;   // v: new id
        uint32_t node = 0u;              // Philox subject
        int w0 = 0;
        uint32_t busy = 0u;
        if (has) {
            const int64_t r = item / nsl;
            w0 = (int)(item - r * nsl) * SWL;
            int4 e;
            if (r < A.n_lane) {
                e = __ldg(A.lane_tab + r);   // the node and its sources in one entry
                v = A.r_lane + (int32_t)r;
            } else {
                v = A.d0_list[r - A.n_lane];
                e = make_int4((int32_t)node_of(A, v), -1, -1, -1);
            }
            node = (uint32_t)e.x;
            const int32_t u[kLaneMaxDeg] = {e.y, e.z, e.w};
            d = (e.y >= 0) + (e.z >= 0) + (e.w >= 0);
            if (!ModelTraits<MODEL>::counts && d > 0) beg = __ldg(A.arc0 + v);   // arc positions key the draws
            const size_t off = (size_t)v * A.Wn + w0;
            // own words and sources' words, 4 (or fewer) words per load; `busy` records
            // whether any lane can change at this step (an infected lane to recover, or a
            // lane that can change with a set source lane in its in-arcs)
#pragma unroll
            for (int q = 0; q < SWL; q += (SWL < 4 ? SWL : 4)) {
                constexpr int VL = SWL < 4 ? SWL : 4;
                const Vec<VL> a = ldg_vec<VL>(A.cur + off + q);
                Vec<VL> bb{}, ee{};
                if (P >= 2) bb = ldg_vec<VL>(A.cur + A.plane_words + off + q);
                if (P >= 3) ee = ldg_vec<VL>(A.cur + 2 * A.plane_words + off + q);
                uint32_t xs[VL];
#pragma unroll
                for (int i = 0; i < VL; ++i) {
                    st.v[0][q + i][tid] = a.w[i];
                    if (P >= 2) st.v[1][q + i][tid] = bb.w[i];
                    if (P >= 3) st.v[2][q + i][tid] = ee.w[i];
                    xs[i] = 0u;
                }
#pragma unroll
                for (int j = 0; j < kLaneMaxDeg; ++j) {
                    Vec<VL> x{};
                    if (u[j] >= 0) x = ldg_vec<VL>(src_plane + (size_t)u[j] * A.Wn + w0 + q);
#pragma unroll
                    for (int i = 0; i < VL; ++i) {
                        st.v[P + j][q + i][tid] = x.w[i];
                        xs[i] |= x.w[i];
                    }
                }
#pragma unroll
                for (int i = 0; i < VL; ++i) {
                    const uint32_t s0 = a.w[i], s1 = P >= 2 ? bb.w[i] : 0u, s2 = P >= 3 ? ee.w[i] : 0u;
                    // a lane changes on its own, or can change with a set source lane
                    busy |= self_lanes<MODEL>(s0, s1, s2) | (need_of<MODEL>(~0u, s0, s1, s2) & xs[i]);
                }
            }
        }
        uint32_t fl = 0u;
        if (has && !busy) {
            // no lane can change: the next state is this one
            const size_t off = (size_t)v * A.Wn + w0;
#pragma unroll
            for (int q = 0; q < SWL; q += (SWL < 4 ? SWL : 4)) {
                constexpr int VL = SWL < 4 ? SWL : 4;
#pragma unroll
                for (int pl = 0; pl < P; ++pl) {
                    uint32_t nw[VL];
#pragma unroll
                    for (int i = 0; i < VL; ++i) nw[i] = st.v[pl][q + i][tid];
                    st_vec<VL>(A.nxt + pl * A.plane_words + off + q, nw);
                }
            }
        } else if (has) {
#pragma unroll 1
            for (int i = 0; i < SWL; ++i) {
                const WordCtx x = word_ctx(A, w0 + i);
                const uint32_t s0 = st.v[0][i][tid];
                const uint32_t s1 = P >= 2 ? st.v[1][i][tid] : 0u;
                const uint32_t s2 = P >= 3 ? st.v[2][i][tid] : 0u;
                const uint32_t x0 = st.v[P][i][tid], x1 = st.v[P + 1][i][tid], x2 = st.v[P + 2][i][tid];
                const uint32_t need = need_of<MODEL>(x.vm, s0, s1, s2);
                uint32_t c[2] = {0u, 0u}, newly = 0u;
                if constexpr (!ModelTraits<MODEL>::counts) {
                    constexpr bool W = ModelTraits<MODEL>::weighted;
                    const uint64_t thr = W ? 0ull : ic_threshold(A, x.s, d);
                    const uint32_t xs[kLaneMaxDeg] = {x0, x1, x2};
#pragma unroll
                    for (int j = 0; j < kLaneMaxDeg; ++j) {
                        const uint32_t m = xs[j] & need & ~newly;
                        if (m)
                            newly |= lanes_u_less(m, W ? arc_threshold(A, x.s, beg + j) : thr, (uint32_t)(beg + j),
                                                  A.t, x.g, W ? TAG_ARC_INFECT : TAG_IC_EDGE, x.k0, x.k1);
                    }
                } else {
                    // counts of set source lanes (at most 3): two bit-planes
                    c[0] = (x0 ^ x1 ^ x2) & need;
                    c[1] = ((x0 & x1) | (x2 & (x0 ^ x1))) & need;
                }
                const WordOut o = update_word<MODEL, 2>(A, node, x, s0, s1, s2, d, c, newly);
                st.v[0][i][tid] = o.n0;
                if (P >= 2) st.v[1][i][tid] = o.n1;
                if (P >= 3) st.v[2][i][tid] = o.n2;
                if (x.s != cur_s) {
                    if (cur_s >= 0) set_acc_add(s_pc, cur_s, dd0, dd1, dd2);
                    cur_s = x.s;
                    dd0 = dd1 = dd2 = 0;
                }
                dd0 += __popc(o.n0) - __popc(s0);
                dd1 += __popc(o.n1) - __popc(s1);
                dd2 += __popc(o.n2) - __popc(s2);
                if (lanes_on) {
                    lane_deltas(s_lane, w0 + i, s0, o.n0);
                    if (P >= 2) lane_deltas(s_lane + nl, w0 + i, s1, o.n1);
                    if (P >= 3) lane_deltas(s_lane + 2 * nl, w0 + i, s2, o.n2);
                }
                fl |= word_flags<MODEL>(o, s0, s1, s2);
            }
            const size_t off = (size_t)v * A.Wn + w0;
#pragma unroll
            for (int q = 0; q < SWL; q += (SWL < 4 ? SWL : 4)) {
                constexpr int VL = SWL < 4 ? SWL : 4;
#pragma unroll
                for (int pl = 0; pl < P; ++pl) {
                    uint32_t nw[VL];
#pragma unroll
                    for (int i = 0; i < VL; ++i) nw[i] = st.v[pl][q + i][tid];
                    st_vec<VL>(A.nxt + pl * A.plane_words + off + q, nw);
                }
            }
        }
        const bool want = has && fl != 0u;
        if (want && (fl & 1u)) acc.push_deg += (unsigned long long)(__ldg(A.out_ptr + node + 1) - __ldg(A.out_ptr + node));
        if (A.prof_bytes && has) acc.bytes += row_bytes(SWL, P, d > 0, d);
        list_append(A, build, want, (int32_t)((uint32_t)v | ((fl & 1u) ? kPushBit : 0u)), list_slot);
    }
    if (cur_s >= 0) set_acc_add(s_pc, cur_s, dd0, dd1, dd2);
    flush_accum(A, acc, list_slot, PK_LANE);
    set_acc_flush(A, s_pc);
    if (lanes_on) flush_lanes(A, s_lane, nl);
}

// Widest slice of the one-thread-per-row kernel: its staging area (planes + 3 sources,
// SWL words, 256 threads) must fit the 48 KB of static shared memory.
template <int MODEL>
constexpr int lane_swl_max() { return ModelTraits<MODEL>::planes >= 3 ? 4 : 8; }

template <int MODEL>
int launch_rows_lane(const StepArgs &A, int swl, int grid, size_t smem, cudaStream_t s) {
    switch (swl) {
        case 1: k_rows_lane<MODEL, 1><<<grid, kBlock, smem, s>>>(A); break;
        case 2: k_rows_lane<MODEL, 2><<<grid, kBlock, smem, s>>>(A); break;
        case 4: k_rows_lane<MODEL, 4><<<grid, kBlock, smem, s>>>(A); break;
        case 8:
            if constexpr (lane_swl_max<MODEL>() >= 8) {
                k_rows_lane<MODEL, 8><<<grid, kBlock, smem, s>>>(A);
                break;
            }
            return fail(FSGP_EINVAL, "lane kernel slice width");
        default: return fail(FSGP_EINVAL, "lane kernel slice width");
    }
    return FSGP_OK;
}

template <int MODEL, int SWL>
int occupancy_lane_w(size_t smem) {
    // the staging area is static; per-lane counters (dynamic) may push the total past the
    // default 48 KB window.  The attribute is process-wide and host threads of a batch set
    // it concurrently, so it is always raised to the largest per-lane counter area any run
    // uses (32 KB), never lowered to this run's need (set before any launch or capture).
    cudaFuncSetAttribute(k_rows_lane<MODEL, SWL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * 1024);
    int z = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&z, k_rows_lane<MODEL, SWL>, kBlock, smem);
    return z;
}

template <int MODEL>
int occupancy_lane(int swl, size_t smem) {
    int z = 1;
    switch (swl) {
        case 1: z = occupancy_lane_w<MODEL, 1>(smem); break;
        case 2: z = occupancy_lane_w<MODEL, 2>(smem); break;
        case 4: z = occupancy_lane_w<MODEL, 4>(smem); break;
        default:
            if constexpr (lane_swl_max<MODEL>() >= 8) z = occupancy_lane_w<MODEL, 8>(smem);
            else z = occupancy_lane_w<MODEL, 4>(smem);
            break;
    }
    return z < 1 ? 1 : z;
}

// ------------------------------------------------------------------------- launch

template <int MODEL, int V, int TEAM>
int launch_rows_vt(const StepArgs &A, const StepLaunch &L, cudaStream_t s) {
    Prof *pr = L.prof;
    if (L.have_hub) {
        if (pr) pr->start(PK_HUB, s);
        if (A.hub_sat) {
            k_hub_chunks<MODEL, V, TEAM><<<L.grid_hub, kBlock, 0, s>>>(A, 1);
            k_hub_chunks<MODEL, V, TEAM><<<L.grid_hub, kBlock, 0, s>>>(A, 2);
        } else {
            k_hub_chunks<MODEL, V, TEAM><<<L.grid_hub, kBlock, 0, s>>>(A, 0);
        }
        if (pr) { pr->stop(s); pr->start(PK_HUBFIN, s); }
        k_hub_finalize<MODEL><<<L.grid_fin, kBlock, L.smem_lanes, s>>>(A);
        if (pr) pr->stop(s);
    }
    if (L.have_mid) {
        if (pr) pr->start(PK_MID, s);
        k_rows<MODEL, V, TEAM, true><<<L.grid_mid, kBlock, L.smem_lanes, s>>>(A, 1);
        if (pr) pr->stop(s);
    }
    if (L.have_small) {
        if (pr) pr->start(PK_SMALL, s);
        k_rows<MODEL, V, TEAM, false><<<L.grid_small, kBlock, L.smem_lanes, s>>>(A, 0);
        if (pr) pr->stop(s);
    }
    if (L.have_small4) {
        if (pr) pr->start(PK_SMALL4, s);
        k_rows<MODEL, V, TEAM, false, 4><<<L.grid_small4, kBlock, L.smem_lanes, s>>>(A, 3);
        if (pr) pr->stop(s);
    }
    if (L.have_lane) {
        if (pr) pr->start(PK_LANE, s);
        const int rc = launch_rows_lane<MODEL>(A, L.swl, L.grid_lane, L.smem_lanes, s);
        if (pr) pr->stop(s);
        if (rc) return rc;
    }
    return FSGP_OK;
}

template <int MODEL, int V, int TEAM>
void occupancy_vt(size_t smem, RowOccupancy *o) {
    int a = 1, m = 1, b = 1, s4 = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s4, k_rows<MODEL, V, TEAM, false, 4>, kBlock, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_rows<MODEL, V, TEAM, false>, kBlock, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_rows<MODEL, V, TEAM, true>, kBlock, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_hub_chunks<MODEL, V, TEAM>, kBlock, 0);
    o->small = a < 1 ? 1 : a;
    o->mid = m < 1 ? 1 : m;
    o->hub = b < 1 ? 1 : b;
    o->small4 = s4 < 1 ? 1 : s4;
}

#define FSGP_VT_SWITCH(MACRO)                          \
    switch (V * 100 + TEAM) {                          \
        case 101: MACRO(1, 1); break;                  \
        case 102: MACRO(1, 2); break;                  \
        case 104: MACRO(1, 4); break;                  \
        case 108: MACRO(1, 8); break;                  \
        case 116: MACRO(1, 16); break;                 \
        case 132: MACRO(1, 32); break;                 \
        case 201: MACRO(2, 1); break;                  \
        case 401: MACRO(4, 1); break;                  \
        case 402: MACRO(4, 2); break;                  \
        case 404: MACRO(4, 4); break;                  \
        case 408: MACRO(4, 8); break;                  \
        case 416: MACRO(4, 16); break;                 \
        case 432: MACRO(4, 32); break;                 \
        case 202: MACRO(2, 2); break;                  \
        case 204: MACRO(2, 4); break;                  \
        case 208: MACRO(2, 8); break;                  \
        case 216: MACRO(2, 16); break;                 \
        case 232: MACRO(2, 32); break;                 \
        default: return fail(FSGP_EINVAL, "unsupported words-per-thread / team combination"); \
    }

template <int MODEL>
int launch_rows(const StepArgs &A, const StepLaunch &L, cudaStream_t s) {
    const int V = L.V, TEAM = L.TEAM;
#define FSGP_L(v_, t_) launch_rows_vt<MODEL, v_, t_>(A, L, s)
    FSGP_VT_SWITCH(FSGP_L)
#undef FSGP_L
    return FSGP_OK;
}

// Only the CTA-split pair (chunks, then finalize), for callers that treat every row as
// a split row.
template <int MODEL, int V, int TEAM>
int launch_split_vt(const StepArgs &A, int grid_chunks, int grid_fin, cudaStream_t s) {
    k_hub_chunks<MODEL, V, TEAM><<<grid_chunks, kBlock, 0, s>>>(A, 0);
    k_hub_finalize<MODEL><<<grid_fin, kBlock, 0, s>>>(A);
    return FSGP_OK;
}

template <int MODEL>
int launch_split_rows(const StepArgs &A, int V, int TEAM, int grid_chunks, int grid_fin,
                      cudaStream_t s) {
#define FSGP_S(v_, t_) launch_split_vt<MODEL, v_, t_>(A, grid_chunks, grid_fin, s)
    FSGP_VT_SWITCH(FSGP_S)
#undef FSGP_S
    return FSGP_OK;
}

template <int MODEL>
int occupancy_rows(int V, int TEAM, size_t smem, RowOccupancy *o) {
#define FSGP_O(v_, t_) occupancy_vt<MODEL, v_, t_>(smem, o)
    FSGP_VT_SWITCH(FSGP_O)
#undef FSGP_O
    o->lane = occupancy_lane<MODEL>(o->swl, smem);
    return FSGP_OK;
}

// Cooperative launch of the persistent step loop (one word per thread, the 8-bit team
// kernel: fused small graphs with in-degrees <= 255).  The grid is capped at the CTAs
// that can be resident at once; *grid_out gets the grid used.  FSGP_EUNSUPPORTED: no
// persistent kernel for this team width (the caller runs the launched loop instead).
template <int MODEL, int TEAM>
int launch_persist_t(const StepArgs &A, const PersistArgs &Q, int grid, size_t smem, int sm_count,
                     cudaStream_t s, int *grid_out) {
    // two teams per row split its arcs (measured on ER n = 10k, R = 64: 2 teams 0.73 ms
    // per run, 4 teams 0.79 ms, 8 teams 0.94 ms)
    constexpr int AG = TEAM >= 32 ? 1 : 2;
    auto kern = k_rows_persist<MODEL, 1, TEAM, false, kSmallBits, AG>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor (persistent)");
    if (per_sm < 1) return FSGP_EUNSUPPORTED;
    // one work item (row slice) per team of AG teams: AG times the launched loop's CTAs
    grid = std::max(1, std::min(grid * AG, per_sm * sm_count));
    StepArgs a = A;
    PersistArgs q = Q;
    void *args[] = {&a, &q};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(kBlock), args, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel (persistent step loop)");
    *grid_out = grid;
    return FSGP_OK;
}

template <int MODEL>
int launch_persist(const StepArgs &A, const PersistArgs &Q, int TEAM, int grid, size_t smem, int sm_count,
                   cudaStream_t s, int *grid_out) {
    switch (TEAM) {
        case 1: return launch_persist_t<MODEL, 1>(A, Q, grid, smem, sm_count, s, grid_out);
        case 2: return launch_persist_t<MODEL, 2>(A, Q, grid, smem, sm_count, s, grid_out);
        case 4: return launch_persist_t<MODEL, 4>(A, Q, grid, smem, sm_count, s, grid_out);
        case 8: return launch_persist_t<MODEL, 8>(A, Q, grid, smem, sm_count, s, grid_out);
        case 16: return launch_persist_t<MODEL, 16>(A, Q, grid, smem, sm_count, s, grid_out);
        case 32: return launch_persist_t<MODEL, 32>(A, Q, grid, smem, sm_count, s, grid_out);
        default: return FSGP_EUNSUPPORTED;
    }
}

}  // namespace fsgp
