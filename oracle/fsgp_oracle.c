/*
 * fsgp_oracle.c -- plain CPU oracle for synchronous batched Monte Carlo propagation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct restatement of
 * what the GPU library computes.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header, table
 * or helper with the CUDA library: it has its own Philox4x32-10, its own survival
 * table and its own update rules, each written from the paper's definitions.
 *
 * Shape (paper, Algorithm 1): for each realization, for each step, for each node,
 * read the step-(k-1) states of the node and its in-neighbours and write the step-k
 * state into a second buffer (the X^{k+1} <- X^k double buffer of Algorithm 1;
 * node-synchronous update, Eq. (all), Eqs. (ms), (agg), (updata) of Sec. 3.1).
 * Realizations are independent (batched Monte Carlo definition, Eq. (batch)), so the
 * only parallelism here is threads over realizations.
 *
 * Integer readings of the paper (all listed in the design notes):
 *  - SIR (Appendix A.1, micro-accelerated SIR): a susceptible node with k infected
 *    in-neighbours is infected with probability 1-(1-beta)^k.  Here the probability
 *    is the exact integer survival table surv[0]=2^32, surv[k]=floor(surv[k-1]*q/2^32),
 *    q=2^32-llrint(beta*2^32), and the node is infected iff its 32-bit uniform
 *    u >= surv[k] (the survival form of "U < m_i").  An infected node recovers iff
 *    u_rec < llrint(gamma*2^32) (delta of the appendix read as gamma).
 *  - SIS: the same with I -> S instead of I -> R (Table 1 model, rules not written
 *    out in the paper).
 *  - IC (Kempe et al., cited in Sec. 2): each in-arc (w -> v) is tried once, at the
 *    step after w activates, if v is still inactive; live iff u*d_in(v) < 2^32
 *    (weighted cascade) or u < llrint(p*2^32) (constant p).
 *  - LT (named in Sec. 1; definition taken from the project statement): per node and
 *    realization threshold theta = u(tag 4, v, t=0, r); an inactive node with k >= 1
 *    active in-arcs activates iff k*2^32 >= theta*d_in(v).
 *  - The discrete-time epidemic rows of Table 1 (named there, rules not written out;
 *    k counts the in-arcs whose source is infectious, I):
 *      SI: SIR without recovery (I absorbing).
 *      SEIR(DT): S -> E iff k >= 1 and u >= surv_beta[k]; E -> I iff u(tag 5) <
 *        llrint(alpha*2^32); I -> R iff u(tag 2) < llrint(gamma*2^32).
 *      SEIS(DT): the same with I -> S.
 *      SWIR: S -> I iff k >= 1 and u >= surv_kappa[k] (kappa = beta), otherwise
 *        S -> W iff k >= 1 and u(tag 6) >= surv_mu[k]; W -> I iff k >= 1 and u >=
 *        surv_nu[k]; I -> R at the next step.
 *    Every node changes state at most once per step, from its step-(t-1) state.
 *  - Weighted graphs (Table 1 lists edge weights for the epidemic models; SIR, SIS and
 *    SI here): arc e = (u -> v) carries weight w_e >= 0 and infects with probability
 *    p_e = beta * w_e per step while u is infectious and v susceptible, independently
 *    over arcs, so that v escapes with probability prod_e (1 - p_e) (the unweighted
 *    1-(1-beta)^k when every w_e = 1).  Each infectious in-arc draws its own uniform
 *    (tag 7, keyed by the arc's position e in col_idx, the step and the realization)
 *    and transmits iff u < thr_e; thr_e is formed in single precision:
 *    p = (float)beta * w_e, thr_e = 0 if p <= 0, 2^32 if p >= 1, else
 *    llrintf(p * 2^32).  Recovery is unchanged.
 *
 * Uniforms (bit-plane contract): P_j = Philox4x32_10(key=(lo32(seed),hi32(seed)),
 * ctr=(a, t, r>>5, (tag<<8)|(j>>2)))[j&3] for j = 0..31, and bit (31-j) of u is bit
 * (r&31) of P_j.  This oracle always assembles all 32 bits.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#define ORC_SIR 0
#define ORC_SIS 1
#define ORC_IC 2
#define ORC_LT 3
#define ORC_SI 4
#define ORC_SEIR 5
#define ORC_SEIS 6
#define ORC_SWIR 7

#define TAG_INFECT 1u
#define TAG_RECOVER 2u
#define TAG_IC_EDGE 3u
#define TAG_LT_THRESH 4u
#define TAG_LATENT 5u
#define TAG_WEAKEN 6u
#define TAG_ARC_INFECT 7u

/* node states (= compartment index).  SIR/SIS: 0=S 1=I 2=R.  IC/LT: 0=inactive 1=newly
 * active (frontier) 2=active since an earlier step.  SI: 0=S 1=I.  SEIR/SEIS: 0=S 1=E
 * 2=I 3=R.  SWIR: 0=S 1=W 2=I 3=R. */
#define ST_0 0
#define ST_1 1
#define ST_2 2
#define ST_3 3

/* compartments reported per model (columns of counts / rows of freq) */
int orc_compartments(int model)
{
    return (model == ORC_SEIR || model == ORC_SWIR) ? 4 : 3;
}

/* state that transmits (counted in k) and the state seeds start in */
static uint8_t infectious_state(int model)
{
    return (model == ORC_SEIR || model == ORC_SEIS || model == ORC_SWIR) ? ST_2 : ST_1;
}

/* ---------------- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) --------------
 * One round: two 32x32->64 multiplies of counter words 0 and 2 by the round
 * multipliers; the high halves are xored with the other counter words and the key,
 * the low halves pass through.  The key is bumped by the Weyl constants (golden ratio
 * and sqrt(3)-1 scaled to 2^32) between rounds.  Ten rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The 32-bit uniform of realization r for (tag, subject a, step t). */
uint32_t orc_uniform(uint64_t rng_seed, uint32_t tag, uint32_t a, uint32_t t, uint32_t r)
{
    uint32_t key[2] = {(uint32_t)(rng_seed & 0xFFFFFFFFu), (uint32_t)(rng_seed >> 32)};
    uint32_t u = 0;
    for (uint32_t call = 0; call < 8; ++call) {
        uint32_t ctr[4] = {a, t, r >> 5, (tag << 8) | call};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        for (uint32_t i = 0; i < 4; ++i) {
            uint32_t j = call * 4 + i;               /* plane index, MSB first */
            uint32_t bit = (out[i] >> (r & 31u)) & 1u;
            u |= bit << (31u - j);
        }
    }
    return u;
}

/* Exact integer survival table: surv[k] ~ 2^32 (1-beta)^k, for k = 0..kmax. */
void orc_survival_table(double beta, int64_t kmax, uint64_t *surv)
{
    uint64_t b = (uint64_t)llrint(beta * 4294967296.0);
    uint64_t q = 4294967296ull - b;
    surv[0] = 4294967296ull;
    for (int64_t k = 1; k <= kmax; ++k) {
        /* q = 2^32 (beta rounds to 0) would overflow the 64-bit product: then the
         * survival probability is exactly 1 at every k. */
        if (q == 4294967296ull) surv[k] = surv[k - 1];
        else surv[k] = (surv[k - 1] * q) >> 32;
    }
}

uint64_t orc_prob_threshold(double p)
{
    return (uint64_t)llrint(p * 4294967296.0);
}

/* ---------------- one simulation ---------------- */

typedef struct {
    int model;
    int32_t n;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    double beta, gamma;
    int ic_mode;          /* 0 = weighted cascade (1/d_in), 1 = constant probability */
    double ic_p;
    const int32_t *seeds;
    int64_t n_seeds;
    int32_t T;
    uint64_t rng_seed;
    double alpha, mu, nu;     /* SEIR/SEIS latent rate; SWIR weakening and weakened infection */
    int C;                    /* compartments */
    const uint8_t *init_state; /* optional [n_real][n] start states (resume); NULL = seeds */
    int32_t t0;               /* absolute index of the starting step */
    int32_t r_lo, n_real;     /* realizations r_lo .. r_lo+n_real-1 */
    /* outputs */
    uint64_t *counts;     /* [T+1][3], summed over the realizations run */
    uint32_t *per_real;   /* optional [n_real][T+1][3] */
    uint32_t *freq;       /* optional [3][n] */
    uint8_t *final_state; /* optional [n_real][n] */
    int32_t *quiet_step;  /* [n_real]: IC/LT first step with an empty frontier (T if never) */
    /* derived */
    uint64_t *surv;
    uint64_t *surv_mu;    /* SWIR */
    uint64_t *surv_nu;    /* SWIR */
    int64_t kmax;
    uint64_t g_rec;
    uint64_t p_const;
    uint64_t a_lat;       /* SEIR/SEIS latent threshold */
    const float *arc_w;   /* optional [nnz] arc weights (SIR/SIS/SI): per-arc infection */
    float beta_f;         /* beta in single precision (weighted threshold) */
} orc_job;

/* Weighted infection threshold of one arc (single precision, see the header). */
static uint64_t arc_threshold(float beta_f, float w)
{
    const float p = beta_f * w;
    if (!(p > 0.0f)) return 0;
    if (p >= 1.0f) return 4294967296ull;
    return (uint64_t)llrintf(p * 4294967296.0f);
}

/* Weighted infection of a susceptible node: some infectious in-arc transmits. */
static int weighted_infected(const orc_job *jb, const uint8_t *X, int32_t beg, int32_t end,
                             uint8_t infectious, uint32_t t, uint32_t r)
{
    for (int32_t e = beg; e < end; ++e) {
        if (X[jb->col_idx[e]] != infectious) continue;
        uint32_t u = orc_uniform(jb->rng_seed, TAG_ARC_INFECT, (uint32_t)e, t, r);
        if ((uint64_t)u < arc_threshold(jb->beta_f, jb->arc_w[e])) return 1;
    }
    return 0;
}

typedef struct {
    orc_job *job;
    int tid, nthreads;
    uint64_t *counts;  /* thread-local [T+1][3] */
    uint32_t *freq;    /* thread-local [3][n] or NULL */
} orc_worker;

/* One synchronous step of node v for realization r: returns the state of v at step t
 * given the states X of step t-1 (Eq. nodestate of Sec. 2). */
static uint8_t node_update(const orc_job *jb, const uint8_t *X, int32_t v, uint32_t t, uint32_t r)
{
    const int32_t beg = jb->row_ptr[v], end = jb->row_ptr[v + 1];
    const int64_t d = (int64_t)end - beg;
    const uint8_t s = X[v];
    switch (jb->model) {
    case ORC_SIR:
    case ORC_SIS: {
        if (s == ST_0 && jb->arc_w) return weighted_infected(jb, X, beg, end, ST_1, t, r) ? ST_1 : ST_0;
        if (s == ST_0) {
            int64_t k = 0;
            for (int32_t e = beg; e < end; ++e)
                if (X[jb->col_idx[e]] == ST_1) ++k;
            if (k == 0) return ST_0;
            uint32_t u = orc_uniform(jb->rng_seed, TAG_INFECT, (uint32_t)v, t, r);
            uint64_t thr = jb->surv[k <= jb->kmax ? k : jb->kmax];
            return ((uint64_t)u >= thr) ? ST_1 : ST_0;
        }
        if (s == ST_1) {
            uint32_t u = orc_uniform(jb->rng_seed, TAG_RECOVER, (uint32_t)v, t, r);
            if ((uint64_t)u < jb->g_rec) return jb->model == ORC_SIR ? ST_2 : ST_0;
            return ST_1;
        }
        return ST_2;
    }
    case ORC_IC: {
        if (s != ST_0) return ST_2;
        for (int32_t e = beg; e < end; ++e) {
            if (X[jb->col_idx[e]] != ST_1) continue;
            uint32_t u = orc_uniform(jb->rng_seed, TAG_IC_EDGE, (uint32_t)e, t, r);
            int live;
            if (jb->ic_mode == 0) live = ((uint64_t)u * (uint64_t)d) < 4294967296ull;
            else live = (uint64_t)u < jb->p_const;
            if (live) return ST_1;
        }
        return ST_0;
    }
    case ORC_LT: {
        if (s != ST_0) return ST_2;
        int64_t k = 0;
        for (int32_t e = beg; e < end; ++e)
            if (X[jb->col_idx[e]] != ST_0) ++k;
        if (k == 0) return ST_0;
        uint32_t theta = orc_uniform(jb->rng_seed, TAG_LT_THRESH, (uint32_t)v, 0u, r);
        /* k*2^32 >= theta*d, both sides < 2^63 for k, d < 2^31 */
        if (((uint64_t)k << 32) >= (uint64_t)theta * (uint64_t)d) return ST_1;
        return ST_0;
    }
    case ORC_SI: {
        if (s != ST_0) return s;
        if (jb->arc_w) return weighted_infected(jb, X, beg, end, ST_1, t, r) ? ST_1 : ST_0;
        int64_t k = 0;
        for (int32_t e = beg; e < end; ++e)
            if (X[jb->col_idx[e]] == ST_1) ++k;
        if (k == 0) return ST_0;
        uint32_t u = orc_uniform(jb->rng_seed, TAG_INFECT, (uint32_t)v, t, r);
        return ((uint64_t)u >= jb->surv[k <= jb->kmax ? k : jb->kmax]) ? ST_1 : ST_0;
    }
    case ORC_SEIR:
    case ORC_SEIS: {
        if (s == ST_0) {
            int64_t k = 0;
            for (int32_t e = beg; e < end; ++e)
                if (X[jb->col_idx[e]] == ST_2) ++k;
            if (k == 0) return ST_0;
            uint32_t u = orc_uniform(jb->rng_seed, TAG_INFECT, (uint32_t)v, t, r);
            return ((uint64_t)u >= jb->surv[k <= jb->kmax ? k : jb->kmax]) ? ST_1 : ST_0;
        }
        if (s == ST_1) {
            uint32_t u = orc_uniform(jb->rng_seed, TAG_LATENT, (uint32_t)v, t, r);
            return ((uint64_t)u < jb->a_lat) ? ST_2 : ST_1;
        }
        if (s == ST_2) {
            uint32_t u = orc_uniform(jb->rng_seed, TAG_RECOVER, (uint32_t)v, t, r);
            if ((uint64_t)u < jb->g_rec) return jb->model == ORC_SEIR ? ST_3 : ST_0;
            return ST_2;
        }
        return ST_3;
    }
    case ORC_SWIR: {
        if (s == ST_0 || s == ST_1) {
            int64_t k = 0;
            for (int32_t e = beg; e < end; ++e)
                if (X[jb->col_idx[e]] == ST_2) ++k;
            if (k == 0) return s;
            const int64_t kk = k <= jb->kmax ? k : jb->kmax;
            uint32_t u = orc_uniform(jb->rng_seed, TAG_INFECT, (uint32_t)v, t, r);
            if (s == ST_0) {
                if ((uint64_t)u >= jb->surv[kk]) return ST_2;
                uint32_t w = orc_uniform(jb->rng_seed, TAG_WEAKEN, (uint32_t)v, t, r);
                return ((uint64_t)w >= jb->surv_mu[kk]) ? ST_1 : ST_0;
            }
            return ((uint64_t)u >= jb->surv_nu[kk]) ? ST_2 : ST_1;
        }
        return ST_3;   /* I -> R after one step; R absorbing */
    }
    }
    return s;
}

static void tally(const orc_job *jb, const uint8_t *X, uint64_t *cnt)
{
    uint64_t c[4] = {0, 0, 0, 0};
    for (int32_t v = 0; v < jb->n; ++v) c[X[v]]++;
    for (int i = 0; i < jb->C; ++i) cnt[i] += c[i];
}

static void *worker_main(void *arg)
{
    orc_worker *w = (orc_worker *)arg;
    orc_job *jb = w->job;
    const int32_t n = jb->n, T = jb->T;
    uint8_t *X = (uint8_t *)malloc((size_t)n > 0 ? (size_t)n : 1);
    uint8_t *Y = (uint8_t *)malloc((size_t)n > 0 ? (size_t)n : 1);
    for (int32_t ri = w->tid; ri < jb->n_real; ri += w->nthreads) {
        const uint32_t r = (uint32_t)(jb->r_lo + ri);
        /* X^0 */
        const int C = jb->C;
        if (jb->init_state) {
            memcpy(X, jb->init_state + (size_t)ri * n, (size_t)n);
        } else {
            memset(X, ST_0, (size_t)n);
            for (int64_t i = 0; i < jb->n_seeds; ++i) X[jb->seeds[i]] = infectious_state(jb->model);
        }
        uint64_t c0[4] = {0, 0, 0, 0};
        tally(jb, X, c0);
        for (int c = 0; c < C; ++c) {
            w->counts[c] += c0[c];
            if (jb->per_real) jb->per_real[((size_t)ri * (T + 1)) * C + c] = (uint32_t)c0[c];
        }
        int quiet = 0;
        int32_t quiet_step = T;
        if (jb->model == ORC_IC || jb->model == ORC_LT) {
            int any_front = 0;
            for (int32_t v = 0; v < n; ++v) if (X[v] == ST_1) { any_front = 1; break; }
            if (!any_front) { quiet = 1; quiet_step = 0; }
        }
        for (int32_t k = 1; k <= T; ++k) {
            if (!quiet) {
                const uint32_t t = (uint32_t)(jb->t0 + k);
                for (int32_t v = 0; v < n; ++v) Y[v] = node_update(jb, X, v, t, r);
                uint8_t *tmp = X; X = Y; Y = tmp;
                if (jb->model == ORC_IC || jb->model == ORC_LT) {
                    int any_front = 0;
                    for (int32_t v = 0; v < n; ++v) if (X[v] == ST_1) { any_front = 1; break; }
                    if (!any_front) { quiet = 1; quiet_step = k; }
                }
            }
            uint64_t ck[4] = {0, 0, 0, 0};
            tally(jb, X, ck);
            for (int c = 0; c < C; ++c) {
                w->counts[(size_t)k * C + c] += ck[c];
                if (jb->per_real) jb->per_real[((size_t)ri * (T + 1) + k) * C + c] = (uint32_t)ck[c];
            }
        }
        if (jb->quiet_step) jb->quiet_step[ri] = quiet_step;
        if (w->freq)
            for (int32_t v = 0; v < n; ++v) w->freq[(size_t)X[v] * n + v]++;
        if (jb->final_state) memcpy(jb->final_state + (size_t)ri * n, X, (size_t)n);
    }
    free(X);
    free(Y);
    return NULL;
}

/*
 * Run n_real realizations (r_lo .. r_lo+n_real-1) of one model from one seed set.
 * Returns 0 on success, -1 on invalid arguments, -2 on allocation failure.
 * With C = orc_compartments(model): counts must hold (T+1)*C u64, per_real (optional)
 * n_real*(T+1)*C u32, freq (optional) C*n u32, final_state (optional) n_real*n u8,
 * quiet_step (optional) n_real i32.
 */
/* As orc_simulate_ext, with optional arc weights (SIR, SIS and SI only; NULL =
 * unweighted). */
int orc_simulate_w(int model, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                   double beta, double gamma, int ic_mode, double ic_p,
                   double alpha, double mu, double nu, const float *arc_w,
                   const int32_t *seeds, int64_t n_seeds, int32_t T, uint64_t rng_seed,
                   const uint8_t *init_state, int32_t t0,
                   int32_t r_lo, int32_t n_real, int nthreads,
                   uint64_t *counts, uint32_t *per_real, uint32_t *freq, uint8_t *final_state,
                   int32_t *quiet_step)
{
    if (model < 0 || model > 7 || n < 0 || T < 0 || n_real < 0 || r_lo < 0 || !counts) return -1;
    if (arc_w && model != ORC_SIR && model != ORC_SIS && model != ORC_SI) return -1;
    if (nthreads < 1) nthreads = 1;
    for (int64_t i = 0; i < n_seeds; ++i)
        if (seeds[i] < 0 || seeds[i] >= n) return -1;
    orc_job jb;
    memset(&jb, 0, sizeof jb);
    jb.model = model; jb.n = n; jb.row_ptr = row_ptr; jb.col_idx = col_idx;
    jb.beta = beta; jb.gamma = gamma; jb.ic_mode = ic_mode; jb.ic_p = ic_p;
    jb.alpha = alpha; jb.mu = mu; jb.nu = nu; jb.C = orc_compartments(model);
    jb.seeds = seeds; jb.n_seeds = n_seeds; jb.T = T; jb.rng_seed = rng_seed;
    jb.init_state = init_state; jb.t0 = t0;
    jb.r_lo = r_lo; jb.n_real = n_real;
    jb.counts = counts; jb.per_real = per_real; jb.freq = freq; jb.final_state = final_state;
    jb.quiet_step = quiet_step;
    jb.arc_w = arc_w;
    jb.beta_f = (float)beta;
    if (arc_w)
        for (int64_t e = 0; e < (int64_t)row_ptr[n]; ++e)
            if (!(arc_w[e] >= 0.0f) || arc_w[e] > 3.4e38f) return -1;   /* finite, >= 0 */
    int64_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t d = (int64_t)row_ptr[v + 1] - row_ptr[v];
        if (d > maxdeg) maxdeg = d;
    }
    jb.kmax = maxdeg;
    jb.surv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(maxdeg + 1));
    jb.surv_mu = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(maxdeg + 1));
    jb.surv_nu = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(maxdeg + 1));
    if (!jb.surv || !jb.surv_mu || !jb.surv_nu) {
        free(jb.surv); free(jb.surv_mu); free(jb.surv_nu);
        return -2;
    }
    orc_survival_table(beta, maxdeg, jb.surv);
    orc_survival_table(mu, maxdeg, jb.surv_mu);
    orc_survival_table(nu, maxdeg, jb.surv_nu);
    jb.g_rec = orc_prob_threshold(gamma);
    jb.p_const = orc_prob_threshold(ic_p);
    jb.a_lat = orc_prob_threshold(alpha);
    const int C = jb.C;

    memset(counts, 0, sizeof(uint64_t) * (size_t)(T + 1) * C);
    if (freq) memset(freq, 0, sizeof(uint32_t) * C * (size_t)n);
    if (nthreads > n_real && n_real > 0) nthreads = n_real;
    orc_worker *ws = (orc_worker *)calloc((size_t)nthreads, sizeof(orc_worker));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int rc = 0;
    for (int i = 0; i < nthreads; ++i) {
        ws[i].job = &jb; ws[i].tid = i; ws[i].nthreads = nthreads;
        ws[i].counts = (uint64_t *)calloc((size_t)(T + 1) * C, sizeof(uint64_t));
        ws[i].freq = freq ? (uint32_t *)calloc((size_t)C * n + 1, sizeof(uint32_t)) : NULL;
        if (!ws[i].counts || (freq && !ws[i].freq)) rc = -2;
    }
    if (rc == 0) {
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, worker_main, &ws[i]);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        for (int i = 0; i < nthreads; ++i) {
            for (size_t j = 0; j < (size_t)(T + 1) * C; ++j) counts[j] += ws[i].counts[j];
            if (freq)
                for (size_t j = 0; j < (size_t)C * n; ++j) freq[j] += ws[i].freq[j];
        }
    }
    for (int i = 0; i < nthreads; ++i) { free(ws[i].counts); free(ws[i].freq); }
    free(ws); free(th); free(jb.surv); free(jb.surv_mu); free(jb.surv_nu);
    return rc;
}

int orc_simulate_ext(int model, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     double beta, double gamma, int ic_mode, double ic_p,
                     double alpha, double mu, double nu,
                     const int32_t *seeds, int64_t n_seeds, int32_t T, uint64_t rng_seed,
                     const uint8_t *init_state, int32_t t0,
                     int32_t r_lo, int32_t n_real, int nthreads,
                     uint64_t *counts, uint32_t *per_real, uint32_t *freq, uint8_t *final_state,
                     int32_t *quiet_step)
{
    return orc_simulate_w(model, n, row_ptr, col_idx, beta, gamma, ic_mode, ic_p, alpha, mu, nu, NULL,
                          seeds, n_seeds, T, rng_seed, init_state, t0, r_lo, n_real, nthreads,
                          counts, per_real, freq, final_state, quiet_step);
}

/* The four models of the first table rows (SIR, SIS, IC, LT): three compartments. */
int orc_simulate(int model, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                 double beta, double gamma, int ic_mode, double ic_p,
                 const int32_t *seeds, int64_t n_seeds, int32_t T, uint64_t rng_seed,
                 const uint8_t *init_state, int32_t t0,
                 int32_t r_lo, int32_t n_real, int nthreads,
                 uint64_t *counts, uint32_t *per_real, uint32_t *freq, uint8_t *final_state,
                 int32_t *quiet_step)
{
    if (model < 0 || model > 3) return -1;
    return orc_simulate_ext(model, n, row_ptr, col_idx, beta, gamma, ic_mode, ic_p, 0.0, 0.0, 0.0,
                            seeds, n_seeds, T, rng_seed, init_state, t0, r_lo, n_real, nthreads,
                            counts, per_real, freq, final_state, quiet_step);
}

/* Step-by-step single-node check used for sampled parity at full size: the state of
 * node v at step t (absolute index) in realization r, from the step-(t-1) states X. */
int orc_node_step(int model, const int32_t *row_ptr, const int32_t *col_idx, int32_t v,
                  const uint8_t *X, double beta, double gamma, int ic_mode, double ic_p,
                  uint32_t t, uint32_t r, uint64_t rng_seed)
{
    orc_job jb;
    memset(&jb, 0, sizeof jb);
    jb.model = model; jb.row_ptr = row_ptr; jb.col_idx = col_idx;
    jb.beta = beta; jb.gamma = gamma; jb.ic_mode = ic_mode; jb.ic_p = ic_p;
    jb.rng_seed = rng_seed;
    int64_t d = (int64_t)row_ptr[v + 1] - row_ptr[v];
    jb.kmax = d;
    jb.surv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(d + 1));
    if (!jb.surv) return -2;
    orc_survival_table(beta, d, jb.surv);
    jb.g_rec = orc_prob_threshold(gamma);
    jb.p_const = orc_prob_threshold(ic_p);
    jb.C = orc_compartments(model);
    int s = (model >= 0 && model <= 3) ? node_update(&jb, X, v, t, r) : -1;
    free(jb.surv);
    return s;
}

/* ---------------- Hegselmann-Krause opinion dynamics (Appendix A.2) ----------------
 * Continuous opinions, no randomness: R independent opinion vectors (realizations)
 * given by the caller.  At step k every node i takes the mean of the opinions of its
 * in-neighbours j (Sec. 2 convention N(i) = N^-(i), arcs with multiplicity, i itself
 * only through a self-loop) whose distance |h_i - h_j| is below eps; with no such
 * neighbour the opinion stays (the NaN case of the appendix).  Readings: the strict
 * "< eps" of the appendix's message definition (its prose says "<= eps"), and single
 * precision throughout (the paper's tensors), with the sum taken in col_idx order and
 * one division, so that an implementation that keeps that order reproduces it exactly.
 */
typedef struct {
    int32_t n;
    const int32_t *row_ptr, *col_idx;
    const float *h0;      /* [R][n] */
    int32_t R, T;
    float eps;
    float *h_out;         /* [R][n] */
    uint64_t *changes;    /* [T+1]: (node, realization) pairs whose opinion changed at step k */
    int tid, nthreads;
    uint64_t *local;      /* thread-local [T+1] */
} orc_hk_job;

static void *hk_worker(void *arg)
{
    orc_hk_job *jb = (orc_hk_job *)arg;
    const int32_t n = jb->n;
    float *X = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float *Y = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int32_t r = jb->tid; r < jb->R; r += jb->nthreads) {
        memcpy(X, jb->h0 + (size_t)r * n, sizeof(float) * (size_t)n);
        for (int32_t k = 1; k <= jb->T; ++k) {
            uint64_t ch = 0;
            for (int32_t i = 0; i < n; ++i) {
                const float hi = X[i];
                float sum = 0.0f;
                int32_t cnt = 0;
                for (int32_t e = jb->row_ptr[i]; e < jb->row_ptr[i + 1]; ++e) {
                    const float hj = X[jb->col_idx[e]];
                    if (fabsf(hi - hj) < jb->eps) {
                        sum = sum + hj;
                        ++cnt;
                    }
                }
                Y[i] = cnt > 0 ? sum / (float)cnt : hi;
                if (Y[i] != hi) ++ch;
            }
            float *tmp = X; X = Y; Y = tmp;
            jb->local[k] += ch;
        }
        memcpy(jb->h_out + (size_t)r * n, X, sizeof(float) * (size_t)n);
    }
    free(X);
    free(Y);
    return NULL;
}

/* Returns 0, -1 (bad arguments: eps negative or not finite, an opinion not finite), or
 * -2 (allocation). */
int orc_hk(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const float *h0, int32_t R, int32_t T,
           float eps, float *h_out, uint64_t *changes, int nthreads)
{
    if (n < 0 || R < 0 || T < 0 || !h0 || !h_out || !changes) return -1;
    if (!(eps >= 0.0f) || isinf(eps)) return -1;
    for (int64_t i = 0; i < (int64_t)R * n; ++i)
        if (!(h0[i] == h0[i]) || isinf(h0[i])) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > R && R > 0) nthreads = R;
    memset(changes, 0, sizeof(uint64_t) * (size_t)(T + 1));
    orc_hk_job *jobs = (orc_hk_job *)calloc((size_t)nthreads, sizeof(orc_hk_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    int rc = 0;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = (orc_hk_job){n, row_ptr, col_idx, h0, R, T, eps, h_out, changes, i, nthreads, NULL};
        jobs[i].local = (uint64_t *)calloc((size_t)T + 1, sizeof(uint64_t));
        if (!jobs[i].local) rc = -2;
    }
    if (rc == 0) {
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, hk_worker, &jobs[i]);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        for (int i = 0; i < nthreads; ++i)
            for (int32_t k = 0; k <= T; ++k) changes[k] += jobs[i].local[k];
    }
    for (int i = 0; i < nthreads; ++i) free(jobs[i].local);
    free(jobs);
    free(th);
    return rc;
}

