/*
 * CPU oracle for exemplar-based clustering (EBC).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the GPU library computes.  It is used by the test suite,
 * by the smoke check and by the benchmark's CPU-baseline leg, and by nothing
 * else.  It shares no code, header, table or helper with the CUDA path.
 *
 * Definitions followed (paper sections):
 *   - dissimilarity d(x, y) = ||x - y||^2, squared Euclidean (Sec. 5, setup);
 *   - k-medoids loss L(S) = |V|^-1 sum_{v in V} min_{s in S} d(v, s)
 *     (Sec. 4, Eq. "k-medoids loss");
 *   - EBC f(S) = L({e0}) - L(S u {e0}) with e0 the all-zero vector
 *     (Sec. 4, Eq. "exemplar-based clustering");
 *   - Algorithm 1 (EBC on the CPU): running minimum over the set, sum over V,
 *     scale by 1/|V|, return the difference of the two losses;
 *   - discrete derivative Delta_f(e|S) = f(S u {e}) - f(S) (Sec. 3, Def. 1);
 *   - Greedy: each step adds the not-yet-selected item of largest marginal
 *     gain (Sec. 3 and Sec. 4.1);
 *   - the threshold sieve of the streaming optimisers the paper names
 *     (Sec. 2, Sec. 4.1, Fig. 4): accept a streamed item when its marginal
 *     gain reaches (v/2 - f(S)) / (K - |S|).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - e0 is fixed to the zero vector;
 *   - Algorithm 1's FLT_MAX start becomes DBL_MAX because the oracle is FP64;
 *   - Greedy breaks equal gains toward the smallest index and keeps picking
 *     (gain 0) when every remaining gain is 0; k > n - |S| is an error;
 *   - "form B" f(S) = |V|^-1 sum_v max(0, ||v||^2 - min_{s in S} d(v, s)) is
 *     the same quantity as Algorithm 1 by algebra (min over S u {e0} equals
 *     min(||v||^2, min over S)); both forms are provided so tests can check
 *     one against the other.
 *
 * Arithmetic: every input is an FP32 array, widened exactly to double.  All
 * distances are computed directly as sum_i (x_i - y_i)^2 in double, never via
 * the norm expansion.  Sums over V use Neumaier's compensated summation
 * (Neumaier 1974).  Build with -ffp-contract=off so the compiler keeps the
 * written operation order.  OpenMP threads split work over candidates or sets
 * only; every per-candidate / per-set sum is serial, so results do not depend
 * on the thread count.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_EINDEX (-2)
#define ORC_ENOMEM (-3)

/* ---- compensated sum (Neumaier 1974) ---------------------------------- */
typedef struct {
    double s;
    double c;
} orc_sum;

static void orc_sum_add(orc_sum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double orc_sum_get(const orc_sum *a) { return a->s + a->c; }

/* ---- the dissimilarity: squared Euclidean, direct ---------------------- */
double orc_sqdist(const float *x, const float *y, int32_t d) {
    double acc = 0.0;
    for (int32_t i = 0; i < d; ++i) {
        double diff = (double)x[i] - (double)y[i];
        acc += diff * diff;
    }
    return acc;
}

/* d(v, e0) with e0 = 0 */
static double orc_sqdist_e0(const float *x, int32_t d) {
    double acc = 0.0;
    for (int32_t i = 0; i < d; ++i) {
        double xi = (double)x[i];
        acc += xi * xi;
    }
    return acc;
}

static const float *row(const float *V, int64_t i, int32_t d) { return V + (size_t)i * (size_t)d; }

static int check_idx(const int32_t *S, int64_t s, int64_t n) {
    for (int64_t j = 0; j < s; ++j)
        if (S[j] < 0 || (int64_t)S[j] >= n) return ORC_EINDEX;
    return ORC_OK;
}

/*
 * k-medoids loss of Algorithm 1, L(V, S u {e0}) when with_e0 != 0, else
 * L(V, S).  t starts at the largest double (Algorithm 1 starts at FLT_MAX)
 * and is lowered by every exemplar in turn; an empty S without e0 therefore
 * has loss DBL_MAX, as the algorithm as written would return.
 */
double orc_loss(const float *V, int64_t n, int32_t d, const int32_t *S, int64_t s, int with_e0) {
    if (n <= 0) return 0.0;
    orc_sum sigma = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        const float *v = row(V, i, d);
        double t = DBL_MAX;
        if (with_e0) {
            double de0 = orc_sqdist_e0(v, d);
            if (de0 < t) t = de0;
        }
        for (int64_t j = 0; j < s; ++j) {
            double dj = orc_sqdist(row(V, S[j], d), v, d);
            if (dj < t) t = dj;
        }
        if (t == DBL_MAX) return DBL_MAX;
        orc_sum_add(&sigma, t);
    }
    return orc_sum_get(&sigma) / (double)n;
}

/* Form A: Algorithm 1 as written, f(S) = L({e0}) - L(S u {e0}). */
int orc_f_alg1(const float *V, int64_t n, int32_t d, const int32_t *S, int64_t s, double *out) {
    if (n < 0 || d <= 0 || s < 0) return ORC_EINVAL;
    if (check_idx(S, s, n)) return ORC_EINDEX;
    double l0 = orc_loss(V, n, d, NULL, 0, 1);
    double ls = orc_loss(V, n, d, S, s, 1);
    *out = l0 - ls;
    return ORC_OK;
}

/* Form B: f(S) = (1/n) sum_v max(0, ||v||^2 - min_{s in S} d(v, s)). */
static double f_relu_one(const float *V, int64_t n, int32_t d, const int32_t *S, int64_t s) {
    if (n <= 0) return 0.0;
    orc_sum acc = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        const float *v = row(V, i, d);
        double nv = orc_sqdist_e0(v, d);
        double t = DBL_MAX;
        for (int64_t j = 0; j < s; ++j) {
            double dj = orc_sqdist(row(V, S[j], d), v, d);
            if (dj < t) t = dj;
        }
        double gain = nv - t;
        if (gain > 0.0) orc_sum_add(&acc, gain);
    }
    return orc_sum_get(&acc) / (double)n;
}

int orc_f(const float *V, int64_t n, int32_t d, const int32_t *S, int64_t s, double *out) {
    if (n < 0 || d <= 0 || s < 0) return ORC_EINVAL;
    if (check_idx(S, s, n)) return ORC_EINDEX;
    *out = f_relu_one(V, n, d, S, s);
    return ORC_OK;
}

/* f(S_j) for every set of a CSR list (the multi-set S_multi of Sec. 4.1). */
int orc_eval_sets(const float *V, int64_t n, int32_t d, const int32_t *idx, const int64_t *off, int64_t l,
                  double *out_f, int nthreads) {
    if (n < 0 || d <= 0 || l < 0) return ORC_EINVAL;
    if (l > 0 && off[0] != 0) return ORC_EINVAL;
    for (int64_t j = 0; j < l; ++j)
        if (off[j + 1] < off[j]) return ORC_EINVAL;
    if (l > 0 && check_idx(idx, off[l], n)) return ORC_EINDEX;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t j = 0; j < l; ++j) out_f[j] = f_relu_one(V, n, d, idx + off[j], off[j + 1] - off[j]);
    (void)nthreads;
    return ORC_OK;
}

/* ||v||^2 for every ground point: the distance to e0. */
void orc_norms(const float *V, int64_t n, int32_t d, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_sqdist_e0(row(V, i, d), d);
}

/*
 * Marginal gain of candidate c given the current per-point minima m_v
 * (m_v = min over S u {e0} of d(v, s)):
 *   Delta_f(c | S) = (1/n) sum_v max(0, m_v - d(v, c)).
 * This is f(S u {c}) - f(S) by Def. 1, because adding c lowers the minimum of
 * point v from m_v to min(m_v, d(v, c)).
 */
static double gain_one(const float *V, int64_t n, int32_t d, const double *m, int64_t c) {
    orc_sum acc = {0.0, 0.0};
    const float *cv = row(V, c, d);
    for (int64_t i = 0; i < n; ++i) {
        double g = m[i] - orc_sqdist(row(V, i, d), cv, d);
        if (g > 0.0) orc_sum_add(&acc, g);
    }
    return orc_sum_get(&acc) / (double)n;
}

int orc_gains(const float *V, int64_t n, int32_t d, const double *m, const int32_t *cand, int64_t mc,
              double *out, int nthreads) {
    if (n <= 0 || d <= 0 || mc < 0) return ORC_EINVAL;
    if (check_idx(cand, mc, n)) return ORC_EINDEX;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t j = 0; j < mc; ++j) out[j] = gain_one(V, n, d, m, cand[j]);
    (void)nthreads;
    return ORC_OK;
}

/* m_v <- min(m_v, d(v, c)) : the minimum after adding c to S. */
int orc_update_m(const float *V, int64_t n, int32_t d, double *m, int32_t c) {
    if (c < 0 || (int64_t)c >= n) return ORC_EINDEX;
    const float *cv = row(V, c, d);
    for (int64_t i = 0; i < n; ++i) {
        double dc = orc_sqdist(row(V, i, d), cv, d);
        if (dc < m[i]) m[i] = dc;
    }
    return ORC_OK;
}

/*
 * Greedy (Sec. 3; Sec. 4.1 describes the step): start from S = {} (m_v =
 * ||v||^2), then k times add argmax over unselected c of Delta_f(c | S),
 * ties to the smallest index.  out_f[t] = f(S_{t+1}) accumulated as the sum
 * of the picked gains (the telescoping sum of discrete derivatives).
 * out_gap[t] = (g1 - g2) / g1, the relative gap between the best and the
 * second-best gain of the step; 0 when g1 == 0, 1 when a single candidate
 * with positive gain remains.
 * m_io (length n) is the per-point minimum and sel_io (length n) marks the
 * points already in S; pass NULL for both to start from S = {}.  When given
 * they are updated in place, so greedy can be continued.  f_start is f(S) of
 * the starting state (0 for S = {}).
 */
int orc_greedy(const float *V, int64_t n, int32_t d, int32_t k, int32_t *out_idx, double *out_f,
               double *out_gap, double *m_io, unsigned char *sel_io, double f_start, int nthreads) {
    if (n <= 0 || d <= 0 || k < 0 || (int64_t)k > n) return ORC_EINVAL;
    if ((m_io == NULL) != (sel_io == NULL)) return ORC_EINVAL;
    double *m = m_io;
    double *g = (double *)malloc(sizeof(double) * (size_t)n);
    unsigned char *sel = sel_io ? sel_io : (unsigned char *)calloc((size_t)n, 1);
    double *mown = NULL;
    if (!m) {
        mown = (double *)malloc(sizeof(double) * (size_t)n);
        m = mown;
        if (m) orc_norms(V, n, d, m);
    }
    if (!g || !sel || !m) {
        free(g);
        if (!sel_io) free(sel);
        free(mown);
        return ORC_ENOMEM;
    }
    int64_t remaining = 0;
    for (int64_t c = 0; c < n; ++c) remaining += sel[c] ? 0 : 1;
    if ((int64_t)k > remaining) {
        free(g);
        if (!sel_io) free(sel);
        free(mown);
        return ORC_EINVAL;
    }
    double f = f_start;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int32_t t = 0; t < k; ++t) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
        for (int64_t c = 0; c < n; ++c) g[c] = sel[c] ? -1.0 : gain_one(V, n, d, m, c);
        int64_t best = -1;
        double g1 = -1.0, g2 = -1.0;
        for (int64_t c = 0; c < n; ++c) {
            if (sel[c]) continue;
            if (g[c] > g1) {
                g2 = g1;
                g1 = g[c];
                best = c;
            } else if (g[c] > g2) {
                g2 = g[c];
            }
        }
        if (best < 0) break;
        sel[best] = 1;
        orc_update_m(V, n, d, m, (int32_t)best);
        f += g1;
        out_idx[t] = (int32_t)best;
        out_f[t] = f;
        if (out_gap) {
            /* a lone remaining candidate with positive gain is a forced pick: gap 1 */
            if (g1 <= 0.0)
                out_gap[t] = 0.0;
            else
                out_gap[t] = (g2 >= 0.0) ? (g1 - g2) / g1 : 1.0;
        }
    }
    free(g);
    if (!sel_io) free(sel);
    free(mown);
    (void)nthreads;
    return ORC_OK;
}

/* Exhaustive optimum of max_{|S| <= k} f(S) (Sec. 3, cardinality-constrained
 * problem) by enumerating every subset of size exactly k (f is monotone, so
 * the optimum has size k when k <= n).  Tiny n only. */
int orc_exhaustive_opt(const float *V, int64_t n, int32_t d, int32_t k, double *out_f, int32_t *out_set) {
    if (n <= 0 || n > 24 || k < 0 || k > n) return ORC_EINVAL;
    int32_t S[24];
    double best = -1.0;
    for (uint32_t mask = 0; mask < (1u << n); ++mask) {
        if (__builtin_popcount(mask) != k) continue;
        int64_t s = 0;
        for (int64_t i = 0; i < n; ++i)
            if (mask & (1u << i)) S[s++] = (int32_t)i;
        double v = f_relu_one(V, n, d, S, s);
        if (v > best) {
            best = v;
            if (out_set) memcpy(out_set, S, sizeof(int32_t) * (size_t)k);
        }
    }
    *out_f = best;
    return ORC_OK;
}

/*
 * Threshold sieve over a stream: the decision rule shared by the streaming
 * optimisers the paper names next to Greedy (Sec. 2 and Sec. 4.1: Sieve
 * Streaming, Badanidiyuru et al. 2014; Three Sieves, Buschjaeger et al.,
 * which the case study of Sec. 6 runs, Fig. 4), written from their
 * published descriptions.  Items arrive in stream order;
 * with s = |S| < K, threshold v = thr[level] and
 *     tau = (v / 2 - f(S)) / (K - s),
 * an item e not in S joins S when Delta_f(e | S) >= tau.  An item in S, or
 * one whose gain is below tau, is a rejection.  After `patience` consecutive
 * rejections the sieve moves to the next threshold (level + 1, staying on
 * the last one) and the count restarts; patience <= 0 never moves (one
 * fixed threshold: one sieve of Sieve Streaming).  Once |S| = K the rest of
 * the stream is ignored.
 *
 * State in / out (so a stream can be fed in pieces): m_io, sel_io (length
 * n, as orc_greedy), f_io = f(S), level_io, rej_io.  Outputs: out_idx /
 * out_f (accepted items and f after each; capacity K), out_count, and
 * out_margin[p] for every stream position p that was decided: |gain - tau|
 * / max(|gain|, |tau|) (1 for items already in S, 0 when both are 0), the
 * relative distance of the decision from a tie.
 */
int orc_sieve(const float *V, int64_t n, int32_t d, const int32_t *items, int64_t len, int32_t K,
              const double *thr, int32_t nthr, int64_t patience, double *m, unsigned char *sel, double *f_io,
              int32_t *level_io, int64_t *rej_io, int32_t *out_idx, double *out_f, double *out_margin,
              int32_t *out_count) {
    if (n <= 0 || d <= 0 || len < 0 || K < 0 || (int64_t)K > n || nthr < 1 || !thr || !m || !sel || !f_io ||
        !level_io || !rej_io || !out_count)
        return ORC_EINVAL;
    if (*level_io < 0 || *level_io >= nthr || *rej_io < 0) return ORC_EINVAL;
    if (check_idx(items, len, n)) return ORC_EINDEX;
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) s += sel[i] ? 1 : 0;
    if (s > (int64_t)K) return ORC_EINVAL;
    double f = *f_io;
    int32_t level = *level_io;
    int64_t rej = *rej_io;
    int32_t cnt = 0;
    for (int64_t p = 0; p < len && s < (int64_t)K; ++p) {
        const int32_t e = items[p];
        int accept = 0;
        double margin = 1.0;
        if (!sel[e]) {
            const double tau = (thr[level] / 2.0 - f) / (double)((int64_t)K - s);
            const double g = gain_one(V, n, d, m, e);
            const double scale = fmax(fabs(g), fabs(tau));
            margin = scale > 0.0 ? fabs(g - tau) / scale : 0.0;
            accept = g >= tau;
            if (accept) {
                sel[e] = 1;
                orc_update_m(V, n, d, m, e);
                f += g;
                s += 1;
                out_idx[cnt] = e;
                out_f[cnt] = f;
                cnt += 1;
                rej = 0;
            }
        }
        if (out_margin) out_margin[p] = margin;
        if (!accept) {
            rej += 1;
            if (patience > 0 && rej >= patience) {
                if (level + 1 < nthr) level += 1;
                rej = 0;
            }
        }
    }
    *f_io = f;
    *level_io = level;
    *rej_io = rej;
    *out_count = cnt;
    return ORC_OK;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
