// C ABI of the threshold sieve over a stream (include/ebc.h:
// ebc_sieve_host, ebc_threshold_ladder): the decision rule of the streaming
// optimisers the paper names beside Greedy (Sec. 2 and Sec. 4.1: Sieve
// Streaming; Three Sieves, which the case study of Sec. 6 runs), driven from
// the host over the bulk bound, exact gain and m_v update kernels.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.cuh"

using namespace ebc::hx;

namespace {

constexpr int kSieveExact = 64;  // items per exact-gain launch

// Scratch of one ebc_sieve_host call (stream-ordered pool memory), freed
// on every return path.
struct SieveBufs {
    cudaStream_t stream = nullptr;
    int32_t *list = nullptr;                // [bcap] unselected items of the batch
    int *cnt = nullptr;                     // [2] device list counts (bounds list, exact list)
    double *ub = nullptr;                   // [bcap] upper bounds of the gains
    double *lo = nullptr;                   // [bcap] FP32 path: lower bounds (not used by the rule)
    double *plo = nullptr, *phi = nullptr;  // FP32 path: [bcap * nchunks] chunk partials
    int32_t *xlist = nullptr;               // [kSieveExact] items given the exact gain
    double *xpart = nullptr;                // [kSieveExact * nchunks]
    double *xg = nullptr;                   // [kSieveExact]
    ~SieveBufs() {
        void *ptrs[] = {list, cnt, ub, lo, plo, phi, xlist, xpart, xg};
        for (void *q : ptrs) ebc::pool_free(q, stream);
    }
};

}  // namespace

extern "C" {

ebc_status ebc_threshold_ladder(double m, int32_t K, double eps, double upper, double *out, int32_t cap,
                                int32_t *count) {
    if (!count || !(m > 0.0) || !std::isfinite(m) || !(eps > 0.0) || !std::isfinite(eps) || K < 1 ||
        !(upper > 0.0) || !std::isfinite(upper) || cap < 0 || (cap > 0 && !out))
        return EBC_EINVAL;
    const double base = 1.0 + eps;
    const double top = upper * K * m;
    if (!(base > 1.0) || !std::isfinite(top)) return EBC_EINVAL;
    // smallest i with base^i >= m, then every i up to base^i <= top
    int64_t i = (int64_t)floor(log(m) / log(base)) - 2;
    while (pow(base, (double)i) < m) ++i;
    int64_t lo_i = i, cnt = 0;
    while (pow(base, (double)i) <= top) {
        ++i;
        if (++cnt > 1000000) return EBC_EINVAL;
    }
    *count = (int32_t)cnt;
    if (cap == 0 && !out) return EBC_OK;
    if (cap < cnt) return EBC_EINVAL;
    for (int64_t j = 0; j < cnt; ++j) out[j] = pow(base, (double)(lo_i + cnt - 1 - j));
    return EBC_OK;
}

ebc_status ebc_sieve_host(ebc_t h, ebc_sieve_state *s, const int32_t *items, int64_t len, int32_t *out_idx,
                          double *out_f, int32_t *out_count) {
    ebc::TraceRange trace_("ebc_sieve_host");
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (!s || !out_count) return fail(h, EBC_EINVAL, "ebc_sieve_host: NULL state or count");
    if (len < 0 || (len > 0 && !items)) return fail(h, EBC_EINVAL, "ebc_sieve_host: bad stream");
    if (s->nthr < 1 || !s->thr) return fail(h, EBC_EINVAL, "ebc_sieve_host: no thresholds");
    for (int32_t j = 0; j < s->nthr; ++j)
        if (!std::isfinite(s->thr[j])) return fail(h, EBC_EINVAL, "ebc_sieve_host: non-finite threshold");
    if (s->level < 0 || s->level >= s->nthr || s->rejections < 0)
        return fail(h, EBC_EINVAL, "ebc_sieve_host: level or rejections out of range");
    if ((int64_t)s->K < h->nsel || (int64_t)s->K > c.n) return fail(h, EBC_EINVAL, "ebc_sieve_host: K outside [|S|, n]");
    const int64_t room = (int64_t)s->K - h->nsel;
    if (room > 0 && (!out_idx || !out_f)) return fail(h, EBC_EINVAL, "ebc_sieve_host: NULL output");
    for (int64_t p = 0; p < len; ++p)
        if (items[p] < 0 || (int64_t)items[p] >= c.n) return fail(h, EBC_EINDEX, "ebc_sieve_host: item outside [0, n)");
    *out_count = 0;
    s->consumed = 0;
    if (len == 0 || room == 0) return EBC_OK;
    if (ebc_status s0 = ebc_sync(h)) return s0;

    // host mirrors of S and f(S)
    std::vector<uint8_t> sel((size_t)c.n);
    double f = 0.0;
    CK(h, cudaMemcpyAsync(sel.data(), c.sel, (size_t)c.n, cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaMemcpyAsync(&f, &c.st->f, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaStreamSynchronize(c.stream));

    const bool tc = c.prec != EBC_FP32;  // tensor-core bounds (FP8 certifies with its BF16 copy)
    const int64_t bmin = tc ? 256 : 64;
    const int64_t bcap = std::min<int64_t>(c.n, tc ? 32768 : 1024);
    const int nchunks = c.cert.nchunks;
    SieveBufs B;
    B.stream = c.stream;
    CK(h, dalloc(&B.list, (size_t)bcap, c));
    CK(h, dalloc(&B.cnt, 2, c));
    CK(h, dalloc(&B.ub, (size_t)bcap, c));
    CK(h, dalloc(&B.xlist, kSieveExact, c));
    CK(h, dalloc(&B.xpart, (size_t)kSieveExact * nchunks, c));
    CK(h, dalloc(&B.xg, kSieveExact, c));
    if (!tc) {
        CK(h, dalloc(&B.lo, (size_t)bcap, c));
        CK(h, dalloc(&B.plo, (size_t)bcap * nchunks, c));
        CK(h, dalloc(&B.phi, (size_t)bcap * nchunks, c));
    }
    const double eta = bulk_eta(c);
    const double *thr = s->thr;
    const int32_t nthr = s->nthr, K = s->K;
    const int64_t patience = s->patience;
    int32_t level = s->level;
    int64_t rej = s->rejections;
    int64_t nsel = h->nsel;
    int32_t cnt = 0;

    // upper bounds of every point's gain, valid while S only grows (kept by
    // the handle across calls; diminishing returns, Def. 3): an item whose
    // bound is below its tau is rejected without device work
    std::vector<double> &ub = h->sieve_ub;
    if ((int64_t)ub.size() != c.n) ub.assign((size_t)c.n, INFINITY);
    if (s->bounds)
        for (int64_t i = 0; i < c.n; ++i) ub[(size_t)i] = std::min(ub[(size_t)i], s->bounds[i]);

    struct Maybe {
        int64_t pos;  // stream position
        double tau;
        int32_t level;
    };
    std::vector<Maybe> U, X;  // positions whose cached bound reaches tau; then those still needing the exact gain
    std::vector<int32_t> hl, xl;
    std::vector<double> hub, xg;

    // batch: up to bsz items to bound within a walk of at most wlen stream
    // positions; both grow while nothing is accepted and restart from the
    // distance to the last acceptance (a walk after an acceptance revisits
    // the positions behind it with the new tau)
    int64_t p = 0, bsz = bmin, wlen = 4096;
    while (p < len && nsel < K) {
        // walk from p as if every item were rejected (the state up to the
        // first acceptance), collecting the positions whose bound reaches
        // their tau
        U.clear();
        int32_t lev = level;
        int64_t r = rej, q = p;
        for (; q < len && (int64_t)U.size() < bsz && q - p < wlen; ++q) {
            const int32_t e = items[q];
            if (!sel[(size_t)e]) {
                const double tau = (thr[lev] / 2.0 - f) / (double)((int64_t)K - nsel);
                if (!(ub[(size_t)e] < tau)) U.push_back({q, tau, lev});
            }
            r += 1;
            if (patience > 0 && r >= patience) {
                if (lev + 1 < nthr) lev += 1;
                r = 0;
            }
        }
        // level 1: fresh bulk upper bounds of those items
        X.clear();
        if (!U.empty()) {
            const int64_t nl = (int64_t)U.size();
            hl.resize((size_t)nl);
            for (int64_t i = 0; i < nl; ++i) hl[(size_t)i] = items[U[(size_t)i].pos];
            hub.resize((size_t)nl);
            CK(h, cudaMemcpyAsync(B.list, hl.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, c.stream));
            if (tc) {
                int nch = h->nch;
                CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc(c, true); }));
                CK(h, launch(h, PK_LIST, 2, [&] { return ebc::launch_gains_tc(c, B.list, nl, true, &nch); }));
                CK(h, launch(h, -1, 1, [&] {
                       return ebc::launch_reduce_select(c, nl, nch, B.list, false, B.ub, h->nblk);
                   }));
            } else {
                const int n32 = (int)nl;
                CK(h, cudaMemcpyAsync(B.cnt, &n32, sizeof(int), cudaMemcpyHostToDevice, c.stream));
                CK(h, launch(h, PK_LIST, 2, [&] {
                       return ebc::launch_bounds_list(c, B.list, B.cnt, (int)nl, B.plo, B.phi, c.cert.chunk, nchunks);
                   }));
                CK(h, launch(h, -1, 1, [&] {
                       return ebc::launch_fold_bounds(c, B.plo, B.phi, B.cnt, (int)nl, B.lo, B.ub);
                   }));
            }
            CK(h, cudaMemcpyAsync(hub.data(), B.ub, sizeof(double) * nl, cudaMemcpyDeviceToHost, c.stream));
            CK(h, cudaStreamSynchronize(c.stream));
            s->bounded += nl;
            for (int64_t i = 0; i < nl; ++i) {
                // rigorous: TC partial sums carry relative error <= eta
                const double b = tc ? hub[(size_t)i] * (1.0 + eta) : hub[(size_t)i];
                double &u = ub[(size_t)hl[(size_t)i]];
                u = std::min(u, b);
                if (!(u < U[(size_t)i].tau)) X.push_back(U[(size_t)i]);
            }
        }
        // level 2: exact gains of the items still undecided, in stream
        // order, up to the first that reaches its tau; groups of 8, 16, ...
        // kSieveExact (one pass over V serves 8 items, and the first
        // candidates usually decide)
        int64_t acc = -1;
        double acc_g = 0.0;
        int32_t acc_lev = level;
        size_t group = 8;
        for (size_t u0 = 0; u0 < X.size() && acc < 0; u0 += group, group = std::min<size_t>(2 * group, kSieveExact)) {
            const int ng = (int)std::min<size_t>(group, X.size() - u0);
            xl.resize((size_t)ng);
            for (int j = 0; j < ng; ++j) xl[(size_t)j] = items[X[u0 + j].pos];
            CK(h, cudaMemcpyAsync(B.xlist, xl.data(), sizeof(int32_t) * ng, cudaMemcpyHostToDevice, c.stream));
            CK(h, cudaMemcpyAsync(B.cnt + 1, &ng, sizeof(int), cudaMemcpyHostToDevice, c.stream));
            CK(h, launch(h, PK_REFINE, 1, [&] {
                   return ebc::launch_exact_list(c, B.xlist, B.cnt + 1, kSieveExact, B.xpart, c.cert.chunk, nchunks);
               }));
            CK(h, launch(h, -1, 1, [&] { return ebc::launch_sieve_fold_exact(c, B.xpart, B.cnt + 1, kSieveExact, B.xg); }));
            xg.resize((size_t)ng);
            CK(h, cudaMemcpyAsync(xg.data(), B.xg, sizeof(double) * ng, cudaMemcpyDeviceToHost, c.stream));
            CK(h, cudaStreamSynchronize(c.stream));
            s->exact += ng;
            for (int j = 0; j < ng; ++j)
                if (xg[(size_t)j] >= X[u0 + j].tau) {
                    acc = X[u0 + j].pos;
                    acc_g = xg[(size_t)j];
                    acc_lev = X[u0 + j].level;
                    break;
                }
        }
        if (acc < 0) {  // every walked position is a rejection
            level = lev;
            rej = r;
            s->consumed += q - p;
            p = q;
            bsz = std::min(bcap, 2 * bsz);
            wlen = std::min<int64_t>(len, 2 * wlen);
            continue;
        }
        const int32_t item = items[acc];
        CK(h, launch(h, -1, 2, [&] {
               cudaError_t e = ebc::launch_sieve_commit(c, item, acc_g);
               return e != cudaSuccess ? e : ebc::launch_update(c);
           }));
        sel[(size_t)item] = 1;
        ub[(size_t)item] = 0.0;
        f += acc_g;  // the device adds the same double to the same f
        nsel += 1;
        h->nsel = nsel;
        out_idx[cnt] = item;
        out_f[cnt] = f;
        cnt += 1;
        level = acc_lev;
        rej = 0;
        int64_t ua = 0;  // items bounded in this walk up to the accepted one
        while (ua < (int64_t)U.size() && U[(size_t)ua].pos <= acc) ++ua;
        s->consumed += acc + 1 - p;
        bsz = std::min(bcap, std::max(bmin, 2 * ua));
        wlen = std::max<int64_t>(4096, 2 * (acc + 1 - p));
        p = acc + 1;
    }
    s->level = level;
    s->rejections = rej;
    *out_count = cnt;
    return ebc_sync(h);
}

}  // extern "C"
