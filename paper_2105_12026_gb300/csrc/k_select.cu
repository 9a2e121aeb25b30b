// Certified pick of a Greedy round (Sec. 3: add the unselected point of
// largest marginal gain; ties to the smallest index), in two levels.
//
// The bulk kernel gives every candidate c an upper bound U_c of its gain
// (exact up to the relative error eta_bulk of its FP32 partial sums).
//  1. The K largest U_c form the top list.  For each, FP32 direct distances
//     give rigorous bounds lo_c <= gain(c) <= hi_c (relative width ~1e-5).
//  2. best_lo = max lo over the list.  If the (K+1)-th bound can reach it,
//     every candidate with U_c (1 + eta_bulk) >= best_lo joins the pool
//     (escalation) and gets bounds the same way.
//  3. Contenders = pool entries with hi >= best_lo (usually one or two).
//     Only these get the exact gain (FP64 direct distances).
//  4. The pick is the contender of largest exact gain, the smallest index
//     among the contenders within kTieRel of it (ties).  Any other candidate
//     has gain <= hi < best_lo (1 - 2 kTieRel) <= the exact gain of the entry
//     attaining best_lo, itself a contender: the pick is the exact argmax, and
//     every candidate tied with it is a contender.
// When every remaining gain is exactly 0 the pick is the smallest
// unselected index.
#include "ebc_internal.cuh"
#include "sel_util.cuh"

namespace ebc {

namespace {
// Relative widening of the folded bounds.  Each bound term is one FP32
// rounding from its exact value; the bound kernels add terms of one sign in
// FP32 along chains of at most 128 additions (k_bounds_fp32: 8 per thread,
// 16 lanes, then up to 16 point tiles, depth 28; the few-candidate kernels:
// 64 terms) before the FP64 sums, so the relative error is at most
// 130 * 2^-24 plus the FP64 part.
double fold_eta(int64_t chunk) {
    (void)chunk;
    return 131.0 * ldexp(1.0, -24) + 1e-12;
}
}  // namespace

// lo[e] / hi[e] = (sum over chunks of the partials) / n, widened by eta.
// One warp per entry, lane-strided partial sums, then a fixed tree.
__global__ void k_fold_bounds(const double *__restrict__ part_lo, const double *__restrict__ part_hi, int nchunks,
                              const int *__restrict__ count, int cap, double inv_n, double eta,
                              double *__restrict__ lo, double *__restrict__ hi) {
    const int cnt = min(*count, cap);
    const int lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    for (int e = blockIdx.x * nw + (threadIdx.x >> 5); e < cnt; e += gridDim.x * nw) {
        double sl = 0.0, sh = 0.0;
        for (int q = lane; q < nchunks; q += 32) {
            sl += part_lo[(int64_t)e * nchunks + q];
            sh += part_hi[(int64_t)e * nchunks + q];
        }
        for (int o = 16; o > 0; o >>= 1) {
            sl += __shfl_xor_sync(0xffffffffu, sl, o);
            sh += __shfl_xor_sync(0xffffffffu, sh, o);
        }
        if (lane == 0) {
            lo[e] = sl * inv_n * (1.0 - eta);
            hi[e] = sh * inv_n * (1.0 + eta);
        }
    }
}

cudaError_t launch_fold_bounds(Ctx &c, const double *part_lo, const double *part_hi, const int *count, int cap,
                               double *lo, double *hi) {
    const int blocks = (int)lmin((cap + 7) / 8, (int64_t)c.num_sms * 2);
    k_fold_bounds<<<blocks, 256, 0, c.stream>>>(part_lo, part_hi, c.cert.nchunks, count, cap, 1.0 / (double)c.n,
                                                fold_eta(c.cert.chunk), lo, hi);
    return cudaGetLastError();
}

// Level 1 on the top list: best certified lower bound and whether any
// candidate outside the list could reach it.
__global__ void k_decide_top(const double *__restrict__ top_lo, const int *__restrict__ top_idx,
                             const double *__restrict__ top_val, double eta_bulk, DevState *st) {
    if (threadIdx.x != 0) return;
    const int cnt = st->top_count;
    double best_lo = 0.0;
    double maxerr = st->max_raw_rel_err;
    for (int e = 0; e < cnt; ++e) {
        best_lo = fmax(best_lo, top_lo[e]);
        if (top_lo[e] > 0.0) maxerr = fmax(maxerr, (top_val[e] - top_lo[e]) / top_lo[e]);
    }
    (void)top_idx;
    st->max_raw_rel_err = maxerr;
    const double thr = st->top_thr;  // (K+1)-th bulk bound, -1 when no other candidate
    // outside candidates have gain <= U (1 + eta_bulk) <= thr (1 + eta_bulk); a
    // zero bound means a zero gain, which can only matter for the all-zero case
    const double tie_lo = best_lo * (1.0 - 2.0 * kTieRel);
    st->need_esc = (thr > 0.0 && thr * (1.0 + eta_bulk) >= tie_lo) ? 1 : 0;
    st->esc_thr = tie_lo;
    st->best_lo = best_lo;
    st->esc_count = 0;
    st->ctd_count = 0;
    st->zero_scan = 0;
}

cudaError_t launch_decide_top(Ctx &c, double eta_bulk) {
    k_decide_top<<<1, 32, 0, c.stream>>>(c.cert.top_lo, c.top_idx, c.top_val, eta_bulk, c.st);
    return cudaGetLastError();
}

// Level 2: final best lower bound over the whole pool and the contenders.
__global__ void k_decide_contenders(const double *__restrict__ top_hi, const double *__restrict__ top_lo,
                                    const int *__restrict__ top_idx, const double *__restrict__ esc_lo,
                                    const double *__restrict__ esc_hi, const double *__restrict__ esc_exact,
                                    const int *__restrict__ esc_idx, int cap, DevState *st,
                                    int *__restrict__ ctd_idx) {
    __shared__ double sbest[32];
    __shared__ int sn;
    const int top_cnt = st->top_count;
    const int esc_cnt = st->need_esc ? st->esc_count : 0;
    const int in_cap = min(esc_cnt, cap);
    double b = 0.0;
    for (int e = threadIdx.x; e < top_cnt; e += blockDim.x) b = fmax(b, top_lo[e]);
    for (int e = threadIdx.x; e < in_cap; e += blockDim.x) b = fmax(b, esc_lo[e]);
    for (int e = cap + threadIdx.x; e < esc_cnt; e += blockDim.x) b = fmax(b, esc_exact[e]);
    for (int o = 16; o > 0; o >>= 1) b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0) sbest[threadIdx.x >> 5] = b;
    if (threadIdx.x == 0) sn = 0;
    __syncthreads();
    double best_lo = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) best_lo = fmax(best_lo, sbest[w]);
    const double tie_lo = best_lo * (1.0 - 2.0 * kTieRel);
    for (int e = threadIdx.x; e < top_cnt; e += blockDim.x)
        if (top_hi[e] >= tie_lo) ctd_idx[atomicAdd(&sn, 1)] = top_idx[e];
    for (int e = threadIdx.x; e < in_cap; e += blockDim.x)
        if (esc_hi[e] >= tie_lo) ctd_idx[atomicAdd(&sn, 1)] = esc_idx[e];
    __syncthreads();
    if (threadIdx.x == 0) {
        st->best_lo = best_lo;
        st->ctd_count = sn;
    }
}

cudaError_t launch_decide_contenders(Ctx &c) {
    k_decide_contenders<<<1, 256, 0, c.stream>>>(c.cert.top_hi, c.cert.top_lo, c.top_idx, c.cert.esc_lo, c.cert.esc_hi,
                                                 c.esc_exact, c.esc_idx, c.cert.cap, c.st, c.cert.ctd_idx);
    return cudaGetLastError();
}

// Exact gains of the contenders (and of escalated entries past the chunked
// capacity, already exact), the pick, and the state update.
__global__ void k_commit_pick(const double *__restrict__ ctd_part, int nchunks, double inv_n,
                              const int *__restrict__ ctd_idx, double *__restrict__ ctd_exact,
                              const double *__restrict__ esc_exact, const int *__restrict__ esc_idx, int cap,
                              uint8_t *__restrict__ sel, int64_t n, int32_t *__restrict__ out_idx,
                              double *__restrict__ out_f, double *__restrict__ ub, DevState *st) {
    const int nc = st->ctd_count;
    const int esc_cnt = st->need_esc ? st->esc_count : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = w; e < nc; e += blockDim.x >> 5) {
        double s = 0.0;
        for (int q = lane; q < nchunks; q += 32) s += ctd_part[(int64_t)e * nchunks + q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) ctd_exact[e] = s * inv_n;
    }
    __syncthreads();
    // largest exact gain, then the smallest index among the entries within
    // kTieRel of it (the pick's own exact gain goes into f)
    double mv = -1.0;
    int mi = INT_MAX;
    for (int e = threadIdx.x; e < nc; e += blockDim.x)
        if (better(ctd_exact[e], ctd_idx[e], mv, mi)) {
            mv = ctd_exact[e];
            mi = ctd_idx[e];
        }
    for (int e = cap + threadIdx.x; e < esc_cnt; e += blockDim.x)
        if (better(esc_exact[e], esc_idx[e], mv, mi)) {
            mv = esc_exact[e];
            mi = esc_idx[e];
        }
    block_best(mv, mi);
    const double tie = mv * (1.0 - kTieRel);
    double bv = -1.0;
    int bi = INT_MAX;
    for (int e = threadIdx.x; e < nc; e += blockDim.x)
        if (ctd_exact[e] >= tie && ctd_idx[e] < bi) {
            bv = ctd_exact[e];
            bi = ctd_idx[e];
        }
    for (int e = cap + threadIdx.x; e < esc_cnt; e += blockDim.x)
        if (esc_exact[e] >= tie && esc_idx[e] < bi) {
            bv = esc_exact[e];
            bi = esc_idx[e];
        }
    block_min_index(bv, bi);
    // every remaining gain is 0 (no escalation, outside bounds 0): smallest unselected index
    const bool zero_scan = bv == 0.0 && st->top_thr >= 0.0 && !st->need_esc;
    if (zero_scan) {
        double zv = 0.0;
        int zi = INT_MAX;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
            if (!sel[j]) {
                zi = (int)j;
                break;
            }
        block_best(zv, zi);
        bi = zi;
    }
    if (threadIdx.x == 0) {
        if (bi == INT_MAX || bi < 0) {
            if (st->err == 0) st->err = (int)EBC_EINVAL;  // no candidate left (host checks prevent this)
            st->pick = -1;
            return;
        }
        const int r = st->round;
        sel[bi] = 1;
        if (ub) ub[bi] = -1.0;  // lazy Greedy: selected candidates leave every list
        st->f += bv;
        st->pick = bi;
        st->pick_gain = bv;
        if (out_idx) out_idx[r] = bi;
        if (out_f) out_f[r] = st->f;
        st->round = r + 1;
        st->rounds += 1;
        st->exact_evals += nc;
        if (st->need_esc) {
            st->escalated_rounds += 1;
            st->escalated_cands += st->esc_count;
        } else {
            st->certified += 1;
        }
    }
}

cudaError_t launch_commit_pick(Ctx &c, int32_t *out_idx, double *out_f) {
    k_commit_pick<<<1, 256, 0, c.stream>>>(c.cert.ctd_part, c.cert.nchunks, 1.0 / (double)c.n, c.cert.ctd_idx,
                                           c.cert.ctd_exact, c.esc_exact, c.esc_idx, c.cert.cap, c.sel, c.n,
                                           out_idx, out_f, c.lazy ? c.ub64 : nullptr, c.st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Threshold sieve over a stream (the streaming optimisers of Sec. 2 / Sec.
// 4.1): exact gains of a short list from the exact kernel's chunk partials,
// and the commit of an accepted item.
// ---------------------------------------------------------------------------
__global__ void k_sieve_fold_exact(const double *__restrict__ part, int nchunks, const int *__restrict__ count,
                                   int cap, double inv_n, double *__restrict__ out) {
    const int nc = min(*count, cap);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = w; e < nc; e += blockDim.x >> 5) {
        double s = 0.0;
        for (int q = lane; q < nchunks; q += 32) s += part[(int64_t)e * nchunks + q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[e] = s * inv_n;
    }
}

cudaError_t launch_sieve_fold_exact(Ctx &c, const double *part, const int *count, int cap, double *out) {
    k_sieve_fold_exact<<<1, 256, 0, c.stream>>>(part, c.cert.nchunks, count, cap, 1.0 / (double)c.n, out);
    return cudaGetLastError();
}

// Add item to S with its exact gain (taken by the host from the fold above);
// the m_v update that follows reads st->pick.
__global__ void k_sieve_commit(int item, double gain, uint8_t *__restrict__ sel, double *__restrict__ ub,
                               DevState *st) {
    sel[item] = 1;
    if (ub) ub[item] = -1.0;  // lazy Greedy bounds: a selected point leaves every list
    st->f += gain;
    st->pick = item;
    st->pick_gain = gain;
    st->round += 1;
}

cudaError_t launch_sieve_commit(Ctx &c, int item, double gain) {
    k_sieve_commit<<<1, 1, 0, c.stream>>>(item, gain, c.sel, c.ub64, c.st);
    return cudaGetLastError();
}

}  // namespace ebc
