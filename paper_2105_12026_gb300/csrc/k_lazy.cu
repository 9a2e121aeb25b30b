// Lazy Greedy round (the "lazy" evaluation of Minoux, applied to the Greedy
// of Sec. 3 on the EBC function of Sec. 4).
//
// As S grows, every m_v can only decrease, so each candidate's marginal gain
// (1/n) sum_v max(0, m_v - d(v, c)) can only decrease (diminishing returns,
// Def. 3).  An upper bound of a candidate's gain obtained in an earlier round
// therefore stays an upper bound.  The handle keeps one such bound per
// candidate, ub[c] (+inf before the first evaluation, -1 once selected).
//
// A round:
//  1. pre-selection: the K largest ub[c] (ties to the smallest index), their
//     rigorous FP32 bounds [lo, hi] (the bound kernel of the certified pick);
//     thr = max lo is a lower bound of the round's best gain; ub <- min(ub, hi);
//  2. list: E = {c unselected : ub[c] >= thr}.  A candidate outside E has
//     gain <= ub < thr <= best gain, so it can be neither the argmax nor tied
//     with it;
//  3. the tensor-core bulk bounds U_c for the candidates of E only, then the
//     usual two-level certification restricted to E; ub[c] <- min(ub[c],
//     U_c (1 + eta)) for every c in E.
// The pick is therefore the exact argmax with the same tie rule as the full
// round, and its exact gain (hence f) is computed by the same kernel: picks
// and f are bitwise those of the full round.  Work per round is |E| * n
// instead of (unselected) * n.
#include <float.h>

#include "ebc_internal.cuh"
#include "sel_util.cuh"

namespace ebc {

__global__ void k_lazy_init(double *__restrict__ ub, const uint8_t *__restrict__ sel, int64_t n) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < n) ub[j] = sel[j] ? -1.0 : DBL_MAX;
}

cudaError_t launch_lazy_init(Ctx &c) {
    k_lazy_init<<<(unsigned)((c.n + 255) / 256), 256, 0, c.stream>>>(c.ub64, c.sel, c.n);
    return cudaGetLastError();
}

// ub <- min(ub, U (1 + eta)) from a full bulk pass (gain_up[c] = U_c, -1 when
// selected): the FP8 pre-screen of the certified FP8 Greedy.
__global__ void k_lazy_from_full(const double *__restrict__ gain_up, int64_t n, double eta, double *__restrict__ ub) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double u = gain_up[j];
    if (u >= 0.0) ub[j] = fmin(ub[j], u * (1.0 + eta));
}

cudaError_t launch_lazy_from_full(Ctx &c, double eta) {
    k_lazy_from_full<<<(unsigned)((c.n + 255) / 256), 256, 0, c.stream>>>(c.gain_up, c.n, eta, c.ub64);
    return cudaGetLastError();
}

// Per-block top (K + 1) of ub among unselected candidates.
__global__ void k_lazy_blocktop(const double *__restrict__ ub, int64_t n, int per_blk, int kk,
                                double *__restrict__ blk_val, int *__restrict__ blk_idx) {
    const int64_t beg = (int64_t)blockIdx.x * per_blk;
    const int64_t end = lmin(beg + per_blk, n);
    block_topk(ub, nullptr, beg, end, kk, blk_val + (int64_t)blockIdx.x * kk, blk_idx + (int64_t)blockIdx.x * kk);
}

cudaError_t launch_lazy_preselect(Ctx &c, int nblk, int K) {
    const int per = (int)((c.n + nblk - 1) / nblk);
    k_lazy_blocktop<<<nblk, 256, 0, c.stream>>>(c.ub64, c.n, per, K + 1, c.blk_val, c.blk_idx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_merge_top(c, nblk, K, 0.0);
}

// thr = max lo over the pre-selected list (lowered by the tie margin);
// tighten their ub with hi.
__global__ void k_lazy_threshold(const double *__restrict__ top_lo, const double *__restrict__ top_hi,
                                 const int *__restrict__ top_idx, double *__restrict__ ub, DevState *st) {
    if (threadIdx.x != 0) return;
    const int cnt = st->top_count;
    double thr = 0.0;
    for (int e = 0; e < cnt; ++e) {
        thr = fmax(thr, top_lo[e]);
        const int c = top_idx[e];
        if (c >= 0) ub[c] = fmin(ub[c], top_hi[e]);
    }
    st->lazy_thr = thr * (1.0 - 2.0 * kTieRel);  // candidates tied with the best stay in the list
    st->list_m = 0;
}

cudaError_t launch_lazy_threshold(Ctx &c) {
    k_lazy_threshold<<<1, 32, 0, c.stream>>>(c.cert.top_lo, c.cert.top_hi, c.top_idx, c.ub64, c.st);
    return cudaGetLastError();
}

// E = {c : ub[c] >= thr, c unselected} (selected candidates have ub = -1).
__global__ void k_lazy_build(const double *__restrict__ ub, int64_t n, DevState *st, int *__restrict__ list) {
    const double thr = st->lazy_thr;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double u = ub[j];
        if (u < 0.0 || u < thr) continue;
        list[atomicAdd(&st->list_m, 1)] = (int)j;
    }
}

cudaError_t launch_lazy_build(Ctx &c) {
    k_lazy_build<<<c.num_sms * 4, 256, 0, c.stream>>>(c.ub64, c.n, c.st, c.lazy_idx);
    return cudaGetLastError();
}

// Sum the list's chunk partials (bulk upper bounds), tighten ub, and each
// block's top (K + 1) by candidate index.
__global__ void k_lazy_select(const double *__restrict__ partial, const int *__restrict__ list,
                              const uint8_t *__restrict__ sel, double inv_n, double eta, int kk,
                              double *__restrict__ gain_up, double *__restrict__ ub, double *__restrict__ blk_val,
                              int *__restrict__ blk_idx, DevState *st) {
    const int64_t m = st->list_m;
    const int nchunks = st->list_nch;
    const int64_t per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t beg = lmin((int64_t)blockIdx.x * per, m);
    const int64_t end = lmin(beg + per, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->bulk_cands += m;
    for (int64_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nchunks; ++q) s += partial[(int64_t)q * m + j];
        s *= inv_n;
        const int c = list[j];
        if (sel[c]) {
            gain_up[j] = -1.0;
            continue;
        }
        gain_up[j] = s;
        ub[c] = fmin(ub[c], s * (1.0 + eta));
    }
    __syncthreads();
    block_topk(gain_up, list, beg, end, kk, blk_val + (int64_t)blockIdx.x * kk, blk_idx + (int64_t)blockIdx.x * kk);
}

cudaError_t launch_lazy_select(Ctx &c, double eta, int nblk) {
    k_lazy_select<<<nblk, 256, 0, c.stream>>>(c.partial, c.lazy_idx, c.sel, 1.0 / (double)c.n, eta, c.refine_k + 1,
                                               c.gain_up, c.ub64, c.blk_val, c.blk_idx, c.st);
    return cudaGetLastError();
}

// Escalation over the list: entries outside the top list whose bulk bound
// could reach the best certified lower bound.
__global__ void k_lazy_collect(const double *__restrict__ gain_up, const int *__restrict__ list,
                               const int *__restrict__ top_idx, double eta, DevState *st, int *__restrict__ esc_idx,
                               int cap) {
    if (!st->need_esc) return;
    const int64_t m = st->list_m;
    const double best = st->esc_thr;
    const int K = st->top_count;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const double u = gain_up[j];
        if (u < 0.0) continue;
        if (best > 0.0 && u * (1.0 + eta) < best) continue;
        const int c = list[j];
        bool in_top = false;
        for (int e = 0; e < K; ++e) in_top |= (top_idx[e] == c);
        if (in_top) continue;
        const int pos = atomicAdd(&st->esc_count, 1);
        if (pos < cap) esc_idx[pos] = c;
    }
}

cudaError_t launch_lazy_collect(Ctx &c, double eta) {
    k_lazy_collect<<<c.num_sms * 2, 256, 0, c.stream>>>(c.gain_up, c.lazy_idx, c.top_idx, eta, c.st, c.esc_idx,
                                                         (int)c.n);
    return cudaGetLastError();
}

}  // namespace ebc
