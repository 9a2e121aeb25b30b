// Kernels shared by every precision: the instance prologue, the per-round
// selection of the leading candidates, their exact FP64 re-evaluation, the
// certified pick and the m_v update.
//
// Arithmetic conventions:
//  * An exact distance is sum_i (v_i - c_i)^2 in FP64, summed in index
//    order with separate multiply and add (__dmul_rn / __dadd_rn, no FMA
//    contraction).  The FP32 inputs widen exactly, the difference and the
//    square are exact in FP64, so only the additions round.
//  * Every sum over V is formed in a fixed order (per-thread, then a fixed
//    tree, then per-chunk partials added in chunk order), so results are
//    bitwise reproducible and do not depend on what else runs on the GPU.
#include <float.h>
#include <math.h>

#include "ebc_internal.cuh"

namespace ebc {

__device__ __forceinline__ double exact_sqdist(const float *__restrict__ v, const float *__restrict__ c, int d) {
    double acc = 0.0;
    for (int i = 0; i < d; ++i) {
        double df = __dsub_rn((double)v[i], (double)c[i]);
        acc = __dadd_rn(acc, __dmul_rn(df, df));
    }
    return acc;
}

// FP32 direct distance; |result - exact| <= (d + 4) * 2^-24 * exact.
__device__ __forceinline__ float screen_sqdist(const float *__restrict__ v, const float *__restrict__ c, int d) {
    float acc = 0.f;
    for (int i = 0; i < d; ++i) {
        float df = v[i] - c[i];
        acc = fmaf(df, df, acc);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// Prologue: ||v||^2 (the distance to e0), m_v = ||v||^2, selection flags,
// finiteness check.  One thread per point so the norm is summed in index
// order, like the distance to any other exemplar.
// ---------------------------------------------------------------------------
__global__ void k_prologue(const float *__restrict__ V, int64_t n, int d, double *__restrict__ nv64,
                           float *__restrict__ nv32, double *__restrict__ m64, uint8_t *__restrict__ sel,
                           DevState *st) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float *v = V + r * d;
    double acc = 0.0;
    bool finite = true;
    for (int i = 0; i < d; ++i) {
        float x = v[i];
        finite = finite && isfinite(x);
        double xd = (double)x;
        acc = __dadd_rn(acc, __dmul_rn(xd, xd));
    }
    nv64[r] = acc;
    nv32[r] = (float)acc;
    m64[r] = acc;
    sel[r] = 0;
    if (!finite) atomicCAS(&st->err, 0, (int)EBC_EINVAL);
}

cudaError_t launch_prologue(Ctx &c) {
    int th = 256;
    int64_t bl = (c.n + th - 1) / th;
    k_prologue<<<(unsigned)bl, th, 0, c.stream>>>(c.V32, c.n, c.d, c.nv64, c.nv32, c.m64, c.sel, c.st);
    return cudaGetLastError();
}

__global__ void k_reset(const double *__restrict__ nv64, double *__restrict__ m64, uint8_t *__restrict__ sel,
                        int64_t n, DevState *st) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) {
        m64[r] = nv64[r];
        sel[r] = 0;
    }
    if (r == 0) {
        DevState z;
        memset(&z, 0, sizeof(z));
        z.top_thr = -1.0;
        *st = z;
    }
}

cudaError_t launch_reset_state(Ctx &c) {
    int th = 256;
    int64_t bl = (c.n + th - 1) / th;
    k_reset<<<(unsigned)bl, th, 0, c.stream>>>(c.nv64, c.m64, c.sel, c.n, c.st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Block-wide argmax in the order (value descending, index ascending).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool better(double va, int ia, double vb, int ib) {
    return va > vb || (va == vb && ia < ib);
}

__device__ void block_best(double &v, int &i) {
    __shared__ double sv[32];
    __shared__ int si[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sv[w] = v;
        si[w] = i;
    }
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        v = lane < nw ? sv[lane] : -DBL_MAX;
        i = lane < nw ? si[lane] : INT_MAX;
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, v, o);
            int oi = __shfl_xor_sync(0xffffffffu, i, o);
            if (better(ov, oi, v, i)) {
                v = ov;
                i = oi;
            }
        }
        if (lane == 0) {
            sv[0] = v;
            si[0] = i;
        }
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
    __syncthreads();
}

// Extract the `cnt` best entries of the thread-strided range [beg, end) of
// (val[], idx[]) in order; entries with value < 0 are never taken.
__device__ void block_topk(const double *__restrict__ val, const int *__restrict__ idx, int64_t beg, int64_t end,
                           int cnt, double *out_v, int *out_i) {
    double lastv = DBL_MAX;
    int lasti = -1;
    for (int r = 0; r < cnt; ++r) {
        double bv = -DBL_MAX;
        int bi = INT_MAX;
        for (int64_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
            double x = val[j];
            int xi = idx ? idx[j] : (int)j;
            if (x < 0.0) continue;
            if (!better(lastv, lasti, x, xi)) continue;  // already taken
            if (better(x, xi, bv, bi)) {
                bv = x;
                bi = xi;
            }
        }
        block_best(bv, bi);
        if (threadIdx.x == 0) {
            out_v[r] = bi == INT_MAX ? -1.0 : bv;
            out_i[r] = bi == INT_MAX ? -1 : bi;
        }
        lastv = bv;
        lasti = bi;
    }
}

// ---------------------------------------------------------------------------
// Sum the per-chunk partials of the bulk gains kernel, scale by 1/n, mask the
// selected points.  Greedy mode writes gain_up and each block's top-(K+1);
// the gains API writes out_gain (0 for selected points).
// ---------------------------------------------------------------------------
__global__ void k_reduce_select(const double *__restrict__ partial, int64_t m, int nchunks, const int *__restrict__ cand,
                                const uint8_t *__restrict__ sel, double inv_n, int greedy, double *__restrict__ gain_up,
                                double *__restrict__ out_gain, int per_blk, int kk, double *__restrict__ blk_val,
                                int *__restrict__ blk_idx) {
    int64_t beg = (int64_t)blockIdx.x * per_blk;
    int64_t end = lmin(beg + per_blk, m);
    for (int64_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nchunks; ++q) s += partial[(int64_t)q * m + j];
        s *= inv_n;
        int c = cand ? cand[j] : (int)j;
        bool masked = c < 0 || sel[c];  // sanitised invalid entries are -1
        if (greedy)
            gain_up[j] = masked ? -1.0 : s;
        else
            out_gain[j] = masked ? 0.0 : s;
    }
    if (!greedy) return;
    __syncthreads();
    block_topk(gain_up, nullptr, beg, end, kk, blk_val + (int64_t)blockIdx.x * kk, blk_idx + (int64_t)blockIdx.x * kk);
}

cudaError_t launch_reduce_select(Ctx &c, int64_t m, int nchunks, const int *cand, bool greedy, double *out_gain,
                                 int nblk) {
    int per = (int)((m + nblk - 1) / nblk);
    k_reduce_select<<<nblk, 256, 0, c.stream>>>(c.partial, m, nchunks, cand, c.sel, 1.0 / (double)c.n, greedy ? 1 : 0,
                                                c.gain_up, out_gain, per, c.refine_k + 1, c.blk_val, c.blk_idx);
    return cudaGetLastError();
}

// Merge the per-block lists into the round's top-K and the (K+1)-th bound.
__global__ void k_merge_top(const double *__restrict__ blk_val, const int *__restrict__ blk_idx, int total, int K,
                            int *__restrict__ top_idx, double *__restrict__ top_val, DevState *st) {
    __shared__ double ov[kMaxRefineK + 1];
    __shared__ int oi[kMaxRefineK + 1];
    block_topk(blk_val, blk_idx, 0, total, K + 1, ov, oi);
    __syncthreads();
    if (threadIdx.x == 0) {
        int cnt = 0;
        for (int r = 0; r < K; ++r) {
            top_idx[r] = oi[r];
            top_val[r] = ov[r];
            if (oi[r] >= 0) cnt = r + 1;
        }
        st->top_count = cnt;
        st->top_thr = oi[K] >= 0 ? ov[K] : -1.0;
        st->esc_count = 0;
        st->need_esc = 0;
    }
}

cudaError_t launch_merge_top(Ctx &c, int nblk, int K, double) {
    k_merge_top<<<1, 1024, 0, c.stream>>>(c.blk_val, c.blk_idx, nblk * (K + 1), K, c.top_idx, c.top_val, c.st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact gains of a candidate list (count read from device memory):
//   out[e * nchunks + q] = sum_{v in chunk q} max(0, m_v - d(v, c_e))
// with d exact in FP64.  A block takes a group of RB candidates (rows staged
// in shared memory) and one V chunk; each point's row is read once for the
// RB FP32 screen distances.  A pair whose screen distance exceeds m_v by
// more than the screen's error bound contributes exactly 0 and skips the
// FP64 work.  Grid-stride over (group, chunk) items.
// ---------------------------------------------------------------------------
constexpr int RB = 8;

template <bool VEC4>
__global__ void __launch_bounds__(256) k_refine(const float *__restrict__ V, int64_t n, int d,
                                                const double *__restrict__ m64, const int *__restrict__ list,
                                                const int *__restrict__ count, int cap, int64_t chunk, int nchunks,
                                                double rho, double *__restrict__ out) {
    extern __shared__ __align__(16) float cs[];  // [RB][d]
    __shared__ double red[RB][8];
    const int cnt = min(*count, cap);
    const int groups = (cnt + RB - 1) / RB;
    const int64_t items = (int64_t)groups * nchunks;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int grp = (int)(it / nchunks);
        const int q = (int)(it % nchunks);
        const int e0 = grp * RB;
        const int ng = min(RB, cnt - e0);
        __syncthreads();
        for (int x = threadIdx.x; x < RB * d; x += blockDim.x) {
            int k = x / d, i = x % d;
            cs[x] = k < ng ? V[(int64_t)list[e0 + k] * d + i] : 0.f;
        }
        __syncthreads();
        const int64_t b = (int64_t)q * chunk, en = lmin(b + chunk, n);
        double acc[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) acc[k] = 0.0;
        for (int64_t v = b + threadIdx.x; v < en; v += blockDim.x) {
            const float *vr = V + v * d;
            float sd[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) sd[k] = 0.f;
            if (VEC4) {
                for (int i = 0; i < d; i += 4) {
                    const float4 x = *reinterpret_cast<const float4 *>(vr + i);
#pragma unroll
                    for (int k = 0; k < RB; ++k) {
                        const float4 c4 = *reinterpret_cast<const float4 *>(cs + k * d + i);
                        float d0 = x.x - c4.x, d1 = x.y - c4.y, d2 = x.z - c4.z, d3 = x.w - c4.w;
                        sd[k] = fmaf(d0, d0, sd[k]);
                        sd[k] = fmaf(d1, d1, sd[k]);
                        sd[k] = fmaf(d2, d2, sd[k]);
                        sd[k] = fmaf(d3, d3, sd[k]);
                    }
                }
            } else {
                for (int i = 0; i < d; ++i) {
                    const float x = vr[i];
#pragma unroll
                    for (int k = 0; k < RB; ++k) {
                        float df = x - cs[k * d + i];
                        sd[k] = fmaf(df, df, sd[k]);
                    }
                }
            }
            const double mv = m64[v];
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                if (k >= ng || (double)sd[k] * (1.0 - rho) >= mv) continue;  // exact distance >= m_v: term 0
                const double de = exact_sqdist(vr, cs + k * d, d);
                const double t = mv - de;
                if (t > 0.0) acc[k] += t;
            }
        }
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            double a = acc[k];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) red[k][w] = a;
        }
        __syncthreads();
        if (threadIdx.x < ng) {
            double s = 0.0;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s += red[threadIdx.x][ww];
            out[(int64_t)(e0 + threadIdx.x) * nchunks + q] = s;
        }
    }
}

cudaError_t launch_refine(Ctx &c, const int *list, const int *count, int list_cap, double *out, int64_t chunk,
                          int nchunks) {
    const double rho = (double)(c.d + 4) * ldexp(1.0, -24);
    const int grid = c.num_sms * 4;
    const size_t sm = sizeof(float) * (size_t)c.d * RB;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_refine<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_refine<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    if (c.d % 4 == 0)
        k_refine<true><<<grid, 256, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, list_cap, chunk, nchunks, rho,
                                                    out);
    else
        k_refine<false><<<grid, 256, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, list_cap, chunk, nchunks,
                                                     rho, out);
    return cudaGetLastError();
}

// Escalated candidates beyond the chunked buffer's capacity: one block per
// candidate over all of V, result written directly.  No work in the usual
// case (count <= cap).
__global__ void __launch_bounds__(256) k_refine_overflow(const float *__restrict__ V, int64_t n, int d,
                                                         const double *__restrict__ m64, const int *__restrict__ list,
                                                         const int *__restrict__ count, int cap, double rho,
                                                         double *__restrict__ out_exact, double inv_n) {
    extern __shared__ float cs1[];
    __shared__ double red[8];
    const int cnt = *count;
    for (int e = cap + blockIdx.x; e < cnt; e += gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i < d; i += blockDim.x) cs1[i] = V[(int64_t)list[e] * d + i];
        __syncthreads();
        double acc = 0.0;
        for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
            const float *vr = V + v * d;
            const double mv = m64[v];
            if ((double)screen_sqdist(vr, cs1, d) * (1.0 - rho) >= mv) continue;
            const double t = mv - exact_sqdist(vr, cs1, d);
            if (t > 0.0) acc += t;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += red[w];
            out_exact[e] = s * inv_n;
        }
    }
}

cudaError_t launch_refine_overflow(Ctx &c, const int *list, const int *count, int cap, double *out_exact) {
    const double rho = (double)(c.d + 4) * ldexp(1.0, -24);
    k_refine_overflow<<<c.num_sms * 2, 256, sizeof(float) * (size_t)c.d, c.stream>>>(
        c.V32, c.n, c.d, c.m64, list, count, cap, rho, out_exact, 1.0 / (double)c.n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Decide the round from the top-K exact gains.  The pick is certified when
// the best exact gain is at least (1 + eta) times the (K+1)-th upper bound,
// because every other candidate's exact gain is at most (1 + eta) times its
// bound and every such bound is at most the (K+1)-th.
// ---------------------------------------------------------------------------
__global__ void k_decide(const double *__restrict__ ref_part, int nchunks, double inv_n, const int *__restrict__ top_idx,
                         const double *__restrict__ top_val, double *__restrict__ top_exact, double eta, DevState *st) {
    if (threadIdx.x != 0) return;
    int cnt = st->top_count;
    double best = -1.0;
    int bi = INT_MAX;
    double maxerr = st->max_raw_rel_err;
    for (int e = 0; e < cnt; ++e) {
        double s = 0.0;
        for (int q = 0; q < nchunks; ++q) s += ref_part[(int64_t)e * nchunks + q];
        s *= inv_n;
        top_exact[e] = s;
        if (better(s, top_idx[e], best, bi)) {
            best = s;
            bi = top_idx[e];
        }
        if (s > 0.0) maxerr = fmax(maxerr, (top_val[e] - s) / s);
    }
    st->max_raw_rel_err = maxerr;
    double thr = st->top_thr;
    int need = 0, zero_scan = 0;
    if (thr < 0.0) {
        need = 0;  // no candidate outside the top list
    } else if (best > 0.0) {
        need = !(best >= thr * (1.0 + eta));
    } else if (thr > 0.0) {
        need = 1;  // best is 0 but some bound is not: evaluate every remaining candidate
    } else {
        zero_scan = 1;  // every gain is 0: the pick is the smallest unselected index
    }
    st->need_esc = need;
    st->zero_scan = zero_scan;
    st->esc_thr = best;
    st->esc_count = 0;
    st->pick_gain = best;
    st->pick = bi;
}

// Collect every unselected candidate outside the top list whose bound could
// reach the best exact gain.
__global__ void k_collect(const double *__restrict__ gain_up, int64_t m, const int *__restrict__ top_idx, double eta,
                          DevState *st, int *__restrict__ esc_idx, int cap) {
    if (!st->need_esc) return;
    double best = st->esc_thr;
    int K = st->top_count;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        double u = gain_up[j];
        if (u < 0.0) continue;  // selected
        if (best > 0.0 && u * (1.0 + eta) < best) continue;
        bool in_top = false;
        for (int e = 0; e < K; ++e) in_top |= (top_idx[e] == (int)j);
        if (in_top) continue;
        int pos = atomicAdd(&st->esc_count, 1);
        if (pos < cap) esc_idx[pos] = (int)j;
    }
}

cudaError_t launch_collect_escalation(Ctx &c, double eta) {
    k_collect<<<kNumSMsHint * 2, 256, 0, c.stream>>>(c.gain_up, c.n, c.top_idx, eta, c.st, c.esc_idx, (int)c.n);
    return cudaGetLastError();
}

// Final pick: best of the top list and the escalated list, then commit.
__global__ void k_commit(const double *__restrict__ esc_part, int nchunks, int cap, double inv_n,
                         const int *__restrict__ esc_idx, double *__restrict__ esc_exact, uint8_t *__restrict__ sel,
                         int64_t n, int32_t *__restrict__ out_idx, double *__restrict__ out_f, DevState *st) {
    double bv = st->pick_gain;
    int bi = st->pick;
    if (st->need_esc) {
        int cnt = st->esc_count;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            double s;
            if (e < cap) {
                s = 0.0;
                for (int q = 0; q < nchunks; ++q) s += esc_part[(int64_t)e * nchunks + q];
                s *= inv_n;
                esc_exact[e] = s;
            } else {
                s = esc_exact[e];  // written by the overflow kernel
            }
            if (better(s, esc_idx[e], bv, bi)) {
                bv = s;
                bi = esc_idx[e];
            }
        }
    }
    if (st->zero_scan) {
        // all remaining gains are exactly 0: smallest unselected index wins
        bv = 0.0;
        bi = INT_MAX;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
            if (!sel[j]) {
                bi = (int)j;
                break;
            }
    }
    block_best(bv, bi);
    if (threadIdx.x == 0) {
        if (bi == INT_MAX || bi < 0) {
            if (st->err == 0) st->err = (int)EBC_EINVAL;  // no candidate left (host checks prevent this)
            return;
        }
        int r = st->round;
        sel[bi] = 1;
        st->f += bv;
        st->pick = bi;
        st->pick_gain = bv;
        if (out_idx) out_idx[r] = bi;
        if (out_f) out_f[r] = st->f;
        st->round = r + 1;
        st->rounds += 1;
        if (st->need_esc) {
            st->escalated_rounds += 1;
            st->escalated_cands += st->esc_count;
        } else {
            st->certified += 1;
        }
    }
}

// m_v <- min(m_v, d(v, c*)) with the exact distance; points whose screen
// distance is clearly above m_v keep m_v unchanged.
__global__ void k_update(const float *__restrict__ V, int64_t n, int d, double *__restrict__ m64, DevState *st,
                         double rho) {
    extern __shared__ float cs[];
    int c = st->pick;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->mmax_bits = 0u;  // the next round recomputes max_v m_v
    if (c < 0 || (int64_t)c >= n) return;  // no valid pick this round (error already recorded)
    for (int i = threadIdx.x; i < d; i += blockDim.x) cs[i] = V[(int64_t)c * d + i];
    __syncthreads();
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const float *vr = V + v * d;
    double mv = m64[v];
    float ds = screen_sqdist(vr, cs, d);
    if ((double)ds * (1.0 - rho) >= mv) return;
    double de = exact_sqdist(vr, cs, d);
    if (de < mv) m64[v] = de;
}

cudaError_t launch_update(Ctx &c) {
    double rho = (double)(c.d + 4) * ldexp(1.0, -24);
    int th = 256;
    int64_t bl = (c.n + th - 1) / th;
    k_update<<<(unsigned)bl, th, sizeof(float) * (size_t)c.d, c.stream>>>(c.V32, c.n, c.d, c.m64, c.st, rho);
    return cudaGetLastError();
}

// f(S) = (1/n) sum_v (||v||^2 - m_v), one block, fixed order.
__global__ void k_current_f(const double *__restrict__ nv64, const double *__restrict__ m64, int64_t n, double inv_n,
                            double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) acc += nv64[v] - m64[v];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = s * inv_n;
    }
}

cudaError_t launch_current_f(Ctx &c, double *d_out) {
    k_current_f<<<1, 1024, 0, c.stream>>>(c.nv64, c.m64, c.n, 1.0 / (double)c.n, d_out);
    return cudaGetLastError();
}

// exported helpers for api.cu ---------------------------------------------------
cudaError_t launch_decide_n(Ctx &c, int nchunks, double eta) {
    k_decide<<<1, 32, 0, c.stream>>>(c.ref_part, nchunks, 1.0 / (double)c.n, c.top_idx, c.top_val, c.top_exact, eta,
                                     c.st);
    return cudaGetLastError();
}

cudaError_t launch_commit_n(Ctx &c, const double *esc_part, int nchunks, int cap, int32_t *out_idx, double *out_f) {
    k_commit<<<1, 256, 0, c.stream>>>(esc_part, nchunks, cap, 1.0 / (double)c.n, c.esc_idx, c.esc_exact, c.sel, c.n,
                                      out_idx, out_f, c.st);
    return cudaGetLastError();
}

}  // namespace ebc
