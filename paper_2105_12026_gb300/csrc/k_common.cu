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
#include "sel_util.cuh"

namespace ebc {

__device__ __forceinline__ double exact_sqdist(const float *__restrict__ v, const float *__restrict__ c, int d) {
    double acc = 0.0;
    for (int i = 0; i < d; ++i) {
        double df = __dsub_rn((double)v[i], (double)c[i]);
        acc = __dadd_rn(acc, __dmul_rn(df, df));
    }
    return acc;
}

// Squared distance in double-FP32 arithmetic: each difference is split
// exactly into s + e (TwoSum), s^2 exactly into p + pe (FMA), and the terms
// are accumulated as an unevaluated pair (hi, lo) with TwoSum.  The result
// hi + lo is within about d * 2^-44 relative of the exact distance, using
// FP32 units only (FP64 throughput is a small fraction of FP32 on this GPU).
__device__ __forceinline__ double df_sqdist(const float *__restrict__ v, const float *__restrict__ c, int d) {
    // explicit _rn intrinsics: the compiler must not contract these into FMAs
    float hi = 0.f, lo = 0.f;
    for (int i = 0; i < d; ++i) {
        const float a = v[i], b = -c[i];
        const float s = __fadd_rn(a, b);
        const float bp = __fsub_rn(s, a);
        const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));  // a - c = s + e
        const float p = __fmul_rn(s, s);
        const float pe = __fmaf_rn(s, s, -p);                  // s^2 = p + pe exactly
        const float t = __fmaf_rn(__fmul_rn(2.f, s), e, pe);   // + 2 s e (e^2 < 2^-48 s^2)
        const float h = __fadd_rn(hi, p);
        const float z = __fsub_rn(h, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(h, z)), __fsub_rn(p, z));  // hi + p = h + err
        lo = __fadd_rn(lo, __fadd_rn(err, t));
        hi = h;
    }
    return (double)hi + (double)lo;
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
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c.ub64) e = launch_lazy_init(c);
    return e;
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

// Bounds on max(0, m_v - d) from the FP32 screen distance s, for which d
// lies in [s / (1 + rho), s / (1 - rho)], inside [s (1 - rho), s (1 + 2 rho)]:
//   hi term max(0, mU - kh s), kh = 1 - rho rounded down, mU = m_v rounded up
//   lo term max(0, mD - kl s), kl = 1 + 2 rho rounded up, mD = m_v rounded down
// formed with one FP32 FMA each.  A term is off by at most one rounding and
// a thread sums at most kBoundTermsPerThread of them in FP32, so the folded
// sums are widened by kEta32 relative (k_select.cu) to stay rigorous.
struct BoundConsts {
    float kh, kl;
};

__host__ __device__ inline BoundConsts bound_consts(int d) {
    const double rho = (double)(d + 4) * ldexp(1.0, -24);
    BoundConsts b;
    b.kh = (float)(1.0 - rho);
    if ((double)b.kh > 1.0 - rho) b.kh = nextafterf(b.kh, 0.f);
    b.kl = (float)(1.0 + 2.0 * rho);
    if ((double)b.kl < 1.0 + 2.0 * rho) b.kl = nextafterf(b.kl, 2.f);
    return b;
}

__device__ __forceinline__ void bound_terms(float mU, float mD, float s, BoundConsts bc, float &lo, float &hi) {
    hi += fmaxf(fmaf(-bc.kh, s, mU), 0.f);
    lo += fmaxf(fmaf(-bc.kl, s, mD), 0.f);
}

template <bool VEC4, bool BOUNDS>
__global__ void __launch_bounds__(256) k_refine(const float *__restrict__ V, int64_t n, int d,
                                                const double *__restrict__ m64, const int *__restrict__ list,
                                                const int *__restrict__ count, int cap, int64_t chunk, int nchunks,
                                                double rho, double *__restrict__ out, double *__restrict__ out_hi) {
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
        double acc[RB], acch[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) acc[k] = acch[k] = 0.0;
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
                if (k >= ng) continue;
                if (BOUNDS) {
                    float l = 0.f, hh = 0.f;
                    bound_terms(__double2float_ru(mv), __double2float_rd(mv), sd[k], bound_consts(d), l, hh);
                    acc[k] += (double)l;
                    acch[k] += (double)hh;
                    continue;
                }
                if ((double)sd[k] * (1.0 - rho) >= mv) continue;  // exact distance >= m_v: term 0
                const double de = exact_sqdist(vr, cs + k * d, d);
                const double t = mv - de;
                if (t > 0.0) acc[k] += t;
            }
        }
        for (int pass = 0; pass < (BOUNDS ? 2 : 1); ++pass) {
            __syncthreads();
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                double a = pass == 0 ? acc[k] : acch[k];
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) red[k][w] = a;
            }
            __syncthreads();
            if (threadIdx.x < ng) {
                double s = 0.0;
                for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s += red[threadIdx.x][ww];
                (pass == 0 ? out : out_hi)[(int64_t)(e0 + threadIdx.x) * nchunks + q] = s;
            }
        }
    }
}

// Same contract as k_refine, for d <= 256: a tile of 64 points is staged in
// shared memory with coalesced loads (rows padded to d + 1 floats so that the
// 32 points a warp handles fall in distinct banks); each thread owns one
// point of the tile and two of the group's 8 candidates, and both the FP32
// screen and the FP64 exact distance read from shared memory.
constexpr int RT = kRefineTile;  // points per staged tile

template <bool BOUNDS>
__global__ void __launch_bounds__(256) k_refine_tiled(const float *__restrict__ V, int64_t n, int d,
                                                      const double *__restrict__ m64, const int *__restrict__ list,
                                                      const int *__restrict__ count, int cap, int64_t chunk,
                                                      int nchunks, double rho, double *__restrict__ out,
                                                      double *__restrict__ out_hi) {
    extern __shared__ __align__(16) float sm[];
    const int dp = d + 1;
    float *cs = sm;                 // [RB][d]
    float *ps = sm + RB * d;        // [RT][d + 1]
    __shared__ double ms[RT];
    __shared__ float msu[RT], msd[RT];
    __shared__ double red[RB][8];
    __shared__ double redh[RB][2];
    const BoundConsts bcst = bound_consts(d);
    const int cnt = min(*count, cap);
    const int groups = (cnt + RB - 1) / RB;
    const int64_t items = (int64_t)groups * nchunks;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int p = tid & (RT - 1);   // point of the tile
    const int k0 = (tid >> 6) * 2;  // first of this thread's two candidates
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int grp = (int)(it / nchunks);
        const int q = (int)(it % nchunks);
        const int e0 = grp * RB;
        const int ng = min(RB, cnt - e0);
        __syncthreads();
        for (int x = tid; x < RB * d; x += blockDim.x) {
            int k = x / d, i = x % d;
            cs[x] = k < ng ? V[(int64_t)list[e0 + k] * d + i] : 0.f;
        }
        const int64_t b = (int64_t)q * chunk, en = lmin(b + chunk, n);
        double acc0 = 0.0, acc1 = 0.0, hi0 = 0.0, hi1 = 0.0;
        float fl0 = 0.f, fl1 = 0.f, fh0 = 0.f, fh1 = 0.f;  // FP32 bound sums of this item
        for (int64_t v0 = b; v0 < en; v0 += RT) {
            const int np = (int)lmin(RT, en - v0);
            __syncthreads();
            for (int x = tid; x < RT * d; x += blockDim.x) {
                int r = x / d, i = x % d;
                ps[r * dp + i] = r < np ? V[(v0 + r) * d + i] : 0.f;
            }
            if (tid < RT) {
                const double mm = tid < np ? m64[v0 + tid] : -1.0;
                ms[tid] = mm;
                msu[tid] = __double2float_ru(mm);
                msd[tid] = __double2float_rd(mm);
            }
            __syncthreads();
            const float *pr = ps + p * dp;
            const float *c0 = cs + k0 * d;
            const float *c1 = c0 + d;
            float s0 = 0.f, s1 = 0.f;
            for (int i = 0; i < d; ++i) {
                const float x = pr[i];
                const float a = x - c0[i], bb = x - c1[i];
                s0 = fmaf(a, a, s0);
                s1 = fmaf(bb, bb, s1);
            }
            const double mv = ms[p];
            if (BOUNDS) {
                if (p < np) {
                    if (k0 < ng) bound_terms(msu[p], msd[p], s0, bcst, fl0, fh0);
                    if (k0 + 1 < ng) bound_terms(msu[p], msd[p], s1, bcst, fl1, fh1);
                }
            } else if (p < np) {
                if (k0 < ng && (double)s0 * (1.0 - rho) < mv) {
                    const double t = mv - exact_sqdist(pr, c0, d);
                    if (t > 0.0) acc0 += t;
                }
                if (k0 + 1 < ng && (double)s1 * (1.0 - rho) < mv) {
                    const double t = mv - exact_sqdist(pr, c1, d);
                    if (t > 0.0) acc1 += t;
                }
            }
        }
        if (BOUNDS) {
            acc0 = fl0;
            acc1 = fl1;
            hi0 = fh0;
            hi1 = fh1;
        }
        // threads 64 j .. 64 j + 63 hold candidates 2 j, 2 j + 1: two warps each
        for (int o = 16; o > 0; o >>= 1) {
            acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
            acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
            if (BOUNDS) {
                hi0 += __shfl_xor_sync(0xffffffffu, hi0, o);
                hi1 += __shfl_xor_sync(0xffffffffu, hi1, o);
            }
        }
        if (lane == 0) {
            red[k0][w & 1] = acc0;
            red[k0 + 1][w & 1] = acc1;
            if (BOUNDS) {
                redh[k0][w & 1] = hi0;
                redh[k0 + 1][w & 1] = hi1;
            }
        }
        __syncthreads();
        if (tid < ng) {
            out[(int64_t)(e0 + tid) * nchunks + q] = red[tid][0] + red[tid][1];
            if (BOUNDS) out_hi[(int64_t)(e0 + tid) * nchunks + q] = redh[tid][0] + redh[tid][1];
        }
    }
}

cudaError_t launch_refine(Ctx &c, const int *list, const int *count, int list_cap, double *out, double *out_hi,
                          int64_t chunk, int nchunks) {
    if (c.d <= 256) {
        const double rho = (double)(c.d + 4) * ldexp(1.0, -24);
        const size_t sm = sizeof(float) * ((size_t)RB * c.d + (size_t)RT * (c.d + 1));
        static size_t configured = 0;
        if (sm > 48 * 1024 && sm > configured) {
            cudaError_t e = cudaFuncSetAttribute(k_refine_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_refine_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            configured = sm;
        }
        if (out_hi)
            k_refine_tiled<true><<<c.num_sms * 4, 256, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, list_cap,
                                                                        chunk, nchunks, rho, out, out_hi);
        else
            k_refine_tiled<false><<<c.num_sms * 4, 256, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, list_cap,
                                                                         chunk, nchunks, rho, out, nullptr);
        return cudaGetLastError();
    }
    return launch_refine_rows(c, list, count, list_cap, out, out_hi, chunk, nchunks);
}

template <bool VEC4, bool BOUNDS>
static cudaError_t refine_rows_one(Ctx &c, const int *list, const int *count, int list_cap, double *out,
                                   double *out_hi, int64_t chunk, int nchunks) {
    const double rho = (double)(c.d + 4) * ldexp(1.0, -24);
    const int grid = c.num_sms * 4;
    const size_t sm = sizeof(float) * (size_t)c.d * RB;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_refine<VEC4, BOUNDS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_refine<VEC4, BOUNDS><<<grid, 256, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, list_cap, chunk, nchunks,
                                                        rho, out, out_hi);
    return cudaGetLastError();
}

cudaError_t launch_refine_rows(Ctx &c, const int *list, const int *count, int list_cap, double *out,
                               double *out_hi, int64_t chunk, int nchunks) {
    const bool v4 = c.d % 4 == 0;
    if (out_hi)
        return v4 ? refine_rows_one<true, true>(c, list, count, list_cap, out, out_hi, chunk, nchunks)
                  : refine_rows_one<false, true>(c, list, count, list_cap, out, out_hi, chunk, nchunks);
    return v4 ? refine_rows_one<true, false>(c, list, count, list_cap, out, nullptr, chunk, nchunks)
              : refine_rows_one<false, false>(c, list, count, list_cap, out, nullptr, chunk, nchunks);
}

// Exact gains of a short list (the contenders), one candidate per item:
// out[e * nchunks + q] = sum over chunk q of max(0, m_v - d(v, c_e)), with d
// from the double-FP32 distance for pairs the FP32 screen cannot exclude.
// Point tiles of 128 rows are staged in shared memory (padded rows); one
// thread per point.  For d <= 256.
constexpr int XT = 128;

__global__ void __launch_bounds__(XT) k_exact_one(const float *__restrict__ V, int64_t n, int d,
                                                  const double *__restrict__ m64, const int *__restrict__ list,
                                                  const int *__restrict__ count, int cap, int64_t chunk, int nchunks,
                                                  double rho, double *__restrict__ out) {
    extern __shared__ __align__(16) float smx[];
    const int dp = d + 1;
    float *cs = smx;       // [d]
    float *ps = smx + d;   // [XT][d + 1]
    __shared__ double red[XT / 32];
    const int cnt = min(*count, cap);
    const int64_t items = (int64_t)cnt * nchunks;
    const int tid = threadIdx.x;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int e = (int)(it / nchunks);
        const int q = (int)(it % nchunks);
        __syncthreads();
        for (int i = tid; i < d; i += XT) cs[i] = V[(int64_t)list[e] * d + i];
        const int64_t b = (int64_t)q * chunk, en = lmin(b + chunk, n);
        double acc = 0.0;
        for (int64_t v0 = b; v0 < en; v0 += XT) {
            const int np = (int)lmin(XT, en - v0);
            __syncthreads();
            for (int x = tid; x < XT * d; x += XT) {
                int r = x / d, i = x % d;
                ps[r * dp + i] = r < np ? V[(v0 + r) * d + i] : 0.f;
            }
            __syncthreads();
            if (tid < np) {
                const float *pr = ps + tid * dp;
                float s = 0.f;
                for (int i = 0; i < d; ++i) {
                    const float df = pr[i] - cs[i];
                    s = fmaf(df, df, s);
                }
                const double mv = m64[v0 + tid];
                if ((double)s * (1.0 - rho) < mv) {
                    const double t = mv - df_sqdist(pr, cs, d);
                    if (t > 0.0) acc += t;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < XT / 32; ++w) s += red[w];
            out[(int64_t)e * nchunks + q] = s;
        }
    }
}

cudaError_t launch_exact_list(Ctx &c, const int *list, const int *count, int cap, double *out, int64_t chunk,
                              int nchunks) {
    if (few_supported(c)) return launch_few_exact(c, list, count, cap, out, chunk, nchunks);
    if (c.d > 256) return launch_refine_rows(c, list, count, cap, out, nullptr, chunk, nchunks);
    const double rho = (double)(c.d + 4) * ldexp(1.0, -24);
    const size_t sm = sizeof(float) * ((size_t)c.d + (size_t)XT * (c.d + 1));
    static size_t configured = 0;
    if (sm > 48 * 1024 && sm > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_exact_one, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        configured = sm;
    }
    k_exact_one<<<c.num_sms * 4, XT, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk, nchunks, rho,
                                                     out);
    return cudaGetLastError();
}

cudaError_t launch_bounds_list(Ctx &c, const int *list, const int *count, int cap, double *out_lo, double *out_hi,
                               int64_t chunk, int nchunks) {
    // short lists (the top-K, most escalations): one warp per point, 8
    // candidates per pass; longer ones: the register-tiled kernel.  The count
    // is on the device, so both are launched and one of them returns at once.
    const BoundConsts bc = bound_consts(c.d);
    if (!few_supported(c)) return launch_bounds_fp32(c, list, count, cap, out_lo, out_hi, chunk, nchunks, bc.kh, bc.kl, 0);
    cudaError_t e = launch_few_bounds(c, list, count, cap, out_lo, out_hi, chunk, nchunks, kFewBoundsMax);
    if (e != cudaSuccess || cap <= kFewBoundsMax) return e;
    return launch_bounds_fp32(c, list, count, cap, out_lo, out_hi, chunk, nchunks, bc.kh, bc.kl, kFewBoundsMax);
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
    if (few_supported(c)) return launch_few_update(c);
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

}  // namespace ebc
