// Kernels for a few candidates over all of V (the per-round tail of the
// certified Greedy pick of Sec. 3 and the m_v update of the incremental
// evaluation of Sec. 4): rigorous FP32 gain bounds of a short list, exact
// gains of the contenders, and m_v <- min(m_v, d(v, c*)).
//
// A group of LPP lanes holds one point: each lane 4 (or 8) of its dimensions
// (float4 loads, coalesced) and the same dimensions of up to 8 candidates in
// registers; a warp holds 32 / LPP points at once (LPP = 8 for d <= 32, 16
// for d <= 64, 32 above, so that few lanes idle at small d).  Per-candidate
// distances are fixed xor-shuffle trees within the group.  Each pass over V
// reads every point once for up to 8 candidates.  Above d = 256 the "wide"
// kernels walk each lane's dimensions in slabs of 256 (8 per lane) with the
// candidate rows staged whole in dynamic shared memory.
//
// Rounding.  An FP32 distance formed this way has, along any term's path,
// the difference's rounding (twice, once squared), at most 8 for the lane's
// fused multiply-adds (d / 32 in the wide kernels; fewer when the lane holds
// fewer non-zero terms) and at most 5 for the tree, so
// |s - d| <= (d + 10) 2^-24 d for every d >= 1 (the terms are non-negative);
// the bound constants below use that.
#include <float.h>
#include <math.h>

#include <mutex>
#include <utility>
#include <vector>

#include "ebc_internal.cuh"

namespace ebc {

namespace {
constexpr int FW = 8;       // warps per block
constexpr int FC = 8;       // candidates per pass
constexpr int FDMAX = 256;  // largest d
constexpr int UNR = 4;      // points in flight per lane group

__host__ __device__ inline double few_rho(int d) { return (double)(d + 10) * ldexp(1.0, -24); }

// Dimension k (0 <= k < DL) of the lane with index `sub` in its group, or -1.
//   VEC4: dims 4 LPP (k / 4) + 4 sub + k % 4 (d a multiple of 4)
//   else: dims LPP k + sub
template <bool VEC4, int LPP>
__device__ __forceinline__ int lane_dim(int k, int sub, int d) {
    const int i = VEC4 ? 4 * LPP * (k >> 2) + 4 * sub + (k & 3) : LPP * k + sub;
    return i < d ? i : -1;
}

template <bool VEC4, int DL, int LPP>
__device__ __forceinline__ void load_point(const float *__restrict__ row, int sub, int d, float (&x)[DL]) {
    if (VEC4) {
#pragma unroll
        for (int j = 0; j < DL / 4; ++j) {
            const int i = 4 * LPP * j + 4 * sub;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < d) a = __ldg(reinterpret_cast<const float4 *>(row + i));
            x[4 * j] = a.x;
            x[4 * j + 1] = a.y;
            x[4 * j + 2] = a.z;
            x[4 * j + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < DL; ++k) {
            const int i = LPP * k + sub;
            x[k] = i < d ? __ldg(row + i) : 0.f;
        }
    }
}

// Float bounds of a non-negative double with integer operations only (the
// FP64 pipe of this GPU is narrow): dn <= x <= up, dn and up adjacent floats
// (or equal when x is a float).  Below the smallest normal float dn = 0 and
// up = FLT_MIN; above the largest, up = inf.
__device__ __forceinline__ void d2f_bounds(double x, float &up, float &dn) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int fe = (int)(b >> 52) - 1023 + 127;  // float biased exponent (x >= 0)
    if (b == 0ull) {
        up = dn = 0.f;
    } else if (fe <= 0) {
        dn = 0.f;
        up = FLT_MIN;
    } else if (fe >= 255) {
        dn = FLT_MAX;
        up = INFINITY;
    } else {
        const unsigned int fb = ((unsigned int)fe << 23) | (unsigned int)((b >> 29) & 0x7FFFFFull);
        dn = __uint_as_float(fb);
        up = (b & ((1ull << 29) - 1)) ? __uint_as_float(fb + 1u) : dn;  // + 1 ulp (carries into the exponent)
    }
}

// Sums over the group's LPP lanes of the 8 per-candidate partials s[0..7],
// as a reduce-scatter: offsets LPP/2, LPP/4 and LPP/8 split the candidates
// between the two halves, smaller offsets add.  The lane with group index
// sub ends with the total of candidate cand_of(sub) (LPP / 8 lanes per
// candidate); every total is still a fixed tree of log2(LPP) pair additions
// over the group's partials.
template <int LPP>
__device__ __forceinline__ int cand_of(int sub) {
    return ((sub & (LPP / 2)) ? 4 : 0) + ((sub & (LPP / 4)) ? 2 : 0) + ((sub & (LPP / 8)) ? 1 : 0);
}

template <int LPP>
__device__ __forceinline__ int sub_of_cand(int e) {
    return ((e >> 2) & 1) * (LPP / 2) + ((e >> 1) & 1) * (LPP / 4) + (e & 1) * (LPP / 8);
}

template <int LPP>
__device__ __forceinline__ float reduce_scatter8(const float (&s)[8], int sub) {
    float t[4], u[2];
    const bool b1 = sub & (LPP / 2), b2 = sub & (LPP / 4), b3 = sub & (LPP / 8);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float send = b1 ? s[j] : s[j + 4];
        const float keep = b1 ? s[j + 4] : s[j];
        t[j] = keep + __shfl_xor_sync(0xffffffffu, send, LPP / 2);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float send = b2 ? t[j] : t[j + 2];
        const float keep = b2 ? t[j + 2] : t[j];
        u[j] = keep + __shfl_xor_sync(0xffffffffu, send, LPP / 4);
    }
    const float send = b3 ? u[0] : u[1];
    const float keep = b3 ? u[1] : u[0];
    float w = keep + __shfl_xor_sync(0xffffffffu, send, LPP / 8);
#pragma unroll
    for (int o = LPP / 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    return w;
}

// Sum over the group's LPP lanes (fixed xor tree).
template <int LPP>
__device__ __forceinline__ float group_sum(float s) {
#pragma unroll
    for (int o = LPP / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// (hi, lo) += (a, b) exactly up to the final rounding of lo (TwoSum on hi).
__device__ __forceinline__ void df_add(float &hi, float &lo, float a, float b) {
    const float h = __fadd_rn(hi, a);
    const float z = __fsub_rn(h, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(h, z)), __fsub_rn(a, z));
    lo = __fadd_rn(lo, __fadd_rn(err, b));
    hi = h;
}

// Double-FP32 squared distance of the group's point to c (TwoSum /
// TwoProduct per dimension with explicit round-to-nearest intrinsics, as in
// the exact gain path), then a fixed xor tree within the group whose pair
// additions are again TwoSum.  Every lane of the warp takes part (the
// shuffles are warp-wide); each group gets its own point's distance.
template <int DL, int LPP>
__device__ __forceinline__ double df_dist_group(const float (&x)[DL], const float (&c)[DL]) {
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int k = 0; k < DL; ++k) {
        const float a = x[k], b = -c[k];
        const float s = __fadd_rn(a, b);
        const float bp = __fsub_rn(s, a);
        const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));  // a - c = s + e
        const float p = __fmul_rn(s, s);
        const float pe = __fmaf_rn(s, s, -p);                 // s^2 = p + pe
        const float t = __fmaf_rn(__fmul_rn(2.f, s), e, pe);  // + 2 s e
        df_add(hi, lo, p, t);
    }
#pragma unroll
    for (int o = LPP / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        df_add(hi, lo, oh, ol);
    }
    // df_add is not symmetric in its low parts, so the lanes of a group end
    // with slightly different values: every lane takes the group's first
    // lane's, and a distance never depends on which lane reads it
    const int first = (threadIdx.x & 31) & ~(LPP - 1);
    hi = __shfl_sync(0xffffffffu, hi, first);
    lo = __shfl_sync(0xffffffffu, lo, first);
    return (double)hi + (double)lo;
}

// Stage the block's candidate rows and give each lane its dimensions.
template <bool VEC4, int DL, int LPP>
__device__ __forceinline__ void stage_candidates(const float *__restrict__ V, int d, const int *__restrict__ list,
                                                 int first, int cnt, float (*cs)[FDMAX], float (&c)[FC][DL],
                                                 int &ng) {
    ng = min(FC, cnt - first);
    for (int x = threadIdx.x; x < FC * d; x += blockDim.x) {
        const int e = x / d, i = x % d;
        cs[e][i] = e < ng ? V[(int64_t)list[first + e] * d + i] : 0.f;
    }
    __syncthreads();
    const int sub = threadIdx.x % LPP;
#pragma unroll
    for (int e = 0; e < FC; ++e)
#pragma unroll
        for (int k = 0; k < DL; ++k) {
            const int i = lane_dim<VEC4, LPP>(k, sub, d);
            c[e][k] = i >= 0 ? cs[e][i] : 0.f;
        }
}
}  // namespace

// Rigorous [lo, hi] bounds of the gains of a short device list, as chunk
// partials out_lo / out_hi[e * nchunks + q] (same contract as the tiled
// bound kernel).  Terms max(0, mU - kh s) and max(0, mD - kl s) in FP32,
// summed per candidate by one lane of each group in FP32 over at most 64
// points (fewer than the 128 terms per FP32 sum the folded bounds are
// widened for), then in FP64, then over the block's groups in a fixed order.
// Lists longer than max_cnt are left to the tiled kernel.
template <bool VEC4, int DL, int LPP>
__global__ void __launch_bounds__(FW * 32, DL == 4 ? 3 : 1) k_few_bounds(const float *__restrict__ V, int64_t n, int d,
                                                        const double *__restrict__ m64, const int *__restrict__ list,
                                                        const int *__restrict__ count, int cap, int64_t chunk,
                                                        int nchunks, float kh, float kl, double *__restrict__ out_lo,
                                                        double *__restrict__ out_hi, int max_cnt) {
    constexpr int PPW = 32 / LPP;  // points per warp
    __shared__ __align__(16) float cs[FC][FDMAX];
    __shared__ double rlo[FW][PPW][FC], rhi[FW][PPW][FC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / LPP, sub = lane % LPP;
    const bool owner = (sub & (LPP / 8 - 1)) == 0;  // holds candidate cand_of(sub)'s total
    const int cnt = min(*count, cap);
    if (cnt > max_cnt) return;
    const int groups = (cnt + FC - 1) / FC;
    const int64_t items = (int64_t)groups * nchunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int g = (int)(it / nchunks), q = (int)(it % nchunks);
        __syncthreads();
        float c[FC][DL];
        int ng;
        stage_candidates<VEC4, DL, LPP>(V, d, list, g * FC, cnt, cs, c, ng);
        double alo = 0.0, ahi = 0.0;
        float flo = 0.f, fhi = 0.f;
        int nterm = 0;
        const int64_t vb = (int64_t)q * chunk, ve = lmin(vb + chunk, n);
        for (int64_t v0 = vb + (int64_t)warp * PPW * UNR; v0 < ve; v0 += (int64_t)FW * PPW * UNR) {
            float x[UNR][DL];
            double mm[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {  // all loads first: UNR points per group in flight
                const int64_t p = v0 + u * PPW + grp;
                const int64_t v = lmin(p, ve - 1);
                load_point<VEC4, DL, LPP>(V + v * d, sub, d, x[u]);
                mm[u] = p < ve ? m64[v] : -1.0;  // -1: no such point, every term 0
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                float mu, md;
                if (__double_as_longlong(mm[u]) < 0) {  // -1: past the chunk, no terms
                    mu = md = -1.f;
                } else {
                    d2f_bounds(mm[u], mu, md);
                }
                float sp[FC];
#pragma unroll
                for (int e = 0; e < FC; ++e) {
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < DL; ++k) {
                        const float df = x[u][k] - c[e][k];
                        s = fmaf(df, df, s);
                    }
                    sp[e] = s;
                }
                const float s = reduce_scatter8<LPP>(sp, sub);  // candidate cand_of(sub)
                if (owner) {
                    fhi += fmaxf(fmaf(-kh, s, mu), 0.f);
                    flo += fmaxf(fmaf(-kl, s, md), 0.f);
                }
            }
            nterm += UNR;
            if (nterm >= 64) {
                ahi += (double)fhi;
                alo += (double)flo;
                fhi = flo = 0.f;
                nterm = 0;
            }
        }
        ahi += (double)fhi;
        alo += (double)flo;
        if (owner) {
            rlo[warp][grp][cand_of<LPP>(sub)] = alo;
            rhi[warp][grp][cand_of<LPP>(sub)] = ahi;
        }
        __syncthreads();
        if (threadIdx.x < ng) {
            double sl = 0.0, sh = 0.0;
            for (int w = 0; w < FW; ++w)
                for (int r = 0; r < PPW; ++r) {
                    sl += rlo[w][r][threadIdx.x];
                    sh += rhi[w][r][threadIdx.x];
                }
            const int64_t e = (int64_t)g * FC + threadIdx.x;
            out_lo[e * nchunks + q] = sl;
            out_hi[e * nchunks + q] = sh;
        }
    }
}

// Exact gains of a device list as chunk partials out[e * nchunks + q] =
// sum over chunk q of max(0, m_v - d(v, c_e)), d in double-FP32 for the
// pairs the FP32 screen cannot exclude (a screen s with RD(s kh) >= m_v
// rounded up, kh = 1 - rho rounded down, proves d >= m_v: the pair
// contributes exactly 0).
template <bool VEC4, int DL, int LPP>
__global__ void __launch_bounds__(FW * 32, DL == 4 ? 3 : 1) k_few_exact(const float *__restrict__ V, int64_t n, int d,
                                                       const double *__restrict__ m64, const int *__restrict__ list,
                                                       const int *__restrict__ count, int cap, int64_t chunk,
                                                       int nchunks, float kh, double *__restrict__ out) {
    constexpr int PPW = 32 / LPP;
    __shared__ __align__(16) float cs[FC][FDMAX];
    __shared__ double red[FW][PPW][FC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / LPP, sub = lane % LPP;
    const bool owner = (sub & (LPP / 8 - 1)) == 0;
    const int cnt = min(*count, cap);
    const int groups = (cnt + FC - 1) / FC;
    const int64_t items = (int64_t)groups * nchunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int g = (int)(it / nchunks), q = (int)(it % nchunks);
        __syncthreads();
        float c[FC][DL];
        int ng;
        stage_candidates<VEC4, DL, LPP>(V, d, list, g * FC, cnt, cs, c, ng);
        double acc = 0.0;  // owner lanes: candidate cand_of(sub)
        const int64_t vb = (int64_t)q * chunk, ve = lmin(vb + chunk, n);
        for (int64_t v0 = vb + (int64_t)warp * PPW * UNR; v0 < ve; v0 += (int64_t)FW * PPW * UNR) {
            float x[UNR][DL];
            double mm[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {  // all loads first: UNR points per group in flight
                const int64_t p = v0 + u * PPW + grp;
                const int64_t v = lmin(p, ve - 1);
                load_point<VEC4, DL, LPP>(V + v * d, sub, d, x[u]);
                mm[u] = p < ve ? m64[v] : -1.0;  // -1: no such point, screened out
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const double mv = mm[u];
                const bool valid = __double_as_longlong(mv) >= 0;  // group-uniform
                float mu = -1.f, md;
                if (valid) d2f_bounds(mv, mu, md);
                float sp[FC];
#pragma unroll
                for (int e = 0; e < FC; ++e) {
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < DL; ++k) {
                        const float df = x[u][k] - c[e][k];
                        s = fmaf(df, df, s);
                    }
                    sp[e] = s;
                }
                const float sall = reduce_scatter8<LPP>(sp, sub);
#pragma unroll
                for (int e = 0; e < FC; ++e) {
                    if (e >= ng) break;  // warp-uniform
                    const float s = __shfl_sync(0xffffffffu, sall, grp * LPP + sub_of_cand<LPP>(e));
                    // d >= s (1 - rho) >= RD(s kh) >= mu >= m_v proves a zero term
                    const bool need = valid && __fmul_rd(s, kh) < mu;  // group-uniform
                    if (__any_sync(0xffffffffu, need)) {               // the tree needs the whole warp
                        const double t = mv - df_dist_group<DL, LPP>(x[u], c[e]);
                        if (need && sub == sub_of_cand<LPP>(e) && t > 0.0) acc += t;
                    }
                }
            }
        }
        if (owner) red[warp][grp][cand_of<LPP>(sub)] = acc;
        __syncthreads();
        if (threadIdx.x < ng) {
            double s = 0.0;
            for (int w = 0; w < FW; ++w)
                for (int r = 0; r < PPW; ++r) s += red[w][r][threadIdx.x];
            out[((int64_t)g * FC + threadIdx.x) * nchunks + q] = s;
        }
    }
}

// m_v <- min(m_v, d(v, c*)) with d the double-FP32 distance (within about
// 2^-44 relative; FP32 units only); points whose FP32 screen distance
// proves d >= m_v keep m_v.
template <bool VEC4, int DL, int LPP>
__global__ void __launch_bounds__(FW * 32) k_few_update(const float *__restrict__ V, int64_t n, int d,
                                                        double *__restrict__ m64, DevState *st, float kh) {
    constexpr int PPW = 32 / LPP;
    __shared__ __align__(16) float cs[FDMAX];
    const int c = st->pick;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->mmax_bits = 0u;  // the next round recomputes max_v m_v
    if (c < 0 || (int64_t)c >= n) return;                           // no valid pick (error already recorded)
    for (int i = threadIdx.x; i < d; i += blockDim.x) cs[i] = V[(int64_t)c * d + i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / LPP, sub = lane % LPP;
    float cr[DL];
#pragma unroll
    for (int k = 0; k < DL; ++k) {
        const int i = lane_dim<VEC4, LPP>(k, sub, d);
        cr[k] = i >= 0 ? cs[i] : 0.f;
    }
    const int64_t gw = (int64_t)blockIdx.x * FW + warp, nw = (int64_t)gridDim.x * FW;
    for (int64_t v0 = gw * PPW * UNR; v0 < n; v0 += nw * PPW * UNR) {
        float x[UNR][DL];
        double mm[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {  // all loads first: UNR points per group in flight
            const int64_t v = lmin(v0 + u * PPW + grp, n - 1);
            load_point<VEC4, DL, LPP>(V + v * d, sub, d, x[u]);
            mm[u] = m64[v];
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int64_t p = v0 + u * PPW + grp;
            const double mv = mm[u];
            float mu, md;
            d2f_bounds(mv, mu, md);
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < DL; ++k) {
                const float df = x[u][k] - cr[k];
                s = fmaf(df, df, s);
            }
            s = group_sum<LPP>(s);
            const bool need = p < n && __fmul_rd(s, kh) < mu;  // else d >= m_v: m_v stays (group-uniform)
            if (__any_sync(0xffffffffu, need)) {               // the tree needs the whole warp
                const double de = df_dist_group<DL, LPP>(x[u], cr);
                if (need && sub == 0 && de < mv) m64[p] = de;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// d > 256: one group of 32 lanes per point; each lane holds 8 dimensions of a
// slab of 256 (the lane layout above, offset by 256 per slab); the block's
// candidate rows are staged whole in dynamic shared memory ([FC][d] floats).
// ---------------------------------------------------------------------------
namespace {
constexpr int SLAB = 256;
constexpr int UNRW = 4;  // points in flight per warp

template <bool VEC4>
__device__ __forceinline__ void smem_slab(const float *__restrict__ row, int lane, int dl, float (&c)[8]) {
    if (VEC4) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int i = 128 * j + 4 * lane;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < dl) a = *reinterpret_cast<const float4 *>(row + i);
            c[4 * j] = a.x;
            c[4 * j + 1] = a.y;
            c[4 * j + 2] = a.z;
            c[4 * j + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = 32 * k + lane;
            c[k] = i < dl ? row[i] : 0.f;
        }
    }
}

// Double-FP32 distance of a point row (global) to a candidate row (shared),
// slab by slab: the per-dimension steps and the xor tree of df_dist_group.
template <bool VEC4>
__device__ __forceinline__ double df_dist_wide(const float *__restrict__ row, const float *__restrict__ crow, int d,
                                               int lane) {
    float hi = 0.f, lo = 0.f;
    for (int s0 = 0; s0 < d; s0 += SLAB) {
        float x[8], c[8];
        load_point<VEC4, 8, 32>(row + s0, lane, d - s0, x);
        smem_slab<VEC4>(crow + s0, lane, d - s0, c);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float a = x[k], b = -c[k];
            const float s = __fadd_rn(a, b);
            const float bp = __fsub_rn(s, a);
            const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));  // a - c = s + e
            const float p = __fmul_rn(s, s);
            const float pe = __fmaf_rn(s, s, -p);                 // s^2 = p + pe
            const float t = __fmaf_rn(__fmul_rn(2.f, s), e, pe);  // + 2 s e
            df_add(hi, lo, p, t);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        df_add(hi, lo, oh, ol);
    }
    hi = __shfl_sync(0xffffffffu, hi, 0);  // lane 0's value for every lane (see df_dist_group)
    lo = __shfl_sync(0xffffffffu, lo, 0);
    return (double)hi + (double)lo;
}

// Per-lane FP32 screen partials of UNRW consecutive points (p0.., rows
// clamped to `last`) against the block's FC staged candidates, over all slabs.
template <bool VEC4>
__device__ __forceinline__ void screen_wide(const float *__restrict__ V, int d, int64_t p0, int64_t last,
                                            const float *__restrict__ csw, int lane, float (&sp)[UNRW][FC]) {
#pragma unroll
    for (int u = 0; u < UNRW; ++u)
#pragma unroll
        for (int e = 0; e < FC; ++e) sp[u][e] = 0.f;
    for (int s0 = 0; s0 < d; s0 += SLAB) {
        float x[UNRW][8];
#pragma unroll
        for (int u = 0; u < UNRW; ++u) load_point<VEC4, 8, 32>(V + lmin(p0 + u, last) * d + s0, lane, d - s0, x[u]);
#pragma unroll
        for (int e = 0; e < FC; ++e) {
            float c[8];
            smem_slab<VEC4>(csw + e * d + s0, lane, d - s0, c);
#pragma unroll
            for (int u = 0; u < UNRW; ++u)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float df = x[u][k] - c[k];
                    sp[u][e] = fmaf(df, df, sp[u][e]);
                }
        }
    }
}

// Stage the block's candidate rows (zero rows past the list); returns how many.
__device__ __forceinline__ int stage_wide(const float *__restrict__ V, int d, const int *__restrict__ list, int first,
                                          int cnt, float *__restrict__ csw) {
    const int ng = min(FC, cnt - first);
    for (int x = threadIdx.x; x < FC * d; x += blockDim.x) {
        const int e = x / d, i = x % d;
        csw[x] = e < ng ? V[(int64_t)list[first + e] * d + i] : 0.f;
    }
    __syncthreads();
    return ng;
}
}  // namespace

// Same contract and bound terms as k_few_bounds.
template <bool VEC4>
__global__ void __launch_bounds__(FW * 32) k_few_bounds_wide(const float *__restrict__ V, int64_t n, int d,
                                                             const double *__restrict__ m64,
                                                             const int *__restrict__ list, const int *__restrict__ count,
                                                             int cap, int64_t chunk, int nchunks, float kh, float kl,
                                                             double *__restrict__ out_lo, double *__restrict__ out_hi,
                                                             int max_cnt) {
    extern __shared__ __align__(16) float csw[];  // [FC][d]
    __shared__ double rlo[FW][FC], rhi[FW][FC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool owner = (lane & 3) == 0;  // holds candidate cand_of(lane)'s total
    const int cnt = min(*count, cap);
    if (cnt > max_cnt) return;
    const int groups = (cnt + FC - 1) / FC;
    const int64_t items = (int64_t)groups * nchunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int g = (int)(it / nchunks), q = (int)(it % nchunks);
        __syncthreads();
        const int ng = stage_wide(V, d, list, g * FC, cnt, csw);
        double alo = 0.0, ahi = 0.0;
        float flo = 0.f, fhi = 0.f;
        int nterm = 0;
        const int64_t vb = (int64_t)q * chunk, ve = lmin(vb + chunk, n);
        for (int64_t v0 = vb + (int64_t)warp * UNRW; v0 < ve; v0 += (int64_t)FW * UNRW) {
            float sp[UNRW][FC];
            screen_wide<VEC4>(V, d, v0, ve - 1, csw, lane, sp);
#pragma unroll
            for (int u = 0; u < UNRW; ++u) {
                float mu = -1.f, md = -1.f;  // no such point: every term 0
                if (v0 + u < ve) d2f_bounds(m64[v0 + u], mu, md);
                const float s = reduce_scatter8<32>(sp[u], lane);
                if (owner) {
                    fhi += fmaxf(fmaf(-kh, s, mu), 0.f);
                    flo += fmaxf(fmaf(-kl, s, md), 0.f);
                }
            }
            nterm += UNRW;
            if (nterm >= 64) {
                ahi += (double)fhi;
                alo += (double)flo;
                fhi = flo = 0.f;
                nterm = 0;
            }
        }
        ahi += (double)fhi;
        alo += (double)flo;
        if (owner) {
            rlo[warp][cand_of<32>(lane)] = alo;
            rhi[warp][cand_of<32>(lane)] = ahi;
        }
        __syncthreads();
        if (threadIdx.x < ng) {
            double sl = 0.0, sh = 0.0;
            for (int w = 0; w < FW; ++w) {
                sl += rlo[w][threadIdx.x];
                sh += rhi[w][threadIdx.x];
            }
            const int64_t e = (int64_t)g * FC + threadIdx.x;
            out_lo[e * nchunks + q] = sl;
            out_hi[e * nchunks + q] = sh;
        }
    }
}

// Same contract and screen as k_few_exact.
template <bool VEC4>
__global__ void __launch_bounds__(FW * 32) k_few_exact_wide(const float *__restrict__ V, int64_t n, int d,
                                                            const double *__restrict__ m64, const int *__restrict__ list,
                                                            const int *__restrict__ count, int cap, int64_t chunk,
                                                            int nchunks, float kh, double *__restrict__ out) {
    extern __shared__ __align__(16) float csw[];  // [FC][d]
    __shared__ double red[FW][FC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cnt = min(*count, cap);
    const int groups = (cnt + FC - 1) / FC;
    const int64_t items = (int64_t)groups * nchunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int g = (int)(it / nchunks), q = (int)(it % nchunks);
        __syncthreads();
        const int ng = stage_wide(V, d, list, g * FC, cnt, csw);
        double acc = 0.0;  // lane sub_of_cand(e): candidate e
        const int64_t vb = (int64_t)q * chunk, ve = lmin(vb + chunk, n);
        for (int64_t v0 = vb + (int64_t)warp * UNRW; v0 < ve; v0 += (int64_t)FW * UNRW) {
            float sp[UNRW][FC];
            screen_wide<VEC4>(V, d, v0, ve - 1, csw, lane, sp);
#pragma unroll
            for (int u = 0; u < UNRW; ++u) {
                const float sall = reduce_scatter8<32>(sp[u], lane);
                if (v0 + u >= ve) continue;  // warp-uniform
                const double mv = m64[v0 + u];
                float mu, md;
                d2f_bounds(mv, mu, md);
                for (int e = 0; e < ng; ++e) {
                    const float s = __shfl_sync(0xffffffffu, sall, sub_of_cand<32>(e));
                    // d >= s (1 - rho) >= RD(s kh) >= mu >= m_v proves a zero term
                    if (__fmul_rd(s, kh) < mu) {  // warp-uniform
                        const double t = mv - df_dist_wide<VEC4>(V + (v0 + u) * d, csw + e * d, d, lane);
                        if (lane == sub_of_cand<32>(e) && t > 0.0) acc += t;
                    }
                }
            }
        }
        if ((lane & 3) == 0) red[warp][cand_of<32>(lane)] = acc;
        __syncthreads();
        if (threadIdx.x < ng) {
            double s = 0.0;
            for (int w = 0; w < FW; ++w) s += red[w][threadIdx.x];
            out[((int64_t)g * FC + threadIdx.x) * nchunks + q] = s;
        }
    }
}

// Same contract as k_few_update.
template <bool VEC4>
__global__ void __launch_bounds__(FW * 32) k_few_update_wide(const float *__restrict__ V, int64_t n, int d,
                                                             double *__restrict__ m64, DevState *st, float kh) {
    extern __shared__ __align__(16) float csw[];  // [d]
    const int c = st->pick;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->mmax_bits = 0u;  // the next round recomputes max_v m_v
    if (c < 0 || (int64_t)c >= n) return;                           // no valid pick (error already recorded)
    for (int i = threadIdx.x; i < d; i += blockDim.x) csw[i] = V[(int64_t)c * d + i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * FW + warp, nw = (int64_t)gridDim.x * FW;
    for (int64_t v0 = gw * UNRW; v0 < n; v0 += nw * UNRW) {
        float s[UNRW];
#pragma unroll
        for (int u = 0; u < UNRW; ++u) s[u] = 0.f;
        for (int s0 = 0; s0 < d; s0 += SLAB) {
            float cr[8];
            smem_slab<VEC4>(csw + s0, lane, d - s0, cr);
#pragma unroll
            for (int u = 0; u < UNRW; ++u) {
                float x[8];
                load_point<VEC4, 8, 32>(V + lmin(v0 + u, n - 1) * d + s0, lane, d - s0, x);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float df = x[k] - cr[k];
                    s[u] = fmaf(df, df, s[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UNRW; ++u) {
            const float su = group_sum<32>(s[u]);
            if (v0 + u >= n) continue;  // warp-uniform
            const double mv = m64[v0 + u];
            float mu, md;
            d2f_bounds(mv, mu, md);
            if (__fmul_rd(su, kh) >= mu) continue;  // d >= m_v: m_v stays (warp-uniform)
            const double de = df_dist_wide<VEC4>(V + (v0 + u) * d, csw, d, lane);
            if (lane == 0 && de < mv) m64[v0 + u] = de;
        }
    }
}

namespace {
// Dynamic shared memory above 48 KB: raise the kernel's limit once per
// (device, kernel) to what d = 4096 needs.
cudaError_t allow_wide_smem(const void *kernel) {
    static std::mutex mu;
    static std::vector<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &p : done)
        if (p.first == dev && p.second == kernel) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float) * FC * 4096));
    if (e == cudaSuccess) done.emplace_back(dev, kernel);
    return e;
}
}  // namespace

// every d up to 4096: the register kernels up to 256, the wide ones above
bool few_supported(const Ctx &c) { return c.d <= 4096; }

// Kernel variant for d: float4 lanes when d is a multiple of 4; lanes per
// point 8 (d <= 32), 16 (d <= 64) or 32; 4 dimensions per lane, 8 above
// d = 128.
#define FEW_DISPATCH(CALL)                \
    do {                                  \
        const bool v4 = c.d % 4 == 0;     \
        if (c.d <= 32) {                  \
            if (v4) CALL(true, 4, 8);     \
            else CALL(false, 4, 8);       \
        } else if (c.d <= 64) {           \
            if (v4) CALL(true, 4, 16);    \
            else CALL(false, 4, 16);      \
        } else if (c.d <= 128) {          \
            if (v4) CALL(true, 4, 32);    \
            else CALL(false, 4, 32);      \
        } else {                          \
            if (v4) CALL(true, 8, 32);    \
            else CALL(false, 8, 32);      \
        }                                 \
    } while (0)

// 1 - rho rounded down: the screen's scale for a proof that d >= m_v
float few_kh(int d) {
    const double rho = few_rho(d);
    float kh = (float)(1.0 - rho);
    if ((double)kh > 1.0 - rho) kh = nextafterf(kh, 0.f);
    return kh;
}

cudaError_t launch_few_bounds(Ctx &c, const int *list, const int *count, int cap, double *out_lo, double *out_hi,
                              int64_t chunk, int nchunks, int max_cnt) {
    // constants of the bound terms for the lane-tree rounding (see above)
    const double rho = few_rho(c.d);
    const float kh = few_kh(c.d);
    float kl = (float)(1.0 + 2.0 * rho);
    if ((double)kl < 1.0 + 2.0 * rho) kl = nextafterf(kl, 2.f);
    const int grid = c.num_sms * 4;
    if (c.d > FDMAX) {
        const size_t sm = sizeof(float) * FC * (size_t)c.d;
        const bool v4 = c.d % 4 == 0;
        const void *k = v4 ? (const void *)k_few_bounds_wide<true> : (const void *)k_few_bounds_wide<false>;
        if (cudaError_t e = allow_wide_smem(k); e != cudaSuccess) return e;
        if (v4)
            k_few_bounds_wide<true><<<grid, FW * 32, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk,
                                                                      nchunks, kh, kl, out_lo, out_hi, max_cnt);
        else
            k_few_bounds_wide<false><<<grid, FW * 32, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk,
                                                                       nchunks, kh, kl, out_lo, out_hi, max_cnt);
        return cudaGetLastError();
    }
#define CALL(V4, D, L)                                                                                          \
    k_few_bounds<V4, D, L><<<grid, FW * 32, 0, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk,       \
                                                           nchunks, kh, kl, out_lo, out_hi, max_cnt)
    FEW_DISPATCH(CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_few_exact(Ctx &c, const int *list, const int *count, int cap, double *out, int64_t chunk,
                             int nchunks) {
    const int grid = c.num_sms * 4;
    const float kh = few_kh(c.d);
    if (c.d > FDMAX) {
        const size_t sm = sizeof(float) * FC * (size_t)c.d;
        const bool v4 = c.d % 4 == 0;
        const void *k = v4 ? (const void *)k_few_exact_wide<true> : (const void *)k_few_exact_wide<false>;
        if (cudaError_t e = allow_wide_smem(k); e != cudaSuccess) return e;
        if (v4)
            k_few_exact_wide<true><<<grid, FW * 32, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk,
                                                                     nchunks, kh, out);
        else
            k_few_exact_wide<false><<<grid, FW * 32, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk,
                                                                      nchunks, kh, out);
        return cudaGetLastError();
    }
#define CALL(V4, D, L)                                                                                         \
    k_few_exact<V4, D, L><<<grid, FW * 32, 0, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk,       \
                                                          nchunks, kh, out)
    FEW_DISPATCH(CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_few_update(Ctx &c) {
    const int grid = c.num_sms * 8;
    const float kh = few_kh(c.d);
    if (c.d > FDMAX) {
        const size_t sm = sizeof(float) * (size_t)c.d;
        if (c.d % 4 == 0)
            k_few_update_wide<true><<<grid, FW * 32, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, c.st, kh);
        else
            k_few_update_wide<false><<<grid, FW * 32, sm, c.stream>>>(c.V32, c.n, c.d, c.m64, c.st, kh);
        return cudaGetLastError();
    }
#define CALL(V4, D, L) k_few_update<V4, D, L><<<grid, FW * 32, 0, c.stream>>>(c.V32, c.n, c.d, c.m64, c.st, kh)
    FEW_DISPATCH(CALL);
#undef CALL
    return cudaGetLastError();
}

#undef FEW_DISPATCH

}  // namespace ebc
