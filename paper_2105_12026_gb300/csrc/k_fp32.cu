// FP32 "plain" kernels on the CUDA cores: the direct (v - c)^2 form of the
// distance, as in the paper's GPU kernel (Algorithm 2), register-tiled.
//
//  * k_gains_fp32: partial[q][j] = sum over the V chunk q of
//        max(0, mu_v - k1 * dhat(v, c_j))
//    where dhat is the FP32 direct distance.  In upper-bound mode (Greedy)
//    mu_v = m_v rounded up to FP32 and k1 = 1 - rho rounded down, with
//    rho = (d + 4) 2^-24 >= the relative error of dhat, so every term bounds
//    max(0, m_v - d(v, c_j)) from above up to one rounding of the FMA.  In
//    plain mode mu_v = m_v rounded to nearest and k1 = 1.
//  * k_eval_sets_fp32: the work-matrix rows W[j, .] of Sec. 4.2 reduced on
//    the fly: for each set j and point v, min over members of dhat, then
//    max(0, ||v||^2 - min), summed over V in FP64.
#include <float.h>
#include <math.h>

#include "ebc_internal.cuh"

namespace ebc {

namespace {
constexpr int TC = 64;   // candidates per block tile
constexpr int TV = 128;  // points per block tile
constexpr int KC = 16;   // dimensions per smem stage
}  // namespace

// 256 threads, a tile of 128 candidates x 128 points: tx = tid % 16 covers 8
// points (two runs of 4), ty = tid / 16 covers 8 candidates (two runs of 4),
// 64 FP32 accumulators per thread.  Dimensions are staged 16 at a time in
// shared memory (dimension-major), double-buffered through registers: the
// next stage's global loads are issued before the current stage's
// arithmetic and stored to the other buffer after it, one barrier per
// stage.  Per (candidate, point) the arithmetic is the FMA chain over the
// dimensions in index order, and per candidate and point tile the 8 terms
// of a thread are summed in FP32, then the 16 lanes; the tile sums are
// added in FP32 over blocks of up to 16 point tiles (a sum of depth at most
// 28, within the bulk partials' error bound), and the blocks in FP64: the
// FP64 pipe, a few lanes per clock on GB300, then adds once per block.
namespace {
constexpr int FC = 128;  // candidates per block
constexpr int FV = 128;  // points per block tile
constexpr int FK = 16;   // dimensions per stage (32 measured slower: 0.69 vs 0.73 of the roof)
constexpr int FPT = FC * FK / 4 / 256;  // float4 pieces of each operand per thread and stage

template <bool VEC>
__device__ __forceinline__ void fp32_stage_load(const float *__restrict__ V, int d, const int *Ci, int64_t v0,
                                                int64_t ve, int k0, int tid, float4 (&cr)[FPT], float4 (&vr)[FPT]) {
    // 128 rows x FK dimensions of each operand in float4 pieces: FPT per thread
#pragma unroll
    for (int s = 0; s < FPT; ++s) {
        const int e = tid + 256 * s;
        const int r = e / (FK / 4), kq = (e % (FK / 4)) * 4;
        const int ci = Ci[r];
        const int64_t v = v0 + r;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (VEC) {  // d % 4 == 0: a piece is inside the row or wholly past it
            if (k0 + kq < d) {
                if (ci >= 0) x = *reinterpret_cast<const float4 *>(V + (int64_t)ci * d + k0 + kq);
                if (v < ve) y = *reinterpret_cast<const float4 *>(V + v * d + k0 + kq);
            }
        } else {
            float xs[4] = {0.f, 0.f, 0.f, 0.f}, ys[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (k0 + kq + i < d) {
                    if (ci >= 0) xs[i] = V[(int64_t)ci * d + k0 + kq + i];
                    if (v < ve) ys[i] = V[v * d + k0 + kq + i];
                }
            x = make_float4(xs[0], xs[1], xs[2], xs[3]);
            y = make_float4(ys[0], ys[1], ys[2], ys[3]);
        }
        cr[s] = x;
        vr[s] = y;
    }
}

// Packed FP32 pairs (sm_100+ f32x2 instructions): each element is computed
// and rounded exactly as the scalar instruction would.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long x, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ void fp32_stage_store(float (*Cs)[FC], float (*Vs)[FV], int tid, const float4 (&cr)[FPT],
                                                 const float4 (&vr)[FPT]) {
#pragma unroll
    for (int s = 0; s < FPT; ++s) {
        const int e = tid + 256 * s;
        const int r = e / (FK / 4), kq = (e % (FK / 4)) * 4;
        Cs[kq][r] = cr[s].x;
        Cs[kq + 1][r] = cr[s].y;
        Cs[kq + 2][r] = cr[s].z;
        Cs[kq + 3][r] = cr[s].w;
        Vs[kq][r] = vr[s].x;
        Vs[kq + 1][r] = vr[s].y;
        Vs[kq + 2][r] = vr[s].z;
        Vs[kq + 3][r] = vr[s].w;
    }
}
}  // namespace

template <bool VEC>
__global__ void __launch_bounds__(256, 1) k_gains_fp32(const float *__restrict__ V, int64_t n, int d,
                                                       const double *__restrict__ m64, const int *__restrict__ cand,
                                                       int64_t m, int upper, float k1, int64_t chunk,
                                                       double *__restrict__ partial) {
    extern __shared__ __align__(16) uint8_t fsm[];
    constexpr int OV = 2 * FK * FC * 4, OA = OV + 2 * FK * FV * 4, OM = OA + 8 * 256 * 8, OC = OM + 2 * FV * 4;
    auto Cs = reinterpret_cast<float (*)[FK][FC]>(fsm);       // [2][FK][FC]
    auto Vs = reinterpret_cast<float (*)[FK][FV]>(fsm + OV);  // [2][FK][FV]
    auto Accd = reinterpret_cast<double (*)[256]>(fsm + OA);  // [8][256]
    auto Ms = reinterpret_cast<float (*)[FV]>(fsm + OM);      // [2][FV]
    int *Ci = reinterpret_cast<int *>(fsm + OC);              // [FC]

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t c0 = (int64_t)blockIdx.x * FC;
    const int q = blockIdx.y;
    const int64_t vb = (int64_t)q * chunk;
    const int64_t ve = lmin(vb + chunk, n);
    const int nks = (d + FK - 1) / FK;                        // stages per point tile
    const int nvt = (int)((ve - vb + FV - 1) / FV);           // point tiles of the chunk
    const int nst = nvt * nks;                                // stages in all

    if (tid < FC) {
        const int64_t j = c0 + tid;
        Ci[tid] = j < m ? (cand ? cand[j] : (int)j) : -1;
    }
    __syncthreads();
    auto load_m = [&](int vt, int buf) {
        if (tid < FV) {
            const int64_t v = vb + (int64_t)vt * FV + tid;
            float mv = -INFINITY;
            if (v < ve) {
                const double md = m64[v];
                mv = upper ? __double2float_ru(md) : __double2float_rn(md);
            }
            Ms[buf][tid] = mv;
        }
    };
#pragma unroll
    for (int i = 0; i < 8; ++i) Accd[i][tid] = 0.0;
    // acc[i][p]: candidate i against the point pair p (points 2p, 2p + 1 of the thread's 8)
    unsigned long long acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[i][p] = 0ull;

    float tacc[8];  // FP32 sums of the current block of point tiles
#pragma unroll
    for (int i = 0; i < 8; ++i) tacc[i] = 0.f;
    int tb = 0;     // point tiles in the block
    float4 cr[FPT], vr[FPT];
    if (nst > 0) {
        fp32_stage_load<VEC>(V, d, Ci, vb, ve, 0, tid, cr, vr);
        fp32_stage_store(Cs[0], Vs[0], tid, cr, vr);
        load_m(0, 0);
    }
    __syncthreads();
    for (int st = 0; st < nst; ++st) {
        const int vt = st / nks, ks = st % nks;
        const int buf = st & 1;
        const bool more = st + 1 < nst;
        if (more) {
            const int vt1 = (st + 1) / nks, ks1 = (st + 1) % nks;
            fp32_stage_load<VEC>(V, d, Ci, vb + (int64_t)vt1 * FV, ve, ks1 * FK, tid, cr, vr);
        }
#pragma unroll
        for (int kk = 0; kk < FK; ++kk) {
            const float4 ca = *reinterpret_cast<const float4 *>(&Cs[buf][kk][ty * 4]);
            const float4 cb = *reinterpret_cast<const float4 *>(&Cs[buf][kk][64 + ty * 4]);
            const ulonglong2 va = *reinterpret_cast<const ulonglong2 *>(&Vs[buf][kk][tx * 4]);
            const ulonglong2 vb2 = *reinterpret_cast<const ulonglong2 *>(&Vs[buf][kk][64 + tx * 4]);
            const float cv[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
            const unsigned long long vv[4] = {va.x, va.y, vb2.x, vb2.y};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const unsigned long long c2 = f2_pack(cv[i], cv[i]);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const unsigned long long df = f2_sub(vv[p], c2);
                    acc[i][p] = f2_fma(df, df, acc[i][p]);
                }
            }
        }
        if (ks == nks - 1) {
            // the point tile is complete: relu terms, summed as described above
            const int mb = vt & 1;
            float mv[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                mv[j] = Ms[mb][tx * 4 + j];
                mv[4 + j] = Ms[mb][64 + tx * 4 + j];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float a[8];
#pragma unroll
                for (int p = 0; p < 4; ++p) f2_unpack(acc[i][p], a[2 * p], a[2 * p + 1]);
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) s += fmaxf(0.f, fmaf(-k1, a[j], mv[j]));
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                s += __shfl_xor_sync(0xffffffffu, s, 8);
                tacc[i] += s;
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[i][p] = 0ull;
            }
            if (++tb == 16 || !more) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    Accd[i][tid] += (double)tacc[i];
                    tacc[i] = 0.f;
                }
                tb = 0;
            }
        }
        if (more) {
            fp32_stage_store(Cs[buf ^ 1], Vs[buf ^ 1], tid, cr, vr);
            if ((st + 1) % nks == 0) load_m((st + 1) / nks, ((st + 1) / nks) & 1);
        }
        __syncthreads();
    }
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t j = c0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (j < m) partial[(int64_t)q * m + j] = Accd[i][tid];
        }
    }
}

cudaError_t launch_gains_fp32(Ctx &c, const int *cand, int64_t m, bool upper, int64_t chunk, int nchunks) {
    float k1 = 1.0f;
    if (upper) {
        double rho = (double)(c.d + 4) * ldexp(1.0, -24);
        double want = 1.0 - rho;
        k1 = (float)want;
        if ((double)k1 > want) k1 = nextafterf(k1, 0.f);  // round down
    }
    dim3 grid((unsigned)((m + FC - 1) / FC), (unsigned)nchunks);
    const size_t smem = (size_t)2 * FK * FC * 4 + (size_t)2 * FK * FV * 4 + (size_t)8 * 256 * 8 + 2 * FV * 4 + FC * 4;
    const void *kfn = c.d % 4 == 0 ? (const void *)k_gains_fp32<true> : (const void *)k_gains_fp32<false>;
    if (cudaError_t e = allow_smem(kfn, (uint32_t)smem); e != cudaSuccess) return e;
    if (c.d % 4 == 0)
        k_gains_fp32<true><<<grid, 256, smem, c.stream>>>(c.V32, c.n, c.d, c.m64, cand, m, upper ? 1 : 0, k1, chunk,
                                                          c.partial);
    else
        k_gains_fp32<false><<<grid, 256, smem, c.stream>>>(c.V32, c.n, c.d, c.m64, cand, m, upper ? 1 : 0, k1,
                                                           chunk, c.partial);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Rigorous [lo, hi] bounds of the gains of a device candidate list (count
// read from device memory), as chunk partials:
//   out_lo[e * nchunks + q] / out_hi[...] = sum over chunk q of the FP32
//   bound terms max(0, mD - kl s) / max(0, mU - kh s), s the FP32 direct
//   distance (see bound_consts in k_common.cu for the constants).
// Same register tiling as k_gains_fp32; grid-stride over (candidate tile of
// 64, chunk) items.  A thread adds its 8 terms per point tile in FP32, then
// the 16 lanes of a candidate in FP32, then tiles in FP64: at most
// 128 terms per FP32 sum.
// ---------------------------------------------------------------------------
// RES: rows of at most 128 dimensions; the candidate tile stays in shared
// memory for a whole (tile, chunk) item instead of being staged again for
// every point tile.  The pair arithmetic uses packed FP32x2 subtract and
// FMA (each element rounded as the scalar instruction would), so the FMA
// chain per pair over the dimensions in index order, and hence every bound,
// is the same in both forms.
constexpr int BF_DMAX = 128;

template <bool RES>
__global__ void __launch_bounds__(256) k_bounds_fp32(const float *__restrict__ V, int64_t n, int d,
                                                     const double *__restrict__ m64, const int *__restrict__ list,
                                                     const int *__restrict__ count, int cap, int64_t chunk,
                                                     int nchunks, float kh, float kl, double *__restrict__ out_lo,
                                                     double *__restrict__ out_hi, int min_cnt) {
    __shared__ __align__(16) float Cs[RES ? BF_DMAX : KC][TC];
    __shared__ __align__(16) float Vs[KC][TV];
    __shared__ float MsU[TV], MsD[TV];
    __shared__ int Ci[TC];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int cnt = min(*count, cap);
    if (cnt <= min_cnt) return;  // short lists: the few-candidate kernel
    const int ctiles = (cnt + TC - 1) / TC;
    const int64_t items = (int64_t)ctiles * nchunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int ct = (int)(it / nchunks);
        const int q = (int)(it % nchunks);
        const int64_t vb = (int64_t)q * chunk;
        const int64_t ve = lmin(vb + chunk, n);
        __syncthreads();
        if (tid < TC) {
            const int e = ct * TC + tid;
            Ci[tid] = e < cnt ? list[e] : -1;
        }
        if constexpr (RES) {
            __syncthreads();
            // the whole candidate tile, dimension-major, zero past d
            for (int e = tid; e < TC * BF_DMAX; e += 256) {
                const int r = e / BF_DMAX, k = e % BF_DMAX;
                const int ci = Ci[r];
                Cs[k][r] = (ci >= 0 && k < d) ? V[(int64_t)ci * d + k] : 0.f;
            }
        }
        double lod[4] = {0.0, 0.0, 0.0, 0.0}, hid[4] = {0.0, 0.0, 0.0, 0.0};
        // FP32 sums of blocks of up to 16 point tiles (depth <= 28, inside the
        // 131 * 2^-24 widening), then FP64: one FP64 add per block, not per tile
        float lob[4] = {0.f, 0.f, 0.f, 0.f}, hib[4] = {0.f, 0.f, 0.f, 0.f};
        int tb = 0;
        for (int64_t v0 = vb; v0 < ve; v0 += TV) {
            __syncthreads();
            if (tid < TV) {
                const int64_t v = v0 + tid;
                float mu = -INFINITY, md = -INFINITY;
                if (v < ve) {
                    const double mm = m64[v];
                    mu = __double2float_ru(mm);
                    md = __double2float_rd(mm);
                }
                MsU[tid] = mu;
                MsD[tid] = md;
            }
            // acc[i][p]: candidate i against the point pair p (points 2p, 2p + 1 of the thread's 8)
            unsigned long long acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int p2 = 0; p2 < 4; ++p2) acc[i][p2] = 0ull;
            for (int k0 = 0; k0 < d; k0 += KC) {
                __syncthreads();
                if constexpr (!RES) {
#pragma unroll
                    for (int s = 0; s < (TC * KC) / 256; ++s) {
                        int e = tid + 256 * s;
                        int r = e / KC, kk = e % KC;
                        int ci = Ci[r];
                        Cs[kk][r] = (ci >= 0 && k0 + kk < d) ? V[(int64_t)ci * d + k0 + kk] : 0.f;
                    }
                }
#pragma unroll
                for (int s = 0; s < (TV * KC) / 256; ++s) {
                    int e = tid + 256 * s;
                    int r = e / KC, kk = e % KC;
                    int64_t v = v0 + r;
                    Vs[kk][r] = (v < ve && k0 + kk < d) ? V[v * d + k0 + kk] : 0.f;
                }
                __syncthreads();
                const int kc0 = RES ? k0 : 0;
#pragma unroll
                for (int kk = 0; kk < KC; ++kk) {
                    const float4 c4 = *reinterpret_cast<const float4 *>(&Cs[kc0 + kk][ty * 4]);
                    const ulonglong2 va = *reinterpret_cast<const ulonglong2 *>(&Vs[kk][tx * 4]);
                    const ulonglong2 vb2 = *reinterpret_cast<const ulonglong2 *>(&Vs[kk][64 + tx * 4]);
                    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
                    const unsigned long long vv[4] = {va.x, va.y, vb2.x, vb2.y};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const unsigned long long c2 = f2_pack(cv[i], cv[i]);
#pragma unroll
                        for (int p2 = 0; p2 < 4; ++p2) {
                            const unsigned long long df = f2_sub(vv[p2], c2);
                            acc[i][p2] = f2_fma(df, df, acc[i][p2]);
                        }
                    }
                }
            }
            float mu[8], md[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                mu[j] = MsU[tx * 4 + j];
                mu[4 + j] = MsU[64 + tx * 4 + j];
                md[j] = MsD[tx * 4 + j];
                md[4 + j] = MsD[64 + tx * 4 + j];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float a[8];
#pragma unroll
                for (int p2 = 0; p2 < 4; ++p2) f2_unpack(acc[i][p2], a[2 * p2], a[2 * p2 + 1]);
                float sl = 0.f, sh = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    sh += fmaxf(fmaf(-kh, a[j], mu[j]), 0.f);
                    sl += fmaxf(fmaf(-kl, a[j], md[j]), 0.f);
                }
                sh += __shfl_xor_sync(0xffffffffu, sh, 1);
                sh += __shfl_xor_sync(0xffffffffu, sh, 2);
                sh += __shfl_xor_sync(0xffffffffu, sh, 4);
                sh += __shfl_xor_sync(0xffffffffu, sh, 8);
                sl += __shfl_xor_sync(0xffffffffu, sl, 1);
                sl += __shfl_xor_sync(0xffffffffu, sl, 2);
                sl += __shfl_xor_sync(0xffffffffu, sl, 4);
                sl += __shfl_xor_sync(0xffffffffu, sl, 8);
                hib[i] += sh;
                lob[i] += sl;
            }
            if (++tb == 16 || v0 + TV >= ve) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    hid[i] += (double)hib[i];
                    lod[i] += (double)lob[i];
                    hib[i] = lob[i] = 0.f;
                }
                tb = 0;
            }
        }
        if (tx == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = ct * TC + ty * 4 + i;
                if (e < cnt) {
                    out_lo[(int64_t)e * nchunks + q] = lod[i];
                    out_hi[(int64_t)e * nchunks + q] = hid[i];
                }
            }
        }
    }
}

cudaError_t launch_bounds_fp32(Ctx &c, const int *list, const int *count, int cap, double *out_lo, double *out_hi,
                               int64_t chunk, int nchunks, float kh, float kl, int min_cnt) {
    if (c.d <= BF_DMAX)
        k_bounds_fp32<true><<<c.num_sms * 4, 256, 0, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk,
                                                                 nchunks, kh, kl, out_lo, out_hi, min_cnt);
    else
        k_bounds_fp32<false><<<c.num_sms * 4, 256, 0, c.stream>>>(c.V32, c.n, c.d, c.m64, list, count, cap, chunk,
                                                                  nchunks, kh, kl, out_lo, out_hi, min_cnt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Multi-set evaluation, FP32 direct distances.
// Block: 128 threads, one point each; the block's 128 points are staged in
// shared memory dimension-major (Vt[i][t]) when d <= 128, otherwise each
// thread reads its own row.  Members are processed four at a time from a
// shared [dim][4] stage so one 16-byte load feeds four distances.
// Grid: (point tiles of 128, groups of SG sets).  Output: set_part[tile][j]
// = sum over the tile's points of max(0, ||v||^2 - min_{s in S_j} dhat(v, s)),
// summed in FP64.
// ---------------------------------------------------------------------------
namespace {
constexpr int ES_T = 128;
constexpr int ES_SG = 8;
constexpr int ES_DMAX_RES = 128;
constexpr int ES_DC = 256;  // member stage depth (dims) for the non-resident path
}  // namespace

template <bool RESIDENT>
__global__ void __launch_bounds__(ES_T) k_eval_sets_fp32(const float *__restrict__ V, int64_t n, int d,
                                                         const float *__restrict__ nv32, const int32_t *__restrict__ idx,
                                                         const int64_t *__restrict__ off, int64_t l,
                                                         double *__restrict__ set_part, DevState *st,
                                                         const int *__restrict__ bad) {
    if (*bad) return;  // offsets failed validation: read nothing
    extern __shared__ __align__(16) float esm[];
    float *Vt = esm;                                        // [d][ES_T] when RESIDENT
    float4 *S4 = reinterpret_cast<float4 *>(esm + (RESIDENT ? d * ES_T : 0));  // [dstage][4]
    const int dstage = RESIDENT ? d : min(d, ES_DC);
    const int t = threadIdx.x;
    const int64_t tile = blockIdx.x;
    const int64_t v = tile * ES_T + t;
    const bool vok = v < n;
    if (RESIDENT) {
        for (int e = t; e < d * ES_T; e += ES_T) {
            int r = e / d, i = e % d;
            int64_t vv = tile * ES_T + r;
            Vt[i * ES_T + r] = vv < n ? V[vv * d + i] : 0.f;
        }
    }
    const float nv = vok ? nv32[v] : 0.f;
    const int64_t j0 = (int64_t)blockIdx.y * ES_SG;
    for (int64_t j = j0; j < lmin(j0 + ES_SG, l); ++j) {
        const int64_t mb = off[j], me = off[j + 1];
        float dmin = INFINITY;
        for (int64_t s0 = mb; s0 < me; s0 += 4) {
            int mi[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t p = s0 + u;
                int x = p < me ? idx[p] : -1;
                if (p < me && (x < 0 || (int64_t)x >= n)) {
                    if (t == 0) atomicCAS(&st->err, 0, (int)EBC_EINDEX);
                    x = -1;
                }
                mi[u] = x;
            }
            float dist[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k0 = 0; k0 < d; k0 += dstage) {
                int kn = min(dstage, d - k0);
                __syncthreads();
                for (int e = t; e < kn * 4; e += ES_T) {
                    int i = e >> 2, u = e & 3;
                    float x = mi[u] >= 0 ? V[(int64_t)mi[u] * d + k0 + i] : 0.f;
                    reinterpret_cast<float *>(S4)[i * 4 + u] = x;
                }
                __syncthreads();
                if (vok) {
                    for (int i = 0; i < kn; ++i) {
                        float x = RESIDENT ? Vt[(k0 + i) * ES_T + t] : V[v * d + k0 + i];
                        float4 s4 = S4[i];
                        float d0 = x - s4.x, d1 = x - s4.y, d2 = x - s4.z, d3 = x - s4.w;
                        dist[0] = fmaf(d0, d0, dist[0]);
                        dist[1] = fmaf(d1, d1, dist[1]);
                        dist[2] = fmaf(d2, d2, dist[2]);
                        dist[3] = fmaf(d3, d3, dist[3]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (mi[u] >= 0) dmin = fminf(dmin, dist[u]);
        }
        double val = vok ? (double)fmaxf(0.f, nv - dmin) : 0.0;
        // block sum in FP64, fixed order
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
        __shared__ double red[ES_T / 32];
        __syncthreads();
        if ((t & 31) == 0) red[t >> 5] = val;
        __syncthreads();
        if (t == 0) {
            double s = 0.0;
            for (int w = 0; w < ES_T / 32; ++w) s += red[w];
            set_part[tile * l + j] = s;
        }
    }
}

// out_f[j0 + j] = (1/n) sum_q set_part[q * l + j]: one warp per set, lanes
// take the rows in a fixed strided assignment, then a fixed xor tree.
__global__ void k_sets_finalize(const double *__restrict__ set_part, int64_t ntiles, int64_t l, int64_t j0,
                                int64_t lall, double inv_n, double *__restrict__ out_f) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= l) return;  // whole warps leave together
    double s = 0.0;
    for (int64_t q = lane; q < ntiles; q += 32) s += set_part[q * l + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out_f[j0 + j] = s * inv_n;
    (void)lall;
}

cudaError_t launch_sets_finalize(Ctx &c, int64_t ntiles, int64_t lb, int64_t j0, int64_t l, double *out_f) {
    k_sets_finalize<<<(unsigned)((lb * 32 + 255) / 256), 256, 0, c.stream>>>(c.set_part, ntiles, lb, j0, l,
                                                                               1.0 / (double)c.n, out_f);
    return cudaGetLastError();
}

cudaError_t launch_eval_sets_fp32(Ctx &c, const int32_t *idx, const int64_t *off, int64_t l, double *out_f,
                                  const int *bad) {
    int64_t ntiles = (c.n + ES_T - 1) / ES_T;
    // process the sets in batches so the partials fit the scratch buffer
    // (and the set groups the grid's y extent, at most 65,535 blocks)
    int64_t batch = min(c.set_part_cap / ntiles, (int64_t)65535 * ES_SG);
    if (batch < 1) return cudaErrorMemoryAllocation;
    bool resident = c.d <= ES_DMAX_RES;
    size_t smem = resident ? (size_t)c.d * ES_T * 4 + (size_t)c.d * 16 : (size_t)min(c.d, ES_DC) * 16;
    if (resident && smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_eval_sets_fp32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    for (int64_t j0 = 0; j0 < l; j0 += batch) {
        int64_t lb = min(batch, l - j0);
        dim3 grid((unsigned)ntiles, (unsigned)((lb + ES_SG - 1) / ES_SG));
        if (resident)
            k_eval_sets_fp32<true><<<grid, ES_T, smem, c.stream>>>(c.V32, c.n, c.d, c.nv32, idx, off + j0, lb,
                                                                   c.set_part, c.st, bad);
        else
            k_eval_sets_fp32<false><<<grid, ES_T, smem, c.stream>>>(c.V32, c.n, c.d, c.nv32, idx, off + j0, lb,
                                                                    c.set_part, c.st, bad);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_sets_finalize(c, ntiles, lb, j0, l, out_f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ebc
