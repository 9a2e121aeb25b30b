// Bulk marginal gains on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For a tile of 128 candidates c (TMEM lanes) and 256 points v (TMEM
// columns) the tensor core forms D = C_hat . V_hat^T in FP32 from BF16/FP16
// rows, and the epilogue turns every entry into one term of
//     gain(c) = (1/n) sum_v max(0, m_v - d(v, c))
// through the norm expansion d_hat = ||v_hat||^2 + ||c_hat||^2 - 2 D:
//     t = 2 D + a_v + dc * w_v + b_c,
//     a_v = m_v - ||v_hat||^2 (+ slack),   b_c = -||c_hat||^2 (+ slack)
// then max(0, t) is summed over the 128 columns a thread owns in FP32 and
// over tiles in FP64.  Candidates sit on the lane axis so each thread's
// sum over V stays in its own registers (no shuffles).
//
// Greedy runs this kernel in upper-bound mode.  For a pair (v, c) that can
// contribute to the exact gain, d(v, c) < m_v, so ||v - c|| < sqrt(m_v), and
// with e = (v_hat - v) - (c_hat - c), |e| <= dv + dc (dv = ||v_hat - v||):
//   | ||v_hat - c_hat||^2 - ||v - c||^2 | = |2 (v - c).e + |e|^2|
//                                        <= (dv + dc)(2 sqrt(m_v) + dv + dc)
//   = [dv (2 sqrt(m_v) + dv)] + dc [2 sqrt(m_v) + 2 dv] + dc^2.
// The first bracket depends on v only and is added to a_v; the last term on
// c only and goes to b_c; the cross term is dc * w_v, one FMA per entry.
// Further slack in b_c: the FP32 accumulation of the tensor core,
// 2 gamma ||v_hat|| ||c_hat|| with gamma = (K/4 + 4) 2^-22 (one unit in the
// last place per four products plus four, far above the behaviour reported
// for NVIDIA tensor cores), bounded with max ||v_hat||; and the three FP32
// roundings of the epilogue, 2^-22 Z_c with Z_c a bound on every
// intermediate magnitude.  a_v and b_c are rounded up, so every term is >=
// the exact term max(0, m_v - d(v, c)): the sum is a rigorous upper bound on
// the exact gain, up to the relative error of the FP32 partial sums, which
// the caller accounts for.

// Warp roles (320 threads, one CTA per SM, persistent over work units):
//   warp 0      TMA producer: candidate tile (A, resident per unit, two
//               buffers) and a ring of point tiles (B stages)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warps 2..9  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, warps
//               2-5 the first 128 columns of an accumulator, 6-9 the rest
// Two 256-column FP32 accumulators (all 512 TMEM columns) let the epilogue
// of tile i overlap the MMAs of tile i+1.
//
// Every wait is bounded (tc_ptx.cuh); on a timeout the CTA records
// EBC_ETIMEOUT, stops issuing, waits (bounded) for its own TMA copies and
// MMAs in flight, frees TMEM and returns.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <float.h>
#include <math.h>

#include <algorithm>

#include "ebc_internal.cuh"
#include "tc_ptx.cuh"

namespace ebc {

namespace {
constexpr int BM = 128;          // candidates per tile
constexpr int BN = 256;          // points per tile
constexpr int KATOM = 64;        // 16-bit elements per 128-byte swizzle atom
constexpr int NTHREADS = 320;
constexpr int NEPI = 256;        // epilogue threads
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_LIMIT = 227 * 1024;

struct TcArgs {
    int64_t m;           // candidates
    int n_vtiles;        // point tiles covering n
    int n_ctiles;        // candidate tiles covering m
    int nchunks;         // V chunks
    int vt_per_chunk;    // point tiles per chunk
    int DP;              // padded K
    int nstages;         // B ring depth
    uint32_t idesc;      // instruction descriptor
    int upper;           // 1: upper-bound mode (Greedy), 0: plain gains
    const float *a32;    // [n_vtiles * BN] a_v, -inf past n
    const float *w32;    // [n_vtiles * BN] w_v
    const int *cand;     // candidate slot -> point index (nullptr: identity)
    const double *qn64;  // ||v_hat||^2
    const float *qerr;   // ||v_hat - v||
    const float *qnorm;  // ||v_hat||
    const float *qmax;   // [2] max qerr, max qnorm
    const unsigned int *mmax_bits;  // max_v m_v, FP32 bits
    double gamma;        // accumulation error factor
    double *partial;     // [nchunks][m]
    int *err;            // device error word
};

struct SmemLayout {
    uint32_t a_bytes, b_bytes, off_b, off_as, off_comb, off_bar, off_misc, total;
};

__host__ __device__ inline SmemLayout smem_layout(int DP, int nstages) {
    SmemLayout L;
    L.a_bytes = (uint32_t)BM * DP * 2;
    L.b_bytes = (uint32_t)BN * DP * 2;
    L.off_b = 2 * L.a_bytes;
    L.off_as = L.off_b + nstages * L.b_bytes;
    L.off_comb = L.off_as + 4 * BN * 4;  // a_s[2][BN], w_s[2][BN]
    L.off_bar = L.off_comb + BM * 8;
    L.off_misc = L.off_bar + (2 * nstages + 8) * 8;
    L.total = L.off_misc + 64 + 1024;  // + alignment slack for the 1024-byte base
    return L;
}

__device__ __forceinline__ void record_timeout(int *err, volatile int *abort) {
    *abort = 1;
    atomicCAS(err, 0, (int)EBC_ETIMEOUT);
}

}  // namespace

__global__ void __launch_bounds__(NTHREADS, 1)
    k_gains_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs args) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int ns = args.nstages;
    const SmemLayout L = smem_layout(args.DP, ns);
    uint8_t *sA = base;
    uint8_t *sB = base + L.off_b;
    float *a_s = reinterpret_cast<float *>(base + L.off_as);
    float *w_s = a_s + 2 * BN;
    double *comb = reinterpret_cast<double *>(base + L.off_comb);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + L.off_bar);
    uint64_t *empty = full + ns;
    uint64_t *a_full = empty + ns;
    uint64_t *a_empty = a_full + 2;
    uint64_t *t_full = a_empty + 2;
    uint64_t *t_empty = t_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + L.off_misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(base + L.off_misc + 4);
    // drain bookkeeping: parity of the last issued phase, -1 if none
    int *last_full = reinterpret_cast<int *>(base + L.off_misc + 8);      // [ns] (ns <= 8)
    int *last_afull = last_full + 8;                                        // [2]
    int *last_tfull = last_afull + 2;                                       // [2]

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int total_units = args.n_ctiles * args.nchunks;
    const int katoms = args.DP / KATOM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ns; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
            last_full[s] = -1;
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&a_full[b], 1);
            tc::mbar_init(&a_empty[b], 1);
            tc::mbar_init(&t_full[b], 1);
            tc::mbar_init(&t_empty[b], NEPI / 32);
            last_afull[b] = -1;
            last_tfull[b] = -1;
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            tc::tma_prefetch_desc(&tmA);
            tc::tma_prefetch_desc(&tmB);
            int g = 0, ua = 0;
            for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x, ++ua) {
                const int ct = u / args.nchunks, ch = u % args.nchunks;
                const int vt0 = ch * args.vt_per_chunk;
                const int vt1 = min(vt0 + args.vt_per_chunk, args.n_vtiles);
                const int ab = ua & 1;
                if (!tc::mbar_wait(&a_empty[ab], ((ua >> 1) & 1) ^ 1, abort_flag)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                tc::mbar_arrive_expect_tx(&a_full[ab], L.a_bytes);
                for (int j = 0; j < katoms; ++j)
                    tc::tma_load_2d(sA + ab * L.a_bytes + j * (BM * 128), &tmA, &a_full[ab], j * KATOM, ct * BM);
                last_afull[ab] = (ua >> 1) & 1;
                bool ok = true;
                for (int vt = vt0; vt < vt1; ++vt, ++g) {
                    const int s = g % ns;
                    const int ph = (g / ns) & 1;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
                        record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&full[s], L.b_bytes);
                    for (int j = 0; j < katoms; ++j)
                        tc::tma_load_2d(sB + s * L.b_bytes + j * (BN * 128), &tmB, &full[s], j * KATOM, vt * BN);
                    last_full[s] = ph;
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int g = 0, t = 0, ua = 0;
            for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x, ++ua) {
                const int ch = u % args.nchunks;
                const int vt0 = ch * args.vt_per_chunk;
                const int vt1 = min(vt0 + args.vt_per_chunk, args.n_vtiles);
                const int ab = ua & 1;
                if (!tc::mbar_wait(&a_full[ab], (ua >> 1) & 1, abort_flag)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                bool ok = true;
                for (int vt = vt0; vt < vt1; ++vt, ++g, ++t) {
                    const int s = g % ns;
                    const int b = t & 1;
                    if (!tc::mbar_wait(&full[s], (g / ns) & 1, abort_flag) ||
                        !tc::mbar_wait(&t_empty[b], ((t >> 1) & 1) ^ 1, abort_flag)) {
                        record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
                    const uint32_t a0 = tc::smem_u32(sA + ab * L.a_bytes);
                    const uint32_t b0 = tc::smem_u32(sB + s * L.b_bytes);
                    for (int kk = 0; kk < args.DP / 16; ++kk) {
                        const uint32_t j = kk >> 2, w = kk & 3;
                        const uint64_t ad = tc::sdesc_sw128(a0 + j * (BM * 128) + w * 32);
                        const uint64_t bd = tc::sdesc_sw128(b0 + j * (BN * 128) + w * 32);
                        tc::mma_f16(d_tmem, ad, bd, args.idesc, kk > 0 ? 1u : 0u);
                    }
                    tc::mma_commit(&empty[s]);
                    tc::mma_commit(&t_full[b]);
                    last_tfull[b] = (t >> 1) & 1;
                }
                if (!ok) break;
                tc::mma_commit(&a_empty[ab]);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2;           // 0..7
        const int q = warp & 3;            // TMEM lane quarter this warp may access
        const int half = ew >> 2;          // column half of the accumulator
        const int row = q * 32 + lane;     // candidate row within the tile
        const int etid = threadIdx.x - 64; // 0..255
        const double inv_big = ldexp(1.0, -22);
        int t = 0;
        bool alive = true;
        for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
            const int ct = u / args.nchunks, ch = u % args.nchunks;
            const int vt0 = ch * args.vt_per_chunk;
            const int vt1 = min(vt0 + args.vt_per_chunk, args.n_vtiles);
            const int64_t j = (int64_t)ct * BM + row;
            int cidx = -1;
            if (j < args.m) cidx = args.cand ? args.cand[j] : (int)j;
            float bc = 0.f, dc = 0.f;
            if (cidx >= 0) {
                const double qn = args.qn64[cidx];
                if (args.upper) {
                    const double M = (double)__uint_as_float(*args.mmax_bits);
                    const double sM = sqrt(M);
                    const double qe = (double)args.qerr[cidx];
                    const double qm = (double)args.qnorm[cidx];
                    const double dmax = (double)args.qmax[0], qmax = (double)args.qmax[1];
                    const double Eacc = 2.0 * args.gamma * qmax * qm;
                    const double Z = 2.0 * qmax * qm + qmax * qmax + M + dmax * (2.0 * sM + dmax) +
                                     qe * (2.0 * sM + 2.0 * dmax) + qn + qe * qe + Eacc;
                    bc = __double2float_ru(-qn + qe * qe + Eacc + Z * inv_big);
                    dc = __double2float_ru(qe);
                } else {
                    bc = __double2float_rn(-qn);
                }
            }
            double acc = 0.0;
            for (int vt = vt0; vt < vt1; ++vt, ++t) {
                const int b = t & 1;
                a_s[b * BN + etid] = args.a32[(int64_t)vt * BN + etid];
                w_s[b * BN + etid] = args.w32[(int64_t)vt * BN + etid];
                tc::named_bar_sync(1, NEPI);
                if (alive) {
                    // the TMEM loads below are warp-collective: decide per warp
                    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&t_full[b], (t >> 1) & 1, abort_flag));
                    if (!ok) {
                        if (lane == 0) record_timeout(args.err, abort_flag);
                        alive = false;
                    }
                }
                if (!alive) continue;
                tc::tc_fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + half * 128);
                const float *ap = a_s + b * BN + half * 128;
                const float *wp = w_s + b * BN + half * 128;
                float s = 0.f;
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    uint32_t r0[32], r1[32];
                    tc::tmem_ld32(taddr + rr * 64, r0);
                    tc::tmem_ld32(taddr + rr * 64 + 32, r1);
                    tc::tmem_ld_wait();
                    if (rr == 1) {
                        // this warp is done with accumulator b
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&t_empty[b]);
                    }
                    const float4 *ap4 = reinterpret_cast<const float4 *>(ap + rr * 64);
                    const float4 *wp4 = reinterpret_cast<const float4 *>(wp + rr * 64);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float4 a4 = ap4[i];
                        const float4 w4 = wp4[i];
                        const uint32_t *r = i < 8 ? &r0[4 * i] : &r1[4 * (i - 8)];
                        s += fmaxf(fmaf(dc, w4.x, fmaf(2.f, __uint_as_float(r[0]), a4.x)) + bc, 0.f);
                        s += fmaxf(fmaf(dc, w4.y, fmaf(2.f, __uint_as_float(r[1]), a4.y)) + bc, 0.f);
                        s += fmaxf(fmaf(dc, w4.z, fmaf(2.f, __uint_as_float(r[2]), a4.z)) + bc, 0.f);
                        s += fmaxf(fmaf(dc, w4.w, fmaf(2.f, __uint_as_float(r[3]), a4.w)) + bc, 0.f);
                    }
                }
                acc += (double)s;
            }
            // combine the two column halves in a fixed order
            if (half == 1) comb[row] = acc;
            tc::named_bar_sync(2, NEPI);
            if (half == 0 && cidx >= 0 && alive) args.partial[(int64_t)ch * args.m + j] = acc + comb[row];
            tc::named_bar_sync(2, NEPI);
        }
    }

    // ---------------------------------------------------------------- teardown
    __syncthreads();
    if (threadIdx.x == 0) {
        // nothing may still write shared memory or TMEM when the CTA leaves:
        // wait (bounded) for the last issued phase of every barrier
        volatile int never = 0;
        for (int s = 0; s < ns; ++s)
            if (last_full[s] >= 0) tc::mbar_wait(&full[s], (uint32_t)last_full[s], &never);
        for (int b = 0; b < 2; ++b) {
            if (last_afull[b] >= 0) tc::mbar_wait(&a_full[b], (uint32_t)last_afull[b], &never);
            if (last_tfull[b] >= 0) tc::mbar_wait(&t_full[b], (uint32_t)last_tfull[b], &never);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// Quantisation: v_hat = RN(v) in bf16 or fp16, zero padded to DP; FP64
// ||v_hat||^2, the quantisation error norm ||v_hat - v|| and ||v_hat||
// (both rounded up) and their maxima.  One thread per row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint16_t to_q(float x, int prec) {
    if (prec == EBC_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float from_q(uint16_t h, int prec) {
    if (prec == EBC_BF16) return __bfloat162float(__ushort_as_bfloat16(h));
    return __half2float(__ushort_as_half(h));
}

__global__ void k_quantize(const float *__restrict__ V, int64_t n, int d, int64_t n_pad, int DP, int prec,
                           uint16_t *__restrict__ Vq, double *__restrict__ qn64, float *__restrict__ qerr,
                           float *__restrict__ qnorm, float *__restrict__ a32, float *__restrict__ w32,
                           unsigned int *__restrict__ qmax_bits, int *__restrict__ err) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    uint16_t *dst = Vq + r * DP;
    if (r >= n) {
        for (int i = 0; i < DP; ++i) dst[i] = 0;
        qn64[r] = 0.0;
        qerr[r] = 0.f;
        qnorm[r] = 0.f;
        a32[r] = -INFINITY;
        w32[r] = 0.f;
        return;
    }
    const float *v = V + r * d;
    double qn = 0.0, e2 = 0.0;
    bool finite = true;
    for (int i = 0; i < DP; ++i) {
        float x = i < d ? v[i] : 0.f;
        uint16_t h = to_q(x, prec);
        dst[i] = h;
        float xq = from_q(h, prec);
        finite = finite && isfinite(xq);
        double xd = (double)xq;
        qn = __dadd_rn(qn, __dmul_rn(xd, xd));
        double e = xd - (double)x;
        e2 = __dadd_rn(e2, __dmul_rn(e, e));
    }
    if (!finite) atomicCAS(err, 0, (int)EBC_EINVAL);
    qn64[r] = qn;
    // the sums above carry at most (DP + 1) relative rounding errors of
    // 2^-53; pad the square roots by 2^-40 relative before rounding up
    float qe = __double2float_ru(__dsqrt_ru(e2) * (1.0 + ldexp(1.0, -40)));
    float qm = __double2float_ru(__dsqrt_ru(qn) * (1.0 + ldexp(1.0, -40)));
    qerr[r] = qe;
    qnorm[r] = qm;
    atomicMax(&qmax_bits[0], __float_as_uint(qe));
    atomicMax(&qmax_bits[1], __float_as_uint(qm));
}

// Per-round point terms.  Upper-bound mode: a_v = m_v - ||v_hat||^2 +
// dv (2 sqrt(m_v) + dv) and w_v = 2 sqrt(m_v) + 2 dv, both rounded up, and
// M = max_v m_v rounded up.  Plain mode: a_v = m_v - ||v_hat||^2 rounded to
// nearest and w_v = 0.
__global__ void k_prep_tc(const double *__restrict__ m64, const double *__restrict__ qn64,
                          const float *__restrict__ qerr, int64_t n, float *__restrict__ a32, float *__restrict__ w32,
                          int upper, unsigned int *__restrict__ mmax_bits) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float mx = 0.f;
    if (v < n) {
        double mv = m64[v];
        if (upper) {
            const double dv = (double)qerr[v];
            const double sq = __dsqrt_ru(mv);
            const double sv = __dmul_ru(dv, __dadd_ru(__dmul_ru(2.0, sq), dv));
            a32[v] = __double2float_ru(__dadd_ru(__dsub_ru(mv, qn64[v]), sv));
            w32[v] = __double2float_ru(__dadd_ru(__dmul_ru(2.0, sq), __dmul_ru(2.0, dv)));
            mx = __double2float_ru(mv);
        } else {
            a32[v] = __double2float_rn(mv - qn64[v]);
            w32[v] = 0.f;
        }
    }
    if (!upper) return;
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(mmax_bits, __float_as_uint(mx));
}

// Gather candidate rows of Vq into Cq (16 bytes per thread); invalid
// (sanitised, -1) candidates get a zero row.
__global__ void k_gather_rows(const uint16_t *__restrict__ Vq, const int *__restrict__ cand, int64_t m, int DP,
                              uint16_t *__restrict__ Cq) {
    const int per_row = DP / 8;  // uint4 per row
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m * per_row) return;
    int64_t j = e / per_row;
    int w = (int)(e % per_row);
    int c = cand[j];
    uint4 val = make_uint4(0, 0, 0, 0);
    if (c >= 0) val = reinterpret_cast<const uint4 *>(Vq + (int64_t)c * DP)[w];
    reinterpret_cast<uint4 *>(Cq + j * DP)[w] = val;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

cudaError_t make_map(CUtensorMap *map, void *gptr, int64_t rows, int DP, int prec, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)DP, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)DP * 2};
    cuuint32_t box[2] = {(cuuint32_t)KATOM, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, prec == EBC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, gptr,
                    dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int pick_stages(int DP) {
    for (int ns = 6; ns >= 2; --ns)
        if ((int)smem_layout(DP, ns).total <= SMEM_LIMIT) return ns;
    return 0;
}

}  // namespace

bool tc_supported(const Ctx &c) { return c.d <= 128; }

void tc_free(Ctx &c) {
    void *ptrs[] = {c.tc.Vq, c.tc.Cq, c.tc.qn64, c.tc.qerr, c.tc.qnorm, c.tc.qmax, c.tc.a32, c.tc.w32};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    c.tc = Ctx::Tc();
}

cudaError_t tc_quantize(Ctx &c) {
    Ctx::Tc &T = c.tc;
    cudaError_t e = cudaMemsetAsync(T.qmax, 0, 2 * sizeof(float), c.stream);
    if (e != cudaSuccess) return e;
    int th = 128;
    k_quantize<<<(unsigned)((T.n_pad + th - 1) / th), th, 0, c.stream>>>(
        c.V32, c.n, c.d, T.n_pad, T.DP, T.prec, T.Vq, T.qn64, T.qerr, T.qnorm, T.a32, T.w32,
        reinterpret_cast<unsigned int *>(T.qmax), &c.st->err);
    return cudaGetLastError();
}

cudaError_t tc_setup(Ctx &c, int prec) {
    Ctx::Tc &T = c.tc;
    if (T.Vq == nullptr) {
        T.n_pad = (c.n + BN - 1) / BN * BN;
        T.DP = (c.d + KATOM - 1) / KATOM * KATOM;
        size_t rows = (size_t)T.n_pad;
        cudaError_t e;
        if ((e = cudaMalloc(&T.Vq, rows * T.DP * 2)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&T.Cq, rows * T.DP * 2)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&T.qn64, rows * 8)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&T.qerr, rows * 4)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&T.qnorm, rows * 4)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&T.qmax, 2 * 4)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&T.a32, rows * 4)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&T.w32, rows * 4)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(T.Cq, 0, rows * T.DP * 2, c.stream)) != cudaSuccess) return e;
    }
    T.prec = prec;
    cudaError_t e = make_map(&T.tmA_V, T.Vq, T.n_pad, T.DP, prec, BM);
    if (e == cudaSuccess) e = make_map(&T.tmB_V, T.Vq, T.n_pad, T.DP, prec, BN);
    if (e == cudaSuccess) e = make_map(&T.tmA_C, T.Cq, T.n_pad, T.DP, prec, BM);
    if (e != cudaSuccess) return e;
    return tc_quantize(c);
}

cudaError_t launch_prep_tc(Ctx &c, bool upper) {
    int th = 256;
    k_prep_tc<<<(unsigned)((c.n + th - 1) / th), th, 0, c.stream>>>(c.m64, c.tc.qn64, c.tc.qerr, c.n, c.tc.a32,
                                                                     c.tc.w32, upper ? 1 : 0, &c.st->mmax_bits);
    return cudaGetLastError();
}

cudaError_t launch_gains_tc(Ctx &c, const int *cand, int64_t m, bool upper, int *nchunks_out) {
    Ctx::Tc &T = c.tc;
    const int DP = T.DP;
    const int ns = pick_stages(DP);
    if (ns == 0) return cudaErrorInvalidConfiguration;
    const SmemLayout L = smem_layout(DP, ns);
    static int configured_smem = 0;
    if (configured_smem < (int)L.total) {
        cudaError_t e = cudaFuncSetAttribute(k_gains_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
        if (e != cudaSuccess) return e;
        configured_smem = (int)L.total;
    }
    if (cand) {
        int64_t tot = m * (DP / 8);
        k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(T.Vq, cand, m, DP, T.Cq);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    TcArgs a;
    a.m = m;
    a.n_vtiles = (int)(T.n_pad / BN);
    a.n_ctiles = (int)((m + BM - 1) / BM);
    // V chunks: balance the persistent grid (units = candidate tiles x chunks)
    const int G = c.num_sms;
    const int64_t cap = c.partial_cap / std::max<int64_t>(m, 1);
    int best = 1;
    double best_eff = 0.0;
    for (int nch = 1; nch <= std::min<int64_t>(16, std::min<int64_t>(cap, a.n_vtiles)); ++nch) {
        int64_t units = (int64_t)a.n_ctiles * nch;
        int64_t per = (units + G - 1) / G;
        double eff = (double)units / (double)(per * std::min<int64_t>(G, units)) * (units < G ? (double)units / G : 1.0);
        eff *= 1.0 - 0.003 * nch;  // per-unit candidate-tile load
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = nch;
        }
    }
    a.nchunks = best;
    a.vt_per_chunk = (a.n_vtiles + best - 1) / best;
    a.nchunks = (a.n_vtiles + a.vt_per_chunk - 1) / a.vt_per_chunk;
    a.DP = DP;
    a.nstages = ns;
    a.idesc = tc::idesc_f16(T.prec == EBC_BF16 ? 1u : 0u, BM, BN);
    a.upper = upper ? 1 : 0;
    a.a32 = T.a32;
    a.w32 = T.w32;
    a.cand = cand;
    a.qn64 = T.qn64;
    a.qerr = T.qerr;
    a.qnorm = T.qnorm;
    a.qmax = T.qmax;
    a.mmax_bits = &c.st->mmax_bits;
    a.gamma = ((double)DP / 4.0 + 4.0) * ldexp(1.0, -22);
    a.partial = c.partial;
    a.err = &c.st->err;
    const int units = a.n_ctiles * a.nchunks;
    const int grid = std::min(units, G);
    k_gains_tc<<<grid, NTHREADS, L.total, c.stream>>>(cand ? T.tmA_C : T.tmA_V, T.tmB_V, a);
    *nchunks_out = a.nchunks;
    return cudaGetLastError();
}

}  // namespace ebc
