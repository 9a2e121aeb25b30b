// Bulk marginal gains on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// A work unit holds 256 candidates as two sub-tiles of 128 (TMEM lanes),
// each with its own 256-column TMEM region; every streamed tile of 256
// points feeds the MMAs of both sub-tiles, so each point byte brought into
// shared memory serves 256 candidates.  For a candidate c and point v the
// accumulator receives, entirely from the tensor core,
//     t(c, v) = c_hat . (2 v_hat) + X_c . Y_v
// where the 16 "extension" columns X (per candidate, static) and Y (per
// point, rewritten every round) carry the remaining terms of
//     m_v - d(v, c) ~= 2 c_hat.v_hat - ||c_hat||^2 + (m_v - ||v_hat||^2)
// plus, in upper-bound mode, a rigorous slack (below), each term split into
// two or three bf16 pieces whose sum is never below the term:
//     X = [q q q | s s | al al al' al' | 1 1 1 | 0..]   q = -||c_hat||^2, s = slack_c,
//     Y = [1 1 1 | sg sg | w w' w w'  | a a a | 0..]    al = ||c_hat - c||, a = a_v,
// giving q + sg*s + (al + al')(w + w') + a.  The epilogue only forms
// sum_v max(0, t) over the 128 columns a thread owns in blocks of up to four
// tiles (FP32, four chains of at most 128 terms each), then over blocks
// (FP64: GB300's FP64 pipe retires about two lanes per clock per SM, so it
// adds once per block, not once per tile).  Candidates sit on the lane axis, so a thread's sum over V stays in
// its registers.  Scaling v_hat by 2 is exact.
//
// Upper-bound mode (Greedy, sg = 1).  For a pair that can contribute to the
// exact gain, d(v, c) < m_v, so ||v - c|| < sqrt(m_v); with dv = ||v_hat - v||,
// dc = ||c_hat - c|| and e = (v_hat - v) - (c_hat - c), |e| <= dv + dc and
//   | ||v_hat - c_hat||^2 - ||v - c||^2 | = |2 (v - c).e + |e|^2|
//       <= dv (2 sqrt(m_v) + dv) + dc (2 sqrt(m_v) + 2 dv) + dc^2.
// The first part goes to a_v, the cross part is al * w with
// w = 2 sqrt(m_v) + 2 dv, and dc^2 goes to s_c.  The FP32 accumulation of the
// tensor core is bounded by gamma * sum |terms| with gamma = (K/4 + 4) 2^-22
// (one unit in the last place per four products plus four, far above the
// behaviour reported for NVIDIA tensor cores); its candidate part is in s_c,
// its point part in a_v.  Every piece is rounded so the sums are upper bounds,
// hence each max(0, t) >= max(0, m_v - d(v, c)) and the gain is a rigorous
// upper bound up to the relative error of the FP32 partial sums, which the
// caller accounts for.  Plain mode (sg = 0, w = 0, a rounded to nearest)
// gives the raw low-precision gain.
//
// Warp roles (352 threads, one CTA per SM, persistent over work units):
//   warp 0      TMA producer: the 256-candidate tile (A, one or two buffers)
//               and a ring of point tiles (B stages), each with its extension
//   warp 1      TMEM allocator and MMA issuer of candidate sub-tile 0 (one
//               thread): for every point tile, its MMAs into region 0
//   warp 10     MMA issuer of sub-tile 1 (one thread), into region 1.  A
//               tcgen05.mma holds its issuing thread for about its own
//               execution time, so each issuer waits and commits while the
//               other issues; with 256-byte rows they take turns (sub-tile 0
//               of a tile, then sub-tile 1), so region 0 completes first
//   warps 2..9  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, warps
//               2-5 the first 128 columns of a region, 6-9 the rest (one
//               128-column load each); they drain region 0 while region 1
//               fills and vice versa
// The two regions use all 512 TMEM columns.  The multi-set kernel and the
// K-blocked kernels use the same roles.
//
// Every wait is bounded (tc_ptx.cuh); on a timeout the CTA records
// EBC_ETIMEOUT, stops issuing, waits (bounded) for its own TMA copies and
// MMAs in flight, frees TMEM and returns.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <float.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "ebc_internal.cuh"
#include "tc_ptx.cuh"

namespace ebc {

namespace {
constexpr int BMS = 128;         // candidates per MMA sub-tile (TMEM lanes)
constexpr int BM = 2 * BMS;      // candidates per work unit (two sub-tiles share every point tile)
constexpr int BN = 256;          // points per tile (TMEM columns per region)
constexpr int NPAD = 256;        // row padding of the quantised arrays
constexpr int KATOM = 64;        // 16-bit elements per 128-byte swizzle atom
constexpr int KEXT = 16;         // extension columns (one MMA K step)
constexpr int NTHREADS_G = 352;  // producer, two MMA issuers, eight epilogue warps
constexpr int NEPI = 256;        // epilogue threads
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr float PAD_A = -1.0e30f;  // a_v of padding points: every term is 0

struct TcArgs {
    int64_t m;           // candidates
    int n_vtiles;        // point tiles covering n
    int n_ctiles;        // candidate tiles covering m
    int nchunks;         // V chunks
    int vt_per_chunk;    // point tiles per chunk
    int RB;              // bytes per row of the main part (whole 128-byte swizzle atoms)
    int xatom;           // elements per 128-byte atom: the TMA x step (64 for 16-bit, 128 for 8-bit)
    int nstages;         // B ring depth
    int na;              // candidate-tile buffers (1 or 2)
    uint32_t idesc;      // instruction descriptor, main part
    uint32_t idesc_ext;  // instruction descriptor, extension (bf16)
    double *partial;     // gains: [nchunks][m]; sets: [point units][lb]
    int *err;            // device error word
    const float *row_scale;  // FP8: factor of each A row's sums (nullptr: 1)
    // multi-set mode only
    const int64_t *chunks;  // [nchunks][4]: first set, end set, first column, end column
    const int *gset;        // per 16-column group: 2 * (set index within its chunk) + (last group of the set)
    int64_t lb;             // sets of this launch (partial row length)
    int64_t j0;             // first set of this launch
    // gains of a list whose length is on the device (lazy Greedy)
    const int *m_dev;       // list length, or nullptr when m and the plan above are final
    int64_t partial_cap;    // doubles of the partial buffer
    int G;                  // persistent CTAs
    int *nch_out;           // chunk count used, for the reduction kernel
    uint64_t wait_ns;       // limit of each pipeline wait (wait_limit_ns())
    // multi-set mode, plan on the device: this launch's chunks are records
    // [sets_bf[sets_batch], sets_bf[sets_batch + 1]) of `chunks`
    const int *sets_bf;
    int sets_batch;
    int turns;  // resident layout with two TMEM regions: issuers take turns (1) or run freely (0)
};

constexpr int MODE_GAINS = 0;
constexpr int MODE_SETS = 1;
constexpr int SET_GROUP = 16;       // members per group: sets are padded to multiples of 16

// The launch's work plan as plain values: from the arguments, or, for a
// list whose length is on the device, derived from that length (every CTA
// and thread computes the same plan).  The argument struct itself is never
// modified in the kernel.
struct Plan {
    int64_t m;         // candidates (gains) / unused (sets)
    int n_ctiles;      // A tiles
    int nchunks;       // units per A tile
    int vt_per_chunk;  // B tiles per unit (gains)
    int chunk0;        // sets: first chunk record of the launch
};

__device__ __forceinline__ Plan make_plan(const TcArgs &a) {
    Plan p;
    if (a.m_dev) {
        p.m = *reinterpret_cast<const volatile int *>(a.m_dev);
        int vpc = 1;
        p.nchunks = pick_chunks(p.m, a.n_vtiles, a.G, a.partial_cap, &vpc);
        p.vt_per_chunk = vpc;
        p.n_ctiles = (int)((p.m + BM - 1) / BM);
    } else {
        p.m = a.m;
        p.n_ctiles = a.n_ctiles;
        p.nchunks = a.nchunks;
        p.vt_per_chunk = a.vt_per_chunk;
    }
    p.chunk0 = 0;
    if (a.sets_bf) {
        const volatile int *bf = a.sets_bf;
        p.chunk0 = bf[a.sets_batch];
        p.nchunks = bf[a.sets_batch + 1] - p.chunk0;
    }
    return p;
}

// Work unit u -> A tile index, chunk, first B row and number of B tiles
// (of TBN points each in gains mode).
template <int MODE, int TBN = BN>
__device__ __forceinline__ void unit_span(const TcArgs &a, const Plan &P, int u, int &at, int &ch, int &b_row0,
                                          int &nb) {
    at = u / P.nchunks;
    ch = u % P.nchunks;
    if constexpr (MODE == MODE_GAINS) {
        const int vt0 = ch * P.vt_per_chunk;
        const int vt1 = min(vt0 + P.vt_per_chunk, a.n_vtiles);
        b_row0 = vt0 * TBN;
        nb = vt1 - vt0;
    } else {
        const int64_t *r = a.chunks + 4 * ((int64_t)P.chunk0 + ch);
        b_row0 = (int)r[2];
        nb = (int)((r[3] - r[2] + BN - 1) / BN);
    }
}

struct SmemLayout {
    uint32_t a_main, a_sub, a_bytes, b_main, b_bytes, off_b, off_comb, off_bar, off_misc, total;
    uint32_t off_ext;  // K-blocked layout: the extension buffer
};

// A buffer: sub-tile 0 (main K atoms, then its extension), sub-tile 1 (same).
// B stage of bn points: main K atoms, then the extension.
__host__ __device__ inline SmemLayout smem_layout(int RB, int nstages, int na, int bn = BN) {
    SmemLayout L;
    L.a_main = (uint32_t)BMS * RB;
    L.a_sub = L.a_main + BMS * KEXT * 2;
    L.a_bytes = 2 * L.a_sub;
    L.b_main = (uint32_t)bn * RB;
    L.b_bytes = L.b_main + bn * KEXT * 2;
    L.off_b = na * L.a_bytes;
    L.off_comb = L.off_b + nstages * L.b_bytes;
    L.off_bar = L.off_comb + 2 * BMS * 8;
    L.off_misc = L.off_bar + (2 * nstages + 8) * 8;
    // misc words, the four-region barriers of 128-point tiles and the
    // issuers' hand-over barriers, then the alignment slack for the
    // 1024-byte base
    L.total = L.off_misc + 160 + 1024;
    L.off_ext = 0;
    return L;
}

// K-blocked layout (candidate rows too long to stay resident): stages of
// one 128-byte K atom of both candidate sub-tiles and of the point tile
// (64 KB), then one buffer for the three extensions of a point tile (16 KB),
// loaded with the tile's last atom.
__host__ __device__ inline SmemLayout smem_layout_kb(int nstages) {
    SmemLayout L;
    L.a_main = 0;
    L.a_sub = 0;
    L.a_bytes = 2 * BMS * KEXT * 2 + BN * KEXT * 2;  // extension buffer
    L.b_main = 2 * BMS * 128 + BN * 128;             // one stage
    L.b_bytes = L.b_main;
    L.off_b = 0;
    L.off_ext = nstages * L.b_bytes;
    L.off_comb = L.off_ext + L.a_bytes;
    L.off_bar = L.off_comb + 2 * BMS * 8;
    L.off_misc = L.off_bar + (2 * nstages + 8) * 8;
    L.total = L.off_misc + 64 + 1024;
    return L;
}
constexpr int KB_STAGES = 3;

__device__ __forceinline__ void record_timeout(int *err, volatile int *abort) {
    *abort = 1;
    atomicCAS(err, 0, (int)EBC_ETIMEOUT);
}

// max of 16 consecutive accumulator words (three-input max, depth 3)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float max16(const uint32_t *x) {
    const float a0 = fmax3(__uint_as_float(x[0]), __uint_as_float(x[1]), __uint_as_float(x[2]));
    const float a1 = fmax3(__uint_as_float(x[3]), __uint_as_float(x[4]), __uint_as_float(x[5]));
    const float a2 = fmax3(__uint_as_float(x[6]), __uint_as_float(x[7]), __uint_as_float(x[8]));
    const float a3 = fmax3(__uint_as_float(x[9]), __uint_as_float(x[10]), __uint_as_float(x[11]));
    const float a4 = fmax3(__uint_as_float(x[12]), __uint_as_float(x[13]), __uint_as_float(x[14]));
    return fmaxf(fmax3(a0, a1, a2), fmax3(a3, a4, __uint_as_float(x[15])));
}

// Sums over the 32 lanes of 16 per-group values, as a reduce-scatter: lane l
// ends with the total of group group_of_lane(l) (2 lanes per group); 16
// shuffles, every total a fixed tree of 5 pair additions.
__device__ __forceinline__ int group_of_lane(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

__device__ __forceinline__ float reduce_scatter16(const float (&v)[16], int lane) {
    float t[8], u[4], w[2];
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4, b2 = lane & 2;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        t[j] = (b16 ? v[j + 8] : v[j]) + __shfl_xor_sync(0xffffffffu, b16 ? v[j] : v[j + 8], 16);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        u[j] = (b8 ? t[j + 4] : t[j]) + __shfl_xor_sync(0xffffffffu, b8 ? t[j] : t[j + 4], 8);
#pragma unroll
    for (int j = 0; j < 2; ++j)
        w[j] = (b4 ? u[j + 2] : u[j]) + __shfl_xor_sync(0xffffffffu, b4 ? u[j] : u[j + 2], 4);
    float x = (b2 ? w[1] : w[0]) + __shfl_xor_sync(0xffffffffu, b2 ? w[0] : w[1], 2);
    return x + __shfl_xor_sync(0xffffffffu, x, 1);
}

// Running sums of max(0, x) over accumulator words with packed FP32x2 adds:
// two 64-bit accumulators hold four FP32 chains, word i of every 32-word
// group going to chain i % 4 (8 terms per group and chain).  Words 0, 1 of
// every four take max(x, 0) (ALU pipe); words 2, 3 take x + |x| = 2 max(x, 0)
// exactly (one FMA-pipe add with an absolute-value operand), so the ALU pipe
// does half of that work; relu_fold halves those chains (exact) when it
// joins them.  A caller that folds after at most 16 groups (4 tiles of 128
// columns, or 8 of 64) keeps every chain an ordinary FP32 sum of at most 128
// non-negative terms.
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

struct ReluAcc {
    unsigned long long a, b;
};

__device__ __forceinline__ void relu_zero(ReluAcc &s) {
    s.a = pack2(0.f, 0.f);
    s.b = pack2(0.f, 0.f);
}

__device__ __forceinline__ float twice_relu(uint32_t w) {
    const float x = __uint_as_float(w);
    return x + fabsf(x);
}

__device__ __forceinline__ void relu_acc32(ReluAcc &s, const uint32_t *r) {
#pragma unroll
    for (int i = 0; i < 32; i += 4) {
        const unsigned long long x = pack2(fmaxf(__uint_as_float(r[i]), 0.f), fmaxf(__uint_as_float(r[i + 1]), 0.f));
        const unsigned long long y = pack2(twice_relu(r[i + 2]), twice_relu(r[i + 3]));
        asm("add.rn.f32x2 %0, %0, %1;" : "+l"(s.a) : "l"(x));
        asm("add.rn.f32x2 %0, %0, %1;" : "+l"(s.b) : "l"(y));
    }
}

__device__ __forceinline__ float relu_fold(const ReluAcc &s) {
    float alo, ahi, blo, bhi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(alo), "=f"(ahi) : "l"(s.a));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(blo), "=f"(bhi) : "l"(s.b));
    return (alo + ahi) + 0.5f * (blo + bhi);
}

}  // namespace

// The warp-specialised TMA -> tcgen05 -> TMEM pipeline, shared by the bulk
// gains (MODE_GAINS: A = candidates, B = points, epilogue = relu row sums)
// and the multi-set evaluation (MODE_SETS: A = points, B = set members,
// epilogue = per-set maxima and sums over the points).
//
// KB: rows longer than the resident layout allows.  Every stage carries one
// K atom of both A sub-tiles and of the B tile; a B tile's MMAs accumulate
// over all K atoms (the same MMA sequence, hence the same FP32
// accumulation, as the resident layout) and the extension step follows the
// last atom.
//
// TBN: points per B tile (TMEM columns per region) of the resident gains
// pipeline, 256 or 128.  At 128 a B stage takes half the shared memory (so
// deeper rings fit), each epilogue thread sums 64 columns per tile, and the
// 512 TMEM columns hold two sets of the two sub-tile regions: tile t
// accumulates into set t % 2, so the MMAs of a tile never wait for the
// epilogue of the previous one.  The MMA sequence over K is the same.
template <int MODE, bool F8, bool KB = false, int TBN = BN, bool ES = false>
__device__ __forceinline__ void tc_pipeline(const CUtensorMap *tmA_p, const CUtensorMap *tmAx_p,
                                            const CUtensorMap *tmB_p, const CUtensorMap *tmBx_p, const TcArgs &args) {
    static_assert(!KB || !F8, "K-blocked layout: 16-bit operands only");
    static_assert(TBN == BN || (TBN == 128 && MODE == MODE_GAINS && !KB), "128-point tiles: resident gains only");
    static_assert(!ES || (MODE == MODE_GAINS && TBN == BN), "region-split drain: 256-point gains only");
    // one MMA issuer per A sub-tile (warp 1 and the last warp), each waiting
    // and committing while the other issues (every variant)
    constexpr bool DUAL = true;
    constexpr int NREG = TBN == 128 ? 4 : 2;  // TMEM regions
    // with two regions the issuers may take turns (sub-tile 0 of a tile, then
    // sub-tile 1, then sub-tile 0 of the next), so region 0 completes half a
    // tile before region 1 and its epilogue overlaps region 1's MMAs (pays
    // off for long rows); otherwise their MMAs interleave freely
    const bool turns = DUAL && NREG == 2 && args.turns != 0;
    static_assert(!DUAL || NTHREADS_G / 32 - 1 >= 10, "the second issuer follows the epilogue warps");
    constexpr int RH = NREG / 2;               // point tiles in flight in TMEM
    constexpr uint32_t kTmemCols = NREG * TBN;
    const CUtensorMap &tmA = *tmA_p, &tmAx = *tmAx_p, &tmB = *tmB_p, &tmBx = *tmBx_p;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int ns = args.nstages;
    const int na = args.na;
    const SmemLayout L = KB ? smem_layout_kb(ns) : smem_layout(args.RB, ns, na, TBN);
    uint8_t *sA = base;
    uint8_t *sB = base + L.off_b;
    double *comb = reinterpret_cast<double *>(base + L.off_comb);  // [2][BMS]
    uint64_t *full = reinterpret_cast<uint64_t *>(base + L.off_bar);
    uint64_t *empty = full + ns;
    uint64_t *a_full = empty + ns;
    uint64_t *a_empty = a_full + 2;
    // per TMEM region: region (t % RH) * 2 + h holds sub-tile h of point tile t
    uint64_t *t_full = NREG == 2 ? a_empty + 2 : reinterpret_cast<uint64_t *>(base + L.off_misc + 64);
    uint64_t *t_empty = t_full + NREG;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + L.off_misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(base + L.off_misc + 4);
    // drain bookkeeping: parity of the last issued phase, -1 if none
    int *last_full = reinterpret_cast<int *>(base + L.off_misc + 8);  // [ns] (ns <= 8)
    int *last_afull = last_full + 8;                                    // [2]
    int *last_tfull = NREG == 2 ? last_afull + 2 : reinterpret_cast<int *>(base + L.off_misc + 128);  // [NREG]
    // teardown: one commit after every MMA this CTA issued (misc + 56 .. 64)
    uint64_t *fin = reinterpret_cast<uint64_t *>(base + L.off_misc + 56);
    // issuer turns: tok[0] "sub-tile 0 of tile t issued", tok[1] "sub-tile 1 of tile t issued"
    uint64_t *tok = reinterpret_cast<uint64_t *>(base + L.off_misc + 144);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t wait_ns = args.wait_ns;  // limit of every pipeline wait (the teardown keeps kWaitNs)
    const Plan P = make_plan(args);
    if (blockIdx.x == 0 && threadIdx.x == 0 && args.nch_out) *args.nch_out = P.nchunks;
    const int total_units = P.n_ctiles * P.nchunks;
    const int katoms = args.RB / 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ns; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], DUAL ? 2 : 1);
            last_full[s] = -1;
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&a_full[b], 1);
            tc::mbar_init(&a_empty[b], DUAL ? 2 : 1);
            last_afull[b] = -1;
        }
        for (int r = 0; r < NREG; ++r) {
            tc::mbar_init(&t_full[r], 1);
            // every epilogue warp drains every region in gains mode, half of them each in sets mode
            tc::mbar_init(&t_empty[r], (MODE == MODE_GAINS && !ES) ? NEPI / 32 : NEPI / 64);
            last_tfull[r] = -1;
        }
        tc::mbar_init(fin, DUAL ? 2 : 1);
        tc::mbar_init(&tok[0], 1);
        tc::mbar_init(&tok[1], 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, kTmemCols);
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
            tc::tma_prefetch_desc(&tmAx);
            tc::tma_prefetch_desc(&tmB);
            tc::tma_prefetch_desc(&tmBx);
            int g = 0, ua = 0;
            if constexpr (KB) {
                // one stage per (point tile, K atom): A atom of both
                // sub-tiles and B atom; with the tile's last atom its
                // extensions into the extension buffer (barriers a_full[0] /
                // a_empty[0], one phase per point tile)
                uint8_t *sx = base + L.off_ext;
                int tt = 0;
                for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x) {
                    int ct, ch, b_row0, nb;
                    unit_span<MODE>(args, P, u, ct, ch, b_row0, nb);
                    bool ok = true;
                    for (int i = 0; i < nb && ok; ++i, ++tt) {
                        const int brow = b_row0 + i * BN;
                        for (int j = 0; j < katoms; ++j, ++g) {
                            const int s = g % ns;
                            const int ph = (g / ns) & 1;
                            if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag, wait_ns)) {
                                record_timeout(args.err, abort_flag);
                                ok = false;
                                break;
                            }
                            uint8_t *st = sB + s * L.b_bytes;
                            tc::mbar_arrive_expect_tx(&full[s], L.b_main);
                            for (int h = 0; h < 2; ++h)
                                tc::tma_load_2d(st + h * (BMS * 128), &tmA, &full[s], j * args.xatom, ct * BM + h * BMS);
                            tc::tma_load_2d(st + 2 * BMS * 128, &tmB, &full[s], j * args.xatom, brow);
                            last_full[s] = ph;
                            if (j == katoms - 1) {
                                if (!tc::mbar_wait(&a_empty[0], (tt & 1) ^ 1, abort_flag, wait_ns)) {
                                    record_timeout(args.err, abort_flag);
                                    ok = false;
                                    break;
                                }
                                tc::mbar_arrive_expect_tx(&a_full[0], L.a_bytes);
                                for (int h = 0; h < 2; ++h)
                                    tc::tma_load_2d(sx + h * (BMS * KEXT * 2), &tmAx, &a_full[0], 0, ct * BM + h * BMS);
                                tc::tma_load_2d(sx + 2 * (BMS * KEXT * 2), &tmBx, &a_full[0], 0, brow);
                                last_afull[0] = tt & 1;
                            }
                        }
                    }
                    if (!ok) break;
                }
            } else
            for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x, ++ua) {
                int ct, ch, b_row0, nb;
                unit_span<MODE, TBN>(args, P, u, ct, ch, b_row0, nb);
                const int ab = ua % na;
                const int aph = (ua / na) & 1;
                if (!tc::mbar_wait(&a_empty[ab], aph ^ 1, abort_flag, wait_ns)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                uint8_t *abuf = sA + ab * L.a_bytes;
                tc::mbar_arrive_expect_tx(&a_full[ab], L.a_bytes);
                for (int h = 0; h < 2; ++h) {
                    uint8_t *sub = abuf + h * L.a_sub;
                    const int row0 = ct * BM + h * BMS;
                    for (int j = 0; j < katoms; ++j)
                        tc::tma_load_2d(sub + j * (BMS * 128), &tmA, &a_full[ab], j * args.xatom, row0);
                    tc::tma_load_2d(sub + L.a_main, &tmAx, &a_full[ab], 0, row0);
                }
                last_afull[ab] = aph;
                bool ok = true;
                for (int i = 0; i < nb; ++i, ++g) {
                    const int s = g % ns;
                    const int ph = (g / ns) & 1;
                    const int brow = b_row0 + i * TBN;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag, wait_ns)) {
                        record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    uint8_t *bbuf = sB + s * L.b_bytes;
                    tc::mbar_arrive_expect_tx(&full[s], L.b_bytes);
                    for (int j = 0; j < katoms; ++j)
                        tc::tma_load_2d(bbuf + j * (TBN * 128), &tmB, &full[s], j * args.xatom, brow);
                    tc::tma_load_2d(bbuf + L.b_main, &tmBx, &full[s], 0, brow);
                    last_full[s] = ph;
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1 || (DUAL && warp == NTHREADS_G / 32 - 1)) {
        // ------------------------------------------------------------ MMA issuer
        // For every point tile: sub-tile 0 into TMEM region 0, then sub-tile 1
        // into region 1.  The epilogue drains one region while the other fills.
        if (lane == 0) {
            int g = 0, t = 0, ua = 0;
            if constexpr (DUAL && KB) {
                // sub-tile h of every point tile, accumulated over all K atoms;
                // both issuers wait for the same stages and extension buffer and
                // both commit their release (count 2)
                const int h = warp == 1 ? 0 : 1;
                const uint32_t sx = tc::smem_u32(base + L.off_ext);
                for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x) {
                    int ct, ch, b_row0, nb;
                    unit_span<MODE>(args, P, u, ct, ch, b_row0, nb);
                    bool ok = true;
                    for (int i = 0; i < nb && ok; ++i, ++t) {
                        const uint32_t d_tmem = tmem_base + (uint32_t)(h * BN);
                        for (int j = 0; j < katoms; ++j, ++g) {
                            const int s = g % ns;
                            if (!tc::mbar_wait(&full[s], (g / ns) & 1, abort_flag, wait_ns)) {
                                record_timeout(args.err, abort_flag);
                                ok = false;
                                break;
                            }
                            const bool last = j == katoms - 1;
                            if (last && !tc::mbar_wait(&a_full[0], t & 1, abort_flag, wait_ns)) {
                                record_timeout(args.err, abort_flag);
                                ok = false;
                                break;
                            }
                            if (j == 0 && !tc::mbar_wait(&t_empty[h], (t & 1) ^ 1, abort_flag, wait_ns)) {
                                record_timeout(args.err, abort_flag);
                                ok = false;
                                break;
                            }
                            tc::tc_fence_after();
                            const uint32_t st = tc::smem_u32(sB + s * L.b_bytes);
                            const uint32_t b0 = st + 2 * BMS * 128;
                            const uint32_t ah = st + h * (BMS * 128);
                            for (int w = 0; w < 4; ++w) {
                                const uint64_t ad = tc::sdesc_sw128(ah + w * 32);
                                const uint64_t bd = tc::sdesc_sw128(b0 + w * 32);
                                tc::mma_f16(d_tmem, ad, bd, args.idesc, (j > 0 || w > 0) ? 1u : 0u);
                            }
                            if (last) {
                                tc::mma_f16(d_tmem, tc::sdesc_sw32(sx + h * (BMS * KEXT * 2)),
                                            tc::sdesc_sw32(sx + 2 * (BMS * KEXT * 2)), args.idesc_ext, 1u);
                                tc::mma_commit(&a_empty[0]);
                            }
                            tc::mma_commit(&empty[s]);
                        }
                        if (!ok) break;
                        tc::mma_commit(&t_full[h]);
                        last_tfull[h] = t & 1;
                    }
                    if (!ok) break;
                }
            } else if constexpr (DUAL) {
                // sub-tile h of every point tile; both issuers wait for the same
                // A and B stages and both commit their release (count 2)
                const int h = warp == 1 ? 0 : 1;
                for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x, ++ua) {
                    int ct, ch, b_row0, nb;
                    unit_span<MODE, TBN>(args, P, u, ct, ch, b_row0, nb);
                    const int ab = ua % na;
                    if (!tc::mbar_wait(&a_full[ab], (ua / na) & 1, abort_flag, wait_ns)) {
                        record_timeout(args.err, abort_flag);
                        break;
                    }
                    const uint32_t ah = tc::smem_u32(sA + ab * L.a_bytes) + h * L.a_sub;
                    bool ok = true;
                    for (int i = 0; i < nb; ++i, ++g, ++t) {
                        const int s = g % ns;
                        if (!tc::mbar_wait(&full[s], (g / ns) & 1, abort_flag, wait_ns)) {
                            record_timeout(args.err, abort_flag);
                            ok = false;
                            break;
                        }
                        const uint32_t b0 = tc::smem_u32(sB + s * L.b_bytes);
                        const uint32_t tpar = (uint32_t)(t / RH) & 1u;
                        const int rg = (t % RH) * 2 + h;
                        if (!tc::mbar_wait(&t_empty[rg], tpar ^ 1u, abort_flag, wait_ns)) {
                            record_timeout(args.err, abort_flag);
                            ok = false;
                            break;
                        }
                        // this issuer's turn: sub-tile 1 of tile t follows sub-tile 0
                        // of tile t, sub-tile 0 of tile t follows sub-tile 1 of t - 1
                        if (turns && (h == 1 || t > 0) &&
                            !tc::mbar_wait(&tok[1 - h], (uint32_t)(h == 1 ? t : t - 1) & 1u, abort_flag, wait_ns)) {
                            record_timeout(args.err, abort_flag);
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t d_tmem = tmem_base + (uint32_t)(rg * TBN);
                        // one MMA per 32 bytes of K (16 16-bit or 32 8-bit elements)
                        for (int kk = 0; kk < args.RB / 32; ++kk) {
                            const uint32_t j = kk >> 2, w = kk & 3;
                            const uint64_t ad = tc::sdesc_sw128(ah + j * (BMS * 128) + w * 32);
                            const uint64_t bd = tc::sdesc_sw128(b0 + j * (TBN * 128) + w * 32);
                            if constexpr (F8)
                                tc::mma_f8(d_tmem, ad, bd, args.idesc, kk > 0 ? 1u : 0u);
                            else
                                tc::mma_f16(d_tmem, ad, bd, args.idesc, kk > 0 ? 1u : 0u);
                        }
                        tc::mma_f16(d_tmem, tc::sdesc_sw32(ah + L.a_main), tc::sdesc_sw32(b0 + L.b_main),
                                    args.idesc_ext, 1u);
                        if (turns) tc::mbar_arrive(&tok[h]);
                        tc::mma_commit(&t_full[rg]);
                        last_tfull[rg] = (int)tpar;
                        tc::mma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    tc::mma_commit(&a_empty[ab]);
                }
            } else if constexpr (KB) {
                // both TMEM regions accumulate one point tile over all K atoms
                for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x) {
                    int ct, ch, b_row0, nb;
                    unit_span<MODE>(args, P, u, ct, ch, b_row0, nb);
                    bool ok = true;
                    for (int i = 0; i < nb && ok; ++i, ++t) {
                        // region h is awaited at its first MMA of the tile: region 0
                        // fills again while the epilogue still drains region 1
                        for (int j = 0; j < katoms; ++j, ++g) {
                            const int s = g % ns;
                            if (!tc::mbar_wait(&full[s], (g / ns) & 1, abort_flag, wait_ns)) {
                                record_timeout(args.err, abort_flag);
                                ok = false;
                                break;
                            }
                            tc::tc_fence_after();
                            const uint32_t st = tc::smem_u32(sB + s * L.b_bytes);
                            const uint32_t b0 = st + 2 * BMS * 128;
                            const bool last = j == katoms - 1;
                            if (last && !tc::mbar_wait(&a_full[0], t & 1, abort_flag, wait_ns)) {
                                record_timeout(args.err, abort_flag);
                                ok = false;
                                break;
                            }
                            if (last) tc::tc_fence_after();
                            const uint32_t sx = tc::smem_u32(base + L.off_ext);
                            for (int h = 0; h < 2 && ok; ++h) {
                                if (j == 0) {
                                    if (!tc::mbar_wait(&t_empty[h], (t & 1) ^ 1, abort_flag, wait_ns)) {
                                        record_timeout(args.err, abort_flag);
                                        ok = false;
                                        break;
                                    }
                                    tc::tc_fence_after();
                                }
                                const uint32_t d_tmem = tmem_base + (uint32_t)(h * BN);
                                const uint32_t ah = st + h * (BMS * 128);
                                for (int w = 0; w < 4; ++w) {
                                    const uint64_t ad = tc::sdesc_sw128(ah + w * 32);
                                    const uint64_t bd = tc::sdesc_sw128(b0 + w * 32);
                                    tc::mma_f16(d_tmem, ad, bd, args.idesc, (j > 0 || w > 0) ? 1u : 0u);
                                }
                                if (last)
                                    tc::mma_f16(d_tmem, tc::sdesc_sw32(sx + h * (BMS * KEXT * 2)),
                                                tc::sdesc_sw32(sx + 2 * (BMS * KEXT * 2)), args.idesc_ext, 1u);
                            }
                            if (!ok) break;
                            if (last) tc::mma_commit(&a_empty[0]);
                            tc::mma_commit(&empty[s]);
                        }
                        if (!ok) break;
                        for (int h = 0; h < 2; ++h) {
                            tc::mma_commit(&t_full[h]);
                            last_tfull[h] = t & 1;
                        }
                    }
                    if (!ok) break;
                }
            } else
            for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x, ++ua) {
                int ct, ch, b_row0, nb;
                unit_span<MODE, TBN>(args, P, u, ct, ch, b_row0, nb);
                const int ab = ua % na;
                if (!tc::mbar_wait(&a_full[ab], (ua / na) & 1, abort_flag, wait_ns)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                const uint32_t a0 = tc::smem_u32(sA + ab * L.a_bytes);
                bool ok = true;
                for (int i = 0; i < nb && ok; ++i, ++g, ++t) {
                    const int s = g % ns;
                    if (!tc::mbar_wait(&full[s], (g / ns) & 1, abort_flag, wait_ns)) {
                        record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    const uint32_t b0 = tc::smem_u32(sB + s * L.b_bytes);
                    const uint32_t tpar = (uint32_t)(t / RH) & 1u;
                    for (int h = 0; h < 2; ++h) {
                        const int rg = (t % RH) * 2 + h;
                        if (!tc::mbar_wait(&t_empty[rg], tpar ^ 1u, abort_flag, wait_ns)) {
                            record_timeout(args.err, abort_flag);
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t d_tmem = tmem_base + (uint32_t)(rg * TBN);
                        const uint32_t ah = a0 + h * L.a_sub;
                        // one MMA per 32 bytes of K (16 16-bit or 32 8-bit elements)
                        for (int kk = 0; kk < args.RB / 32; ++kk) {
                            const uint32_t j = kk >> 2, w = kk & 3;
                            const uint64_t ad = tc::sdesc_sw128(ah + j * (BMS * 128) + w * 32);
                            const uint64_t bd = tc::sdesc_sw128(b0 + j * (TBN * 128) + w * 32);
                            if constexpr (F8)
                                tc::mma_f8(d_tmem, ad, bd, args.idesc, kk > 0 ? 1u : 0u);
                            else
                                tc::mma_f16(d_tmem, ad, bd, args.idesc, kk > 0 ? 1u : 0u);
                        }
                        tc::mma_f16(d_tmem, tc::sdesc_sw32(ah + L.a_main), tc::sdesc_sw32(b0 + L.b_main),
                                    args.idesc_ext, 1u);
                        tc::mma_commit(&t_full[rg]);
                        last_tfull[rg] = (int)tpar;
                    }
                    if (!ok) break;
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&a_empty[ab]);
            }
        }
    } else if constexpr (MODE == MODE_GAINS && ES) {
        // ------------------------------------------------ region-split epilogue
        // Warps 2-5 drain region 0 (sub-tile 0), warps 6-9 region 1; a thread
        // owns one candidate row and all 256 columns of its region, read as
        // two 128-column loads (the first half summed while the second
        // loads), and hands the region back after the second load.  The two
        // regions drain at the same time, which suits issuers that run freely
        // (both regions complete together); no join of column halves.
        const int ew = warp - 2;        // 0..7
        const int q = warp & 3;         // TMEM lane quarter this warp may access
        const int h = ew >> 2;          // region (candidate sub-tile)
        const int row = q * 32 + lane;  // candidate row within the sub-tile
        int t = 0;
        bool alive = true;
        constexpr int kBlk = 2;  // 64 terms per chain and tile: chains of at most 128 terms
        for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
            int ct, ch, b_row0, nb;
            unit_span<MODE, TBN>(args, P, u, ct, ch, b_row0, nb);
            double acc = 0.0;
            ReluAcc ra;
            relu_zero(ra);
            int inblk = 0;
            for (int i = 0; i < nb; ++i, ++t) {
                if (alive) {
                    // the TMEM loads below are warp-collective: decide per warp
                    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&t_full[h], t & 1, abort_flag, wait_ns));
                    if (!ok) {
                        if (lane == 0) record_timeout(args.err, abort_flag);
                        alive = false;
                    }
                }
                if (!alive) continue;
                tc::tc_fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * TBN);
                uint32_t r[128];
                tc::tmem_ld128(taddr, r);
                tc::tmem_ld_wait();
#pragma unroll
                for (int l = 0; l < 4; ++l) relu_acc32(ra, r + 32 * l);
                tc::tmem_ld128(taddr + 128, r);
                tc::tmem_ld_wait();
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&t_empty[h]);
#pragma unroll
                for (int l = 0; l < 4; ++l) relu_acc32(ra, r + 32 * l);
                if (++inblk == kBlk || i == nb - 1) {
                    acc += (double)relu_fold(ra);
                    relu_zero(ra);
                    inblk = 0;
                }
            }
            if (alive) {
                const int64_t j = (int64_t)ct * BM + h * BMS + row;
                if (j < P.m) {
                    double v = acc;
                    if (F8) v *= (double)args.row_scale[j];  // a power of two: exact
                    args.partial[(int64_t)ch * P.m + j] = v;
                }
            }
        }
    } else if constexpr (MODE == MODE_GAINS) {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2;        // 0..7
        const int q = warp & 3;         // TMEM lane quarter this warp may access
        const int half = ew >> 2;       // column half of a region
        const int row = q * 32 + lane;  // candidate row within a sub-tile
        int t = 0;
        bool alive = true;
        // FP32 blocks of kBlk tiles (chains of at most 128 terms), then FP64
        // over the blocks: the FP64 pipe does one add per block, not per tile
        constexpr int kBlk = 512 / TBN;
        for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
            int ct, ch, b_row0, nb;
            unit_span<MODE, TBN>(args, P, u, ct, ch, b_row0, nb);
            double acc[2] = {0.0, 0.0};
            ReluAcc ra[2];
            relu_zero(ra[0]);
            relu_zero(ra[1]);
            int inblk = 0;
            for (int i = 0; i < nb; ++i, ++t) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int rg = (t % RH) * 2 + h;
                    if (alive) {
                        // the TMEM loads below are warp-collective: decide per warp
                        const bool ok =
                            __all_sync(0xffffffffu, tc::mbar_wait(&t_full[rg], (t / RH) & 1, abort_flag, wait_ns));
                        if (!ok) {
                            if (lane == 0) record_timeout(args.err, abort_flag);
                            alive = false;
                        }
                    }
                    if (!alive) continue;
                    tc::tc_fence_after();
                    const uint32_t taddr =
                        tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(rg * TBN + half * (TBN / 2));
                    // all TBN / 2 columns into registers, then hand the region
                    // back to the MMA issuer before doing any arithmetic
                    if constexpr (TBN == 256) {
                        uint32_t r[128];
                        tc::tmem_ld128(taddr, r);
                        tc::tmem_ld_wait();
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&t_empty[rg]);
#pragma unroll
                        for (int l = 0; l < 4; ++l) relu_acc32(ra[h], r + 32 * l);
                    } else {
                        uint32_t r0[32], r1[32];
                        tc::tmem_ld32(taddr, r0);
                        tc::tmem_ld32(taddr + 32, r1);
                        tc::tmem_ld_wait();
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&t_empty[rg]);
                        relu_acc32(ra[h], r0);
                        relu_acc32(ra[h], r1);
                    }
                }
                if (++inblk == kBlk || i == nb - 1) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        acc[h] += (double)relu_fold(ra[h]);
                        relu_zero(ra[h]);
                    }
                    inblk = 0;
                }
            }
            // combine the two column halves in a fixed order
            if (half == 1) {
                comb[row] = acc[0];
                comb[BMS + row] = acc[1];
            }
            tc::named_bar_sync(2, NEPI);
            if (half == 0 && alive) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t j = (int64_t)ct * BM + h * BMS + row;
                    if (j < P.m) {
                        double v = acc[h] + comb[h * BMS + row];
                        if (F8) v *= (double)args.row_scale[j];  // a power of two: exact
                        args.partial[(int64_t)ch * P.m + j] = v;
                    }
                }
            }
            tc::named_bar_sync(2, NEPI);
        }
    } else {
        // ------------------------------------------------------ set epilogue
        // Warps 2-5 drain region 0 (points 0-127 of the unit), warps 6-9
        // region 1 (points 128-255); a thread owns one point and all 256
        // member columns of its region.  acc(v, s) = ||v||^2 - dhat(v, s), so
        // the set's term is max(0, max over its members of acc).  Groups of
        // 16 columns belong to one set.  The 16 group maxima of a tile are
        // formed first (independent three-input max trees) and the region is
        // handed back before the serial part: the set's running maximum
        // (carried over tiles) and, for every set ending in the tile, the sum
        // of the 32 lanes' terms (FP32, one batched reduce-scatter with fixed
        // trees), written as this warp's partial of the set:
        // partial[(unit * 8 + warp)][set].
        const int ew = warp - 2;  // 0..7
        const int q = warp & 3;
        const int h = ew >> 2;
        int t = 0;
        bool alive = true;
        for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
            int at, ch, b_row0, nb;
            unit_span<MODE>(args, P, u, at, ch, b_row0, nb);
            const int64_t *rec = args.chunks + 4 * ((int64_t)P.chunk0 + ch);
            const int64_t set_b = rec[0], col_e = rec[3];
            double *prow = args.partial + ((int64_t)at * 8 + ew) * args.lb + (set_b - args.j0);
            float run = -INFINITY;
            // group table entries of the next tile are loaded one tile ahead
            int ge_next = lane < (int)(min((int64_t)BN, col_e - b_row0) / SET_GROUP)
                              ? __ldg(args.gset + b_row0 / SET_GROUP + lane)
                              : 0;
            for (int i = 0; i < nb; ++i, ++t) {
                const int64_t c0 = (int64_t)b_row0 + (int64_t)i * BN;
                const int ngr = (int)(min((int64_t)BN, col_e - c0) / SET_GROUP);
                const int ge = ge_next;
                if (i + 1 < nb) {
                    const int64_t c1 = c0 + BN;
                    ge_next = lane < (int)(min((int64_t)BN, col_e - c1) / SET_GROUP)
                                  ? __ldg(args.gset + c1 / SET_GROUP + lane)
                                  : 0;
                }
                const unsigned lastmask = __ballot_sync(0xffffffffu, lane < ngr && (ge & 1));  // groups ending a set
                if (alive) {
                    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&t_full[h], t & 1, abort_flag, wait_ns));
                    if (!ok) {
                        if (lane == 0) record_timeout(args.err, abort_flag);
                        alive = false;
                    }
                }
                if (!alive) continue;
                tc::tc_fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * BN);
                uint32_t r[128];
                float gm[16];
                tc::tmem_ld128(taddr, r);
                tc::tmem_ld_wait();
#pragma unroll
                for (int gg = 0; gg < 8; ++gg) gm[gg] = max16(&r[gg * 16]);
                if (ngr > 8) {
                    tc::tmem_ld128(taddr + 128, r);
                    tc::tmem_ld_wait();
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&t_empty[h]);
                if (ngr > 8) {
#pragma unroll
                    for (int gg = 0; gg < 8; ++gg) gm[8 + gg] = max16(&r[gg * 16]);
                }
                // running maximum over the groups (reset after a set's last
                // group); val[g] = the set's term where group g ends it
                float val[16];
#pragma unroll
                for (int g = 0; g < 16; ++g) {
                    val[g] = 0.f;
                    if (g < ngr) {
                        run = fmaxf(run, gm[g]);
                        const bool last = (lastmask >> g) & 1u;
                        val[g] = last ? fmaxf(run, 0.f) : 0.f;
                        run = last ? -INFINITY : run;
                    }
                }
                if (lastmask) {  // one batched lane reduction for all sets ending in this tile
                    const float tot = reduce_scatter16(val, lane);
                    const int gv = group_of_lane(lane);
                    const int gev = __shfl_sync(0xffffffffu, ge, gv);
                    if ((lane & 1) == 0 && ((lastmask >> gv) & 1u)) prow[gev >> 1] = (double)tot;
                }
            }
        }
    }

    // ---------------------------------------------------------------- teardown
    __syncthreads();
    if ((warp == 1 || (DUAL && warp == NTHREADS_G / 32 - 1)) && lane == 0) {
        // every MMA this thread issued, committed or not (a timeout can stop
        // the issuer between a region's MMAs and their commit), completes
        // before the tensor memory is released
        volatile int never = 0;
        tc::mma_commit(fin);
        tc::mbar_wait(fin, 0u, &never);
    }
    if (threadIdx.x == 0) {
        // nothing may still write shared memory or TMEM when the CTA leaves:
        // wait (bounded) for the last issued phase of every barrier
        volatile int never = 0;
        for (int s = 0; s < ns; ++s)
            if (last_full[s] >= 0) tc::mbar_wait(&full[s], (uint32_t)last_full[s], &never);
        for (int b = 0; b < 2; ++b)
            if (last_afull[b] >= 0) tc::mbar_wait(&a_full[b], (uint32_t)last_afull[b], &never);
        for (int r = 0; r < NREG; ++r)
            if (last_tfull[r] >= 0) tc::mbar_wait(&t_full[r], (uint32_t)last_tfull[r], &never);
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, kTmemCols);
    }
}

__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_gains_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
               const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx, const TcArgs args) {
    tc_pipeline<MODE_GAINS, false>(&tmA, &tmAx, &tmB, &tmBx, args);
}

// Region-split drain (a variant the autotuner may choose).
__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_gains_tc_es(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
                  const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx, const TcArgs args) {
    tc_pipeline<MODE_GAINS, false, false, BN, true>(&tmA, &tmAx, &tmB, &tmBx, args);
}

__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_gains_tc8_es(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
                   const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx,
                   const TcArgs args) {
    tc_pipeline<MODE_GAINS, true, false, BN, true>(&tmA, &tmAx, &tmB, &tmBx, args);
}

// 128-point B tiles (a tile shape the autotuner may choose).
__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_gains_tc_n128(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
                    const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx,
                    const TcArgs args) {
    tc_pipeline<MODE_GAINS, false, false, 128>(&tmA, &tmAx, &tmB, &tmBx, args);
}

// The K-blocked kernel with the region-split drain: the resident kernel's
// default for 128-byte rows, so a forced K-blocked launch there gives the
// same sums.
__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_gains_tc_kb_es(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
                     const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx,
                     const TcArgs args) {
    tc_pipeline<MODE_GAINS, false, true, BN, true>(&tmA, &tmAx, &tmB, &tmBx, args);
}

// Candidate rows too long for the resident layout (d > 128 at 16 bits).
__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_gains_tc_kb(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
                  const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx, const TcArgs args) {
    tc_pipeline<MODE_GAINS, false, true>(&tmA, &tmAx, &tmB, &tmBx, args);
}

// FP8 e4m3 operands (kind::f8f6f4), BF16 extension step; full candidate
// ranges or host-sized lists only.
__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_gains_tc8(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
                const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx, const TcArgs args) {
    tc_pipeline<MODE_GAINS, true>(&tmA, &tmAx, &tmB, &tmBx, args);
}

__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_gains_tc8_n128(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
                     const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx,
                     const TcArgs args) {
    tc_pipeline<MODE_GAINS, true, false, 128>(&tmA, &tmAx, &tmB, &tmBx, args);
}

__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_sets_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
              const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx, const TcArgs args) {
    tc_pipeline<MODE_SETS, false>(&tmA, &tmAx, &tmB, &tmBx, args);
}

// Multi-set evaluation with point and member rows streamed in K blocks (d > 128).
__global__ void __launch_bounds__(NTHREADS_G, 1)
    k_sets_tc_kb(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAx,
                 const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBx, const TcArgs args) {
    tc_pipeline<MODE_SETS, false, true>(&tmA, &tmAx, &tmB, &tmBx, args);
}

// ---------------------------------------------------------------------------
// One persistent launch over the Greedy rounds of several handles (the
// instance-batched bulk gains of an uneven mix of ground sets).
//
// The same warp roles and MMA sequence as the resident MODE_GAINS pipeline,
// with the work units of all handles in one table: a unit is (handle,
// candidate tile, V chunk).  The producer takes the next unit from a device
// counter (the table is ordered largest first, so the last units to start are
// short) and passes its index to the MMA issuer and the epilogue warps
// through a small ring of shared-memory slots; each handle's tensor maps are
// read by TMA from device memory.  Shared-memory buffers are laid out for the
// widest row of the launch (RBmax); a unit of narrower rows fills only the
// first K atoms of each buffer and expects only its own bytes, so its MMAs,
// and hence its sums, are those of the single-handle kernel.
//
// Every wait is bounded; a CTA that gives up records EBC_ETIMEOUT in the
// launch's error word and stops, and the other warps of the CTA see its
// abort flag at their next wait.  The two column halves of a unit are joined
// through mbarriers (no block-wide barrier), so an aborted warp cannot leave
// the others waiting.
// ---------------------------------------------------------------------------
namespace {
constexpr int UR = 4;                // unit ring slots
constexpr uint32_t GROUP_EXTRA = 128;  // shared bytes past the resident layout: ring and join barriers

struct GroupArgs {
    const GroupInst *inst;
    const GroupUnit *units;
    int total_units;
    int *counter;
    int *err;
    int RBmax, nstages, na;
    uint64_t wait_ns;
};
}  // namespace

__global__ void __launch_bounds__(NTHREADS_G, 1) k_gains_tc_group(const GroupArgs args) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int ns = args.nstages;
    const int na = args.na;
    const uint64_t wait_ns = args.wait_ns;
    const SmemLayout L = smem_layout(args.RBmax, ns, na);
    uint8_t *sA = base;
    uint8_t *sB = base + L.off_b;
    double *comb = reinterpret_cast<double *>(base + L.off_comb);  // [2][BMS]
    uint64_t *full = reinterpret_cast<uint64_t *>(base + L.off_bar);
    uint64_t *empty = full + ns;
    uint64_t *a_full = empty + ns;
    uint64_t *a_empty = a_full + 2;
    uint64_t *t_full = a_empty + 2;
    uint64_t *t_empty = t_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + L.off_misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(base + L.off_misc + 4);
    int *last_full = reinterpret_cast<int *>(base + L.off_misc + 8);  // [ns] (ns <= 8)
    int *last_afull = last_full + 8;                                    // [2]
    int *last_tfull = last_afull + 2;                                   // [2]
    uint64_t *fin = reinterpret_cast<uint64_t *>(base + L.off_misc + 56);
    uint64_t *u_full = reinterpret_cast<uint64_t *>(base + L.off_misc + 64);  // [UR]
    uint64_t *u_empty = u_full + UR;                                          // [UR]
    uint64_t *c_full = u_empty + UR;   // column half 1 -> half 0: comb written
    uint64_t *c_empty = c_full + 1;    // half 0 -> half 1: comb read
    volatile int *u_id = reinterpret_cast<volatile int *>(c_empty + 1);  // [UR]
    uint64_t *tok = reinterpret_cast<uint64_t *>(base + L.off_misc + 160);  // [2] issuer turns

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ns; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 2);  // both MMA issuers
            last_full[s] = -1;
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&a_full[b], 1);
            tc::mbar_init(&a_empty[b], 2);
            tc::mbar_init(&t_full[b], 1);
            tc::mbar_init(&t_empty[b], NEPI / 32);
            last_afull[b] = -1;
            last_tfull[b] = -1;
        }
        for (int r = 0; r < UR; ++r) {
            tc::mbar_init(&u_full[r], 1);
            tc::mbar_init(&u_empty[r], 2 + NEPI / 32);  // both MMA issuers and every epilogue warp
        }
        tc::mbar_init(c_full, NEPI / 2);  // every thread of the column-half-1 warps
        tc::mbar_init(c_empty, NEPI / 2);
        tc::mbar_init(fin, 2);
        tc::mbar_init(&tok[0], 1);
        tc::mbar_init(&tok[1], 1);
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
            int g = 0, ua = 0, last_inst = -1;
            for (int i = 0;; ++i) {
                const int r = i % UR;
                if (!tc::mbar_wait(&u_empty[r], ((i / UR) & 1) ^ 1, abort_flag, wait_ns)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                int u = atomicAdd(args.counter, 1);
                if (u >= args.total_units) u = -1;
                u_id[r] = u;
                tc::mbar_arrive(&u_full[r]);  // release: the slot's index is visible to its waiters
                if (u < 0) break;
                const GroupUnit w = args.units[u];
                const GroupInst *I = args.inst + w.inst;
                const int RB = I->RB;
                const int katoms = RB / 128;
                const uint32_t a_tx = 2u * (uint32_t)(BMS * RB + BMS * KEXT * 2);
                const uint32_t b_tx = (uint32_t)(BN * RB + BN * KEXT * 2);
                if (w.inst != last_inst) {  // maps written by a copy before the launch
                    tc::tensormap_acquire(&I->tmA);
                    tc::tensormap_acquire(&I->tmAx);
                    tc::tensormap_acquire(&I->tmB);
                    tc::tensormap_acquire(&I->tmBx);
                    last_inst = w.inst;
                }
                const int ab = ua % na;
                const int aph = (ua / na) & 1;
                if (!tc::mbar_wait(&a_empty[ab], aph ^ 1, abort_flag, wait_ns)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                uint8_t *abuf = sA + ab * L.a_bytes;
                tc::mbar_arrive_expect_tx(&a_full[ab], a_tx);
                for (int h = 0; h < 2; ++h) {
                    uint8_t *sub = abuf + h * L.a_sub;
                    const int row0 = w.ctile * BM + h * BMS;
                    for (int j = 0; j < katoms; ++j)
                        tc::tma_load_2d(sub + j * (BMS * 128), &I->tmA, &a_full[ab], j * KATOM, row0);
                    tc::tma_load_2d(sub + L.a_main, &I->tmAx, &a_full[ab], 0, row0);
                }
                last_afull[ab] = aph;
                bool ok = true;
                const int vt0 = w.chunk * I->vt_per_chunk;
                for (int t = 0; t < w.ntiles; ++t, ++g) {
                    const int s = g % ns;
                    const int ph = (g / ns) & 1;
                    const int brow = (vt0 + t) * BN;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag, wait_ns)) {
                        record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    uint8_t *bbuf = sB + s * L.b_bytes;
                    tc::mbar_arrive_expect_tx(&full[s], b_tx);
                    for (int j = 0; j < katoms; ++j)
                        tc::tma_load_2d(bbuf + j * (BN * 128), &I->tmB, &full[s], j * KATOM, brow);
                    tc::tma_load_2d(bbuf + L.b_main, &I->tmBx, &full[s], 0, brow);
                    last_full[s] = ph;
                }
                if (!ok) break;
                ++ua;
            }
        }
    } else if (warp == 1 || warp == NTHREADS_G / 32 - 1) {
        // ------------------------------------------------------------ MMA issuers
        // warp 1 issues sub-tile 0 of every point tile, the last warp sub-tile
        // 1 (each waits and commits while the other issues); in units of
        // 256-byte rows they take turns, so region 0 completes half a tile
        // before region 1
        if (lane == 0) {
            const int h = warp == 1 ? 0 : 1;
            int g = 0, t = 0, ua = 0;
            int tk = 0;  // tiles of units that take turns (both issuers count the same ones)
            for (int i = 0;; ++i) {
                const int r = i % UR;
                if (!tc::mbar_wait(&u_full[r], (i / UR) & 1, abort_flag, wait_ns)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                const int u = u_id[r];
                tc::mbar_arrive(&u_empty[r]);
                if (u < 0) break;
                const GroupUnit w = args.units[u];
                const GroupInst *I = args.inst + w.inst;
                const int nmma = I->RB / 32;  // one MMA per 32 bytes of K
                const uint32_t idesc = I->idesc, idesc_ext = I->idesc_ext;
                const bool turns = I->RB >= 256;  // rows of 256 bytes: turns; shorter rows: free issue
                const int ab = ua % na;
                if (!tc::mbar_wait(&a_full[ab], (ua / na) & 1, abort_flag, wait_ns)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                const uint32_t a0 = tc::smem_u32(sA + ab * L.a_bytes);
                bool ok = true;
                for (int tt = 0; tt < w.ntiles && ok; ++tt, ++g, ++t) {
                    const int s = g % ns;
                    if (!tc::mbar_wait(&full[s], (g / ns) & 1, abort_flag, wait_ns)) {
                        record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    const uint32_t b0 = tc::smem_u32(sB + s * L.b_bytes);
                    if (!tc::mbar_wait(&t_empty[h], (t & 1) ^ 1, abort_flag, wait_ns)) {
                        record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    if (turns && (h == 1 || tk > 0) &&
                        !tc::mbar_wait(&tok[1 - h], (uint32_t)(h == 1 ? tk : tk - 1) & 1u, abort_flag, wait_ns)) {
                        record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(h * BN);
                    const uint32_t ah = a0 + h * L.a_sub;
                    for (int kk = 0; kk < nmma; ++kk) {
                        const uint32_t j = kk >> 2, w4 = kk & 3;
                        const uint64_t ad = tc::sdesc_sw128(ah + j * (BMS * 128) + w4 * 32);
                        const uint64_t bd = tc::sdesc_sw128(b0 + j * (BN * 128) + w4 * 32);
                        tc::mma_f16(d_tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                    tc::mma_f16(d_tmem, tc::sdesc_sw32(ah + L.a_main), tc::sdesc_sw32(b0 + L.b_main), idesc_ext,
                                1u);
                    if (turns) {
                        tc::mbar_arrive(&tok[h]);
                        ++tk;
                    }
                    tc::mma_commit(&t_full[h]);
                    last_tfull[h] = t & 1;
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&a_empty[ab]);
                ++ua;
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2;        // 0..7
        const int q = warp & 3;         // TMEM lane quarter this warp may access
        const int half = ew >> 2;       // column half of a region
        const int row = q * 32 + lane;  // candidate row within a sub-tile
        int t = 0, ie = 0;
        for (int i = 0;; ++i) {
            const int r = i % UR;
            int u = -1;
            bool ok = true;
            if (lane == 0) {
                ok = tc::mbar_wait(&u_full[r], (i / UR) & 1, abort_flag, wait_ns);
                if (ok) {
                    u = u_id[r];
                    tc::mbar_arrive(&u_empty[r]);
                } else {
                    record_timeout(args.err, abort_flag);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            u = __shfl_sync(0xffffffffu, u, 0);
            if (!ok || u < 0) break;
            const GroupUnit w = args.units[u];
            const GroupInst *I = args.inst + w.inst;
            double acc[2] = {0.0, 0.0};
            ReluAcc ra[2];
            relu_zero(ra[0]);
            relu_zero(ra[1]);
            for (int tt = 0; tt < w.ntiles && ok; ++tt, ++t) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // the TMEM loads below are warp-collective: decide per warp
                    if (!__all_sync(0xffffffffu, tc::mbar_wait(&t_full[h], t & 1, abort_flag, wait_ns))) {
                        if (lane == 0) record_timeout(args.err, abort_flag);
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * BN + half * 128);
                    uint32_t r[128];
                    tc::tmem_ld128(taddr, r);
                    tc::tmem_ld_wait();
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&t_empty[h]);
#pragma unroll
                    for (int l = 0; l < 4; ++l) relu_acc32(ra[h], r + 32 * l);
                }
                // FP32 blocks of four tiles (chains of at most 128 terms), then FP64
                if (ok && ((tt & 3) == 3 || tt == w.ntiles - 1)) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        acc[h] += (double)relu_fold(ra[h]);
                        relu_zero(ra[h]);
                    }
                }
            }
            if (!ok) break;
            // join the column halves in a fixed order: half 1 hands its sums to half 0
            const uint32_t cph = ie & 1;
            if (half == 1) {
                if (!tc::mbar_wait(c_empty, cph ^ 1, abort_flag, wait_ns)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
                comb[row] = acc[0];
                comb[BMS + row] = acc[1];
                tc::mbar_arrive(c_full);
            } else {
                if (!tc::mbar_wait(c_full, cph, abort_flag, wait_ns)) {
                    record_timeout(args.err, abort_flag);
                    break;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t j = (int64_t)w.ctile * BM + h * BMS + row;
                    if (j < I->m) I->partial[(int64_t)w.chunk * I->m + j] = acc[h] + comb[h * BMS + row];
                }
                tc::mbar_arrive(c_empty);
            }
            ++ie;
        }
    }

    // ---------------------------------------------------------------- teardown
    __syncthreads();
    if ((warp == 1 || warp == NTHREADS_G / 32 - 1) && lane == 0) {
        volatile int never = 0;
        tc::mma_commit(fin);
        tc::mbar_wait(fin, 0u, &never);
    }
    if (threadIdx.x == 0) {
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
// bf16 pieces.  hi is the nearest bf16; each residual is exact in FP64
// (Sterbenz); the last piece is rounded up (or to nearest) so that the sum of
// the pieces is >= x with an error of about 2^-24 |x|.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint16_t bf16_bits(__nv_bfloat16 h) { return __bfloat16_as_ushort(h); }

__device__ __forceinline__ void split3(double x, bool up, uint16_t *out) {
    __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
    double r1 = x - (double)__bfloat162float(hi);
    __nv_bfloat16 mid = __float2bfloat16_rn((float)r1);
    double r2 = r1 - (double)__bfloat162float(mid);
    __nv_bfloat16 lo = up ? __float2bfloat16_ru(__double2float_ru(r2)) : __float2bfloat16_rn((float)r2);
    out[0] = bf16_bits(hi);
    out[1] = bf16_bits(mid);
    out[2] = bf16_bits(lo);
}

__device__ __forceinline__ void split2_up(double x, uint16_t *out) {
    __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
    double r1 = x - (double)__bfloat162float(hi);
    __nv_bfloat16 lo = __float2bfloat16_ru(__double2float_ru(r1));
    out[0] = bf16_bits(hi);
    out[1] = bf16_bits(lo);
}

__device__ __forceinline__ uint16_t to_q(float x, int prec) {
    if (prec == EBC_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float from_q(uint16_t h, int prec) {
    if (prec == EBC_BF16) return __bfloat162float(__ushort_as_bfloat16(h));
    return __half2float(__ushort_as_half(h));
}

// Quantisation: v_hat = RN(v) in bf16 or fp16 (zero padded to DP) and 2 v_hat;
// FP64 ||v_hat||^2, ||v_hat - v|| and ||v_hat|| (rounded up) and their maxima.
// One thread per row, sums in index order.
__global__ void k_quantize(const float *__restrict__ V, int64_t n, int d, int64_t n_pad, int DP, int prec,
                           uint16_t *__restrict__ Vq, uint16_t *__restrict__ Vq2, double *__restrict__ qn64,
                           float *__restrict__ qerr, float *__restrict__ qnorm, unsigned int *__restrict__ qmax_bits,
                           int *__restrict__ err) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    uint16_t *dst = Vq + r * DP;
    uint16_t *dst2 = Vq2 + r * DP;
    if (r >= n) {
        for (int i = 0; i < DP; ++i) dst[i] = dst2[i] = 0;
        qn64[r] = 0.0;
        qerr[r] = 0.f;
        qnorm[r] = 0.f;
        return;
    }
    const float *v = V + r * d;
    double qn = 0.0, e2 = 0.0;
    bool finite = true;
    for (int i = 0; i < DP; ++i) {
        float x = i < d ? v[i] : 0.f;
        uint16_t h = to_q(x, prec);
        float xq = from_q(h, prec);
        dst[i] = h;
        dst2[i] = to_q(2.f * xq, prec);  // exact: a power-of-two scaling
        finite = finite && isfinite(2.f * xq);
        double xd = (double)xq;
        qn = __dadd_rn(qn, __dmul_rn(xd, xd));
        double e = xd - (double)x;
        e2 = __dadd_rn(e2, __dmul_rn(e, e));
    }
    if (!finite) atomicCAS(err, 0, (int)EBC_EINVAL);
    qn64[r] = qn;
    // the sums above carry at most (DP + 1) relative roundings of 2^-53;
    // pad the square roots by 2^-40 relative before rounding up
    float qe = __double2float_ru(__dsqrt_ru(e2) * (1.0 + ldexp(1.0, -40)));
    float qm = __double2float_ru(__dsqrt_ru(qn) * (1.0 + ldexp(1.0, -40)));
    qerr[r] = qe;
    qnorm[r] = qm;
    atomicMax(&qmax_bits[0], __float_as_uint(qe));
    atomicMax(&qmax_bits[1], __float_as_uint(qm));
}

// Static candidate extension X and the padding rows of the point extension.
// Also the point-side extension of the multi-set evaluation,
// Px = [1 1 1 | b b b | 0..] with b = ||v||^2 - ||v_hat||^2 (to nearest), so
// that with a member's [q q q | 1 1 1 | 0..], q = -||s_hat||^2, the
// accumulator holds 2 v_hat.s_hat + b + q = ||v||^2 - ||v_hat - s_hat||^2.
// Padding points get b = -1e30 and no ones: every term of theirs is <= 0.
__global__ void k_make_aext(int64_t n, int64_t n_pad, const double *__restrict__ qn64, const float *__restrict__ qerr,
                            const float *__restrict__ qnorm, const float *__restrict__ qmax, double gamma,
                            const double *__restrict__ nv64, uint16_t *__restrict__ Aext, uint16_t *__restrict__ Bext,
                            uint16_t *__restrict__ Px) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    {
        __align__(16) uint16_t prow[KEXT];
        for (int i = 0; i < KEXT; ++i) prow[i] = 0;
        if (r < n) {
            prow[0] = prow[1] = prow[2] = bf16_bits(__float2bfloat16_rn(1.f));
            split3(nv64[r] - qn64[r], false, prow + 3);
        } else {
            prow[3] = bf16_bits(__float2bfloat16_rn(PAD_A));
        }
        uint4 *pd = reinterpret_cast<uint4 *>(Px + r * KEXT);
        const uint4 *ps = reinterpret_cast<const uint4 *>(prow);
        pd[0] = ps[0];
        pd[1] = ps[1];
    }
    __align__(16) uint16_t row[KEXT];
    for (int i = 0; i < KEXT; ++i) row[i] = 0;
    const uint16_t one = bf16_bits(__float2bfloat16_rn(1.f));
    if (r < n) {
        const double qn = qn64[r], dc = (double)qerr[r], qm = (double)qnorm[r], qmx = (double)qmax[1];
        // s_c = dc^2 + gamma (2 max||v_hat|| ||c_hat|| + ||c_hat||^2 + 1)
        const double sc = __dadd_ru(__dmul_ru(dc, dc),
                                    __dmul_ru(gamma, __dadd_ru(__dadd_ru(__dmul_ru(2.0 * qmx, qm), qn), 1.0)));
        split3(-qn, true, row + 0);
        split2_up(sc, row + 3);
        uint16_t al[2];
        split2_up(dc, al);
        row[5] = al[0];
        row[6] = al[0];
        row[7] = al[1];
        row[8] = al[1];
        row[9] = row[10] = row[11] = one;
    }
    uint4 *dst = reinterpret_cast<uint4 *>(Aext + r * KEXT);
    const uint4 *src = reinterpret_cast<const uint4 *>(row);
    dst[0] = src[0];
    dst[1] = src[1];
    if (r >= n) {
        // padding points: a_v = -1e30 makes every term of the column 0
        __align__(16) uint16_t prow[KEXT];
        for (int i = 0; i < KEXT; ++i) prow[i] = 0;
        prow[9] = bf16_bits(__float2bfloat16_rn(PAD_A));
        uint4 *bd = reinterpret_cast<uint4 *>(Bext + r * KEXT);
        const uint4 *ps = reinterpret_cast<const uint4 *>(prow);
        bd[0] = ps[0];
        bd[1] = ps[1];
    }
}

// Per-round point extension Y.  Upper-bound mode: sg = 1,
// w = 2 sqrt(m_v) + 2 dv and a_v = m_v - ||v_hat||^2 + dv (2 sqrt(m_v) + dv)
// + gamma (|m_v - ||v_hat||^2| + dv (2 sqrt(m_v) + dv) + max(dc) w), all
// rounded up.  Plain mode: sg = 0, w = 0, a_v = m_v - ||v_hat||^2 to nearest.
__global__ void k_prep_tc(const double *__restrict__ m64, const double *__restrict__ qn64,
                          const float *__restrict__ qerr, const float *__restrict__ qmax, int64_t n, int upper,
                          double gamma, uint16_t *__restrict__ Bext) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    __align__(16) uint16_t row[KEXT];
    for (int i = 0; i < KEXT; ++i) row[i] = 0;
    const uint16_t one = bf16_bits(__float2bfloat16_rn(1.f));
    row[0] = row[1] = row[2] = one;
    const double mv = m64[v];
    if (upper) {
        const double dv = (double)qerr[v];
        const double sq = __dsqrt_ru(mv);
        const double beta = __dmul_ru(dv, __dadd_ru(__dmul_ru(2.0, sq), dv));
        const double w = __dadd_ru(__dmul_ru(2.0, sq), __dmul_ru(2.0, dv));
        const double base = __dsub_ru(mv, qn64[v]);
        const double acc = __dmul_ru(gamma, __dadd_ru(__dadd_ru(fabs(base), beta), __dmul_ru((double)qmax[0], w)));
        const double a = __dadd_ru(__dadd_ru(base, beta), acc);
        row[3] = row[4] = one;
        uint16_t wp[2];
        split2_up(w, wp);
        row[5] = wp[0];
        row[6] = wp[1];
        row[7] = wp[0];
        row[8] = wp[1];
        split3(a, true, row + 9);
    } else {
        split3(mv - qn64[v], false, row + 9);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(Bext + v * KEXT);
    const uint4 *src = reinterpret_cast<const uint4 *>(row);
    dst[0] = src[0];
    dst[1] = src[1];
}

// Gather candidate rows of Vq and Aext into Cq / Cqx (16 bytes per thread);
// invalid (sanitised, -1) candidates get zero rows.
__global__ void k_gather_rows(const uint16_t *__restrict__ Vq, const uint16_t *__restrict__ Aext,
                              const int *__restrict__ cand, int64_t m, const int *__restrict__ m_dev, int DP,
                              uint16_t *__restrict__ Cq, uint16_t *__restrict__ Cqx) {
    const int per_row = DP / 8 + 2;  // uint4 per row: main part, then 2 for the extension
    if (m_dev) m = lmin(m, *m_dev);
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m * per_row) return;
    int64_t j = e / per_row;
    int w = (int)(e % per_row);
    int c = cand[j];
    uint4 val = make_uint4(0, 0, 0, 0);
    if (w < DP / 8) {
        if (c >= 0) val = reinterpret_cast<const uint4 *>(Vq + (int64_t)c * DP)[w];
        reinterpret_cast<uint4 *>(Cq + j * DP)[w] = val;
    } else {
        int x = w - DP / 8;
        if (c >= 0) val = reinterpret_cast<const uint4 *>(Aext + (int64_t)c * KEXT)[x];
        reinterpret_cast<uint4 *>(Cqx + j * KEXT)[x] = val;
    }
}

// Members of the sets, each set padded to a multiple of 16 columns, as
// B rows of the multi-set evaluation: Mq = 2 s_hat (copied from Vq2) and
// Mx = [q q q | 1 1 1 | 0..], q = -||s_hat||^2.  Padding columns get a zero
// row and Mx = [-1e30 | 0..], so their term is -1e30 for every real point.
// One thread per 16 bytes of a row; the set of padded column p is found by
// binary search in the padded offsets.  Members outside [0, n) are reported
// as EINDEX and treated as padding.
// Member rows of the sets, padded per set to 16-column groups: column p of
// Mq holds 2 s_hat of its set's member (zeros for padding), Mx its
// extension [-||s_hat||^2 in three pieces | 1 1 1 | 0..] (padding: -1e30).
// The column count is the device plan's poff[l]; grid-stride over columns.
__global__ void k_gather_members(const uint16_t *__restrict__ Vq2, const double *__restrict__ qn64, int64_t n, int DP,
                                 const int32_t *__restrict__ idx, const int64_t *__restrict__ off,
                                 const int64_t *__restrict__ poff, int64_t l, int64_t ncap,
                                 uint16_t *__restrict__ Mq, uint16_t *__restrict__ Mx, int *__restrict__ err) {
    const int per_row = DP / 8 + 2;
    const int64_t ncols = min(poff[l], ncap);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ncols * per_row;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / per_row;
        const int w = (int)(e % per_row);
        int64_t lo = 0, hi = l;  // the last set with poff[set] <= p (the non-empty one holding p)
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (poff[mid] <= p) lo = mid;
            else hi = mid;
        }
        const int64_t r = p - poff[lo];
        const int64_t mb = off[lo];
        int64_t src = -1;
        if (r < off[lo + 1] - mb) {
            src = idx[mb + r];
            if (src < 0 || src >= n) {
                if (w == 0) atomicCAS(err, 0, (int)EBC_EINDEX);
                src = -1;
            }
        }
        if (w < DP / 8) {
            uint4 val = make_uint4(0, 0, 0, 0);
            if (src >= 0) val = reinterpret_cast<const uint4 *>(Vq2 + src * DP)[w];
            reinterpret_cast<uint4 *>(Mq + p * DP)[w] = val;
        } else {
            __align__(16) uint16_t row[KEXT];
            for (int i = 0; i < KEXT; ++i) row[i] = 0;
            if (src >= 0) {
                split3(-qn64[src], false, row);
                row[3] = row[4] = row[5] = bf16_bits(__float2bfloat16_rn(1.f));
            } else {
                row[0] = bf16_bits(__float2bfloat16_rn(PAD_A));
            }
            const int x = w - DP / 8;
            reinterpret_cast<uint4 *>(Mx + p * KEXT)[x] = reinterpret_cast<const uint4 *>(row)[x];
        }
    }
}

// ---------------------------------------------------------------------------
// Device plan of a multi-set evaluation (one block; nothing is read back to
// the host).  The sets are the rows of the work matrix of Sec. 4.2 given as
// CSR index lists; each set's members are padded to 16-column groups.
//  1. poff[j]: padded start column of set j (exclusive scan, poff[l] = total);
//     offsets that do not start at 0 or decrease, a NULL member list with
//     members, or more columns than the buffers hold leave no work (poff[l] =
//     0, no chunks) and record EINVAL.
//  2. chunks: a run of sets starts a new chunk where the set's start column
//     enters a new window of SP_WIN columns, and at every launch batch's
//     first set (batches of lbmax sets); rec[k] = {first set, end set, first
//     column, end column}, cj[j] = chunk of set j, bf[b] = first chunk of
//     batch b (bf[batches] = chunk count).
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t SP_WIN = 2048;
constexpr int SP_T = 1024;

// Exclusive scan over the block (SP_T threads) of one value per thread; the
// block total goes to *total.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T *warp_tot, T *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive prefix of the warp totals
        if (lane == 31) *total = t;
    }
    __syncthreads();
    const T r = (w > 0 ? warp_tot[w - 1] : (T)0) + x - v;
    __syncthreads();
    return r;
}
}  // namespace

__global__ void __launch_bounds__(SP_T) k_sets_plan(const int32_t *__restrict__ idx, const int64_t *__restrict__ off,
                                                    int64_t l, int64_t lbmax, int64_t col_cap,
                                                    int64_t *__restrict__ poff, int64_t *__restrict__ rec,
                                                    int *__restrict__ cj, int *__restrict__ bf, int64_t nbatch,
                                                    int *__restrict__ err) {
    __shared__ int64_t wt64[32];
    __shared__ int wt32[32];
    __shared__ int64_t tot64;
    __shared__ int tot32;
    __shared__ int s_bad;
    const int t = threadIdx.x;
    if (t == 0) s_bad = off[0] != 0 || (idx == nullptr && off[l] != off[0]);
    __syncthreads();
    int64_t col = 0;
    for (int64_t base = 0; base < l; base += SP_T) {
        const int64_t j = base + t;
        int64_t pad = 0;
        if (j < l) {
            const int64_t o0 = off[j], o1 = off[j + 1];
            if (o1 < o0) s_bad = 1;  // every writer writes 1
            else pad = (o1 - o0 + 15) / 16 * 16;
        }
        const int64_t c = block_excl_scan<int64_t>(pad, wt64, &tot64);
        if (j < l) poff[j] = col + c;
        col += tot64;
        __syncthreads();
    }
    if (t == 0 && col > col_cap) s_bad = 1;
    __syncthreads();
    if (s_bad) {
        if (t == 0) {
            poff[l] = 0;
            atomicCAS(err, 0, (int)EBC_EINVAL);
        }
        for (int64_t b = t; b <= nbatch; b += SP_T) bf[b] = 0;
        return;
    }
    if (t == 0) poff[l] = col;
    __syncthreads();
    int kbase = 0;
    for (int64_t base = 0; base < l; base += SP_T) {
        const int64_t j = base + t;
        int flag = 0;
        if (j < l) flag = (j % lbmax == 0) || (poff[j] / SP_WIN != poff[j - 1] / SP_WIN);
        const int pos = block_excl_scan<int>(flag, wt32, &tot32);
        if (j < l) {
            const int k = kbase + pos + flag - 1;  // chunk of set j
            cj[j] = k;
            if (flag) {
                rec[4 * (int64_t)k] = j;
                rec[4 * (int64_t)k + 2] = poff[j];
                if (j % lbmax == 0) bf[j / lbmax] = k;
            }
        }
        kbase += tot32;
        __syncthreads();
    }
    if (t == 0) bf[nbatch] = kbase;
    __syncthreads();
    for (int k = t; k < kbase; k += SP_T) {
        const int64_t se = k + 1 < kbase ? rec[4 * (int64_t)(k + 1)] : l;
        rec[4 * (int64_t)k + 1] = se;
        rec[4 * (int64_t)k + 3] = poff[se];
    }
}

// Per 16-column group of the padded members: 2 * (its set's index within the
// set's chunk) + 1 if it is the set's last group.
__global__ void k_sets_gset(const int64_t *__restrict__ poff, int64_t l, const int64_t *__restrict__ rec,
                            const int *__restrict__ cj, int64_t gcap, int *__restrict__ gset) {
    const int64_t ng = min(poff[l] / 16, gcap);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = g * 16;
        int64_t lo = 0, hi = l;  // the last set with poff[set] <= col
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (poff[mid] <= col) lo = mid;
            else hi = mid;
        }
        const int64_t sb = rec[4 * (int64_t)cj[lo]];
        gset[g] = (int)(2 * (lo - sb) + (col + 16 == poff[lo + 1] ? 1 : 0));
    }
}

// ---------------------------------------------------------------------------
// FP8 e4m3.  The candidate operand is q_c = RN(c / s_c) with a per-row
// power-of-two scale s_c (the smallest with max_i |c_i| / s_c <= 448), the
// point operand q_v = RN(v / t) with one power-of-two scale t for all of V;
// c_hat = s_c q_c and v_hat = t q_v exactly.  The MMA accumulates
// q_c . q_v = c_hat . v_hat / (s_c t); the extension columns are divided by
// s_c (candidate side) and 2 t (point side), both exact, so the accumulator
// holds t(c, v) / (2 s_c t) and every candidate's sums are multiplied by
// fc = 2 s_c t at the end (exact).  The rigorous slack of the BF16 path
// applies with dc = ||c_hat - c||, dv = ||v_hat - v||.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint8_t to_e4m3(float x) {
    return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float from_e4m3(uint8_t q) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3)));
}

// smallest power of two s with a / s <= 448 (1 for a == 0)
__device__ __forceinline__ float e4m3_scale(float a) {
    if (!(a > 0.f) || !isfinite(a)) return 1.f;
    int e;
    const float m = frexpf(a / 448.f, &e);  // a / 448 = m 2^e, m in [0.5, 1)
    float sc = ldexpf(1.f, m == 0.5f ? e - 1 : e);
    while (a / sc > 448.f) sc *= 2.f;  // guard against the rounding of a / 448
    return sc;
}

__global__ void k_amax(const float *__restrict__ V, int64_t total, unsigned int *__restrict__ out_bits) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(V[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));
}

// One thread per row; FP64 norms and errors in index order.  qmax_bits:
// [0] max qerr_c, [1] max qnorm_c, [2] max qerr_p, [3] max qnorm_p, [4] amax(V).
__global__ void k_quantize8(const float *__restrict__ V, int64_t n, int d, int64_t n_pad, int DP,
                            unsigned int *__restrict__ qmax_bits, uint8_t *__restrict__ Qc, uint8_t *__restrict__ Qp,
                            float *__restrict__ fc, double *__restrict__ qn_c, double *__restrict__ qn_p,
                            float *__restrict__ qerr_c, float *__restrict__ qerr_p, float *__restrict__ qnorm_c,
                            float *__restrict__ qnorm_p, float *__restrict__ tscale, int *__restrict__ err) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const float t = e4m3_scale(__uint_as_float(qmax_bits[4]));
    if (r == 0) *tscale = t;
    if (r >= n_pad) return;
    uint8_t *qc = Qc + r * DP, *qp = Qp + r * DP;
    if (r >= n) {
        for (int i = 0; i < DP; ++i) qc[i] = qp[i] = 0;
        fc[r] = 1.f;
        qn_c[r] = qn_p[r] = 0.0;
        qerr_c[r] = qerr_p[r] = qnorm_c[r] = qnorm_p[r] = 0.f;
        return;
    }
    const float *v = V + r * d;
    float am = 0.f;
    for (int i = 0; i < d; ++i) am = fmaxf(am, fabsf(v[i]));
    const float sc = e4m3_scale(am);
    double nc = 0.0, np = 0.0, ec = 0.0, ep = 0.0;
    bool finite = true;
    for (int i = 0; i < DP; ++i) {
        const float x = i < d ? v[i] : 0.f;
        finite = finite && isfinite(x);
        const uint8_t a = to_e4m3(x / sc), b = to_e4m3(x / t);  // divisions by powers of two: exact
        qc[i] = a;
        qp[i] = b;
        const double xc = (double)from_e4m3(a) * (double)sc, xp = (double)from_e4m3(b) * (double)t;
        const double xd = (double)x;
        nc = __dadd_rn(nc, __dmul_rn(xc, xc));
        np = __dadd_rn(np, __dmul_rn(xp, xp));
        ec = __dadd_rn(ec, __dmul_rn(xc - xd, xc - xd));
        ep = __dadd_rn(ep, __dmul_rn(xp - xd, xp - xd));
    }
    if (!finite) atomicCAS(err, 0, (int)EBC_EINVAL);
    fc[r] = 2.f * sc * t;
    qn_c[r] = nc;
    qn_p[r] = np;
    const double pad = 1.0 + ldexp(1.0, -40);  // (DP + 1) roundings of 2^-53, see k_quantize
    const float a0 = __double2float_ru(__dsqrt_ru(ec) * pad), a1 = __double2float_ru(__dsqrt_ru(nc) * pad);
    const float a2 = __double2float_ru(__dsqrt_ru(ep) * pad), a3 = __double2float_ru(__dsqrt_ru(np) * pad);
    qerr_c[r] = a0;
    qnorm_c[r] = a1;
    qerr_p[r] = a2;
    qnorm_p[r] = a3;
    atomicMax(&qmax_bits[0], __float_as_uint(a0));
    atomicMax(&qmax_bits[1], __float_as_uint(a1));
    atomicMax(&qmax_bits[2], __float_as_uint(a2));
    atomicMax(&qmax_bits[3], __float_as_uint(a3));
}

// Candidate extension / s_c (FP8): [q q q | s s | al al al' al' | 1 1 1 | 0..] / s_c
// with q = -||c_hat||^2, s = dc^2 + gamma (2 max||v_hat|| ||c_hat|| + ||c_hat||^2 + 1),
// al = dc; the padding rows of the point extension as in k_make_aext.
__global__ void k_make_aext8(int64_t n, int64_t n_pad, const double *__restrict__ qn_c, const float *__restrict__ qerr_c,
                             const float *__restrict__ qnorm_c, const float *__restrict__ qmax, const float *__restrict__ fc,
                             const float *__restrict__ tscale, double gamma, uint16_t *__restrict__ Aext,
                             uint16_t *__restrict__ Bext) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    __align__(16) uint16_t row[KEXT];
    for (int i = 0; i < KEXT; ++i) row[i] = 0;
    if (r < n) {
        const double inv = 1.0 / ((double)fc[r] / (2.0 * (double)*tscale));  // 1 / s_c, a power of two
        const double qn = qn_c[r], dc = (double)qerr_c[r], qm = (double)qnorm_c[r], qmx = (double)qmax[3];
        const double sc = __dadd_ru(__dmul_ru(dc, dc),
                                    __dmul_ru(gamma, __dadd_ru(__dadd_ru(__dmul_ru(2.0 * qmx, qm), qn), 1.0)));
        split3(-qn * inv, true, row + 0);
        split2_up(sc * inv, row + 3);
        uint16_t al[2];
        split2_up(dc * inv, al);
        row[5] = row[6] = al[0];
        row[7] = row[8] = al[1];
        row[9] = row[10] = row[11] = bf16_bits(__float2bfloat16_rn((float)inv));
    }
    uint4 *dst = reinterpret_cast<uint4 *>(Aext + r * KEXT);
    const uint4 *src = reinterpret_cast<const uint4 *>(row);
    dst[0] = src[0];
    dst[1] = src[1];
    if (r >= n) {
        __align__(16) uint16_t prow[KEXT];
        for (int i = 0; i < KEXT; ++i) prow[i] = 0;
        prow[9] = bf16_bits(__float2bfloat16_rn(PAD_A));
        uint4 *bd = reinterpret_cast<uint4 *>(Bext + r * KEXT);
        const uint4 *ps = reinterpret_cast<const uint4 *>(prow);
        bd[0] = ps[0];
        bd[1] = ps[1];
    }
}

// Per-round point extension / (2 t) (FP8): as k_prep_tc with the point-side
// norms and errors and max dc of the candidate side.
__global__ void k_prep_tc8(const double *__restrict__ m64, const double *__restrict__ qn_p,
                           const float *__restrict__ qerr_p, const float *__restrict__ qmax,
                           const float *__restrict__ tscale, int64_t n, int upper, double gamma,
                           uint16_t *__restrict__ Bext) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const double inv = 1.0 / (2.0 * (double)*tscale);  // a power of two
    __align__(16) uint16_t row[KEXT];
    for (int i = 0; i < KEXT; ++i) row[i] = 0;
    const uint16_t one = bf16_bits(__float2bfloat16_rn((float)inv));
    row[0] = row[1] = row[2] = one;
    const double mv = m64[v];
    if (upper) {
        const double dv = (double)qerr_p[v];
        const double sq = __dsqrt_ru(mv);
        const double beta = __dmul_ru(dv, __dadd_ru(__dmul_ru(2.0, sq), dv));
        const double w = __dadd_ru(__dmul_ru(2.0, sq), __dmul_ru(2.0, dv));
        const double base = __dsub_ru(mv, qn_p[v]);
        const double acc = __dmul_ru(gamma, __dadd_ru(__dadd_ru(fabs(base), beta), __dmul_ru((double)qmax[0], w)));
        const double a = __dadd_ru(__dadd_ru(base, beta), acc);
        row[3] = row[4] = one;
        uint16_t wp[2];
        split2_up(w * inv, wp);
        row[5] = wp[0];
        row[6] = wp[1];
        row[7] = wp[0];
        row[8] = wp[1];
        split3(a * inv, true, row + 9);
    } else {
        split3((mv - qn_p[v]) * inv, false, row + 9);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(Bext + v * KEXT);
    const uint4 *src = reinterpret_cast<const uint4 *>(row);
    dst[0] = src[0];
    dst[1] = src[1];
}

// Gather FP8 candidate rows, their extension and scale (16 bytes per thread).
__global__ void k_gather_rows8(const uint8_t *__restrict__ Qc, const uint16_t *__restrict__ Aext,
                               const float *__restrict__ fc, const int *__restrict__ cand, int64_t m, int DP,
                               uint8_t *__restrict__ Cq, uint16_t *__restrict__ Cqx, float *__restrict__ Cfc) {
    const int per_row = DP / 16 + 2;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m * per_row) return;
    const int64_t j = e / per_row;
    const int w = (int)(e % per_row);
    const int c = cand[j];
    uint4 val = make_uint4(0, 0, 0, 0);
    if (w < DP / 16) {
        if (c >= 0) val = reinterpret_cast<const uint4 *>(Qc + (int64_t)c * DP)[w];
        reinterpret_cast<uint4 *>(Cq + j * DP)[w] = val;
    } else {
        const int x = w - DP / 16;
        if (c >= 0) val = reinterpret_cast<const uint4 *>(Aext + (int64_t)c * KEXT)[x];
        reinterpret_cast<uint4 *>(Cqx + j * KEXT)[x] = val;
        if (x == 0) Cfc[j] = c >= 0 ? fc[c] : 1.f;
    }
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

// 2-D map over a row-major [rows, cols] array of 16-bit elements; box of
// box_cols x box_rows with the given swizzle.
cudaError_t make_map(CUtensorMap *map, void *gptr, int64_t rows, int cols, bool bf16, int box_cols, int box_rows,
                     CUtensorMapSwizzle swz) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, gptr, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 2-D map over a row-major [rows, cols] array of bytes (FP8 operands).
cudaError_t make_map_u8(CUtensorMap *map, void *gptr, int64_t rows, int cols, int box_cols, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, gptr, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Pipeline shape: candidate-tile buffers (na) and point-tile stages (ns).
// Two point stages are enough (each tile feeds two sub-tiles' MMAs, twice
// the time of its load); a second candidate buffer removes the reload
// bubble at unit changes when it fits; deeper point rings use what is left.
void pick_pipeline(int RB, int *na, int *ns) {
    *na = 0;
    *ns = 0;
    for (int a = 2; a >= 1; --a)
        for (int s = 6; s >= 2; --s)
            if ((int)smem_layout(RB, s, a).total <= SMEM_LIMIT) {
                *na = a;
                *ns = s;
                return;
            }
}


// Default issue and drain of the 256-point kernels by row width, as measured
// (n = 20k to 400k, BF16 and FP8): 128-byte rows drain fastest split by
// region with the issuers taking turns (7 % over column halves), longer rows
// split by column halves with turns.
void default_issue(int RB, int *turns, int *es) {
    *turns = 1;
    *es = RB <= 128 ? 1 : 0;
}

// Pipeline shape, point-tile width and chunk policy for a bulk launch: 256-
// point tiles in the largest shape that fits shared memory, unless the
// tuning table (or the autotuner) says otherwise.
void choose_config(const Ctx &c, int prec, int RB, int *na, int *ns, int *chunk_mode, int *bn, int *turns,
                   int *es) {
    pick_pipeline(RB, na, ns);
    *chunk_mode = 0;
    *bn = BN;
    default_issue(RB, turns, es);
    TuneCfg t;
    if (tune_lookup(c, prec, RB, c.n, &t)) {
        const int tbn = t.bn == 128 ? 128 : BN;
        if (t.ns >= 2 && t.ns <= 6 && t.na >= 1 && t.na <= 2 &&
            (int)smem_layout(RB, t.ns, t.na, tbn).total <= SMEM_LIMIT) {
            *na = t.na;
            *ns = t.ns;
            *bn = tbn;
        }
        *chunk_mode = t.chunk;
        if (t.turns == 0 || t.turns == 1) *turns = t.turns;
        *es = (t.es == 1 && *bn == BN) ? 1 : 0;
    }
}

// The K-blocked bulk kernel: when a candidate tile and two point stages of
// whole rows do not fit shared memory (d > 128 at 16 bits), or when forced.
bool use_kb(const Ctx &c, int RB) {
    if (c.force_kb) return true;
    int na = 0, ns = 0;
    pick_pipeline(RB, &na, &ns);
    return ns == 0;
}

double gamma_for(int DP) { return ((double)(DP + KEXT) / 4.0 + 4.0) * ldexp(1.0, -22); }

// FP8: the tensor core's internal sum of each 32-product block is assumed
// exact to 13 bits below its largest product (32 x 2^-13 = 2^-8 of the
// block's absolute sum), plus the FP32 accumulation of the BF16 bound.
double gamma8_for(int DP) { return ldexp(1.0, -8) + gamma_for(DP); }

}  // namespace

// Allow a kernel the largest dynamic shared memory any of its launches uses
// (the per-CTA limit), once per (device, kernel): every launch then only
// states its own size, whatever the order of launches with different sizes.
cudaError_t allow_smem(const void *kernel, uint32_t bytes) {
    if (bytes > (uint32_t)SMEM_LIMIT) return cudaErrorInvalidValue;
    static std::mutex mu;
    static std::vector<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &p : done)
        if (p.first == dev && p.second == kernel) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    if (e == cudaSuccess) done.emplace_back(dev, kernel);
    return e;
}

// 16-bit tensor-core bulk bounds and multi-set evaluation: any d (K-blocked
// above 128); the FP8 kernel keeps whole rows resident: d <= 128.
bool tc_supported(const Ctx &c) { return c.d <= 4096; }
bool tc_resident_supported(const Ctx &c) { return c.d <= 128; }

bool tc_config_fits(int RB, int na, int ns, int bn) {
    return na >= 1 && na <= 2 && ns >= 2 && ns <= 6 && (bn == 128 || bn == BN) &&
           (int)smem_layout(RB, ns, na, bn).total <= SMEM_LIMIT;
}

int tc_row_bytes(const Ctx &c) {
    if (c.prec == EBC_FP8E4M3) return (c.d + 127) / 128 * 128;
    return 2 * ((c.d + KATOM - 1) / KATOM * KATOM);
}

void tc8_free(Ctx &c) {
    Ctx::Tc8 &T = c.tc8;
    void *ptrs[] = {T.Qc, T.Qp, T.Cq, T.Aext, T.Cqx, T.Bext, T.fc, T.Cfc, T.qn_c, T.qn_p,
                    T.qerr_c, T.qerr_p, T.qnorm_c, T.qnorm_p, T.qmax, T.tscale};
    for (void *p : ptrs) pool_free(p, c.stream);
    c.tc8 = Ctx::Tc8();
}

cudaError_t tc8_quantize(Ctx &c) {
    Ctx::Tc8 &T = c.tc8;
    cudaError_t e = cudaMemsetAsync(T.qmax, 0, 5 * sizeof(float), c.stream);
    if (e != cudaSuccess) return e;
    k_amax<<<c.num_sms * 4, 256, 0, c.stream>>>(c.V32, c.n * c.d, reinterpret_cast<unsigned int *>(T.qmax) + 4);
    const int th = 128;
    const unsigned g = (unsigned)((T.n_pad + th - 1) / th);
    k_quantize8<<<g, th, 0, c.stream>>>(c.V32, c.n, c.d, T.n_pad, T.DP, reinterpret_cast<unsigned int *>(T.qmax), T.Qc,
                                        T.Qp, T.fc, T.qn_c, T.qn_p, T.qerr_c, T.qerr_p, T.qnorm_c, T.qnorm_p, T.tscale,
                                        &c.st->err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_make_aext8<<<g, th, 0, c.stream>>>(c.n, T.n_pad, T.qn_c, T.qerr_c, T.qnorm_c, T.qmax, T.fc, T.tscale,
                                         gamma8_for(T.DP), T.Aext, T.Bext);
    return cudaGetLastError();
}

cudaError_t tc8_setup(Ctx &c) {
    Ctx::Tc8 &T = c.tc8;
    if (!T.Qc) {
        T.n_pad = (c.n + NPAD - 1) / NPAD * NPAD;
        T.DP = (c.d + 127) / 128 * 128;
        const size_t rows = (size_t)T.n_pad;
        cudaError_t e;
        void **bufs[] = {(void **)&T.Qc, (void **)&T.Qp, (void **)&T.Cq, (void **)&T.Aext, (void **)&T.Cqx,
                         (void **)&T.Bext, (void **)&T.fc, (void **)&T.Cfc, (void **)&T.qn_c, (void **)&T.qn_p,
                         (void **)&T.qerr_c, (void **)&T.qerr_p, (void **)&T.qnorm_c, (void **)&T.qnorm_p,
                         (void **)&T.qmax, (void **)&T.tscale};
        const size_t sizes[] = {rows * T.DP, rows * T.DP, rows * T.DP, rows * KEXT * 2, rows * KEXT * 2,
                                rows * KEXT * 2, rows * 4, rows * 4, rows * 8, rows * 8, rows * 4, rows * 4,
                                rows * 4, rows * 4, 5 * 4, 4};
        for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i)
            if ((e = pool_alloc(bufs[i], sizes[i], c.stream, c.device)) != cudaSuccess) {
                // leave no half-built set: the next call allocates all of them again
                for (size_t j = 0; j < i; ++j) {
                    pool_free(*bufs[j], c.stream);
                    *bufs[j] = nullptr;
                }
                return e;
            }
        if ((e = cudaMemsetAsync(T.Cq, 0, rows * T.DP, c.stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(T.Cqx, 0, rows * KEXT * 2, c.stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(T.Bext, 0, rows * KEXT * 2, c.stream)) != cudaSuccess) return e;
        if ((e = make_map_u8(&T.tmA, T.Qc, T.n_pad, T.DP, 128, BMS)) != cudaSuccess) return e;
        if ((e = make_map_u8(&T.tmA_C, T.Cq, T.n_pad, T.DP, 128, BMS)) != cudaSuccess) return e;
        if ((e = make_map_u8(&T.tmB, T.Qp, T.n_pad, T.DP, 128, BN)) != cudaSuccess) return e;
        if ((e = make_map(&T.tmAx, T.Aext, T.n_pad, KEXT, true, KEXT, BMS, CU_TENSOR_MAP_SWIZZLE_32B)) != cudaSuccess)
            return e;
        if ((e = make_map(&T.tmAx_C, T.Cqx, T.n_pad, KEXT, true, KEXT, BMS, CU_TENSOR_MAP_SWIZZLE_32B)) != cudaSuccess)
            return e;
        if ((e = make_map(&T.tmBx, T.Bext, T.n_pad, KEXT, true, KEXT, BN, CU_TENSOR_MAP_SWIZZLE_32B)) != cudaSuccess)
            return e;
        if ((e = make_map_u8(&T.tmB128, T.Qp, T.n_pad, T.DP, 128, 128)) != cudaSuccess) return e;
        if ((e = make_map(&T.tmBx128, T.Bext, T.n_pad, KEXT, true, KEXT, 128, CU_TENSOR_MAP_SWIZZLE_32B)) !=
            cudaSuccess)
            return e;
    }
    T.ready = true;
    return tc8_quantize(c);
}

cudaError_t launch_prep_tc8(Ctx &c, bool upper) {
    const int th = 256;
    Ctx::Tc8 &T = c.tc8;
    k_prep_tc8<<<(unsigned)((c.n + th - 1) / th), th, 0, c.stream>>>(c.m64, T.qn_p, T.qerr_p, T.qmax, T.tscale, c.n,
                                                                      upper ? 1 : 0, gamma8_for(T.DP), T.Bext);
    return cudaGetLastError();
}

cudaError_t launch_gains_tc8(Ctx &c, const int *cand, int64_t m, int *nchunks_out) {
    Ctx::Tc8 &T = c.tc8;
    int na = 0, ns = 0, chunk_mode = 0, bn = BN, turns = 0, es = 0;
    choose_config(c, EBC_FP8E4M3, T.DP, &na, &ns, &chunk_mode, &bn, &turns, &es);
    if (ns == 0) return cudaErrorInvalidConfiguration;
    const SmemLayout L = smem_layout(T.DP, ns, na, bn);
    const void *kfn = bn != BN ? (const void *)k_gains_tc8_n128
                               : (es ? (const void *)k_gains_tc8_es : (const void *)k_gains_tc8);
    if (cudaError_t e = allow_smem(kfn, L.total); e != cudaSuccess) return e;
    if (cand) {
        const int64_t tot = m * (T.DP / 16 + 2);
        k_gather_rows8<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(T.Qc, T.Aext, T.fc, cand, m, T.DP, T.Cq,
                                                                             T.Cqx, T.Cfc);
        if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return e;
    }
    TcArgs a{};
    a.wait_ns = wait_limit_ns();
    a.m = m;
    a.n_vtiles = (int)(T.n_pad / bn);
    a.n_ctiles = (int)((m + BM - 1) / BM);
    const int G = (c.max_ctas > 0 && c.max_ctas < c.num_sms) ? c.max_ctas : c.num_sms;
    a.nchunks = pick_chunks(m, a.n_vtiles, G, c.partial_cap, &a.vt_per_chunk);
    if (chunk_mode)
        a.nchunks = apply_chunk_mode(a.nchunks, chunk_mode, a.n_vtiles, c.partial_cap / std::max<int64_t>(m, 1),
                                     &a.vt_per_chunk);
    a.RB = T.DP;
    a.xatom = 128;
    a.nstages = ns;
    a.na = na;
    a.turns = turns;
    a.idesc = tc::idesc_f16(0u, BMS, (uint32_t)bn);  // kind::f8f6f4 with format 0: e4m3 x e4m3
    a.idesc_ext = tc::idesc_f16(1u, BMS, (uint32_t)bn);
    a.partial = c.partial;
    a.err = &c.st->err;
    a.row_scale = cand ? T.Cfc : T.fc;
    a.partial_cap = c.partial_cap;
    a.G = G;
    const int units = a.n_ctiles * a.nchunks;
    if (bn == BN && es)
        k_gains_tc8_es<<<std::min(units, G), NTHREADS_G, L.total, c.stream>>>(
            cand ? T.tmA_C : T.tmA, cand ? T.tmAx_C : T.tmAx, T.tmB, T.tmBx, a);
    else if (bn == BN)
        k_gains_tc8<<<std::min(units, G), NTHREADS_G, L.total, c.stream>>>(cand ? T.tmA_C : T.tmA,
                                                                         cand ? T.tmAx_C : T.tmAx, T.tmB, T.tmBx, a);
    else
        k_gains_tc8_n128<<<std::min(units, G), NTHREADS_G, L.total, c.stream>>>(
            cand ? T.tmA_C : T.tmA, cand ? T.tmAx_C : T.tmAx, T.tmB128, T.tmBx128, a);
    *nchunks_out = a.nchunks;
    return cudaGetLastError();
}

void tc_free(Ctx &c) {
    tc8_free(c);
    void *ptrs[] = {c.tc.Vq,   c.tc.Vq2,   c.tc.Aext, c.tc.Bext, c.tc.Cq,   c.tc.Cqx,      c.tc.qn64,
                    c.tc.qerr, c.tc.qnorm, c.tc.qmax, c.tc.Px,   c.tc.Mq,   c.tc.Mx,       c.tc.gset,
                    c.tc.sp_aux, c.tc.sp_rec, c.tc.sp_cj, c.tc.sp_bf};
    for (void *p : ptrs) pool_free(p, c.stream);
    c.tc = Ctx::Tc();
}

cudaError_t tc_quantize(Ctx &c) {
    Ctx::Tc &T = c.tc;
    cudaError_t e = cudaMemsetAsync(T.qmax, 0, 2 * sizeof(float), c.stream);
    if (e != cudaSuccess) return e;
    int th = 128;
    unsigned g = (unsigned)((T.n_pad + th - 1) / th);
    k_quantize<<<g, th, 0, c.stream>>>(c.V32, c.n, c.d, T.n_pad, T.DP, T.prec, T.Vq, T.Vq2, T.qn64, T.qerr, T.qnorm,
                                       reinterpret_cast<unsigned int *>(T.qmax), &c.st->err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_make_aext<<<g, th, 0, c.stream>>>(c.n, T.n_pad, T.qn64, T.qerr, T.qnorm, T.qmax, gamma_for(T.DP), c.nv64, T.Aext,
                                        T.Bext, T.Px);
    return cudaGetLastError();
}

cudaError_t tc_setup(Ctx &c, int prec) {
    Ctx::Tc &T = c.tc;
    if (T.Vq == nullptr) {
        T.n_pad = (c.n + NPAD - 1) / NPAD * NPAD;
        T.DP = (c.d + KATOM - 1) / KATOM * KATOM;
        size_t rows = (size_t)T.n_pad;
        cudaError_t e;
        void **bufs[] = {(void **)&T.Vq,   (void **)&T.Vq2,  (void **)&T.Aext,  (void **)&T.Bext,
                         (void **)&T.Cq,   (void **)&T.Cqx,  (void **)&T.qn64,  (void **)&T.qerr,
                         (void **)&T.qnorm, (void **)&T.qmax, (void **)&T.Px};
        const size_t sizes[] = {rows * T.DP * 2, rows * T.DP * 2, rows * KEXT * 2, rows * KEXT * 2,
                                rows * T.DP * 2, rows * KEXT * 2, rows * 8,        rows * 4,
                                rows * 4,        2 * 4,           rows * KEXT * 2};
        for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i)
            if ((e = pool_alloc(bufs[i], sizes[i], c.stream, c.device)) != cudaSuccess) {
                // leave no half-built set: the next call allocates all of them again
                for (size_t j = 0; j < i; ++j) {
                    pool_free(*bufs[j], c.stream);
                    *bufs[j] = nullptr;
                }
                return e;
            }
        if ((e = cudaMemsetAsync(T.Cq, 0, rows * T.DP * 2, c.stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(T.Cqx, 0, rows * KEXT * 2, c.stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(T.Bext, 0, rows * KEXT * 2, c.stream)) != cudaSuccess) return e;
    }
    T.prec = prec;
    const bool bf = prec == EBC_BF16;
    cudaError_t e = make_map(&T.tmA_V, T.Vq, T.n_pad, T.DP, bf, KATOM, BMS, CU_TENSOR_MAP_SWIZZLE_128B);
    if (e == cudaSuccess) e = make_map(&T.tmB_V, T.Vq2, T.n_pad, T.DP, bf, KATOM, BN, CU_TENSOR_MAP_SWIZZLE_128B);
    if (e == cudaSuccess) e = make_map(&T.tmA_C, T.Cq, T.n_pad, T.DP, bf, KATOM, BMS, CU_TENSOR_MAP_SWIZZLE_128B);
    if (e == cudaSuccess) e = make_map(&T.tmAx_V, T.Aext, T.n_pad, KEXT, true, KEXT, BMS, CU_TENSOR_MAP_SWIZZLE_32B);
    if (e == cudaSuccess) e = make_map(&T.tmAx_C, T.Cqx, T.n_pad, KEXT, true, KEXT, BMS, CU_TENSOR_MAP_SWIZZLE_32B);
    if (e == cudaSuccess) e = make_map(&T.tmBx, T.Bext, T.n_pad, KEXT, true, KEXT, BN, CU_TENSOR_MAP_SWIZZLE_32B);
    if (e == cudaSuccess) e = make_map(&T.tmPx, T.Px, T.n_pad, KEXT, true, KEXT, BMS, CU_TENSOR_MAP_SWIZZLE_32B);
    if (e == cudaSuccess) e = make_map(&T.tmB_V128, T.Vq2, T.n_pad, T.DP, bf, KATOM, 128, CU_TENSOR_MAP_SWIZZLE_128B);
    if (e == cudaSuccess) e = make_map(&T.tmBx128, T.Bext, T.n_pad, KEXT, true, KEXT, 128, CU_TENSOR_MAP_SWIZZLE_32B);
    if (e != cudaSuccess) return e;
    return tc_quantize(c);
}

cudaError_t launch_prep_tc(Ctx &c, bool upper) {
    int th = 256;
    k_prep_tc<<<(unsigned)((c.n + th - 1) / th), th, 0, c.stream>>>(c.m64, c.tc.qn64, c.tc.qerr, c.tc.qmax, c.n,
                                                                     upper ? 1 : 0, gamma_for(c.tc.DP), c.tc.Bext);
    return cudaGetLastError();
}

cudaError_t launch_gains_tc(Ctx &c, const int *cand, int64_t m, bool upper, int *nchunks_out) {
    (void)upper;  // the mode is carried by the point extension written by launch_prep_tc
    Ctx::Tc &T = c.tc;
    const int DP = T.DP;
    const bool kb = use_kb(c, 2 * DP);
    int na = 1, ns = KB_STAGES, chunk_mode = 0, bn = BN, turns = 0, es = 0;
    if (kb)
        default_issue(2 * DP, &turns, &es);
    else
        choose_config(c, T.prec, 2 * DP, &na, &ns, &chunk_mode, &bn, &turns, &es);
    if (ns == 0) return cudaErrorInvalidConfiguration;
    const SmemLayout L = kb ? smem_layout_kb(ns) : smem_layout(2 * DP, ns, na, bn);
    const void *kfn = kb ? (es ? (const void *)k_gains_tc_kb_es : (const void *)k_gains_tc_kb)
                         : (bn != BN ? (const void *)k_gains_tc_n128
                                     : (es ? (const void *)k_gains_tc_es : (const void *)k_gains_tc));
    if (cudaError_t e = allow_smem(kfn, L.total); e != cudaSuccess) return e;
    if (cand) {
        int64_t tot = m * (DP / 8 + 2);
        k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(T.Vq, T.Aext, cand, m, nullptr, DP, T.Cq,
                                                                            T.Cqx);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    TcArgs a{};
    a.wait_ns = wait_limit_ns();
    a.m = m;
    a.n_vtiles = (int)(T.n_pad / bn);
    a.n_ctiles = (int)((m + BM - 1) / BM);
    // V chunks: balance the persistent grid (units = candidate tiles x chunks)
    const int G = (c.max_ctas > 0 && c.max_ctas < c.num_sms) ? c.max_ctas : c.num_sms;
    a.nchunks = pick_chunks(m, a.n_vtiles, G, c.partial_cap, &a.vt_per_chunk);
    if (chunk_mode)
        a.nchunks = apply_chunk_mode(a.nchunks, chunk_mode, a.n_vtiles, c.partial_cap / std::max<int64_t>(m, 1),
                                     &a.vt_per_chunk);
    a.m_dev = nullptr;
    a.partial_cap = c.partial_cap;
    a.G = G;
    a.nch_out = nullptr;
    a.chunks = nullptr;
    a.gset = nullptr;
    a.lb = 0;
    a.j0 = 0;
    a.RB = 2 * DP;
    a.xatom = KATOM;
    a.row_scale = nullptr;
    a.nstages = ns;
    a.na = na;
    a.turns = turns;
    a.idesc = tc::idesc_f16(T.prec == EBC_BF16 ? 1u : 0u, BMS, (uint32_t)bn);
    a.idesc_ext = tc::idesc_f16(1u, BMS, (uint32_t)bn);
    a.partial = c.partial;
    a.err = &c.st->err;
    const int units = a.n_ctiles * a.nchunks;
    const int grid = std::min(units, G);
    if (kb && es)
        k_gains_tc_kb_es<<<grid, NTHREADS_G, L.total, c.stream>>>(cand ? T.tmA_C : T.tmA_V, cand ? T.tmAx_C : T.tmAx_V,
                                                                T.tmB_V, T.tmBx, a);
    else if (kb)
        k_gains_tc_kb<<<grid, NTHREADS_G, L.total, c.stream>>>(cand ? T.tmA_C : T.tmA_V, cand ? T.tmAx_C : T.tmAx_V,
                                                             T.tmB_V, T.tmBx, a);
    else if (bn == BN && es)
        k_gains_tc_es<<<grid, NTHREADS_G, L.total, c.stream>>>(cand ? T.tmA_C : T.tmA_V, cand ? T.tmAx_C : T.tmAx_V,
                                                             T.tmB_V, T.tmBx, a);
    else if (bn == BN)
        k_gains_tc<<<grid, NTHREADS_G, L.total, c.stream>>>(cand ? T.tmA_C : T.tmA_V, cand ? T.tmAx_C : T.tmAx_V, T.tmB_V,
                                                          T.tmBx, a);
    else
        k_gains_tc_n128<<<grid, NTHREADS_G, L.total, c.stream>>>(cand ? T.tmA_C : T.tmA_V, cand ? T.tmAx_C : T.tmAx_V,
                                                               T.tmB_V128, T.tmBx128, a);
    *nchunks_out = a.nchunks;
    return cudaGetLastError();
}

bool tc_group_supported(const Ctx &c) {
    return (c.tc.prec == EBC_BF16 || c.tc.prec == EBC_FP16) && !use_kb(c, 2 * c.tc.DP);
}

int tc_group_row_bytes(const Ctx &c) { return 2 * c.tc.DP; }

void group_inst_fill(const Ctx &c, int nchunks, int vt_per_chunk, GroupInst *out) {
    const Ctx::Tc &T = c.tc;
    out->tmA = T.tmA_V;
    out->tmAx = T.tmAx_V;
    out->tmB = T.tmB_V;
    out->tmBx = T.tmBx;
    out->partial = c.partial;
    out->err = &c.st->err;
    out->m = c.n;
    out->n_vtiles = (int)(T.n_pad / BN);
    out->vt_per_chunk = vt_per_chunk;
    out->nchunks = nchunks;
    out->RB = 2 * T.DP;
    out->idesc = tc::idesc_f16(T.prec == EBC_BF16 ? 1u : 0u, BMS, BN);
    out->idesc_ext = tc::idesc_f16(1u, BMS, BN);
}

// A timeout anywhere in the shared launch leaves units of any handle
// unfinished: every handle of the launch gets the error.
__global__ void k_group_err(const GroupInst *__restrict__ inst, int count, const int *__restrict__ err) {
    const int e = *err;
    if (e == 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        atomicCAS(inst[i].err, 0, e);
}

cudaError_t launch_group_err(const GroupInst *d_inst, int count, const int *d_err, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_group_err<<<(count + 255) / 256, 256, 0, s>>>(d_inst, count, d_err);
    return cudaGetLastError();
}

cudaError_t launch_gains_tc_group(const GroupInst *d_inst, const GroupUnit *d_units, int total_units,
                                  int *d_counter, int *d_err, int RBmax, int G, cudaStream_t s) {
    if (total_units <= 0) return cudaSuccess;
    int na = 0, ns = 0;
    for (int a = 2; a >= 1 && ns == 0; --a)
        for (int st = 6; st >= 2; --st)
            if (smem_layout(RBmax, st, a).total + GROUP_EXTRA <= (uint32_t)SMEM_LIMIT) {
                na = a;
                ns = st;
                break;
            }
    if (ns == 0) return cudaErrorInvalidConfiguration;
    const uint32_t bytes = smem_layout(RBmax, ns, na).total + GROUP_EXTRA;
    if (cudaError_t e = allow_smem((const void *)k_gains_tc_group, bytes); e != cudaSuccess) return e;
    GroupArgs a{};
    a.inst = d_inst;
    a.units = d_units;
    a.total_units = total_units;
    a.counter = d_counter;
    a.err = d_err;
    a.RBmax = RBmax;
    a.nstages = ns;
    a.na = na;
    a.wait_ns = wait_limit_ns();
    k_gains_tc_group<<<std::min(total_units, G), NTHREADS_G, bytes, s>>>(a);
    return cudaGetLastError();
}

// Bulk upper bounds of a candidate list whose length is on the device (the
// lazy Greedy round): rows gathered for at most m_cap entries, the plan
// (chunks) derived inside the kernel, the chunk count left in
// st->list_nch for the reduction.
cudaError_t launch_gains_tc_list(Ctx &c, const int *cand, const int *m_dev, int64_t m_cap) {
    Ctx::Tc &T = c.tc;
    const int DP = T.DP;
    const bool kb = use_kb(c, 2 * DP);
    int na = 1, ns = KB_STAGES;
    if (!kb) pick_pipeline(2 * DP, &na, &ns);
    if (ns == 0) return cudaErrorInvalidConfiguration;
    const SmemLayout L = kb ? smem_layout_kb(ns) : smem_layout(2 * DP, ns, na);
    int turns = 1, es = 0;
    default_issue(2 * DP, &turns, &es);
    const void *kfn = kb ? (es ? (const void *)k_gains_tc_kb_es : (const void *)k_gains_tc_kb)
                         : (es ? (const void *)k_gains_tc_es : (const void *)k_gains_tc);
    if (cudaError_t e = allow_smem(kfn, L.total); e != cudaSuccess) return e;
    const int64_t tot = m_cap * (DP / 8 + 2);
    k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(T.Vq, T.Aext, cand, m_cap, m_dev, DP, T.Cq,
                                                                        T.Cqx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int G = (c.max_ctas > 0 && c.max_ctas < c.num_sms) ? c.max_ctas : c.num_sms;
    TcArgs a{};
    a.wait_ns = wait_limit_ns();
    a.m = m_cap;
    a.n_vtiles = (int)(T.n_pad / BN);
    a.n_ctiles = 0;
    a.nchunks = 1;
    a.vt_per_chunk = a.n_vtiles;
    a.RB = 2 * DP;
    a.xatom = KATOM;
    a.row_scale = nullptr;
    a.nstages = ns;
    a.na = na;
    a.turns = turns;
    a.idesc = tc::idesc_f16(T.prec == EBC_BF16 ? 1u : 0u, BMS, BN);
    a.idesc_ext = tc::idesc_f16(1u, BMS, BN);
    a.partial = c.partial;
    a.err = &c.st->err;
    a.m_dev = m_dev;
    a.partial_cap = c.partial_cap;
    a.G = G;
    a.nch_out = &c.st->list_nch;
    if (kb && es)
        k_gains_tc_kb_es<<<G, NTHREADS_G, L.total, c.stream>>>(T.tmA_C, T.tmAx_C, T.tmB_V, T.tmBx, a);
    else if (kb)
        k_gains_tc_kb<<<G, NTHREADS_G, L.total, c.stream>>>(T.tmA_C, T.tmAx_C, T.tmB_V, T.tmBx, a);
    else if (es)
        k_gains_tc_es<<<G, NTHREADS_G, L.total, c.stream>>>(T.tmA_C, T.tmAx_C, T.tmB_V, T.tmBx, a);
    else
        k_gains_tc<<<G, NTHREADS_G, L.total, c.stream>>>(T.tmA_C, T.tmAx_C, T.tmB_V, T.tmBx, a);
    return cudaGetLastError();
}

// Multi-set evaluation on the tensor cores.  Host plan (from the offsets):
// padded offsets (each set rounded up to 16 columns), chunks of whole sets
// (at most 128 sets and about 2048 columns each) and the group table.  Work
// units are (256 points, chunk); set partials [point unit][warp][set] are
// reduced in a fixed order by k_sets_finalize.  Sets are processed in batches whose
// partials fit the scratch.
// Buffers of the multi-set evaluation for up to `sets` sets with `members`
// members in all (padded columns <= members + 15 sets).
cudaError_t tc_sets_reserve(Ctx &c, int64_t sets, int64_t members) {
    Ctx::Tc &T = c.tc;
    cudaError_t e;
    const int64_t cols = std::max<int64_t>((members + 15 * sets + BN - 1) / BN * BN, BN);
    if (T.mcap < cols) {
        pool_free(T.Mq, c.stream);
        pool_free(T.Mx, c.stream);
        pool_free(T.gset, c.stream);
        T.Mq = T.Mx = nullptr;
        T.gset = nullptr;
        T.mcap = 0;
        if ((e = pool_alloc((void **)&T.Mq, (size_t)cols * T.DP * 2, c.stream, c.device)) != cudaSuccess ||
            (e = pool_alloc((void **)&T.Mx, (size_t)cols * KEXT * 2, c.stream, c.device)) != cudaSuccess ||
            (e = pool_alloc((void **)&T.gset, (size_t)cols / SET_GROUP * 4, c.stream, c.device)) != cudaSuccess) {
            pool_free(T.Mq, c.stream);
            pool_free(T.Mx, c.stream);
            T.Mq = T.Mx = nullptr;
            T.gset = nullptr;
            return e;
        }
        T.mcap = cols;
    }
    if (T.sp_sets < sets) {
        void *old[] = {T.sp_aux, T.sp_rec, T.sp_cj};
        for (void *p : old) pool_free(p, c.stream);
        T.sp_aux = T.sp_rec = nullptr;
        T.sp_cj = nullptr;
        T.sp_sets = 0;
        if ((e = pool_alloc((void **)&T.sp_aux, (size_t)(sets + 1) * 8, c.stream, c.device)) != cudaSuccess ||
            (e = pool_alloc((void **)&T.sp_rec, (size_t)(sets + 1) * 32, c.stream, c.device)) != cudaSuccess ||
            (e = pool_alloc((void **)&T.sp_cj, (size_t)sets * 4, c.stream, c.device)) != cudaSuccess) {
            pool_free(T.sp_aux, c.stream);
            pool_free(T.sp_rec, c.stream);
            T.sp_aux = T.sp_rec = nullptr;
            T.sp_cj = nullptr;
            return e;
        }
        T.sp_sets = sets;
    }
    return cudaSuccess;
}

cudaError_t launch_eval_sets_tc(Ctx &c, const int32_t *idx, const int64_t *off, int64_t l, int64_t members,
                                double *out_f, int64_t *nlaunch) {
    Ctx::Tc &T = c.tc;
    *nlaunch = 0;
    if (l <= 0) return cudaSuccess;
    const bool kb = use_kb(c, 2 * T.DP);
    int na = 1, ns = KB_STAGES;
    if (!kb) pick_pipeline(2 * T.DP, &na, &ns);
    if (ns == 0) return cudaErrorInvalidConfiguration;
    const SmemLayout L = kb ? smem_layout_kb(ns) : smem_layout(2 * T.DP, ns, na);
    const void *kfn = kb ? (const void *)k_sets_tc_kb : (const void *)k_sets_tc;
    cudaError_t e = allow_smem(kfn, L.total);
    if (e != cudaSuccess) return e;
    const int npu = (int)(T.n_pad / BM);
    const int64_t rows = (int64_t)npu * 8;  // partial rows: (point unit, epilogue warp)
    const int64_t lbmax = std::min<int64_t>(l, c.set_part_cap / rows);
    if (lbmax < 1) return cudaErrorMemoryAllocation;
    const int64_t nbatch = (l + lbmax - 1) / lbmax;
    if ((e = tc_sets_reserve(c, l, members)) != cudaSuccess) return e;
    if (T.sp_batches < nbatch + 1) {
        pool_free(T.sp_bf, c.stream);
        T.sp_bf = nullptr;
        T.sp_batches = 0;
        if ((e = pool_alloc((void **)&T.sp_bf, (size_t)(nbatch + 1) * 4, c.stream, c.device)) != cudaSuccess) return e;
        T.sp_batches = nbatch + 1;
    }
    const bool bf = T.prec == EBC_BF16;
    CUtensorMap tmM, tmMx;
    if ((e = make_map(&tmM, T.Mq, T.mcap, T.DP, bf, KATOM, BN, CU_TENSOR_MAP_SWIZZLE_128B)) != cudaSuccess) return e;
    if ((e = make_map(&tmMx, T.Mx, T.mcap, KEXT, true, KEXT, BN, CU_TENSOR_MAP_SWIZZLE_32B)) != cudaSuccess) return e;
    // the plan, the group table and the member rows, all on the device
    k_sets_plan<<<1, SP_T, 0, c.stream>>>(idx, off, l, lbmax, T.mcap, T.sp_aux, T.sp_rec, T.sp_cj, T.sp_bf, nbatch,
                                          &c.st->err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned gs = (unsigned)std::max(1, c.num_sms * 4);
    k_sets_gset<<<gs, 256, 0, c.stream>>>(T.sp_aux, l, T.sp_rec, T.sp_cj, T.mcap / SET_GROUP, T.gset);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_gather_members<<<gs * 2, 256, 0, c.stream>>>(T.Vq2, T.qn64, c.n, T.DP, idx, off, T.sp_aux, l, T.mcap, T.Mq,
                                                   T.Mx, &c.st->err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *nlaunch += 3;
    const int G = (c.max_ctas > 0 && c.max_ctas < c.num_sms) ? c.max_ctas : c.num_sms;
    for (int64_t b = 0; b < nbatch; ++b) {
        const int64_t j0 = b * lbmax;
        const int64_t lb = std::min(lbmax, l - j0);
        TcArgs a{};
        a.wait_ns = wait_limit_ns();
        a.m = 0;
        a.n_vtiles = 0;
        a.n_ctiles = npu;
        a.nchunks = 0;  // from the device plan (sets_bf)
        a.vt_per_chunk = 0;
        a.RB = 2 * T.DP;
        a.xatom = KATOM;
        a.row_scale = nullptr;
        a.nstages = ns;
        a.na = na;
        a.turns = 1;  // measured: free issue 0.34 ms, turns 0.30 ms per C1 call
        a.idesc = tc::idesc_f16(bf ? 1u : 0u, BMS, BN);
        a.idesc_ext = tc::idesc_f16(1u, BMS, BN);
        a.partial = c.set_part;
        a.err = &c.st->err;
        a.chunks = T.sp_rec;
        a.gset = T.gset;
        a.lb = lb;
        a.j0 = j0;
        a.sets_bf = T.sp_bf;
        a.sets_batch = (int)b;
        // empty sets get no partial from any warp
        if ((e = cudaMemsetAsync(c.set_part, 0, sizeof(double) * rows * lb, c.stream)) != cudaSuccess) return e;
        if (kb)
            k_sets_tc_kb<<<G, NTHREADS_G, L.total, c.stream>>>(T.tmA_V, T.tmPx, tmM, tmMx, a);
        else
            k_sets_tc<<<G, NTHREADS_G, L.total, c.stream>>>(T.tmA_V, T.tmPx, tmM, tmMx, a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_sets_finalize(c, rows, lb, j0, l, out_f)) != cudaSuccess) return e;
        *nlaunch += 2;
    }
    return cudaSuccess;
}

}  // namespace ebc
