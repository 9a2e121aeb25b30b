// Internal declarations shared by the library's translation units.
// Nothing here is part of the public ABI (include/ebc.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ebc.h"
#include <nvtx3/nvToolsExt.h>


namespace ebc {

// A named NVTX range over one C-ABI call (visible in Nsight Systems; a no-op
// without an attached tool).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};


constexpr int kMaxRefineK = 31;  // K + 1 <= 32: one warp lane per list entry
constexpr int kRefineTile = 64;  // points per shared-memory tile of the exact / bound kernels
// Exact gains whose computed values lie within this relative distance of the
// round's largest are ties, decided by the smallest index.  The exact gains
// are double-FP32 sums (about 2^-44 relative per term), so a tie in real
// arithmetic (duplicate points, mirror-symmetric pairs) can come out a few
// units apart; every threshold that decides which candidates reach the exact
// stage is lowered by 2 kTieRel so that all tied candidates do.
constexpr double kTieRel = 1e-10;

// Limit of each wait inside the tensor-core pipeline, in ns (1 s unless
// ebc_set_wait_limit_ns changed it); read when a kernel is launched.
uint64_t wait_limit_ns();

__host__ __device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }
constexpr int kNumSMsHint = 152;

// Device-resident scalar state of one handle (Greedy state + certification).
struct DevState {
    double f;               // f(S) of the current Greedy state
    double pick_gain;       // exact gain of the last pick
    double top_thr;         // (K+1)-th largest upper bound, -1 if none
    double esc_thr;         // escalation threshold on upper bounds
    double max_raw_rel_err; // max (bound - exact)/exact over re-evaluated leaders
    long long certified;    // rounds certified by the top-K alone
    long long escalated_rounds;
    long long escalated_cands;
    long long rounds;
    long long exact_evals;  // contenders whose exact FP64 gain was computed
    int round;              // picks made so far (index into out arrays)
    int pick;               // last pick
    int top_count;          // entries in the top-K list this round
    int esc_count;          // entries in the escalation list this round
    int need_esc;           // 1 when this round needs escalation
    int err;                // first device-detected error (ebc_status), 0 if none
    unsigned int mmax_bits; // max_v m_v as FP32 bits (rounded up), for the TC slack
    int zero_scan;          // 1 when every remaining gain is exactly 0
    int ctd_count;          // contenders needing the exact FP64 gain this round
    double best_lo;         // largest certified lower bound of the round
    // lazy Greedy
    double lazy_thr;        // certified lower bound of the round's best gain (pre-selection)
    int list_m;             // candidates in this round's list (lazy mode)
    int list_nch;           // V chunks the bulk kernel used for that list
    long long bulk_cands;   // candidates given a bulk bound, summed over rounds
};

// Points per V chunk of the refine kernels (bounds and exact gains of short
// lists): about 4 chunks per SM for large n; for d > 128 chunks shrink (to
// 32 points at d >= 2048) so that a short list over a small n still spreads
// over the SMs.
__host__ __device__ inline int64_t refine_chunk(int64_t n, int d) {
    const int64_t per_sm = (n + 607) / 608;
    if (d <= 128) return lmax(512, (per_sm + 255) / 256 * 256);
    return lmax(lmax(32, (int64_t)(65536 / d) / 32 * 32), (per_sm + 31) / 32 * 32);
}

// V chunking of the bulk gains kernel for m candidates: the chunk count
// (1..16, bounded by the partial buffer) that best balances
// (candidate tiles x chunks) units over G persistent CTAs.  Used on the host
// and, for lists whose length lives on the device, inside the kernels.
__host__ __device__ inline int pick_chunks(int64_t m, int n_vtiles, int G, int64_t partial_cap, int *vt_per_chunk) {
    const int64_t n_ctiles = (m + 255) / 256;
    const int64_t cap = partial_cap / (m > 0 ? m : 1);
    int best = 1;
    double best_eff = 0.0;
    const int64_t lim = lmin(16, lmin(cap, n_vtiles));
    for (int nch = 1; nch <= lim; ++nch) {
        const int64_t units = n_ctiles * nch;
        const int64_t per = (units + G - 1) / G;
        double eff = (double)units / (double)(per * lmin(G, units)) * (units < G ? (double)units / G : 1.0);
        eff *= 1.0 - 0.003 * nch;  // per-unit candidate-tile load
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = nch;
        }
    }
    const int vpc = (n_vtiles + best - 1) / best;
    *vt_per_chunk = vpc;
    return (n_vtiles + vpc - 1) / vpc;
}

// A tuned configuration of the tensor-core bulk kernel (tune.cu).
struct TuneCfg {
    int na = 0;     // candidate-tile buffers (1, 2)
    int ns = 0;     // point-tile stages (2..6)
    int chunk = 0;  // V-chunk policy: 0 load-balance model, 1 twice the chunks, 2 half
    int bn = 256;   // points per B tile (TMEM columns per region): 256 or 128
    int turns = -1; // 256-point tiles: MMA issuers take turns (1), run freely (0), by row width (-1)
    int es = 0;     // 256-point tiles: drain split by column halves (0) or by region (1)
};

// Scratch / resident buffers of one handle.
struct Ctx {
    int64_t n = 0;
    int32_t d = 0;
    int32_t dpad = 0;  // d rounded up to the tensor-core K tile (64)
    int device = 0;
    cudaStream_t stream = nullptr;
    ebc_prec prec = EBC_FP32;
    int32_t refine_k = 8;
    bool owns_stream = false;

    // resident ground set
    float *V32 = nullptr;    // [n, d] FP32 row-major, exact copy of the input
    double *nv64 = nullptr;  // [n] ||v||^2 in FP64
    float *nv32 = nullptr;   // [n] ||v||^2 rounded to nearest FP32
    // Greedy state
    double *m64 = nullptr;   // [n] m_v = min over S u {e0} of d(v, s)
    uint8_t *sel = nullptr;  // [n] 1 if v is in S
    DevState *st = nullptr;  // device scalars

    // quantised ground set (tensor-core precisions)
    struct Tc {
        int prec = -1;            // precision Vq holds (EBC_BF16 / EBC_FP16), -1 = none
        int64_t n_pad = 0;        // n rounded up to the point tile (256)
        int DP = 0;               // d rounded up to the 64-element swizzle atom
        uint16_t *Vq = nullptr;   // [n_pad, DP] quantised rows v_hat (candidate operand), zero padded
        uint16_t *Vq2 = nullptr;  // [n_pad, DP] 2 v_hat (point operand; exact scaling)
        uint16_t *Aext = nullptr; // [n_pad, 16] bf16 candidate-side extension columns (static)
        uint16_t *Bext = nullptr; // [n_pad, 16] bf16 point-side extension columns (per round)
        uint16_t *Cq = nullptr;   // [n_pad, DP] gathered candidate rows (ebc_gains with a list)
        uint16_t *Cqx = nullptr;  // [n_pad, 16] gathered candidate extension rows
        double *qn64 = nullptr;   // [n_pad] ||v_hat||^2 (FP64)
        float *qerr = nullptr;    // [n_pad] ||v_hat - v|| rounded up
        float *qnorm = nullptr;   // [n_pad] ||v_hat|| rounded up
        float *qmax = nullptr;    // [2] max qerr, max qnorm (as floats, via bit-pattern atomics)
        CUtensorMap tmA_V;        // candidate tiles over Vq (box 64 x 128)
        CUtensorMap tmB_V;        // point tiles over Vq2 (box 64 x 256)
        CUtensorMap tmA_C;        // candidate tiles over Cq
        CUtensorMap tmAx_V;       // candidate extension over Aext (box 16 x 128)
        CUtensorMap tmAx_C;       // candidate extension over Cqx
        CUtensorMap tmBx;         // point extension over Bext (box 16 x 256)
        CUtensorMap tmB_V128;     // 128-point tiles over Vq2 (box 64 x 128)
        CUtensorMap tmBx128;      // point extension over Bext (box 16 x 128)
        // multi-set evaluation (ebc_eval_sets at a tensor-core precision)
        uint16_t *Px = nullptr;   // [n_pad, 16] point-side extension: ||v||^2 - ||v_hat||^2 (static)
        // device plan of a multi-set call (k_sets_plan): padded offsets [l + 1], chunk records
        // [l + 1][4], each set's chunk [l], first chunk of each launch batch [batches + 1]
        int64_t *sp_aux = nullptr, *sp_rec = nullptr;
        int *sp_cj = nullptr, *sp_bf = nullptr;
        int64_t sp_sets = 0, sp_batches = 0;  // capacities
        int64_t res_sets = 0, res_members = 0;  // ebc_reserve_sets
        CUtensorMap tmPx;         // box 16 x 128 over Px
        uint16_t *Mq = nullptr;   // [mcap, DP] 2 s_hat of the gathered set members, padded per set
        uint16_t *Mx = nullptr;   // [mcap, 16] member extension: -||s_hat||^2
        int *gset = nullptr;      // [mcap / 16] per 16-member group: 2 * (set index in its chunk) + last
        int64_t mcap = 0;         // rows of Mq / Mx
    } tc;
    // FP8 e4m3 copy (ebc_set_precision EBC_FP8E4M3): candidate operand with a
    // per-row power-of-two scale s_c, point operand with one power-of-two
    // scale t; both quantised to nearest.  The certified Greedy at FP8 also
    // uses the BF16 copy above (second level).
    struct Tc8 {
        bool ready = false;
        int64_t n_pad = 0;
        int DP = 0;                   // d rounded up to 128 (bytes per row)
        uint8_t *Qc = nullptr;        // [n_pad, DP] candidate operand q_c = RN(c / s_c)
        uint8_t *Qp = nullptr;        // [n_pad, DP] point operand q_v = RN(v / t)
        uint8_t *Cq = nullptr;        // [n_pad, DP] gathered candidate rows
        uint16_t *Aext = nullptr;     // [n_pad, 16] candidate extension / s_c
        uint16_t *Cqx = nullptr;      // [n_pad, 16] gathered candidate extension
        uint16_t *Bext = nullptr;     // [n_pad, 16] point extension / (2 t), per round
        float *fc = nullptr;          // [n_pad] 2 s_c t: scale of a candidate's accumulated sums
        float *Cfc = nullptr;         // [n_pad] gathered fc
        double *qn_c = nullptr, *qn_p = nullptr;  // [n_pad] ||c_hat||^2, ||v_hat||^2
        float *qerr_c = nullptr, *qerr_p = nullptr, *qnorm_c = nullptr, *qnorm_p = nullptr;  // [n_pad], rounded up
        float *qmax = nullptr;        // [5] max qerr_c, max qnorm_c, max qerr_p, max qnorm_p, amax(V)
        float *tscale = nullptr;      // [1] t
        CUtensorMap tmA, tmAx, tmA_C, tmAx_C, tmB, tmBx;
        CUtensorMap tmB128, tmBx128;  // 128-point tiles
    } tc8;
    int num_sms = 152;
    int max_ctas = 0;  // cap on persistent-kernel CTAs (0 = one per SM)
    const TuneCfg *tune_force = nullptr;  // set by the autotuner while it times a configuration

    // scratch
    double *partial = nullptr;  // [nchunk_cap, n] per-V-chunk partial sums of the bulk gains
    int64_t partial_cap = 0;    // doubles
    double *gain_up = nullptr;  // [n] bulk gains (upper bounds in Greedy)
    int *blk_idx = nullptr;     // per-block top lists
    double *blk_val = nullptr;
    int blk_cap = 0;
    int *top_idx = nullptr;     // [kMaxRefineK + 1]
    double *top_val = nullptr;  // [kMaxRefineK + 1] upper bounds of the top list
    int *esc_idx = nullptr;     // [n] escalation list
    double *esc_exact = nullptr;// [n]
    int *cand_buf = nullptr;    // [n] gathered candidate list for ebc_gains
    // lazy Greedy: stale upper bounds of every candidate's gain (gains never
    // increase as S grows) and the round's candidate list
    bool lazy = false;
    bool force_kb = false;  // K-blocked bulk kernel even where whole rows fit (ebc_set_kblocked)
    double *ub64 = nullptr;     // [n]
    int *lazy_idx = nullptr;    // [n]
    double *set_part = nullptr; // eval_sets partials
    int64_t set_part_cap = 0;
    int32_t h_err_store[4] = {0, 0, 0, 0};
    int32_t *h_err = h_err_store;  // host words for error read-back

    // two-level certification of the Greedy pick (k_select.cu)
    struct Sel {
        int cap = 0;               // escalated entries with chunked bounds
        int nchunks = 0;           // V chunks of the refine kernels
        int64_t chunk = 0;         // points per chunk
        double *top_lo = nullptr, *top_hi = nullptr;    // [kMaxRefineK] bounds of the top list
        double *esc_lo = nullptr, *esc_hi = nullptr;    // [cap] bounds of the escalated entries
        double *part_lo = nullptr, *part_hi = nullptr;  // [(kMaxRefineK + cap) * nchunks] chunk partials
        int *ctd_idx = nullptr;                         // [kMaxRefineK + cap] contenders
        double *ctd_part = nullptr;                     // [(kMaxRefineK + cap) * nchunks]
        double *ctd_exact = nullptr;                    // [kMaxRefineK + cap]
    } cert;

    std::string last_error;
};

// ---- device memory: one stream-ordered pool per device (api.cu) ----------
// Handles allocate and free through it (cudaMallocFromPoolAsync /
// cudaFreeAsync on their stream), so creating and destroying instances never
// synchronises the device.  Freed memory stays cached in the pool.
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s, int dev);
void pool_free(void *p, cudaStream_t s);

// ---- handle helpers shared with the batch runtime (api.cu) ---------------
ebc_status create_handle(const float *V, int64_t n, int32_t d, int32_t v_on_device, void *stream, bool sync,
                         ebc_t *out);
ebc_status set_precision_handle(ebc_t h, ebc_prec prec, int32_t refine_k, bool sync);
// time the bulk kernel's configurations for this handle's precision and n
// bucket and store the fastest (only_if_missing: skip a bucket already tuned)
ebc_status autotune_handle(ebc_t h, int32_t reps, bool only_if_missing);
int64_t handle_bytes(int64_t n, int32_t d, ebc_prec prec);

// ---- launchers (defined in the .cu files) --------------------------------
cudaError_t launch_prologue(Ctx &c);
cudaError_t launch_reset_state(Ctx &c);
cudaError_t launch_gains_fp32(Ctx &c, const int *cand, int64_t m, bool upper, int64_t chunk, int nchunks);
cudaError_t launch_reduce_select(Ctx &c, int64_t m, int nchunks, const int *cand, bool greedy,
                                 double *out_gain, int nblk);
// tuning table (tune.cu)
bool tune_lookup(const Ctx &c, int prec, int RB, int64_t n, TuneCfg *cfg);
bool tune_has(int prec, int RB, int64_t n);
bool tune_get(int prec, int RB, int64_t n, TuneCfg *cfg, double *ms);
void tune_store(int prec, int RB, int64_t n, const TuneCfg &cfg, double ms);
int apply_chunk_mode(int nchunks, int mode, int n_vtiles, int64_t cap, int *vt_per_chunk);
bool tc_config_fits(int RB, int na, int ns, int bn);  // k_tc.cu: shared memory of a pipeline shape fits
int tc_row_bytes(const Ctx &c);              // k_tc.cu: row bytes of the current precision's bulk operand

// few-candidate passes over V, one warp per point (k_few.cu); d <= 256
bool few_supported(const Ctx &c);
// lists longer than max_cnt are skipped (left to the tiled bound kernel)
cudaError_t launch_few_bounds(Ctx &c, const int *list, const int *count, int cap, double *out_lo, double *out_hi,
                              int64_t chunk, int nchunks, int max_cnt);
constexpr int kFewBoundsMax = 64;  // list length up to which the few-candidate bound kernel runs
cudaError_t launch_few_exact(Ctx &c, const int *list, const int *count, int cap, double *out, int64_t chunk,
                             int nchunks);
cudaError_t launch_few_update(Ctx &c);
// lazy Greedy (k_lazy.cu)
cudaError_t launch_lazy_preselect(Ctx &c, int nblk, int K);   // top-K of ub64 among unselected -> top list
cudaError_t launch_lazy_threshold(Ctx &c);                     // st->lazy_thr = max folded lo of the top list
cudaError_t launch_lazy_build(Ctx &c);                         // lazy_idx = {c : ub64[c] >= lazy_thr}, st->list_m
cudaError_t launch_lazy_select(Ctx &c, double eta, int nblk);  // list sums, ub64 update, per-block tops
cudaError_t launch_lazy_collect(Ctx &c, double eta);           // escalation over the list
cudaError_t launch_lazy_init(Ctx &c);                          // ub64 = +inf
cudaError_t launch_lazy_from_full(Ctx &c, double eta);         // ub64 <- min(ub64, gain_up (1 + eta))
cudaError_t launch_merge_top(Ctx &c, int nblk, int K, double eta);
// Exact FP64 gains (out_hi == nullptr) or rigorous FP32 [lo, hi] bounds of
// the gains (out holds lo, out_hi hi) of a device list, as chunk partials.
cudaError_t launch_refine(Ctx &c, const int *list, const int *count, int list_cap, double *out, double *out_hi,
                          int64_t chunk, int nchunks);
cudaError_t launch_collect_escalation(Ctx &c, double eta);
cudaError_t launch_refine_overflow(Ctx &c, const int *list, const int *count, int cap, double *out_exact);
cudaError_t launch_refine_rows(Ctx &c, const int *list, const int *count, int list_cap, double *out,
                               double *out_hi, int64_t chunk, int nchunks);
// lists of at most min_cnt entries are skipped (left to the few-candidate kernel)
cudaError_t launch_bounds_fp32(Ctx &c, const int *list, const int *count, int cap, double *out_lo, double *out_hi,
                               int64_t chunk, int nchunks, float kh, float kl, int min_cnt);
// [lo, hi] gain bounds (register-tiled FP32) / exact gains (one candidate per
// block) of a device list with device count, as chunk partials
cudaError_t launch_bounds_list(Ctx &c, const int *list, const int *count, int cap, double *out_lo, double *out_hi,
                               int64_t chunk, int nchunks);
cudaError_t launch_exact_list(Ctx &c, const int *list, const int *count, int cap, double *out, int64_t chunk,
                              int nchunks);
// two-level certified pick (k_select.cu)
cudaError_t launch_fold_bounds(Ctx &c, const double *part_lo, const double *part_hi, const int *count, int cap,
                               double *lo, double *hi);
cudaError_t launch_decide_top(Ctx &c, double eta_bulk);
cudaError_t launch_decide_contenders(Ctx &c);
cudaError_t launch_commit_pick(Ctx &c, int32_t *out_idx, double *out_f);
cudaError_t launch_update(Ctx &c);
// threshold sieve (k_select.cu): exact gains of a list from chunk partials; commit of an accepted item
cudaError_t launch_sieve_fold_exact(Ctx &c, const double *part, const int *count, int cap, double *out);
cudaError_t launch_sieve_commit(Ctx &c, int item, double gain);
cudaError_t launch_current_f(Ctx &c, double *d_out);
cudaError_t launch_eval_sets_fp32(Ctx &c, const int32_t *idx, const int64_t *off, int64_t l, double *out_f,
                                  const int *bad);
// out_f[j0 + j] = (1/n) sum over ntiles rows of set_part[row][j], j < lb
cudaError_t launch_sets_finalize(Ctx &c, int64_t ntiles, int64_t lb, int64_t j0, int64_t l, double *out_f);

// tensor-core path
bool tc_supported(const Ctx &c);           // 16-bit bulk bounds and sets (K-blocked kernels above d = 128)
bool tc_resident_supported(const Ctx &c);  // FP8 bulk: d <= 128
cudaError_t tc_setup(Ctx &c, int prec);          // allocate, quantise, build tensor maps
cudaError_t tc_quantize(Ctx &c);                 // (re)quantise V into Vq
cudaError_t launch_prep_tc(Ctx &c, bool upper);  // a_v for every point (+ max m_v)
// bulk gains on tensor cores; returns the number of V chunks used in *nchunks
cudaError_t launch_gains_tc(Ctx &c, const int *cand, int64_t m, bool upper, int *nchunks);
// bulk gains of the list (cand, *m_dev) whose length is on the device (m_cap bounds it)
cudaError_t launch_gains_tc_list(Ctx &c, const int *cand, const int *m_dev, int64_t m_cap);
// multi-set evaluation on tensor cores, planned on the device: `members` is
// an upper bound of off[l] (more members record EINVAL and evaluate nothing);
// set_part must hold at least 8 n_pad / 256 rows
cudaError_t launch_eval_sets_tc(Ctx &c, const int32_t *idx, const int64_t *off, int64_t l, int64_t members,
                                double *out_f, int64_t *nlaunch);
// grow the multi-set buffers for `sets` sets of `members` members in all
cudaError_t tc_sets_reserve(Ctx &c, int64_t sets, int64_t members);
void tc_free(Ctx &c);
// allow a kernel the per-CTA maximum of dynamic shared memory on the current
// device (once per device and kernel); bytes is the launch's own size
cudaError_t allow_smem(const void *kernel, uint32_t bytes);

// ---- one persistent bulk launch over several handles (k_tc.cu, group.cu) ----
// A handle's part of a shared Greedy round: its tensor maps (read by TMA from
// device memory) and the plan of its bulk gains over all n candidates.  The
// maps keep CUtensorMap's own alignment (at least the 64 bytes TMA needs).
struct GroupInst {
    CUtensorMap tmA, tmAx, tmB, tmBx;  // candidate rows / extension, point rows / extension
    double *partial;                   // [nchunks][m] the handle's chunk partials
    int *err;                          // the handle's device error word
    int64_t m;                         // candidates: every point (selected ones are masked later)
    int n_vtiles;                      // point tiles of 256
    int vt_per_chunk;                  // point tiles per V chunk
    int nchunks;                       // V chunks
    int RB;                            // bytes per row of the main part (128 or 256)
    uint32_t idesc, idesc_ext;         // MMA instruction descriptors (precision), extension (BF16)
};
// One work unit: a 256-candidate tile of one handle against one of its V chunks.
struct GroupUnit {
    int inst, ctile, chunk, ntiles;  // ntiles = point tiles of the chunk (the unit's cost)
};
bool tc_group_supported(const Ctx &c);  // BF16 / FP16 with whole rows resident (d <= 128)
int tc_group_row_bytes(const Ctx &c);   // RB of the handle (2 * padded d)
void group_inst_fill(const Ctx &c, int nchunks, int vt_per_chunk, GroupInst *out);
// the persistent kernel over units [0, total_units) handed out by *d_counter
// (zero on entry); a timeout is recorded in *d_err
cudaError_t launch_gains_tc_group(const GroupInst *d_inst, const GroupUnit *d_units, int total_units,
                                  int *d_counter, int *d_err, int RBmax, int G, cudaStream_t s);
// copy a nonzero *d_err into the error word of handles [0, count) of d_inst
cudaError_t launch_group_err(const GroupInst *d_inst, int count, const int *d_err, cudaStream_t s);

// FP8 e4m3 (k_tc.cu)
cudaError_t tc8_setup(Ctx &c);                    // allocate, quantise, build tensor maps
cudaError_t launch_prep_tc8(Ctx &c, bool upper);  // per-round point extension
cudaError_t launch_gains_tc8(Ctx &c, const int *cand, int64_t m, int *nchunks);

}  // namespace ebc
