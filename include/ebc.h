/*
 * ebc.h -- C ABI of the GB300 exemplar-based clustering (EBC) library.
 *
 * What is computed (paper: "Providing Meaningful Data Summarizations Using
 * Exemplar-based Clustering in Industry 4.0"):
 *
 *   d(x, y) = ||x - y||^2                         squared Euclidean (Sec. 5)
 *   L(S)    = (1/|V|) sum_{v in V} min_{s in S} d(v, s)   k-medoids loss (Sec. 4)
 *   f(S)    = L({e0}) - L(S u {e0}),  e0 = 0      EBC function (Sec. 4)
 *           = (1/n) sum_v max(0, ||v||^2 - min_{s in S} d(v, s))
 *   Delta_f(c | S) = f(S u {c}) - f(S)            discrete derivative (Sec. 3, Def. 1)
 *                  = (1/n) sum_v max(0, m_v - d(v, c)),  m_v = min_{s in S u {e0}} d(v, s)
 *
 * A handle owns one ground set V (n points of dimension d) resident on the
 * GPU, its norms, quantised copies and the Greedy state (S, m_v, f).  Every
 * call is enqueued on the handle's CUDA stream.  Nothing here falls back to
 * the CPU: a handle can only be created on an sm_103 device.
 *
 * Conventions for every function below:
 *   - Indices are 0-based int32 in [0, n).
 *   - "device pointer" arguments must point to device memory that stays
 *     valid until the stream reaches the call; the caller owns them.
 *     "_host" variants take ordinary host pointers and return after the
 *     results are in host memory (they synchronise the stream).
 *   - Calls on one handle must not run concurrently from several host
 *     threads.  Different handles are independent.
 *   - On failure a negative ebc_status is returned and ebc_last_error(h)
 *     holds a one-line description.  Errors that only the device can detect
 *     (an out-of-range index inside a device CSR list) are recorded in the
 *     handle and returned by the next ebc_sync().
 */
#ifndef EBC_H
#define EBC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ebc_ctx *ebc_t;

typedef enum {
    EBC_OK = 0,
    EBC_EINVAL = -1,   /* bad argument: sizes, NULL pointers, non-monotone CSR offsets,
                          k larger than the unselected points, non-finite V */
    EBC_EINDEX = -2,   /* an index outside [0, n) */
    EBC_ENOMEM = -3,   /* a device or host allocation failed */
    EBC_ECUDA = -4,    /* a CUDA runtime call failed (text in ebc_last_error) */
    EBC_ETIMEOUT = -5, /* a bounded device-side wait ran out */
    EBC_EBUSY = -6,    /* resource temporarily unavailable */
    EBC_ENODEV = -7    /* no sm_103 device is current */
} ebc_status;

/* Arithmetic used for the bulk distance work (Sec. 5 compares FP32 with
 * half precision; here the low-precision paths run on tcgen05 tensor cores
 * with FP32 accumulation and exact re-evaluation of the leaders). */
typedef enum {
    EBC_FP32 = 0,    /* direct (v - c)^2 in FP32 on the CUDA cores */
    EBC_BF16 = 1,    /* V.C^T in BF16 on tensor cores, FP32 accumulate */
    EBC_FP16 = 2,    /* V.C^T in FP16 on tensor cores, FP32 accumulate */
    EBC_FP8E4M3 = 3  /* V.C^T in FP8 e4m3: candidate rows with a per-row power-of-two
                        scale, points with one power-of-two scale; Greedy certifies with
                        BF16 bounds of the candidates the FP8 bounds cannot exclude */
} ebc_prec;

/* Counters of the certified Greedy pick (see ebc_greedy). */
typedef struct {
    int64_t rounds;               /* Greedy rounds run since create / reset */
    int64_t certified_rounds;     /* rounds decided by the top-K exact re-evaluation alone */
    int64_t escalated_rounds;     /* rounds that exactly re-evaluated further candidates */
    int64_t escalated_candidates; /* total such extra candidates */
    double max_raw_rel_err;       /* max (bulk bound - lower bound) / lower bound over the top
                                     list: how loose the bulk upper bounds were */
    int64_t exact_evaluations;    /* candidates whose exact gain was computed */
    int32_t prec;                 /* current ebc_prec */
    int32_t refine_k;             /* current K */
    int64_t bulk_candidates;      /* lazy Greedy: candidates given a bulk bound, summed over rounds */
    int32_t lazy;                 /* 1 when lazy Greedy is on (ebc_set_lazy) */
    int32_t reserved;
} ebc_stats;

/* Library version, (major << 16) | minor. */
int32_t ebc_version(void);

/*
 * Create a handle for the ground set V (Sec. 4.2 "Memory Layout": V is copied
 * to the GPU once at initialisation and stays resident).
 *   V            n x d FP32, row-major (point i is V[i*d .. i*d+d-1]).
 *   v_on_device  0: V is a host pointer; 1: V is a device pointer.
 *   stream       cudaStream_t to enqueue on (NULL = the legacy default stream).
 *   out          receives the handle.
 * The library copies V; the caller may free it when this returns.  The
 * prologue computes ||v||^2 (= d(v, e0)), L({e0}) (computed once and shared,
 * Sec. 4.2 "Algorithm"), the quantised copies and m_v = ||v||^2 (S = {}).
 * Synchronises the stream once.  EINVAL for n <= 0, d <= 0, d > 4096 or a
 * non-finite entry of V; ENODEV when the current device is not sm_103.
 */
ebc_status ebc_create(const float *V, int64_t n, int32_t d, int32_t v_on_device, void *stream, ebc_t *out);

/*
 * Replace the ground set of an existing handle by a new V of the same n and
 * d (same layout and pointer kinds as ebc_create), rerun the prologue and
 * return the Greedy state to S = {}.  Allocates nothing, so a resident slot
 * can be reused for the next instance.  Asynchronous; a non-finite entry of
 * V is reported by the next ebc_sync() as EINVAL.
 */
ebc_status ebc_reload(ebc_t h, const float *V, int32_t v_on_device);

/* Release every resource of the handle (NULL is accepted). */
ebc_status ebc_destroy(ebc_t h);

/* Change the stream later calls are enqueued on. */
ebc_status ebc_set_stream(ebc_t h, void *stream);

/*
 * Select the bulk arithmetic and K, the number of leading candidates that
 * Greedy re-evaluates exactly each round (1 <= K <= 31; default FP32, K = 8).
 * EBC_BF16 / EBC_FP16 take any d (above d = 128 the bulk and multi-set
 * kernels stream the rows in 64-element K blocks, see ebc_set_kblocked);
 * EBC_FP8E4M3 needs d <= 128.  EBC_FP8E4M3 also keeps the BF16
 * copy: ebc_gains returns the raw FP8 gains, ebc_greedy bounds every
 * candidate with FP8 and then certifies as the lazy Greedy does with BF16
 * bounds (same picks as every other precision), ebc_eval_sets uses BF16.
 * EINVAL for an unsupported precision or d, K outside [1, 31], or a V that
 * overflows the requested format (FP16) or is not finite.
 */
ebc_status ebc_set_precision(ebc_t h, ebc_prec prec, int32_t refine_k);

/*
 * f(S_j) for a list of l sets (the multi-set S_multi = {S_1..S_l} of
 * Sec. 4.1, evaluated as the work matrix W and its row sums W.1 of
 * Sec. 4.2, Eq. "work matrix"; W is never materialised).
 *   csr_idx  device int32[csr_off[l]]: members of set j are
 *            csr_idx[csr_off[j] .. csr_off[j+1]-1]; duplicates allowed.
 *   csr_off  device int64[l+1], csr_off[0] = 0, non-decreasing.
 *   out_f    device double[l]; an empty set gives 0.
 * Independent of the Greedy state.  With EBC_FP32 the distances are direct
 * FP32; with a tensor-core precision the minimum per set is formed from
 * V.S^T products (K-blocked above d = 128), the members padded per set to
 * 16-column groups; the plan (padding, chunks, member gather) is made on the
 * device.  Asynchronous at EBC_FP32; at a tensor-core precision too when a
 * reservation (ebc_reserve_sets) covers l sets, and then nothing is read back
 * to the host, so the call can be captured in a CUDA graph; without one the
 * call first reads csr_off[l] (8 bytes, one wait for the stream) to size its
 * buffers.  Offsets that do not start at 0 or decrease, a NULL csr_idx with
 * members, or more members than a reservation holds give EINVAL from the
 * next ebc_sync() and no member is read; out-of-range members are detected
 * on the device: the set is evaluated without them and ebc_sync() returns
 * EINDEX.  l = 0 is OK.
 */
ebc_status ebc_eval_sets(ebc_t h, const int32_t *csr_idx, const int64_t *csr_off, int64_t l, double *out_f);

/*
 * Reserve the device buffers of ebc_eval_sets at a tensor-core precision for
 * calls of up to max_sets sets with up to max_members members in all
 * (csr_off[l]).  Such calls then allocate nothing and read nothing back to
 * the host.  max_sets = 0 drops the reservation (the buffers stay).  EINVAL
 * for negative sizes or at EBC_FP32; ENOMEM when the buffers do not fit.
 */
ebc_status ebc_reserve_sets(ebc_t h, int64_t max_sets, int64_t max_members);

/* Host-pointer form of ebc_eval_sets; validates offsets and indices on the host. */
ebc_status ebc_eval_sets_host(ebc_t h, const int32_t *csr_idx, const int64_t *csr_off, int64_t l, double *out_f);

/*
 * Marginal gains Delta_f(c | S) (Sec. 3, Def. 1) for m candidates, relative
 * to the handle's current Greedy state S (S = {} after create / reset).
 *   cand_idx  device int32[m], or NULL for all n points (then m must be n).
 *   out_gain  device double[m].  Candidates already in S get 0.
 * EBC_FP32 gives direct-FP32 distances with FP64 sums over V; tensor-core
 * precisions give the raw low-precision gain (no re-evaluation).
 */
ebc_status ebc_gains(ebc_t h, const int32_t *cand_idx, int64_t m, double *out_gain);

/* Host-pointer form of ebc_gains. */
ebc_status ebc_gains_host(ebc_t h, const int32_t *cand_idx, int64_t m, double *out_gain);

/*
 * k rounds of Greedy (Sec. 3; the step is described in Sec. 4.1): each round
 * adds the not-yet-selected point of largest marginal gain, ties to the
 * smallest index (see below for what counts as a tie), continuing from the
 * handle's current state.
 *   out_idx  device int32[k]: the picks in order.
 *   out_f    device double[k]: out_f[t] = f(S) after pick t (cumulative).
 * Each round evaluates the gain of every unselected point with the bulk
 * precision as a rigorous upper bound; the K largest get rigorous FP32
 * direct-distance bounds [lo, hi]; if the (K+1)-th bulk bound can reach the
 * best lo, every candidate whose bulk bound reaches it gets [lo, hi] too;
 * the candidates whose hi reaches the best lo get the exact gain, and the
 * pick is the best of those.  Exact gains are computed from the FP32 inputs
 * with double-FP32 arithmetic (error-free TwoSum / TwoProduct steps, about
 * 2^-44 relative per distance) and FP64 sums over V; an escalation of more
 * than 4,096 candidates computes the exact gains past that capacity with
 * FP64 distances.  Gains within 1e-10 relative of the round's largest exact
 * gain are ties and go to the smallest index (so duplicate points and
 * mirror-image pairs, whose gains agree in real arithmetic, are ordered by
 * index, not by rounding); the pick is therefore the exact argmax wherever
 * the best two gains differ by more than that, at every precision.  When
 * every remaining gain is 0 the pick is the smallest unselected index.
 * EINVAL when k < 0 or k exceeds the number of unselected points.
 */
ebc_status ebc_greedy(ebc_t h, int32_t k, int32_t *out_idx, double *out_f);

/* Cap the CTAs of the persistent bulk kernel (0 = one per SM).  Leaves SMs
 * free for other work on the GPU, e.g. small requests in a serving batch. */
ebc_status ebc_set_max_ctas(ebc_t h, int32_t max_ctas);

/*
 * Lazy Greedy (Minoux's lazy evaluation of the Greedy of Sec. 3): the handle
 * keeps, for every candidate, an upper bound of its marginal gain from the
 * round it was last bounded; by diminishing returns (Def. 3) such a bound
 * stays valid as S grows.  Each round first certifies a lower bound of the
 * best gain from the candidates with the largest stale bounds, then bounds
 * only the candidates whose stale bound reaches it on the tensor cores, and
 * certifies the pick among them as ebc_greedy does.  Picks and f values are
 * the same as without it (the exact argmax, same tie rule, same exact gain);
 * only the work per round changes.  Applies at the tensor-core precisions;
 * at EBC_FP32 every round evaluates all candidates.  on = 1 enables, 0
 * disables; the bounds restart from the current state when enabled, and
 * ebc_reset / ebc_reload restart them.  Allocates 12 bytes per point on first
 * use.
 */
ebc_status ebc_set_lazy(ebc_t h, int32_t on);

/*
 * Autotuner of the tensor-core bulk kernel.  The kernel's point-tile width
 * (256 or 128 points per MMA, i.e. the N of the 128 x N tile), at 256
 * points whether its two MMA-issuing threads take turns or issue freely and
 * whether its drain warps split the TMEM regions by columns or by region,
 * its pipeline shape (candidate-tile buffers x point-tile stages that fit
 * shared memory at that width) and its V-chunk policy (load-balance model,
 * twice or half as many chunks) are timed with CUDA events on this handle (reps timed
 * launches each, fastest kept) and the fastest is stored in a process-wide
 * table keyed by (precision, padded d, floor(log2 n)); later bulk launches
 * of any handle in that bucket use it.  Rows longer than the resident layout
 * allows (d > 128 at 16 bits) have one K-blocked shape and store nothing.
 * Synchronises the handle's stream; leaves the Greedy state unchanged.
 * Results (picks, f) do not depend on the configuration.  EINVAL at EBC_FP32
 * or reps outside [1, 100].
 */
ebc_status ebc_autotune(ebc_t h, int32_t reps);

/*
 * The tuning-table entry that bulk launches of this handle use at its
 * current precision: cfg[0] = points per tile (256 or 128), cfg[1] =
 * candidate-tile buffers, cfg[2] = point-tile stages, cfg[3] = chunk policy
 * (0, 1, 2), cfg[4] = issuer turns (1 on, 0 off, -1 by row width: on from
 * 256 bytes per row), cfg[5] = drain split (0 by column halves, 1 by
 * region), and *ms (may be NULL) the time the autotuner measured for it.
 * All zero when the bucket has no entry (the default shape is used).  Host
 * only; EINVAL for a NULL handle or cfg.
 */
ebc_status ebc_tune_query(ebc_t h, int32_t cfg[6], double *ms);

/* The tuning table: save as JSON, merge a saved file (EINVAL for an
 * unreadable or malformed file; the table is then unchanged; an entry
 * without "bn" means 256-point tiles, without "turns" turns by row width, without "es" the drain split by
 * column halves),
 * count and clear its entries. */
ebc_status ebc_tune_save(const char *path);
ebc_status ebc_tune_load(const char *path);
int64_t ebc_tune_count(void);
ebc_status ebc_tune_clear(void);

/* Tensor-core layout of the bulk and multi-set kernels at EBC_BF16 /
 * EBC_FP16: 1 streams both operands' rows in 64-element K blocks (always
 * used for d > 128, where whole rows do not fit shared memory); 0 (the
 * default) keeps a tile of whole rows resident where it fits.  Both issue
 * the same MMA sequence, so bounds, picks, f and set values are bitwise
 * the same. */
ebc_status ebc_set_kblocked(ebc_t h, int32_t on);

/* Replay Greedy rounds from a captured CUDA graph (1, the default) or issue
 * every kernel directly (0).  Graph replay needs a non-NULL stream and is
 * not used while profiling is on. */
ebc_status ebc_set_graphs(ebc_t h, int32_t on);

/* Host-pointer form of ebc_greedy. */
ebc_status ebc_greedy_host(ebc_t h, int32_t k, int32_t *out_idx, double *out_f);

/*
 * Threshold sieve over a stream: the decision rule of the streaming
 * optimisers the paper names beside Greedy (Sec. 2 and Sec. 4.1: Sieve
 * Streaming, Badanidiyuru et al. 2014; Three Sieves, Buschjaeger et al.,
 * which the case study of Sec. 6 runs for Fig. 4).  Items (indices into V)
 * arrive in stream order.  With s = |S| < K and the current threshold
 * v = thr[level],
 *     tau = (v / 2 - f(S)) / (K - s),
 * an item not in S joins S when its exact marginal gain Delta_f(e | S) >= tau
 * (S, m_v and f then update as after a Greedy pick).  An item already in S,
 * or one whose gain is below tau, is a rejection; after `patience`
 * consecutive rejections the sieve moves to the next threshold (staying on
 * the last) and the count restarts; patience <= 0 never moves.  Once
 * |S| = K the rest of the stream is left undecided.
 *   Three Sieves:   thr = ebc_threshold_ladder(m, K, eps, 1), patience T.
 *   Sieve Streaming: one handle (or one reset state) per value v of
 *                   ebc_threshold_ladder(m, K, eps, 2), thr = {v}, patience 0;
 *                   keep the best f.
 * Decisions use certified gains: upper bounds reject the items they can and
 * the exact gain (as in Greedy's pick) decides the rest, so decisions and f
 * match the FP64 definition except where the gain and tau agree to about
 * 1e-12 relative.  The handle keeps an upper bound of every point's gain
 * while S only grows (diminishing returns, Sec. 3, Def. 3): an item whose
 * bound is below its tau is rejected without device work; the others get a
 * fresh bulk bound (tensor cores at BF16 / FP16 / FP8, rigorous FP32 bounds
 * at EBC_FP32) before any exact gain.  ebc_reset, ebc_reload and
 * ebc_state_load drop the kept bounds.
 */
typedef struct {
    int32_t K;           /* summary size bound, counting the points already in S */
    int32_t nthr;        /* number of thresholds, >= 1 */
    const double *thr;   /* host array [nthr] of threshold values v (finite), walked in order */
    int64_t patience;    /* consecutive rejections before the next threshold; <= 0: never move */
    int32_t level;       /* in/out: index of the current threshold, in [0, nthr) */
    int32_t reserved;
    int64_t rejections;  /* in/out: consecutive rejections so far, >= 0 */
    int64_t consumed;    /* out: stream positions decided by the last call (len unless |S| reached K) */
    int64_t bounded;     /* in/out counter: items given a bulk upper bound */
    int64_t exact;       /* in/out counter: items whose exact gain was computed */
    const double *bounds; /* optional host [n]: upper bounds of every point's gain valid for the
                             current S and every larger one (e.g. ebc_gain_bounds at S = {});
                             NULL: none */
} ebc_sieve_state;

/*
 * One pass of the threshold sieve over items[0 .. len) (host array),
 * continuing from the handle's state (S, m_v, f) and from s->level /
 * s->rejections, so a stream can be fed in pieces.  Accepted items and f
 * after each go to out_idx / out_f (host arrays, capacity K - |S|), their
 * number to *out_count.  Synchronises the handle's stream.
 * EINVAL: NULL state or outputs, nthr < 1, a non-finite threshold, level or
 * rejections out of range, K < |S| or K > n, len < 0; EINDEX: an item
 * outside [0, n).  The state is unchanged on an argument error.
 */
ebc_status ebc_sieve_host(ebc_t h, ebc_sieve_state *s, const int32_t *items, int64_t len, int32_t *out_idx,
                          double *out_f, int32_t *out_count);

/*
 * Rigorous upper bounds of Delta_f(c | S) for m candidates (same arguments
 * as ebc_gains): the bulk kernel in its upper-bound mode (the per-pair slack
 * of the certified Greedy pick), widened by the relative error of its
 * partial sums; 0 for candidates in S.  Bounds at S = {} stay valid for
 * every S (Sec. 3, Def. 3): the ebc_sieve_state.bounds of a fresh stream.
 */
ebc_status ebc_gain_bounds(ebc_t h, const int32_t *cand_idx, int64_t m, double *out_ub);

/* Host-pointer form of ebc_gain_bounds. */
ebc_status ebc_gain_bounds_host(ebc_t h, const int32_t *cand_idx, int64_t m, double *out_ub);

/*
 * Threshold ladder of the streaming optimisers: every value (1 + eps)^i (i an
 * integer, computed as pow(1 + eps, i) in double) with
 * m <= (1 + eps)^i <= upper * K * m, largest first; m is the largest singleton
 * value max_e f({e}).  Writes at most cap values to out (out may be NULL with
 * cap 0 to size) and the full count to *count.  Host only, no device work.
 * EINVAL: m or eps not finite and > 0, K < 1, upper not finite and > 0,
 * count NULL, more than 1,000,000 values, or cap smaller than the count.
 */
ebc_status ebc_threshold_ladder(double m, int32_t K, double eps, double upper, double *out, int32_t cap,
                                int32_t *count);

/* Return the Greedy state to S = {} (m_v = ||v||^2, f = 0, counters zeroed). */
ebc_status ebc_reset(ebc_t h);

/* Wait for the handle's stream; returns the first device-detected error. */
ebc_status ebc_sync(ebc_t h);

/* Certification counters (synchronises the stream). */
ebc_status ebc_get_stats(ebc_t h, ebc_stats *out);

/*
 * The candidates that reached the certified stage of the last Greedy round
 * (Sec. 3's argmax, step a4): the K entries of the top list by bulk upper
 * bound, then, when the round escalated, every candidate whose bulk bound
 * could reach the best certified lower bound.  Every candidate left out has
 * an upper bound below the pick's gain.  out_idx is host memory of capacity
 * cap; *count receives the full number, and nothing is copied when cap is
 * smaller (call with cap 0 to size).  *count = 0 before the first round.
 * Synchronises the stream.  For inspection and tests.
 */
ebc_status ebc_last_round_candidates(ebc_t h, int32_t *out_idx, int64_t cap, int64_t *count);

/* Launch and device-time counters of one handle.  Device times are
 * measured with CUDA events on the handle's stream around each launch while
 * profiling is on (ebc_set_profiling); launch counts are always kept. */
typedef struct {
    int64_t launches;      /* kernels launched by this handle */
    int64_t bulk_launches; /* launches of the bulk gains kernel (any precision) */
    double bulk_ms;        /* summed device time of those launches (profiling on) */
    int64_t bulk_evals;    /* (candidate, point) pairs those launches evaluated */
    int64_t refine_launches;
    double refine_ms;      /* rigorous bounds and exact re-evaluation of the leaders */
    int64_t eval_launches; /* launches of the multi-set kernel */
    double eval_ms;
    int64_t list_launches; /* lazy and FP8 Greedy: row gather + bulk bounds of the round's list */
    double list_ms;
} ebc_profile;

/* Turn per-launch event timing on (1) or off (0); counters keep running. */
ebc_status ebc_set_profiling(ebc_t h, int32_t on);

/* Read the counters (synchronises the stream). */
ebc_status ebc_get_profile(ebc_t h, ebc_profile *out);

/* Zero the counters. */
ebc_status ebc_reset_profile(ebc_t h);

/*
 * Snapshot of the Greedy state (the per-point minima m_v of Sec. 4's
 * incremental evaluation, the selected set S, f(S) and the round counters),
 * for pre-empting an instance and resuming it later in this or another
 * handle over the same V: a Greedy continued from a loaded snapshot makes the
 * same picks with the same f as one that was never interrupted.  The buffer
 * is host memory of ebc_state_size bytes, owned by the caller.  Save
 * synchronises the stream (and reports a pending device error instead of
 * saving); load checks the snapshot (EINVAL for another shape, a truncated
 * buffer or inconsistent contents) and restarts lazy bounds.
 */
ebc_status ebc_state_size(ebc_t h, int64_t *bytes);
ebc_status ebc_state_save(ebc_t h, void *host_buf, int64_t bytes);
ebc_status ebc_state_load(ebc_t h, const void *host_buf, int64_t bytes);

/* f(S) of the current Greedy state, computed on the device (synchronises). */
ebc_status ebc_current_f(ebc_t h, double *out_f);

/*
 * Multi-set evaluation that allocates nothing (the paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory at
 * run time, such as a control loop with a fixed latency budget, where
 * cudaMalloc can synchronise the device, or a program whose device memory is
 * owned by another allocator).  Same result as ebc_eval_sets at EBC_FP32,
 * without a handle:
 *   V        device float[n * d], row-major;  n >= 1, 1 <= d <= 4096
 *   csr_idx  device int32[csr_off[l]];  csr_off device int64[l + 1]
 *   out_f    device double[l]
 *   stream   cudaStream_t (NULL = legacy default stream)
 * Scratch is a static 8 MiB device array held by every GPU that loads the
 * library until exit; n may be at most 134,217,728 (1,048,576 tiles of 128
 * points), larger n is rejected with EINVAL.  Sets are evaluated in passes
 * that fit the array (and at most 524,280 sets per pass).  All calls share
 * the array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU race and must not be issued.  The first call on a
 * device looks up the array's address with that device current; make that
 * first call before any stream capture.  Every call reads its device-side
 * error words back into host memory and waits for the stream before it
 * returns; it returns EINDEX for a member outside [0, n), EINVAL for offsets
 * that do not start at 0 or decrease, or for a NULL csr_idx with a
 * non-empty set (then no member is read).  An empty set gives 0.  Text of
 * the last failure: ebc_noalloc_last_error().
 */
ebc_status ebc_eval_sets_noalloc(const float *V, int64_t n, int32_t d, const int32_t *csr_idx,
                                 const int64_t *csr_off, int64_t l, double *out_f, void *stream);

/* Text of the last ebc_eval_sets_noalloc failure on this host thread. */
const char *ebc_noalloc_last_error(void);

/*
 * Failure injection, for testing how callers handle the library's error
 * paths without faulting the GPU (the paper has no counterpart).
 *
 * ebc_set_wait_limit_ns: the limit of each wait inside the tensor-core
 * kernels (a CTA waiting for its TMA copies, its MMAs or its epilogue; 0
 * restores the default of 1 s, at most 60 s).  A wait that runs out makes
 * the CTA record EBC_ETIMEOUT, stop issuing work, wait (with the default
 * limit) for the copies and MMAs it already issued, free its tensor memory
 * and return; the next ebc_sync() of the handle returns EBC_ETIMEOUT, the
 * results of that call are undefined, and the handle stays usable (a Greedy
 * state that saw a timeout should be reset).  Applies to kernels launched
 * after the call (a captured Greedy round is captured again).  Process-wide.
 *
 * ebc_inject_alloc_failure: the device allocation after `after` more
 * successful ones (all of the library's device memory comes from one pool)
 * fails as if the device were out of memory, once; -1 disarms.  Calls that
 * allocate return EBC_ENOMEM and leave nothing allocated behind; a batch
 * request whose admission fails finishes with EBC_ENOMEM (ebc_batch_poll)
 * while the other requests go on.  Process-wide.  EINVAL for after < -1.
 */
ebc_status ebc_set_wait_limit_ns(int64_t ns);
ebc_status ebc_inject_alloc_failure(int64_t after);

/* Text of the last error on this handle ("" if none); h may be NULL for
 * errors from ebc_create.  The pointer stays valid until the next call. */
const char *ebc_last_error(ebc_t h);

/* Handles allocate device memory from a stream-ordered pool owned by the
 * library (one per device), so creating and destroying handles does not
 * synchronise the device; freed memory stays cached for later handles.
 * This returns the cached, unused memory of the current device's pool. */
ebc_status ebc_release_cached_memory(void);

/* Device bytes a handle for (n, d, prec) allocates (an estimate the batch
 * runtime uses for admission); -1 for bad sizes. */
int64_t ebc_estimate_bytes(int64_t n, int32_t d, int32_t prec);

/* ------------------------------------------------------------------------
 * Groups: Greedy on many handles with one persistent bulk launch per round.
 * Not in the paper, which runs one optimiser at a time; this is the Greedy
 * step of Sec. 4.1 batched over an uneven mix of instances.  Each round, the
 * bulk gains of every handle still running are computed by ONE persistent
 * tensor-core launch whose work units (handle, 256-candidate tile, V chunk)
 * are handed out largest first from a device queue; each handle's tensor
 * maps are read from device memory.  The certified pick and the m_v update
 * of each handle then run on that handle's own stream.
 * ---------------------------------------------------------------------- */
typedef struct ebc_group_ctx *ebc_group_t;

/* A group on the current device (its own stream and tables).  One host
 * thread at a time per group. */
ebc_status ebc_group_create(ebc_group_t *out);

/*
 * k[i] Greedy rounds on handle h[i] for i < count, continuing from each
 * handle's state, exactly as ebc_greedy(h[i], k[i], out_idx[i], out_f[i])
 * would: the same picks (certified exact argmax, same tie rule) and the same
 * f values.  out_idx[i] / out_f[i] are device arrays of k[i] entries.
 * Handles at EBC_BF16 / EBC_FP16 with d <= 128, lazy Greedy off and no CTA
 * cap share the launches; any other handle runs its rounds through
 * ebc_greedy on its own stream.  Handles on their own streams overlap their
 * per-round tails; handles sharing one stream serialise them.
 * Asynchronous: a handle's outputs are ready when its stream reaches them
 * (ebc_sync); a timeout in a shared launch is reported by ebc_sync of every
 * handle in it.  EINVAL for a NULL or repeated handle, a handle on another
 * device, k[i] < 0 or above the handle's unselected points, or a NULL
 * output with k[i] > 0; on any error the handles' Greedy states are
 * undefined (reset them).
 */
ebc_status ebc_group_greedy(ebc_group_t g, const ebc_t *h, int32_t count, const int32_t *k, int32_t *const *out_idx,
                            double *const *out_f);

/* Lanes (1 to 4, default 1): the handles of a call are dealt round-robin to
 * this many lanes, each with its own stream and shared launch per round, so
 * the per-handle picks of one lane overlap the shared launch of another.
 * ebc_group_set_lanes_by_row_width(g, 1) instead uses two lanes by row width
 * (d <= 64 and 64 < d <= 128), each launch laid out for its own rows.
 * Results do not depend on either.  EINVAL outside [1, 4]. */
ebc_status ebc_group_set_lanes(ebc_group_t g, int32_t lanes);
ebc_status ebc_group_set_lanes_by_row_width(ebc_group_t g, int32_t on);

/* Cap the CTAs of the shared launch (0 = one per SM), leaving SMs to the
 * per-handle picks of other lanes.  EINVAL for a negative cap. */
ebc_status ebc_group_set_max_ctas(ebc_group_t g, int32_t max_ctas);

/* Time every shared launch with CUDA events on its lane's stream (on = 1);
 * ebc_group_profile waits for the timed launches and returns their summed
 * device time, the summed time from the end of one timed launch to the start
 * of the next (in issue order: with one lane, the time the shared launches
 * wait for the per-handle picks and preparations) and the (candidate, point)
 * pairs they evaluated; ebc_group_reset_profile zeroes all three.  Any
 * output may be NULL. */
ebc_status ebc_group_set_profiling(ebc_group_t g, int32_t on);
ebc_status ebc_group_profile(ebc_group_t g, double *launch_ms, double *gap_ms, int64_t *pairs);
ebc_status ebc_group_reset_profile(ebc_group_t g);

/* Shared launches issued, work units they processed and rounds, summed over
 * the group's calls (any pointer may be NULL). */
ebc_status ebc_group_stats(ebc_group_t g, int64_t *launches, int64_t *units, int64_t *rounds);
const char *ebc_group_last_error(ebc_group_t g);
/* Waits for the group's stream, then frees it (NULL is accepted). */
ebc_status ebc_group_destroy(ebc_group_t g);

/* ------------------------------------------------------------------------
 * Batch runtime: many independent instances on one GPU.  Not in the paper,
 * which evaluates one optimiser at a time; it serves the many-request case
 * its optimisers generate.  Each admitted instance gets its own handle and
 * stream; ebc_batch_step() advances every active instance by one Greedy
 * round, so their work overlaps on the device; finished instances free
 * their slot and memory and queued requests are admitted in arrival order
 * while a slot is free and the device-memory budget allows (a request
 * larger than the whole budget runs when nothing else does).
 * Single host thread per batch.
 * ---------------------------------------------------------------------- */
typedef struct ebc_batch_ctx *ebc_batch_t;

typedef struct {
    int64_t submitted, completed, active, queued;
    int64_t bytes_in_use, bytes_peak; /* estimated device bytes of admitted instances */
    int64_t rounds_issued;
    int64_t evals_full;      /* completed instances: (candidate, point) pairs of full rounds,
                                sum over rounds t of (n - t) n, whether or not the rounds were lazy */
    int64_t evals_performed; /* completed instances: pairs the bulk kernels evaluated (lazy rounds
                                bound only the candidates whose stale bound can still win) */
} ebc_batch_info;

/* max_slots concurrent instances, device_budget_bytes for their handles, K
 * leaders re-evaluated per round (as ebc_set_precision). */
ebc_status ebc_batch_create(int32_t max_slots, int64_t device_budget_bytes, int32_t refine_k, ebc_batch_t *out);

/* Queue one Greedy summary of k picks over the host array V (n x d FP32,
 * row-major, copied).  *ticket identifies the request.  EINVAL for bad
 * sizes, k > n, or a tensor-core precision with d > 128. */
ebc_status ebc_batch_submit(ebc_batch_t b, const float *V, int64_t n, int32_t d, int32_t k, ebc_prec prec,
                            int64_t *ticket);

/* (Each slot has its own streams; a process serving many instances does
 * well to set CUDA_DEVICE_MAX_CONNECTIONS=32 before its first CUDA call so
 * that the streams do not share a few hardware queues.)
 * Reap finished instances, admit queued ones, issue one round for every
 * active instance that has at most one round still running (each
 * instance's stream is kept at most two rounds deep, so short requests are
 * not queued behind hundreds of rounds of a long one).  Asynchronous;
 * reports active and queued counts. */
ebc_status ebc_batch_step(ebc_batch_t b, int32_t *n_active, int32_t *n_queued);

/* *done = 1 and the k picks / f values copied out (out arrays of capacity
 * cap) once the request finished; returns that request's status.  *done = 0
 * while pending.  A finished result is handed out once. */
ebc_status ebc_batch_poll(ebc_batch_t b, int64_t ticket, int32_t *out_idx, double *out_f, int32_t cap,
                          int32_t *done);

/* Step until every submitted request has finished. */
ebc_status ebc_batch_run(ebc_batch_t b);

/* Instances with n >= large_n ("large") run their bulk kernel on at most
 * max_ctas CTAs (see ebc_set_max_ctas; 0 = no cap) and at most max_active
 * of them run at once (0 = no limit), so smaller instances keep SMs and slots.
 * Admission goes in arrival order, but a request that cannot start yet
 * (memory or this limit) does not hold back later requests that can. */
ebc_status ebc_batch_set_large(ebc_batch_t b, int64_t large_n, int32_t max_ctas, int32_t max_active);

/* Autotune (ebc_autotune with `reps`) the first instance of every new
 * (precision, d, n bucket) at admission; 0 (the default) disables.
 * Admitting such an instance then blocks the caller for the search. */
ebc_status ebc_batch_set_autotune(ebc_batch_t b, int32_t reps);

/* Lazy Greedy (ebc_set_lazy) for the instances admitted from now on whose
 * n >= min_n (on = 1), or for none (on = 0, the default).  Results are
 * unchanged; lazy rounds pay off for large n (their fixed per-round work
 * outweighs the saving on small instances).  EINVAL if min_n < 0. */
ebc_status ebc_batch_set_lazy(ebc_batch_t b, int32_t on, int64_t min_n);

ebc_status ebc_batch_stats(ebc_batch_t b, ebc_batch_info *out);
const char *ebc_batch_last_error(ebc_batch_t b);
ebc_status ebc_batch_destroy(ebc_batch_t b);

#ifdef __cplusplus
}
#endif

#endif /* EBC_H */
