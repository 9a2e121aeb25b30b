// Batch runtime: many independent summarisation instances sharing one GPU.
//
// Each admitted instance occupies a slot: its own handle (resident V,
// norms, quantised copies, Greedy state) and its own non-blocking stream;
// instances marked large (ebc_batch_set_large) use the lowest stream
// priority, all others the highest, so ordinary requests' kernels get SMs
// first whenever SMs free up.
// ebc_batch_step() advances every active instance by one Greedy round
// (a graph replay after the first round), so rounds of different instances
// overlap on the device; finished instances are detected with events,
// their results copied to pinned host memory and their slot and memory
// released; queued requests are admitted first-come first-served while a
// slot is free and the device-memory budget allows.  This is continuous
// batching at round granularity: a request arriving while others run is
// admitted as soon as a slot and memory free up, without waiting for the
// batch to drain.
#include <string.h>

#include <deque>
#include <string>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

struct ebc_batch_ctx {
    struct Req {
        int64_t ticket;
        std::vector<float> V;
        int64_t n;
        int32_t d, k;
        ebc_prec prec;
        int64_t bytes;
    };
    struct Slot {
        bool busy = false, finishing = false, large = false;
        ebc_t h = nullptr;
        cudaStream_t stream = nullptr;     // current instance's stream (one of the two below)
        cudaStream_t stream_hi = nullptr;  // highest priority: ordinary instances
        cudaStream_t stream_lo = nullptr;  // lowest priority: large instances
        cudaEvent_t done = nullptr;
        cudaEvent_t round_ev[2] = {nullptr, nullptr};  // ends of the last two issued rounds
        int64_t ticket = -1;
        int32_t k = 0, issued = 0, cap = 0;
        int32_t *d_idx = nullptr;
        double *d_f = nullptr;
        int32_t *h_idx = nullptr;  // pinned
        double *h_f = nullptr;     // pinned
        int64_t bytes = 0;
    };
    struct Result {
        ebc_status status;
        std::vector<int32_t> idx;
        std::vector<double> f;
    };
    int32_t refine_k = 8;
    int64_t large_n = 0;      // instances with n >= large_n get at most large_ctas CTAs per kernel
    int32_t large_ctas = 0;
    int32_t lazy = 0;         // lazy Greedy for admitted instances with n >= lazy_min_n (ebc_batch_set_lazy)
    int64_t lazy_min_n = 0;
    int32_t tune_reps = 0;    // autotune each new (precision, d, n bucket) on admission (ebc_batch_set_autotune)
    int32_t max_large = 0;    // at most this many large instances at once (0 = no limit)
    int64_t budget = 0, used = 0, peak = 0;
    int64_t next_ticket = 1, submitted = 0, completed = 0, rounds = 0;
    int64_t evals_full = 0, evals_performed = 0;
    std::deque<Req> queue;
    std::vector<Slot> slots;
    std::unordered_map<int64_t, Result> results;
    std::string err;
};

namespace {

ebc_status bfail(ebc_batch_t b, ebc_status s, const std::string &m) {
    if (b) b->err = m;
    return s;
}

void release_slot(ebc_batch_ctx::Slot &s) {
    if (s.h) ebc_destroy(s.h);
    s.h = nullptr;
    s.busy = s.finishing = false;
    s.ticket = -1;
    s.issued = s.k = 0;
    s.bytes = 0;
}

// Per-slot output buffers, grown (rarely) to the largest k seen.  Device
// buffers come from the library's stream-ordered pool on the slot's
// high-priority stream; both streams of the slot wait for that stream before
// the buffers are used.
ebc_status ensure_outputs(ebc_batch_t b, ebc_batch_ctx::Slot &s, int32_t k) {
    if (s.cap >= k) return EBC_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    const int32_t cap = k > 256 ? k : 256;
    if (s.d_idx || s.d_f) {
        cudaStreamSynchronize(s.stream_hi);
        cudaStreamSynchronize(s.stream_lo);
    }
    ebc::pool_free(s.d_idx, s.stream_hi);
    ebc::pool_free(s.d_f, s.stream_hi);
    if (s.h_idx) cudaFreeHost(s.h_idx);
    if (s.h_f) cudaFreeHost(s.h_f);
    s.d_idx = nullptr;
    s.d_f = nullptr;
    s.h_idx = nullptr;
    s.h_f = nullptr;
    s.cap = 0;
    if (ebc::pool_alloc((void **)&s.d_idx, sizeof(int32_t) * cap, s.stream_hi, dev) != cudaSuccess ||
        ebc::pool_alloc((void **)&s.d_f, sizeof(double) * cap, s.stream_hi, dev) != cudaSuccess ||
        cudaMallocHost(&s.h_idx, sizeof(int32_t) * cap) != cudaSuccess ||
        cudaMallocHost(&s.h_f, sizeof(double) * cap) != cudaSuccess || cudaStreamSynchronize(s.stream_hi) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, EBC_ENOMEM, "ebc_batch: output buffers");
    }
    s.cap = cap;
    return EBC_OK;
}

// Move finished instances to the result table and free their slots.
void reap(ebc_batch_t b) {
    for (auto &s : b->slots) {
        if (!s.busy || !s.finishing) continue;
        cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) continue;
        ebc_batch_ctx::Result r;
        r.status = q == cudaSuccess ? ebc_sync(s.h) : EBC_ECUDA;
        cudaGetLastError();
        if (r.status == EBC_OK) {
            ebc_stats hs;
            if (ebc_get_stats(s.h, &hs) == EBC_OK) {
                const int64_t n = s.h->c.n, k = s.k;
                const int64_t full = (n * k - k * (k - 1) / 2) * n;  // sum over t < k of (n - t) n
                b->evals_full += full;
                b->evals_performed += hs.lazy ? hs.bulk_candidates * n : full;
            }
        }
        r.idx.assign(s.h_idx, s.h_idx + s.k);
        r.f.assign(s.h_f, s.h_f + s.k);
        b->results[s.ticket] = std::move(r);
        b->used -= s.bytes;
        b->completed += 1;
        release_slot(s);
    }
}

// Admit queued requests in arrival order.  A request that cannot start yet
// (memory, or the cap on concurrent large instances) keeps its place, and
// later requests that fit may start before it; slots are the only hard stop.
void admit(ebc_batch_t b) {
    int32_t active_large = 0;
    for (auto &s : b->slots)
        if (s.busy && s.large) active_large += 1;
    for (auto it = b->queue.begin(); it != b->queue.end();) {
        ebc_batch_ctx::Req &r = *it;
        ebc_batch_ctx::Slot *free_slot = nullptr;
        for (auto &s : b->slots)
            if (!s.busy) {
                free_slot = &s;
                break;
            }
        if (!free_slot) return;
        const bool large = b->large_n > 0 && r.n >= b->large_n;
        const bool mem_ok = b->used + r.bytes <= b->budget || b->used == 0;  // an oversize request runs alone
        const bool cls_ok = !large || b->max_large <= 0 || active_large < b->max_large;
        if (!mem_ok || !cls_ok) {
            ++it;
            continue;
        }
        ebc_batch_ctx::Slot &s = *free_slot;
        ebc_status st = ensure_outputs(b, s, r.k);
        ebc_t h = nullptr;
        s.stream = large ? s.stream_lo : s.stream_hi;
        if (st == EBC_OK) st = ebc::create_handle(r.V.data(), r.n, r.d, 0, s.stream, false, &h);
        if (st == EBC_OK && (r.prec != EBC_FP32 || b->refine_k != 8))
            st = ebc::set_precision_handle(h, r.prec, b->refine_k, false);
        if (st == EBC_OK && large && b->large_ctas > 0) st = ebc_set_max_ctas(h, b->large_ctas);
        if (st == EBC_OK && b->lazy && r.n >= b->lazy_min_n) st = ebc_set_lazy(h, 1);
        if (st == EBC_OK && b->tune_reps > 0 && r.prec != EBC_FP32) st = ebc::autotune_handle(h, b->tune_reps, true);
        if (st != EBC_OK) {
            ebc_batch_ctx::Result res;
            res.status = st;
            b->results[r.ticket] = std::move(res);
            b->completed += 1;
            if (h) ebc_destroy(h);
            it = b->queue.erase(it);
            continue;
        }
        s.busy = true;
        s.finishing = false;
        s.large = large;
        s.h = h;
        s.ticket = r.ticket;
        s.k = r.k;
        s.issued = 0;
        s.bytes = r.bytes;
        b->used += r.bytes;
        if (b->used > b->peak) b->peak = b->used;
        active_large += large ? 1 : 0;
        it = b->queue.erase(it);
    }
}

// One Greedy round for every active instance that has at most one round in
// flight; the last round also queues the copy of the results and the
// completion event.  Keeping each stream at most two rounds deep bounds how
// long any instance's kernels can wait behind another's in the device's
// shared hardware queues (many streams map onto few): a request that needs
// hundreds of rounds cannot place all of them ahead of later, shorter ones.
ebc_status issue(ebc_batch_t b) {
    for (auto &s : b->slots) {
        if (!s.busy || s.finishing) continue;
        if (s.issued >= 2 && cudaEventQuery(s.round_ev[s.issued & 1]) == cudaErrorNotReady) continue;
        cudaGetLastError();
        ebc_status st = ebc_greedy(s.h, 1, s.d_idx + s.issued, s.d_f + s.issued);
        if (st != EBC_OK) {
            // record the failure as this instance's result
            ebc_batch_ctx::Result res;
            res.status = st;
            b->results[s.ticket] = std::move(res);
            b->used -= s.bytes;
            b->completed += 1;
            release_slot(s);
            continue;
        }
        cudaEventRecord(s.round_ev[s.issued & 1], s.stream);
        s.issued += 1;
        b->rounds += 1;
        if (s.issued == s.k) {
            cudaMemcpyAsync(s.h_idx, s.d_idx, sizeof(int32_t) * s.k, cudaMemcpyDeviceToHost, s.stream);
            cudaMemcpyAsync(s.h_f, s.d_f, sizeof(double) * s.k, cudaMemcpyDeviceToHost, s.stream);
            cudaEventRecord(s.done, s.stream);
            s.finishing = true;
        }
    }
    return EBC_OK;
}

}  // namespace

extern "C" {

ebc_status ebc_batch_create(int32_t max_slots, int64_t device_budget_bytes, int32_t refine_k, ebc_batch_t *out) {
    if (!out) return EBC_EINVAL;
    *out = nullptr;
    if (max_slots < 1 || max_slots > 4096 || device_budget_bytes <= 0 || refine_k < 1 || refine_k > ebc::kMaxRefineK)
        return EBC_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return EBC_ENODEV;
    }
    ebc_batch_ctx *b = new (std::nothrow) ebc_batch_ctx();
    if (!b) return EBC_ENOMEM;
    b->budget = device_budget_bytes;
    b->refine_k = refine_k;
    b->slots.resize(max_slots);
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (auto &s : b->slots) {
        if (cudaStreamCreateWithPriority(&s.stream_hi, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s.stream_lo, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.round_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.round_ev[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ebc_batch_destroy(b);
            return EBC_ECUDA;
        }
        if (ensure_outputs(b, s, 256) != EBC_OK) {
            ebc_batch_destroy(b);
            return EBC_ENOMEM;
        }
    }
    *out = b;
    return EBC_OK;
}

ebc_status ebc_batch_submit(ebc_batch_t b, const float *V, int64_t n, int32_t d, int32_t k, ebc_prec prec,
                            int64_t *ticket) {
    if (!b) return EBC_EINVAL;
    if (!V || !ticket || n <= 0 || n > (int64_t)INT32_MAX - 1 || d <= 0 || d > 4096 || k < 1 || (int64_t)k > n)
        return bfail(b, EBC_EINVAL, "ebc_batch_submit: bad V, n, d, k or ticket");
    if (prec != EBC_FP32 && !(prec == EBC_BF16 || prec == EBC_FP16 || (prec == EBC_FP8E4M3 && d <= 128)))
        return bfail(b, EBC_EINVAL, "ebc_batch_submit: unsupported precision for this d");
    ebc_batch_ctx::Req r;
    r.ticket = b->next_ticket++;
    r.V.assign(V, V + (size_t)n * d);
    r.n = n;
    r.d = d;
    r.k = k;
    r.prec = prec;
    r.bytes = ebc::handle_bytes(n, d, prec);
    *ticket = r.ticket;
    b->queue.push_back(std::move(r));
    b->submitted += 1;
    return EBC_OK;
}

ebc_status ebc_batch_step(ebc_batch_t b, int32_t *n_active, int32_t *n_queued) {
    ebc::TraceRange trace_("ebc_batch_step");
    if (!b) return EBC_EINVAL;
    reap(b);
    admit(b);
    ebc_status st = issue(b);
    int32_t act = 0;
    for (auto &s : b->slots) act += s.busy ? 1 : 0;
    if (n_active) *n_active = act;
    if (n_queued) *n_queued = (int32_t)b->queue.size();
    return st;
}

ebc_status ebc_batch_poll(ebc_batch_t b, int64_t ticket, int32_t *out_idx, double *out_f, int32_t cap,
                          int32_t *done) {
    if (!b || !done) return EBC_EINVAL;
    *done = 0;
    auto it = b->results.find(ticket);
    if (it == b->results.end()) {
        if (ticket <= 0 || ticket >= b->next_ticket) return bfail(b, EBC_EINVAL, "ebc_batch_poll: unknown ticket");
        return EBC_OK;  // pending
    }
    ebc_batch_ctx::Result &r = it->second;
    if (r.status == EBC_OK) {
        if ((int64_t)cap < (int64_t)r.idx.size() || !out_idx || !out_f)
            return bfail(b, EBC_EINVAL, "ebc_batch_poll: output capacity below k");
        memcpy(out_idx, r.idx.data(), sizeof(int32_t) * r.idx.size());
        memcpy(out_f, r.f.data(), sizeof(double) * r.f.size());
    }
    const ebc_status st = r.status;
    b->results.erase(it);
    *done = 1;
    return st;
}

ebc_status ebc_batch_run(ebc_batch_t b) {
    if (!b) return EBC_EINVAL;
    while (true) {
        int32_t act = 0, q = 0;
        ebc_status st = ebc_batch_step(b, &act, &q);
        if (st != EBC_OK) return st;
        if (act == 0 && q == 0) return EBC_OK;
        // when every active instance has all its rounds queued, wait for one to end
        bool all_finishing = true;
        for (auto &s : b->slots)
            if (s.busy && !s.finishing) all_finishing = false;
        if (all_finishing)
            for (auto &s : b->slots)
                if (s.busy) {
                    cudaEventSynchronize(s.done);
                    break;
                }
    }
}

ebc_status ebc_batch_stats(ebc_batch_t b, ebc_batch_info *out) {
    if (!b || !out) return EBC_EINVAL;
    int64_t act = 0;
    for (auto &s : b->slots) act += s.busy ? 1 : 0;
    out->submitted = b->submitted;
    out->completed = b->completed;
    out->active = act;
    out->queued = (int64_t)b->queue.size();
    out->bytes_in_use = b->used;
    out->bytes_peak = b->peak;
    out->rounds_issued = b->rounds;
    out->evals_full = b->evals_full;
    out->evals_performed = b->evals_performed;
    return EBC_OK;
}

ebc_status ebc_batch_set_autotune(ebc_batch_t b, int32_t reps) {
    if (!b || reps < 0 || reps > 100) return EBC_EINVAL;
    b->tune_reps = reps;
    return EBC_OK;
}

ebc_status ebc_batch_set_lazy(ebc_batch_t b, int32_t on, int64_t min_n) {
    if (!b || min_n < 0) return EBC_EINVAL;
    b->lazy = on != 0;
    b->lazy_min_n = min_n;
    return EBC_OK;
}

ebc_status ebc_batch_set_large(ebc_batch_t b, int64_t large_n, int32_t max_ctas, int32_t max_active) {
    if (!b || large_n < 0 || max_ctas < 0 || max_active < 0) return EBC_EINVAL;
    b->large_n = large_n;
    b->large_ctas = max_ctas;
    b->max_large = max_active;
    return EBC_OK;
}

const char *ebc_batch_last_error(ebc_batch_t b) { return b ? b->err.c_str() : ""; }

ebc_status ebc_batch_destroy(ebc_batch_t b) {
    if (!b) return EBC_OK;
    for (auto &s : b->slots) {
        if (s.stream_hi) cudaStreamSynchronize(s.stream_hi);
        if (s.stream_lo) cudaStreamSynchronize(s.stream_lo);
        release_slot(s);
        ebc::pool_free(s.d_idx, s.stream_hi);
        ebc::pool_free(s.d_f, s.stream_hi);
        if (s.stream_hi) cudaStreamSynchronize(s.stream_hi);
        if (s.h_idx) cudaFreeHost(s.h_idx);
        if (s.h_f) cudaFreeHost(s.h_f);
        if (s.done) cudaEventDestroy(s.done);
        for (cudaEvent_t ev : s.round_ev)
            if (ev) cudaEventDestroy(ev);
        if (s.stream_hi) cudaStreamDestroy(s.stream_hi);
        if (s.stream_lo) cudaStreamDestroy(s.stream_lo);
    }
    delete b;
    return EBC_OK;
}

}  // extern "C"
