// Internals of a handle (struct ebc_ctx) and the helpers shared by the C-ABI
// entry points: api.cu (life cycle, sets, gains, Greedy) and sieve.cu (the
// threshold sieve over a stream).  Not part of the public interface.
#pragma once

#include <string>
#include <vector>

#include "ebc_internal.cuh"

struct Prof {
    bool on = false;
    ebc_profile p{};
    std::vector<cudaEvent_t> pool;
    // (start, end, kind) of launches not yet folded into p
    struct Rec {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<Rec> pending;
};

enum { PK_BULK = 0, PK_REFINE = 1, PK_EVAL = 2, PK_LIST = 3 };

struct ebc_ctx {
    ebc::Ctx c;
    Prof prof;
    int64_t nsel = 0;       // points picked since create / reset (host mirror)
    int64_t ch = 0;         // bulk-gains V chunk (points)
    int nch = 0;            // number of bulk-gains chunks
    int64_t ref_ch = 0;     // refine V chunk
    int nref = 0;           // number of refine chunks
    int nblk = 0;           // select blocks
    int esc_cap = 0;        // escalated candidates with chunked partials
    double *d_scalar = nullptr;  // one device double for ebc_current_f
    int *d_bad = nullptr;
    // one Greedy round captured as a CUDA graph, replayed for later rounds
    int32_t *g_idx = nullptr;    // [n] picks by round (graph outputs)
    double *g_f = nullptr;       // [n] f by round
    cudaGraphExec_t round_exec = nullptr;
    cudaStream_t round_stream = nullptr;  // stream the graph was captured on
    int64_t round_launches = 0;  // kernels in one round
    int prec_at_capture = -1;
    int ctas_at_capture = -1;
    int lazy_at_capture = -1;
    uint64_t wait_at_capture = 0;  // pipeline wait limit baked into the captured round
    // the tail of a round in a shared group launch (reduction of the bulk
    // partials, certified pick, m_v update, next round's point extension),
    // captured once per (V chunks, precision, K, wait limit)
    cudaGraphExec_t tail_exec = nullptr;
    int64_t tail_key[4] = {-1, -1, -1, -1};
    int64_t tail_launches = 0;
    bool graphs = true;          // replay rounds from a graph when possible
    bool attrs_ready = false;    // one direct round has run (kernel attributes are set)
    // threshold sieve: upper bounds of every point's gain, valid while S only
    // grows (emptied whenever S is reset or replaced)
    std::vector<double> sieve_ub;
};

namespace ebc {
namespace hx {

// Record msg as the handle's last error (or the create error for h = NULL)
// and return s.
ebc_status fail(ebc_t h, ebc_status s, const std::string &msg);
// EBC_ENOMEM for an allocation failure, EBC_ECUDA otherwise, with the CUDA text.
ebc_status cuda_fail(ebc_t h, cudaError_t e, const char *where);
ebc_status check_handle(ebc_t h);
// Relative error bound of the bulk kernel's partial sums (its upper bounds
// are rigorous after a factor 1 + bulk_eta).
double bulk_eta(const Ctx &c);
cudaEvent_t take_event(Prof &p);

template <class T>
cudaError_t dalloc(T **p, size_t count, const ebc::Ctx &c) {
    *p = nullptr;
    if (count == 0) count = 1;
    return ebc::pool_alloc((void **)p, sizeof(T) * count, c.stream, c.device);
}

// Run one launcher; count it and, with profiling on, bracket it with events.
template <class F>
cudaError_t launch(ebc_t h, int kind, int64_t nlaunch, F &&fn) {
    Prof &p = h->prof;
    cudaEvent_t a = nullptr, b = nullptr;
    if (p.on && kind >= 0) {
        a = take_event(p);
        b = take_event(p);
        if (a && b) cudaEventRecord(a, h->c.stream);
    }
    cudaError_t e = fn();
    p.p.launches += nlaunch;
    if (kind == PK_BULK) p.p.bulk_launches += nlaunch;
    if (kind == PK_REFINE) p.p.refine_launches += nlaunch;
    if (kind == PK_EVAL) p.p.eval_launches += nlaunch;
    if (kind == PK_LIST) p.p.list_launches += nlaunch;
    if (a && b) {
        cudaEventRecord(b, h->c.stream);
        p.pending.push_back({a, b, kind});
    } else {
        if (a) p.pool.push_back(a);
        if (b) p.pool.push_back(b);
    }
    return e;
}

}  // namespace hx

// The certified pick of a Greedy round whose bulk bounds are reduced into the
// per-block top lists (or the lazy list's), then the m_v update (api.cu).
ebc_status round_certify(ebc_t h, int32_t *out_idx_base, double *out_f_base, bool lazy);

}  // namespace ebc

#define CK(h, expr)                                   \
    do {                                              \
        cudaError_t _e = (expr);                      \
        if (_e != cudaSuccess) return cuda_fail(h, _e, #expr); \
    } while (0)
