// Greedy rounds of several handles with one persistent bulk launch per round
// (ebc_group_*): the instance-batched form of the Greedy step of Sec. 4.1
// for an uneven mix of ground sets.
//
// Every round, each handle still running prepares its point extension on its
// own stream; the group's stream waits for all of them and runs ONE
// persistent tensor-core launch over the work units (handle, candidate tile,
// V chunk) of every handle (k_gains_tc_group: units handed out largest first
// from a device counter, per-handle tensor maps in device memory); each
// handle's stream then waits for that launch and runs the certified pick and
// the m_v update of its own round.  The host enqueues all rounds without
// waiting.  Handles are ordered by their number of rounds, so the handles
// still running in round r are a prefix and their units a prefix of one
// table uploaded once per call.
//
// The V chunking of the shared launch differs from a handle's own launch,
// which changes the bulk bounds only in the last bits; picks and f come from
// the exact re-evaluation, which does not depend on it, so they equal those
// of ebc_greedy on each handle alone.
#include <algorithm>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace ebc::hx;

struct ebc_group_ctx {
    int device = 0;
    int num_sms = 152;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_bulk = nullptr;    // end of the current round's shared launch
    cudaEvent_t ev_staged = nullptr;  // the staging buffers' last upload finished
    bool staged_pending = false;
    std::vector<cudaEvent_t> ev_inst;  // per handle: its point extension is ready
    ebc::GroupInst *h_inst = nullptr;  // pinned staging
    ebc::GroupUnit *h_units = nullptr;
    int64_t h_inst_cap = 0, h_unit_cap = 0;
    ebc::GroupInst *d_inst = nullptr;
    ebc::GroupUnit *d_units = nullptr;
    int64_t d_inst_cap = 0, d_unit_cap = 0;
    int *d_words = nullptr;  // [0] next unit, [1] error of the launch
    int64_t launches = 0, units = 0, rounds = 0;
    std::string err;
};

namespace {

constexpr int kTilesPerUnit = 48;  // target point tiles per work unit

ebc_status gfail(ebc_group_t g, ebc_status s, const std::string &m) {
    if (g) g->err = m;
    return s;
}

ebc_status gcuda(ebc_group_t g, cudaError_t e, const char *where) {
    cudaGetLastError();
    return gfail(g, e == cudaErrorMemoryAllocation ? EBC_ENOMEM : EBC_ECUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define GK(g, expr)                                   \
    do {                                              \
        cudaError_t _e = (expr);                      \
        if (_e != cudaSuccess) return gcuda(g, _e, #expr); \
    } while (0)

bool group_eligible(ebc_t h) {
    const ebc::Ctx &c = h->c;
    return (c.prec == EBC_BF16 || c.prec == EBC_FP16) && c.tc.prec == (int)c.prec && !c.lazy && c.max_ctas == 0 &&
           ebc::tc_group_supported(c);
}

// staging and device tables large enough for ni handles and nu units
ebc_status ensure_tables(ebc_group_t g, int64_t ni, int64_t nu) {
    if (g->staged_pending) {  // the previous call's upload still reads the staging buffers
        GK(g, cudaEventSynchronize(g->ev_staged));
        g->staged_pending = false;
    }
    if (g->h_inst_cap < ni) {
        if (g->h_inst) cudaFreeHost(g->h_inst);
        g->h_inst = nullptr;
        g->h_inst_cap = 0;
        const int64_t cap = std::max<int64_t>(ni, 64);
        GK(g, cudaMallocHost((void **)&g->h_inst, sizeof(ebc::GroupInst) * cap));
        g->h_inst_cap = cap;
    }
    if (g->h_unit_cap < nu) {
        if (g->h_units) cudaFreeHost(g->h_units);
        g->h_units = nullptr;
        g->h_unit_cap = 0;
        const int64_t cap = std::max<int64_t>(nu, 4096);
        GK(g, cudaMallocHost((void **)&g->h_units, sizeof(ebc::GroupUnit) * cap));
        g->h_unit_cap = cap;
    }
    if (g->d_inst_cap < ni) {
        ebc::pool_free(g->d_inst, g->stream);
        g->d_inst = nullptr;
        g->d_inst_cap = 0;
        const int64_t cap = std::max<int64_t>(ni, 64);
        GK(g, ebc::pool_alloc((void **)&g->d_inst, sizeof(ebc::GroupInst) * cap, g->stream, g->device));
        g->d_inst_cap = cap;
    }
    if (g->d_unit_cap < nu) {
        ebc::pool_free(g->d_units, g->stream);
        g->d_units = nullptr;
        g->d_unit_cap = 0;
        const int64_t cap = std::max<int64_t>(nu, 4096);
        GK(g, ebc::pool_alloc((void **)&g->d_units, sizeof(ebc::GroupUnit) * cap, g->stream, g->device));
        g->d_unit_cap = cap;
    }
    if (!g->d_words) GK(g, ebc::pool_alloc((void **)&g->d_words, 2 * sizeof(int), g->stream, g->device));
    while ((int64_t)g->ev_inst.size() < ni) {
        cudaEvent_t ev = nullptr;
        GK(g, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        g->ev_inst.push_back(ev);
    }
    return EBC_OK;
}

}  // namespace

extern "C" {

ebc_status ebc_group_create(ebc_group_t *out) {
    if (!out) return EBC_EINVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return EBC_ENODEV;
    }
    ebc_group_ctx *g = new (std::nothrow) ebc_group_ctx();
    if (!g) return EBC_ENOMEM;
    g->device = dev;
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_bulk, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_staged, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ebc_group_destroy(g);
        return EBC_ECUDA;
    }
    *out = g;
    return EBC_OK;
}

ebc_status ebc_group_greedy(ebc_group_t g, const ebc_t *hs, int32_t count, const int32_t *k, int32_t *const *out_idx,
                            double *const *out_f) {
    ebc::TraceRange trace_("ebc_group_greedy");
    if (!g) return EBC_EINVAL;
    if (count < 0 || (count > 0 && (!hs || !k || !out_idx || !out_f)))
        return gfail(g, EBC_EINVAL, "ebc_group_greedy: bad arguments");
    std::vector<int> shared, own;
    {
        std::vector<ebc_t> seen(hs, hs + count);
        std::sort(seen.begin(), seen.end());
        if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
            return gfail(g, EBC_EINVAL, "ebc_group_greedy: a handle appears twice");
    }
    for (int i = 0; i < count; ++i) {
        ebc_t h = hs[i];
        if (check_handle(h)) return gfail(g, EBC_EINVAL, "ebc_group_greedy: NULL handle");
        if (h->c.device != g->device) return gfail(g, EBC_EINVAL, "ebc_group_greedy: a handle on another device");
        if (k[i] < 0 || (int64_t)k[i] > h->c.n - h->nsel)
            return gfail(g, EBC_EINVAL, "ebc_group_greedy: k exceeds a handle's unselected points");
        if (k[i] == 0) continue;
        if (!out_idx[i] || !out_f[i]) return gfail(g, EBC_EINVAL, "ebc_group_greedy: NULL output");
        (group_eligible(h) ? shared : own).push_back(i);
    }
    // handles the shared launch does not serve run their rounds on their own
    for (int i : own) {
        ebc_status s = ebc_greedy(hs[i], k[i], out_idx[i], out_f[i]);
        if (s != EBC_OK) return gfail(g, s, std::string("ebc_group_greedy: ") + ebc_last_error(hs[i]));
    }
    if (shared.empty()) return EBC_OK;
    // most rounds first: the handles running in round r are a prefix
    std::stable_sort(shared.begin(), shared.end(), [&](int a, int b) { return k[a] > k[b]; });
    const int ni = (int)shared.size();
    std::vector<int> nch(ni), vpc(ni), RB(ni);
    std::vector<int64_t> first_unit(ni + 1, 0);
    for (int e = 0; e < ni; ++e) {
        const ebc::Ctx &c = hs[shared[e]]->c;
        const int n_vtiles = (int)(c.tc.n_pad / 256);
        const int n_ctiles = (int)((c.n + 255) / 256);
        const int max_ch = (int)std::max<int64_t>(1, std::min<int64_t>(c.partial_cap / c.n, n_vtiles));
        int want = std::min(max_ch, std::max(1, (n_vtiles + kTilesPerUnit - 1) / kTilesPerUnit));
        vpc[e] = (n_vtiles + want - 1) / want;
        nch[e] = (n_vtiles + vpc[e] - 1) / vpc[e];
        RB[e] = ebc::tc_group_row_bytes(c);
        first_unit[e + 1] = first_unit[e] + (int64_t)n_ctiles * nch[e];
    }
    const int64_t nu = first_unit[ni];
    if (nu > INT32_MAX / 2) return gfail(g, EBC_EINVAL, "ebc_group_greedy: too many work units");
    ebc_status s = ensure_tables(g, ni, nu);
    if (s != EBC_OK) return s;
    // unit table: handles in order of rounds, within equal rounds largest units first
    {
        int64_t w = 0;
        for (int e0 = 0; e0 < ni;) {
            int e1 = e0;
            while (e1 < ni && k[shared[e1]] == k[shared[e0]]) ++e1;
            const int64_t b = w;
            for (int e = e0; e < e1; ++e) {
                const ebc::Ctx &c = hs[shared[e]]->c;
                const int n_vtiles = (int)(c.tc.n_pad / 256);
                const int n_ctiles = (int)((c.n + 255) / 256);
                for (int ct = 0; ct < n_ctiles; ++ct)
                    for (int ch = 0; ch < nch[e]; ++ch) {
                        const int vt0 = ch * vpc[e];
                        g->h_units[w++] = {e, ct, ch, std::min(vt0 + vpc[e], n_vtiles) - vt0};
                    }
            }
            std::stable_sort(g->h_units + b, g->h_units + w,
                             [](const ebc::GroupUnit &x, const ebc::GroupUnit &y) { return x.ntiles > y.ntiles; });
            e0 = e1;
        }
    }
    for (int e = 0; e < ni; ++e) ebc::group_inst_fill(hs[shared[e]]->c, nch[e], vpc[e], &g->h_inst[e]);
    GK(g, cudaMemcpyAsync(g->d_inst, g->h_inst, sizeof(ebc::GroupInst) * ni, cudaMemcpyHostToDevice, g->stream));
    GK(g, cudaMemcpyAsync(g->d_units, g->h_units, sizeof(ebc::GroupUnit) * nu, cudaMemcpyHostToDevice, g->stream));
    GK(g, cudaEventRecord(g->ev_staged, g->stream));
    g->staged_pending = true;

    // output bases: the commit kernel writes out[round since reset]
    std::vector<int32_t *> ib(ni);
    std::vector<double *> fb(ni);
    for (int e = 0; e < ni; ++e) {
        ebc_t h = hs[shared[e]];
        ib[e] = out_idx[shared[e]] - h->nsel;
        fb[e] = out_f[shared[e]] - h->nsel;
    }
    const int kmax = k[shared[0]];
    int active = ni;
    for (int r = 0; r < kmax; ++r) {
        while (active > 0 && k[shared[active - 1]] <= r) --active;
        int RBmax = 0;
        for (int e = 0; e < active; ++e) RBmax = std::max(RBmax, RB[e]);
        for (int e = 0; e < active; ++e) {
            ebc_t h = hs[shared[e]];
            CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc(h->c, true); }));
            GK(g, cudaEventRecord(g->ev_inst[e], h->c.stream));
            GK(g, cudaStreamWaitEvent(g->stream, g->ev_inst[e], 0));
        }
        GK(g, cudaMemsetAsync(g->d_words, 0, 2 * sizeof(int), g->stream));
        GK(g, ebc::launch_gains_tc_group(g->d_inst, g->d_units, (int)first_unit[active], g->d_words, g->d_words + 1,
                                         RBmax, g->num_sms, g->stream));
        GK(g, ebc::launch_group_err(g->d_inst, active, g->d_words + 1, g->stream));
        GK(g, cudaEventRecord(g->ev_bulk, g->stream));
        g->launches += 1;
        g->units += first_unit[active];
        g->rounds += 1;
        for (int e = 0; e < active; ++e) {
            ebc_t h = hs[shared[e]];
            ebc::Ctx &c = h->c;
            GK(g, cudaStreamWaitEvent(c.stream, g->ev_bulk, 0));
            h->prof.p.bulk_launches += 1;
            h->prof.p.bulk_evals += (c.n - h->nsel) * c.n;
            const int nchunks = nch[e];
            CK(h, launch(h, -1, 1, [&] {
                   return ebc::launch_reduce_select(c, c.n, nchunks, nullptr, true, nullptr, h->nblk);
               }));
            s = ebc::round_certify(h, ib[e], fb[e], false);
            if (s != EBC_OK) return gfail(g, s, std::string("ebc_group_greedy: ") + ebc_last_error(h));
            h->nsel += 1;
            h->attrs_ready = true;
        }
    }
    return EBC_OK;
}

ebc_status ebc_group_stats(ebc_group_t g, int64_t *launches, int64_t *units, int64_t *rounds) {
    if (!g) return EBC_EINVAL;
    if (launches) *launches = g->launches;
    if (units) *units = g->units;
    if (rounds) *rounds = g->rounds;
    return EBC_OK;
}

const char *ebc_group_last_error(ebc_group_t g) { return g ? g->err.c_str() : ""; }

ebc_status ebc_group_destroy(ebc_group_t g) {
    if (!g) return EBC_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    ebc::pool_free(g->d_inst, g->stream);
    ebc::pool_free(g->d_units, g->stream);
    ebc::pool_free(g->d_words, g->stream);
    if (g->stream) {
        cudaStreamSynchronize(g->stream);
        cudaStreamDestroy(g->stream);
    }
    if (g->h_inst) cudaFreeHost(g->h_inst);
    if (g->h_units) cudaFreeHost(g->h_units);
    for (cudaEvent_t ev : g->ev_inst) cudaEventDestroy(ev);
    if (g->ev_bulk) cudaEventDestroy(g->ev_bulk);
    if (g->ev_staged) cudaEventDestroy(g->ev_staged);
    delete g;
    return EBC_OK;
}

}  // extern "C"
