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

// One lane: a stream with its own tables; the handles of a call are dealt
// round-robin to the lanes, whose rounds interleave on the device (the
// per-handle tails of one lane overlap the shared launch of another).
struct GroupLane {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_bulk = nullptr;    // end of the current round's shared launch
    cudaEvent_t ev_staged = nullptr;  // the staging buffers' last upload finished
    bool staged_pending = false;
    ebc::GroupInst *h_inst = nullptr;  // pinned staging
    ebc::GroupUnit *h_units = nullptr;
    int64_t h_inst_cap = 0, h_unit_cap = 0;
    ebc::GroupInst *d_inst = nullptr;
    ebc::GroupUnit *d_units = nullptr;
    int64_t d_inst_cap = 0, d_unit_cap = 0;
    int *d_words = nullptr;  // [0] next unit, [1] error of the launch
};

struct ebc_group_ctx {
    int device = 0;
    int num_sms = 152;
    int nlanes = 1;
    int max_ctas = 0;           // CTAs of the shared launch (0: one per SM)
    bool by_row_width = false;  // lanes by row width (d <= 64 / d <= 128) instead of round-robin
    GroupLane lanes[4];
    std::vector<cudaEvent_t> ev_inst;  // per handle: its point extension is ready
    int64_t launches = 0, units = 0, rounds = 0;
    // shared-launch timing (ebc_group_set_profiling): event pairs not yet folded
    bool prof = false;
    double launch_ms = 0.0;
    double gap_ms = 0.0;  // from the end of one shared launch to the start of the next (lane 0)
    cudaEvent_t last_end = nullptr;
    int64_t launch_evals = 0;  // (candidate, point) pairs of the timed launches
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending, spare;
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

// staging and device tables of a lane large enough for ni handles and nu units
ebc_status ensure_tables(ebc_group_t g, GroupLane *l, int64_t ni, int64_t nu) {
    if (l->staged_pending) {  // the previous call's upload still reads the staging buffers
        GK(g, cudaEventSynchronize(l->ev_staged));
        l->staged_pending = false;
    }
    if (l->h_inst_cap < ni) {
        if (l->h_inst) cudaFreeHost(l->h_inst);
        l->h_inst = nullptr;
        l->h_inst_cap = 0;
        const int64_t cap = std::max<int64_t>(ni, 64);
        GK(g, cudaMallocHost((void **)&l->h_inst, sizeof(ebc::GroupInst) * cap));
        l->h_inst_cap = cap;
    }
    if (l->h_unit_cap < nu) {
        if (l->h_units) cudaFreeHost(l->h_units);
        l->h_units = nullptr;
        l->h_unit_cap = 0;
        const int64_t cap = std::max<int64_t>(nu, 4096);
        GK(g, cudaMallocHost((void **)&l->h_units, sizeof(ebc::GroupUnit) * cap));
        l->h_unit_cap = cap;
    }
    if (l->d_inst_cap < ni) {
        ebc::pool_free(l->d_inst, l->stream);
        l->d_inst = nullptr;
        l->d_inst_cap = 0;
        const int64_t cap = std::max<int64_t>(ni, 64);
        GK(g, ebc::pool_alloc((void **)&l->d_inst, sizeof(ebc::GroupInst) * cap, l->stream, g->device));
        l->d_inst_cap = cap;
    }
    if (l->d_unit_cap < nu) {
        ebc::pool_free(l->d_units, l->stream);
        l->d_units = nullptr;
        l->d_unit_cap = 0;
        const int64_t cap = std::max<int64_t>(nu, 4096);
        GK(g, ebc::pool_alloc((void **)&l->d_units, sizeof(ebc::GroupUnit) * cap, l->stream, g->device));
        l->d_unit_cap = cap;
    }
    if (!l->d_words) GK(g, ebc::pool_alloc((void **)&l->d_words, 2 * sizeof(int), l->stream, g->device));
    return EBC_OK;
}

// The tail of a handle's round after the shared launch: reduce the bulk
// partials (nch V chunks), certify the pick into the handle's by-round
// buffers, update m_v, and prepare the next round's point extension.
ebc_status round_tail(ebc_t h, int nch) {
    ebc::Ctx &c = h->c;
    CK(h, launch(h, -1, 1, [&] { return ebc::launch_reduce_select(c, c.n, nch, nullptr, true, nullptr, h->nblk); }));
    ebc_status s = ebc::round_certify(h, h->g_idx, h->g_f, false);
    if (s != EBC_OK) return s;
    CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc(c, true); }));
    return EBC_OK;
}

// Capture round_tail as a graph for later rounds (a capture failure keeps
// direct launches).
void capture_tail(ebc_t h, int nch) {
    ebc::Ctx &c = h->c;
    if (h->tail_exec) {
        cudaGraphExecDestroy(h->tail_exec);
        h->tail_exec = nullptr;
    }
    const ebc_profile saved = h->prof.p;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const ebc_status s = round_tail(h, nch);
    const cudaError_t e = cudaStreamEndCapture(c.stream, &graph);
    h->tail_launches = h->prof.p.launches - saved.launches;
    h->prof.p = saved;
    if (s != EBC_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return;
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->tail_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        h->tail_exec = nullptr;
        return;
    }
    h->tail_key[0] = nch;
    h->tail_key[1] = (int64_t)c.prec;
    h->tail_key[2] = c.refine_k;
    h->tail_key[3] = (int64_t)ebc::wait_limit_ns();
}

bool tail_graph_ok(ebc_t h, int nch) {
    const ebc::Ctx &c = h->c;
    return h->tail_exec && h->tail_key[0] == nch && h->tail_key[1] == (int64_t)c.prec &&
           h->tail_key[2] == c.refine_k && h->tail_key[3] == (int64_t)ebc::wait_limit_ns();
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
    for (GroupLane &l : g->lanes)
        if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&l.ev_bulk, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&l.ev_staged, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ebc_group_destroy(g);
            return EBC_ECUDA;
        }
    *out = g;
    return EBC_OK;
}

ebc_status ebc_group_set_lanes(ebc_group_t g, int32_t lanes) {
    if (!g || lanes < 1 || lanes > 4) return EBC_EINVAL;
    g->nlanes = lanes;
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
    // most rounds first; dealt to the lanes in that order, so in every lane
    // the handles running in round r are a prefix
    std::stable_sort(shared.begin(), shared.end(), [&](int a, int b) { return k[a] > k[b]; });
    const int ni = (int)shared.size();
    int L = std::min(g->nlanes, ni);
    if (g->by_row_width) L = 2;
    while ((int)g->ev_inst.size() < ni) {
        cudaEvent_t ev = nullptr;
        GK(g, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        g->ev_inst.push_back(ev);
    }
    struct LanePlan {
        std::vector<int> members;  // indices into `shared`, rounds descending
        std::vector<int> nch, vpc, RB;
        std::vector<int64_t> first_unit;
    };
    std::vector<LanePlan> plan(L);
    for (int e = 0; e < ni; ++e) {
        const int lane = g->by_row_width ? (ebc::tc_group_row_bytes(hs[shared[e]]->c) > 128 ? 0 : 1) : e % L;
        plan[lane].members.push_back(e);
    }
    for (int li = 0; li < L; ++li) {
        LanePlan &P = plan[li];
        GroupLane &lane = g->lanes[li];
        const int nm = (int)P.members.size();
        if (nm == 0) continue;
        P.nch.resize(nm);
        P.vpc.resize(nm);
        P.RB.resize(nm);
        P.first_unit.assign(nm + 1, 0);
        for (int x = 0; x < nm; ++x) {
            const ebc::Ctx &c = hs[shared[P.members[x]]]->c;
            const int n_vtiles = (int)(c.tc.n_pad / 256);
            const int n_ctiles = (int)((c.n + 255) / 256);
            const int max_ch = (int)std::max<int64_t>(1, std::min<int64_t>(c.partial_cap / c.n, n_vtiles));
            const int want = std::min(max_ch, std::max(1, (n_vtiles + kTilesPerUnit - 1) / kTilesPerUnit));
            P.vpc[x] = (n_vtiles + want - 1) / want;
            P.nch[x] = (n_vtiles + P.vpc[x] - 1) / P.vpc[x];
            P.RB[x] = ebc::tc_group_row_bytes(c);
            P.first_unit[x + 1] = P.first_unit[x] + (int64_t)n_ctiles * P.nch[x];
        }
        const int64_t nu = P.first_unit[nm];
        if (nu > INT32_MAX / 2) return gfail(g, EBC_EINVAL, "ebc_group_greedy: too many work units");
        ebc_status s = ensure_tables(g, &lane, nm, nu);
        if (s != EBC_OK) return s;
        // unit table: handles in order of rounds, within equal rounds largest units first
        int64_t w = 0;
        for (int x0 = 0; x0 < nm;) {
            int x1 = x0;
            while (x1 < nm && k[shared[P.members[x1]]] == k[shared[P.members[x0]]]) ++x1;
            const int64_t b = w;
            for (int x = x0; x < x1; ++x) {
                const ebc::Ctx &c = hs[shared[P.members[x]]]->c;
                const int n_vtiles = (int)(c.tc.n_pad / 256);
                const int n_ctiles = (int)((c.n + 255) / 256);
                for (int ct = 0; ct < n_ctiles; ++ct)
                    for (int ch = 0; ch < P.nch[x]; ++ch) {
                        const int vt0 = ch * P.vpc[x];
                        lane.h_units[w++] = {x, ct, ch, std::min(vt0 + P.vpc[x], n_vtiles) - vt0};
                    }
            }
            std::stable_sort(lane.h_units + b, lane.h_units + w,
                             [](const ebc::GroupUnit &a, const ebc::GroupUnit &c) { return a.ntiles > c.ntiles; });
            x0 = x1;
        }
        for (int x = 0; x < nm; ++x)
            ebc::group_inst_fill(hs[shared[P.members[x]]]->c, P.nch[x], P.vpc[x], &lane.h_inst[x]);
        GK(g, cudaMemcpyAsync(lane.d_inst, lane.h_inst, sizeof(ebc::GroupInst) * nm, cudaMemcpyHostToDevice,
                              lane.stream));
        GK(g, cudaMemcpyAsync(lane.d_units, lane.h_units, sizeof(ebc::GroupUnit) * nu, cudaMemcpyHostToDevice,
                              lane.stream));
        GK(g, cudaEventRecord(lane.ev_staged, lane.stream));
        lane.staged_pending = true;
    }

    // picks and f go to each handle's by-round buffers (written by round since
    // reset), copied to the caller's outputs at the end
    std::vector<int64_t> first(ni);
    for (int e = 0; e < ni; ++e) {
        ebc_t h = hs[shared[e]];
        ebc::Ctx &c = h->c;
        first[e] = h->nsel;
        if (!h->g_idx) {
            cudaError_t ea = dalloc(&h->g_idx, c.n, c);
            if (ea == cudaSuccess) ea = dalloc(&h->g_f, c.n, c);
            if (ea != cudaSuccess) {
                ebc::pool_free(h->g_idx, c.stream);
                h->g_idx = nullptr;
                h->g_f = nullptr;
                return gcuda(g, ea, "ebc_group_greedy: by-round buffers");
            }
        }
        // the first round's point extension (later rounds: the previous tail)
        CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc(c, true); }));
    }
    const int kmax = k[shared[0]];
    std::vector<int> active(L);
    for (int li = 0; li < L; ++li) active[li] = (int)plan[li].members.size();
    for (int r = 0; r < kmax; ++r) {
        for (int li = 0; li < L; ++li) {
            LanePlan &P = plan[li];
            GroupLane &lane = g->lanes[li];
            if (P.members.empty()) continue;
            int &na = active[li];
            while (na > 0 && k[shared[P.members[na - 1]]] <= r) --na;
            if (na == 0) continue;
            int RBmax = 0;
            for (int x = 0; x < na; ++x) RBmax = std::max(RBmax, P.RB[x]);
            for (int x = 0; x < na; ++x) {
                const int e = P.members[x];
                ebc_t h = hs[shared[e]];
                GK(g, cudaEventRecord(g->ev_inst[e], h->c.stream));
                GK(g, cudaStreamWaitEvent(lane.stream, g->ev_inst[e], 0));
            }
            GK(g, cudaMemsetAsync(lane.d_words, 0, 2 * sizeof(int), lane.stream));
            std::pair<cudaEvent_t, cudaEvent_t> evp{nullptr, nullptr};
            if (g->prof) {
                if (!g->spare.empty()) {
                    evp = g->spare.back();
                    g->spare.pop_back();
                } else {
                    GK(g, cudaEventCreate(&evp.first));
                    GK(g, cudaEventCreate(&evp.second));
                }
                GK(g, cudaEventRecord(evp.first, lane.stream));
            }
            const int G = (g->max_ctas > 0 && g->max_ctas < g->num_sms) ? g->max_ctas : g->num_sms;
            GK(g, ebc::launch_gains_tc_group(lane.d_inst, lane.d_units, (int)P.first_unit[na], lane.d_words,
                                             lane.d_words + 1, RBmax, G, lane.stream));
            if (g->prof) {
                GK(g, cudaEventRecord(evp.second, lane.stream));
                g->pending.push_back(evp);
                for (int x = 0; x < na; ++x) {
                    const ebc::Ctx &c = hs[shared[P.members[x]]]->c;
                    g->launch_evals += c.n * c.n;
                }
            }
            GK(g, ebc::launch_group_err(lane.d_inst, na, lane.d_words + 1, lane.stream));
            GK(g, cudaEventRecord(lane.ev_bulk, lane.stream));
            g->launches += 1;
            g->units += P.first_unit[na];
            for (int x = 0; x < na; ++x) {
                const int e = P.members[x];
                ebc_t h = hs[shared[e]];
                ebc::Ctx &c = h->c;
                GK(g, cudaStreamWaitEvent(c.stream, lane.ev_bulk, 0));
                h->prof.p.bulk_launches += 1;
                h->prof.p.bulk_evals += (c.n - h->nsel) * c.n;
                const int nchunks = P.nch[x];
                const bool graphs = h->graphs && !h->prof.on && c.stream != nullptr;
                if (graphs && tail_graph_ok(h, nchunks)) {
                    GK(g, cudaGraphLaunch(h->tail_exec, c.stream));
                    h->prof.p.launches += h->tail_launches;
                } else {
                    ebc_status s = round_tail(h, nchunks);
                    if (s != EBC_OK) return gfail(g, s, std::string("ebc_group_greedy: ") + ebc_last_error(h));
                    // after one direct tail (kernel attributes set), capture for the next rounds
                    if (graphs && k[shared[e]] - r > 1) capture_tail(h, nchunks);
                }
                h->nsel += 1;
                h->attrs_ready = true;
            }
        }
        g->rounds += 1;
    }
    for (int e = 0; e < ni; ++e) {
        ebc_t h = hs[shared[e]];
        ebc::Ctx &c = h->c;
        const int64_t cnt = k[shared[e]];
        GK(g, cudaMemcpyAsync(out_idx[shared[e]], h->g_idx + first[e], sizeof(int32_t) * cnt,
                              cudaMemcpyDeviceToDevice, c.stream));
        GK(g, cudaMemcpyAsync(out_f[shared[e]], h->g_f + first[e], sizeof(double) * cnt, cudaMemcpyDeviceToDevice,
                              c.stream));
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

ebc_status ebc_group_set_profiling(ebc_group_t g, int32_t on) {
    if (!g) return EBC_EINVAL;
    g->prof = on != 0;
    return EBC_OK;
}

ebc_status ebc_group_set_max_ctas(ebc_group_t g, int32_t max_ctas) {
    if (!g || max_ctas < 0) return EBC_EINVAL;
    g->max_ctas = max_ctas;
    return EBC_OK;
}

ebc_status ebc_group_set_lanes_by_row_width(ebc_group_t g, int32_t on) {
    if (!g) return EBC_EINVAL;
    g->by_row_width = on != 0;
    return EBC_OK;
}

ebc_status ebc_group_profile(ebc_group_t g, double *launch_ms, double *gap_ms, int64_t *pairs) {
    if (!g) return EBC_EINVAL;
    for (auto &p : g->pending) {
        if (cudaEventSynchronize(p.second) != cudaSuccess) return gcuda(g, cudaGetLastError(), "ebc_group_profile");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.first, p.second);
        g->launch_ms += ms;
        if (g->last_end) {
            float gms = 0.f;
            if (cudaEventElapsedTime(&gms, g->last_end, p.first) == cudaSuccess && gms >= 0.f) g->gap_ms += gms;
            cudaGetLastError();
        }
        g->last_end = p.second;
    }
    for (auto &p : g->pending) g->spare.push_back(p);
    g->pending.clear();
    g->last_end = nullptr;
    if (launch_ms) *launch_ms = g->launch_ms;
    if (gap_ms) *gap_ms = g->gap_ms;
    if (pairs) *pairs = g->launch_evals;
    return EBC_OK;
}

ebc_status ebc_group_reset_profile(ebc_group_t g) {
    if (!g) return EBC_EINVAL;
    double ms = 0.0;
    ebc_status s = ebc_group_profile(g, &ms, nullptr, nullptr);
    g->launch_ms = 0.0;
    g->gap_ms = 0.0;
    g->launch_evals = 0;
    return s;
}

const char *ebc_group_last_error(ebc_group_t g) { return g ? g->err.c_str() : ""; }

ebc_status ebc_group_destroy(ebc_group_t g) {
    if (!g) return EBC_OK;
    for (GroupLane &l : g->lanes) {
        if (l.stream) cudaStreamSynchronize(l.stream);
        ebc::pool_free(l.d_inst, l.stream);
        ebc::pool_free(l.d_units, l.stream);
        ebc::pool_free(l.d_words, l.stream);
        if (l.stream) {
            cudaStreamSynchronize(l.stream);
            cudaStreamDestroy(l.stream);
        }
        if (l.h_inst) cudaFreeHost(l.h_inst);
        if (l.h_units) cudaFreeHost(l.h_units);
        if (l.ev_bulk) cudaEventDestroy(l.ev_bulk);
        if (l.ev_staged) cudaEventDestroy(l.ev_staged);
    }
    for (cudaEvent_t ev : g->ev_inst) cudaEventDestroy(ev);
    for (auto *v : {&g->pending, &g->spare})
        for (auto &p : *v) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
    delete g;
    return EBC_OK;
}

}  // extern "C"
