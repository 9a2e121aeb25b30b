// Tuning table of the tensor-core bulk kernel: for a (precision, row bytes,
// n bucket) key, the point-tile width (256 or 128 points), whether the two
// MMA issuers take turns, how the drain is split, the pipeline shape (candidate-tile buffers,
// point-tile stages) and the V-chunk policy found fastest by ebc_autotune
// (api.cu).
// Process-wide, guarded by a mutex; saved to and loaded from a small JSON
// file.  Entries only change how the bulk bounds are scheduled and summed
// (chunk grouping); picks and f do not depend on them.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "ebc_internal.cuh"

namespace ebc {
namespace {

struct Entry {
    TuneCfg cfg;
    double ms = 0.0;
};

using Key = std::tuple<int, int, int>;  // precision, row bytes, floor(log2 n)

std::mutex g_mu;
std::map<Key, Entry> g_table;

int n_bucket(int64_t n) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << (b + 1)) <= n) ++b;
    return b;
}

}  // namespace

bool tune_lookup(const Ctx &c, int prec, int RB, int64_t n, TuneCfg *cfg) {
    if (c.tune_force) {
        *cfg = *c.tune_force;
        return true;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(Key(prec, RB, n_bucket(n)));
    if (it == g_table.end()) return false;
    *cfg = it->second.cfg;
    return true;
}

bool tune_get(int prec, int RB, int64_t n, TuneCfg *cfg, double *ms) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(Key(prec, RB, n_bucket(n)));
    if (it == g_table.end()) return false;
    *cfg = it->second.cfg;
    *ms = it->second.ms;
    return true;
}

bool tune_has(int prec, int RB, int64_t n) {
    std::lock_guard<std::mutex> lock(g_mu);
    return g_table.count(Key(prec, RB, n_bucket(n))) != 0;
}

void tune_store(int prec, int RB, int64_t n, const TuneCfg &cfg, double ms) {
    std::lock_guard<std::mutex> lock(g_mu);
    Entry e;
    e.cfg = cfg;
    e.ms = ms;
    g_table[Key(prec, RB, n_bucket(n))] = e;
}

int apply_chunk_mode(int nchunks, int mode, int n_vtiles, int64_t cap, int *vt_per_chunk) {
    int nch = nchunks;
    if (mode == 1) nch = (int)lmin(lmin(2 * (int64_t)nchunks, 32), lmin(cap, n_vtiles));
    if (mode == 2) nch = nchunks / 2;
    if (nch < 1) nch = 1;
    const int vpc = (n_vtiles + nch - 1) / nch;
    *vt_per_chunk = vpc;
    return (n_vtiles + vpc - 1) / vpc;
}

}  // namespace ebc

extern "C" {

int64_t ebc_tune_count(void) {
    std::lock_guard<std::mutex> lock(ebc::g_mu);
    return (int64_t)ebc::g_table.size();
}

ebc_status ebc_tune_clear(void) {
    std::lock_guard<std::mutex> lock(ebc::g_mu);
    ebc::g_table.clear();
    return EBC_OK;
}

ebc_status ebc_tune_save(const char *path) {
    if (!path) return EBC_EINVAL;
    std::lock_guard<std::mutex> lock(ebc::g_mu);
    FILE *f = fopen(path, "w");
    if (!f) return EBC_EINVAL;
    fprintf(f, "{\"version\": 1, \"entries\": [");
    bool first = true;
    for (const auto &kv : ebc::g_table) {
        const auto &k = kv.first;
        const auto &e = kv.second;
        fprintf(f,
                "%s\n  {\"prec\": %d, \"rb\": %d, \"nbucket\": %d, \"na\": %d, \"ns\": %d, \"chunk\": %d, "
                "\"bn\": %d, \"turns\": %d, \"es\": %d, \"ms\": %.6f}",
                first ? "" : ",", std::get<0>(k), std::get<1>(k), std::get<2>(k), e.cfg.na, e.cfg.ns, e.cfg.chunk,
                e.cfg.bn, e.cfg.turns, e.cfg.es, e.ms);
        first = false;
    }
    fprintf(f, "\n]}\n");
    return fclose(f) == 0 ? EBC_OK : EBC_EINVAL;
}

// Reads files written by ebc_tune_save (one object per entry, the keys
// above in any order); entries replace those with the same key.  EINVAL if
// the file cannot be read or an entry is incomplete or out of range (the
// table is then left unchanged).
ebc_status ebc_tune_load(const char *path) {
    if (!path) return EBC_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f) return EBC_EINVAL;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    fclose(f);
    const size_t ent = text.find("\"entries\"");
    if (ent == std::string::npos) return EBC_EINVAL;
    std::map<ebc::Key, ebc::Entry> add;
    size_t pos = text.find('[', ent);
    if (pos == std::string::npos) return EBC_EINVAL;
    while (true) {
        const size_t a = text.find('{', pos), end = text.find(']', pos);
        if (a == std::string::npos || (end != std::string::npos && end < a)) break;
        const size_t b = text.find('}', a);
        if (b == std::string::npos) return EBC_EINVAL;
        const std::string obj = text.substr(a, b - a + 1);
        auto field = [&](const char *name, double *out) {
            const std::string key = std::string("\"") + name + "\"";
            const size_t p = obj.find(key);
            if (p == std::string::npos) return false;
            const size_t colon = obj.find(':', p + key.size());
            return colon != std::string::npos && sscanf(obj.c_str() + colon + 1, "%lf", out) == 1;
        };
        double prec, rb, nb, na, ns, chunk, bn = 256, turns = -1, es = 0, ms = 0.0;
        if (!field("prec", &prec) || !field("rb", &rb) || !field("nbucket", &nb) || !field("na", &na) ||
            !field("ns", &ns) || !field("chunk", &chunk))
            return EBC_EINVAL;
        field("ms", &ms);
        field("bn", &bn);        // absent: 256-point tiles
        field("turns", &turns);  // absent: by row width
        field("es", &es);        // absent: drain split by column halves
        if (prec < 1 || prec > 3 || rb < 128 || rb > 512 || nb < 0 || nb > 62 || na < 1 || na > 2 || ns < 2 ||
            ns > 6 || chunk < 0 || chunk > 2 || (bn != 256 && bn != 128) || turns < -1 || turns > 1 ||
            (es != 0 && es != 1) || (es == 1 && bn != 256))
            return EBC_EINVAL;
        ebc::Entry e;
        e.cfg.na = (int)na;
        e.cfg.ns = (int)ns;
        e.cfg.chunk = (int)chunk;
        e.cfg.bn = (int)bn;
        e.cfg.turns = (int)turns;
        e.cfg.es = (int)es;
        e.ms = ms;
        add[ebc::Key((int)prec, (int)rb, (int)nb)] = e;
        pos = b + 1;
    }
    std::lock_guard<std::mutex> lock(ebc::g_mu);
    for (const auto &kv : add) ebc::g_table[kv.first] = kv.second;
    return EBC_OK;
}

}  // extern "C"
