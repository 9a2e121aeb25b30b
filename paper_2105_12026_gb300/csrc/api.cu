// C ABI of the library (include/ebc.h): handle life cycle, argument checks,
// and the per-round orchestration of Greedy.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace ebc::hx;

namespace {

thread_local std::string g_create_error;

constexpr int kPoolDevices = 64;
cudaMemPool_t g_pools[kPoolDevices] = {};
std::mutex g_pool_mu;

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= kPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;  // keep freed memory cached for the next instance
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

constexpr int32_t kMaxD = 4096;


void free_all(ebc::Ctx &c, ebc_ctx *h) {
    ebc::tc_free(c);
    void *ptrs[] = {c.V32, c.nv64, c.nv32, c.m64, c.sel, c.st, c.partial, c.gain_up, c.blk_idx, c.blk_val, c.top_idx, c.top_val,
                    c.esc_idx, c.esc_exact, c.cand_buf, c.set_part, c.ub64, c.lazy_idx,
                    c.cert.top_lo, c.cert.top_hi, c.cert.esc_lo, c.cert.esc_hi, c.cert.part_lo, c.cert.part_hi,
                    c.cert.ctd_idx, c.cert.ctd_part, c.cert.ctd_exact,
                    h ? h->d_scalar : nullptr, h ? h->d_bad : nullptr};
    for (void *p : ptrs) ebc::pool_free(p, c.stream);
}

__global__ void k_sanitize(const int32_t *__restrict__ in, int64_t m, int64_t n, int32_t *__restrict__ out,
                           ebc::DevState *st) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    int x = in ? in[j] : (int)j;
    if (x < 0 || (int64_t)x >= n) {
        atomicCAS(&st->err, 0, (int)EBC_EINDEX);
        x = -1;
    }
    out[j] = x;
}

__global__ void k_zero_masked(const int32_t *__restrict__ cand, int64_t m, double *__restrict__ out) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < m && cand[j] < 0) out[j] = 0.0;
}

__global__ void k_scale(double *__restrict__ x, int64_t m, double a) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < m) x[j] *= a;
}

__global__ void k_check_csr(const int64_t *__restrict__ off, int64_t l, ebc::DevState *st, int *bad) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j == 0 && off[0] != 0) {
        atomicCAS(&st->err, 0, (int)EBC_EINVAL);
        atomicExch(bad, 1);
    }
    if (j < l && off[j + 1] < off[j]) {
        atomicCAS(&st->err, 0, (int)EBC_EINVAL);
        atomicExch(bad, 1);
    }
}

cudaError_t fold_profile(ebc_t h) {
    Prof &p = h->prof;
    cudaError_t e = cudaStreamSynchronize(h->c.stream);
    if (e != cudaSuccess) return e;
    for (auto &r : p.pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        if (r.kind == PK_BULK) p.p.bulk_ms += ms;
        if (r.kind == PK_REFINE) p.p.refine_ms += ms;
        if (r.kind == PK_EVAL) p.p.eval_ms += ms;
        if (r.kind == PK_LIST) p.p.list_ms += ms;
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.pending.clear();
    return cudaSuccess;
}

// Lazy Greedy bounds and list, both or neither.
cudaError_t alloc_lazy(ebc::Ctx &c) {
    cudaError_t e = dalloc(&c.ub64, c.n, c);
    if (e == cudaSuccess) e = dalloc(&c.lazy_idx, c.n, c);
    if (e != cudaSuccess) {
        ebc::pool_free(c.ub64, c.stream);
        c.ub64 = nullptr;
        c.lazy_idx = nullptr;
    }
    return e;
}

ebc_status ensure_set_part(ebc_t h, int64_t want) {
    ebc::Ctx &c = h->c;
    if (c.set_part_cap >= want) return EBC_OK;
    ebc::pool_free(c.set_part, c.stream);
    c.set_part = nullptr;
    c.set_part_cap = 0;
    CK(h, dalloc(&c.set_part, (size_t)want, c));
    c.set_part_cap = want;
    return EBC_OK;
}

}  // namespace

namespace ebc {
namespace hx {

ebc_status fail(ebc_t h, ebc_status s, const std::string &msg) {
    if (h)
        h->c.last_error = msg;
    else
        g_create_error = msg;
    return s;
}

ebc_status cuda_fail(ebc_t h, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? EBC_ENOMEM : EBC_ECUDA, m);
}

double bulk_eta(const ebc::Ctx &c) {
    (void)c;
    // each bulk partial is an FP64 sum of FP32 block sums; a block sum joins
    // four chains of at most 128 non-negative FP32 terms with two additions,
    // each term one rounding from its bound: relative error <= 130 * 2^-24
    // (the FP64 additions are covered by the last term)
    return 131.0 * ldexp(1.0, -24) + 1e-12;
}

ebc_status check_handle(ebc_t h) {
    if (!h) return EBC_EINVAL;
    return EBC_OK;
}

cudaEvent_t take_event(Prof &p) {
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace hx
}  // namespace ebc

// Device bytes one handle allocates (create + tensor-core buffers + graph
// outputs), mirroring the allocations of create_handle and tc_setup.
int64_t ebc::handle_bytes(int64_t n, int32_t d, ebc_prec prec) {
    const int64_t ch = std::max<int64_t>(4096, ((n + 63) / 64 + 127) / 128 * 128);
    const int64_t nch = (n + ch - 1) / ch;
    const int64_t ref_ch = ebc::refine_chunk(n, d);
    const int64_t nref = (n + ref_ch - 1) / ref_ch;
    const int64_t nblk = std::min<int64_t>(512, std::max<int64_t>(1, (n + 2047) / 2048));
    const int64_t cap = std::min<int64_t>(n, 4096);
    const int64_t pool = ebc::kMaxRefineK + cap;
    int64_t b = n * d * 4 + n * (8 + 4 + 8 + 1 + 8 + 4 + 8 + 4 + 4 + 8) + std::max<int64_t>(nch, 16) * n * 8;
    b += nblk * (ebc::kMaxRefineK + 1) * 12 + 4096;
    b += 2 * cap * 8 + 3 * pool * nref * 8 + pool * 12 + 2 * ebc::kMaxRefineK * 8;
    if (prec == EBC_BF16 || prec == EBC_FP16 || prec == EBC_FP8E4M3) {
        const int64_t n_pad = (n + 255) / 256 * 256, DP = (d + 63) / 64 * 64;
        b += 3 * n_pad * DP * 2 + 4 * n_pad * 16 * 2 + n_pad * (8 + 4 + 4);
    }
    if (prec == EBC_FP8E4M3) {  // FP8 operands, extensions, scales, norms; lazy bounds and list
        const int64_t n_pad = (n + 255) / 256 * 256, DP8 = (d + 127) / 128 * 128;
        b += 3 * n_pad * DP8 + 3 * n_pad * 16 * 2 + n_pad * (4 + 4 + 8 + 8 + 4 * 4) + n * (8 + 4);
    }
    return b + 64 * 1024;  // allocation granularity and small buffers
}

namespace {
// Injected allocation failure: the allocation after this many more
// successful ones fails (-1: none).
std::atomic<int64_t> g_alloc_fail_after{-1};
std::atomic<uint64_t> g_wait_limit_ns{1000000000ull};
}  // namespace

uint64_t ebc::wait_limit_ns() { return g_wait_limit_ns.load(std::memory_order_relaxed); }

cudaError_t ebc::pool_alloc(void **p, size_t bytes, cudaStream_t s, int dev) {
    *p = nullptr;
    for (int64_t a = g_alloc_fail_after.load(); a >= 0;) {
        if (g_alloc_fail_after.compare_exchange_weak(a, a - 1)) {
            if (a == 0) return cudaErrorMemoryAllocation;  // the injected failure (now disarmed)
            break;
        }
    }
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, s);
}

void ebc::pool_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

extern "C" {

ebc_status ebc_inject_alloc_failure(int64_t after) {
    if (after < -1) return EBC_EINVAL;
    g_alloc_fail_after.store(after);
    return EBC_OK;
}

ebc_status ebc_set_wait_limit_ns(int64_t ns) {
    if (ns < 0 || ns > 60000000000ll) return EBC_EINVAL;
    g_wait_limit_ns.store(ns == 0 ? 1000000000ull : (uint64_t)ns);
    return EBC_OK;
}

ebc_status ebc_release_cached_memory(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return EBC_ENODEV;
    }
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return EBC_ECUDA;
    return cudaMemPoolTrimTo(pool, 0) == cudaSuccess ? EBC_OK : EBC_ECUDA;
}

int64_t ebc_estimate_bytes(int64_t n, int32_t d, int32_t prec) {
    if (n <= 0 || d <= 0) return -1;
    return ebc::handle_bytes(n, d, (ebc_prec)prec);
}

int32_t ebc_version(void) { return (0 << 16) | 1; }

const char *ebc_last_error(ebc_t h) { return h ? h->c.last_error.c_str() : g_create_error.c_str(); }

ebc_status ebc_create(const float *V, int64_t n, int32_t d, int32_t v_on_device, void *stream, ebc_t *out) {
    return ebc::create_handle(V, n, d, v_on_device, stream, true, out);
}

}  // extern "C"

ebc_status ebc::create_handle(const float *V, int64_t n, int32_t d, int32_t v_on_device, void *stream, bool sync,
                              ebc_t *out) {
    ebc::TraceRange trace_("ebc_create");
    g_create_error.clear();
    if (!out) return fail(nullptr, EBC_EINVAL, "ebc_create: out is NULL");
    *out = nullptr;
    if (!V) return fail(nullptr, EBC_EINVAL, "ebc_create: V is NULL");
    if (n <= 0) return fail(nullptr, EBC_EINVAL, "ebc_create: n must be > 0");
    if (n > (int64_t)INT32_MAX - 1) return fail(nullptr, EBC_EINVAL, "ebc_create: n exceeds int32 indexing");
    if (d <= 0 || d > kMaxD) return fail(nullptr, EBC_EINVAL, "ebc_create: d must be in [1, 4096]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, EBC_ENODEV, std::string("ebc_create: ") + cudaGetErrorString(e));
    int maj = 0, min = 0;
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
    if (!(maj == 10 && min == 3)) {
        char b[128];
        snprintf(b, sizeof b, "ebc_create: device %d is sm_%d%d; this library is built for sm_103a only", dev, maj,
                 min);
        return fail(nullptr, EBC_ENODEV, b);
    }
    ebc_ctx *h = new (std::nothrow) ebc_ctx();
    if (!h) return fail(nullptr, EBC_ENOMEM, "ebc_create: host allocation failed");
    ebc::Ctx &c = h->c;
    c.n = n;
    c.d = d;
    c.dpad = (d + 63) / 64 * 64;
    c.device = dev;
    c.stream = (cudaStream_t)stream;

    // chunking of the V axis
    h->ch = std::max<int64_t>(4096, ((n + 63) / 64 + 127) / 128 * 128);
    h->nch = (int)((n + h->ch - 1) / h->ch);
    h->ref_ch = ebc::refine_chunk(n, d);
    h->nref = (int)((n + h->ref_ch - 1) / h->ref_ch);
    h->esc_cap = (int)std::min<int64_t>(n, 4096);
    h->nblk = (int)std::min<int64_t>(512, std::max<int64_t>(1, (n + 2047) / 2048));

    auto bail = [&](ebc_status s, const std::string &m) {
        free_all(c, h);
        delete h;
        return fail(nullptr, s, m);
    };
#define CKC(expr)                                                                                  \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess)                                                                     \
            return bail(_e == cudaErrorMemoryAllocation ? EBC_ENOMEM : EBC_ECUDA,                  \
                        std::string("ebc_create: ") + #expr + ": " + cudaGetErrorString(_e));     \
    } while (0)
    CKC(dalloc(&c.V32, (size_t)n * d, c));
    CKC(dalloc(&c.nv64, n, c));
    CKC(dalloc(&c.nv32, n, c));
    CKC(dalloc(&c.m64, n, c));
    CKC(dalloc(&c.sel, n, c));
    CKC(dalloc(&c.st, 1, c));
    cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
    c.partial_cap = (int64_t)std::max(h->nch, 16) * n;
    CKC(dalloc(&c.partial, (size_t)c.partial_cap, c));
    CKC(dalloc(&c.gain_up, n, c));
    c.blk_cap = h->nblk * (ebc::kMaxRefineK + 1);
    CKC(dalloc(&c.blk_idx, c.blk_cap, c));
    CKC(dalloc(&c.blk_val, c.blk_cap, c));
    CKC(dalloc(&c.top_idx, ebc::kMaxRefineK + 1, c));
    CKC(dalloc(&c.top_val, ebc::kMaxRefineK + 1, c));
    CKC(dalloc(&c.esc_idx, n, c));
    CKC(dalloc(&c.esc_exact, n, c));
    {
        ebc::Ctx::Sel &S = c.cert;
        S.cap = h->esc_cap;
        S.nchunks = h->nref;
        S.chunk = h->ref_ch;
        const size_t pool = (size_t)ebc::kMaxRefineK + S.cap;
        CKC(dalloc(&S.top_lo, ebc::kMaxRefineK, c));
        CKC(dalloc(&S.top_hi, ebc::kMaxRefineK, c));
        CKC(dalloc(&S.esc_lo, S.cap, c));
        CKC(dalloc(&S.esc_hi, S.cap, c));
        CKC(dalloc(&S.part_lo, pool * S.nchunks, c));
        CKC(dalloc(&S.part_hi, pool * S.nchunks, c));
        CKC(dalloc(&S.ctd_idx, pool, c));
        CKC(dalloc(&S.ctd_part, pool * S.nchunks, c));
        CKC(dalloc(&S.ctd_exact, pool, c));
    }
    CKC(dalloc(&c.cand_buf, n, c));
    CKC(dalloc(&h->d_scalar, 1, c));
    CKC(dalloc(&h->d_bad, 1, c));

    CKC(cudaMemcpyAsync(c.V32, V, sizeof(float) * (size_t)n * d,
                        v_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.stream));
    CKC(ebc::launch_reset_state(c));
    CKC(ebc::launch_prologue(c));
    if (sync) {
        CKC(cudaMemcpyAsync(c.h_err, &c.st->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
        CKC(cudaStreamSynchronize(c.stream));
        if (c.h_err[0]) return bail(EBC_EINVAL, "ebc_create: V has a non-finite entry");
    }
#undef CKC
    *out = h;
    return EBC_OK;
}

extern "C" {

ebc_status ebc_destroy(ebc_t h) {
    if (!h) return EBC_OK;
    cudaStreamSynchronize(h->c.stream);
    if (h->round_exec) cudaGraphExecDestroy(h->round_exec);
    if (h->tail_exec) cudaGraphExecDestroy(h->tail_exec);
    ebc::pool_free(h->g_idx, h->c.stream);
    ebc::pool_free(h->g_f, h->c.stream);
    for (auto &r : h->prof.pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->prof.pool) cudaEventDestroy(e);
    free_all(h->c, h);
    delete h;
    return EBC_OK;
}

ebc_status ebc_reload(ebc_t h, const float *V, int32_t v_on_device) {
    if (check_handle(h)) return EBC_EINVAL;
    if (!V) return fail(h, EBC_EINVAL, "ebc_reload: V is NULL");
    ebc::Ctx &c = h->c;
    CK(h, cudaMemcpyAsync(c.V32, V, sizeof(float) * (size_t)c.n * c.d,
                          v_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.stream));
    CK(h, launch(h, -1, 1, [&] { return ebc::launch_reset_state(c); }));
    CK(h, launch(h, -1, 1, [&] { return ebc::launch_prologue(c); }));
    if (c.tc.prec >= 0) CK(h, launch(h, -1, 1, [&] { return ebc::tc_quantize(c); }));
    if (c.tc8.ready) CK(h, launch(h, -1, 3, [&] { return ebc::tc8_setup(c); }));
    h->nsel = 0;
    h->sieve_ub.clear();
    return EBC_OK;
}

ebc_status ebc_set_profiling(ebc_t h, int32_t on) {
    if (check_handle(h)) return EBC_EINVAL;
    h->prof.on = on != 0;
    return EBC_OK;
}

ebc_status ebc_get_profile(ebc_t h, ebc_profile *out) {
    if (check_handle(h) || !out) return fail(h, EBC_EINVAL, "ebc_get_profile: NULL argument");
    CK(h, fold_profile(h));
    *out = h->prof.p;
    return EBC_OK;
}

ebc_status ebc_reset_profile(ebc_t h) {
    if (check_handle(h)) return EBC_EINVAL;
    CK(h, fold_profile(h));
    h->prof.p = ebc_profile{};
    return EBC_OK;
}

ebc_status ebc_set_stream(ebc_t h, void *stream) {
    if (check_handle(h)) return EBC_EINVAL;
    CK(h, cudaStreamSynchronize(h->c.stream));  // stream-ordered allocations become visible to the new stream
    h->c.stream = (cudaStream_t)stream;
    return EBC_OK;
}

ebc_status ebc_set_precision(ebc_t h, ebc_prec prec, int32_t refine_k) {
    return ebc::set_precision_handle(h, prec, refine_k, true);
}

}  // extern "C"

ebc_status ebc::set_precision_handle(ebc_t h, ebc_prec prec, int32_t refine_k, bool sync) {
    if (check_handle(h)) return EBC_EINVAL;
    if (refine_k < 1 || refine_k > ebc::kMaxRefineK) return fail(h, EBC_EINVAL, "ebc_set_precision: K must be in [1, 31]");
    ebc::Ctx &c = h->c;
    if (prec == EBC_BF16 || prec == EBC_FP16) {
        if (!ebc::tc_supported(c))
            return fail(h, EBC_EINVAL, "ebc_set_precision: the tensor-core path supports d <= 4096");
        if (c.tc.prec != (int)prec) {
            if (!sync) {
                // errors (a format overflow) surface at the next ebc_sync
                CK(h, ebc::tc_setup(c, (int)prec));
            } else {
                // flush earlier device errors so a quantisation failure is seen on its own
                ebc_status s0 = ebc_sync(h);
                if (s0 != EBC_OK) return s0;
                CK(h, ebc::tc_setup(c, (int)prec));
                CK(h, cudaMemcpyAsync(c.h_err, &c.st->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
                CK(h, cudaStreamSynchronize(c.stream));
                if (c.h_err[0]) {
                    CK(h, cudaMemsetAsync(&c.st->err, 0, sizeof(int), c.stream));
                    c.tc.prec = -1;
                    return fail(h, EBC_EINVAL, "ebc_set_precision: V overflows the requested 16-bit format");
                }
            }
        }
    } else if (prec == EBC_FP8E4M3) {
        // FP8 bulk bounds pre-screen; the BF16 copy certifies (second level)
        if (!ebc::tc_resident_supported(c))
            return fail(h, EBC_EINVAL, "ebc_set_precision: the FP8 path supports d <= 128");
        if (sync) {
            ebc_status s0 = ebc_sync(h);
            if (s0 != EBC_OK) return s0;
        }
        if (c.tc.prec != EBC_BF16) CK(h, ebc::tc_setup(c, EBC_BF16));
        if (!c.tc8.ready) CK(h, ebc::tc8_setup(c));
        if (!c.ub64) {
            CK(h, alloc_lazy(c));
            CK(h, ebc::launch_lazy_init(c));
        }
        if (sync) {
            CK(h, cudaMemcpyAsync(c.h_err, &c.st->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
            CK(h, cudaStreamSynchronize(c.stream));
            if (c.h_err[0]) {
                CK(h, cudaMemsetAsync(&c.st->err, 0, sizeof(int), c.stream));
                return fail(h, EBC_EINVAL, "ebc_set_precision: V has a non-finite entry");
            }
        }
    } else if (prec != EBC_FP32) {
        return fail(h, EBC_EINVAL, "ebc_set_precision: unknown precision");
    }
    c.prec = prec;
    c.refine_k = refine_k;
    return EBC_OK;
}

extern "C" {

ebc_status ebc_reset(ebc_t h) {
    if (check_handle(h)) return EBC_EINVAL;
    CK(h, ebc::launch_reset_state(h->c));
    h->nsel = 0;
    h->sieve_ub.clear();
    return EBC_OK;
}

ebc_status ebc_sync(ebc_t h) {
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    CK(h, cudaMemcpyAsync(c.h_err, &c.st->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaStreamSynchronize(c.stream));
    int err = c.h_err[0];
    if (err) {
        CK(h, cudaMemsetAsync(&c.st->err, 0, sizeof(int), c.stream));
        CK(h, cudaStreamSynchronize(c.stream));
        return fail(h, (ebc_status)err,
                    err == EBC_EINDEX     ? "device: index outside [0, n)"
                    : err == EBC_ETIMEOUT ? "device: a bounded wait in the tensor-core pipeline ran out"
                                          : "device: invalid argument");
    }
    return EBC_OK;
}

ebc_status ebc_get_stats(ebc_t h, ebc_stats *out) {
    if (check_handle(h) || !out) return fail(h, EBC_EINVAL, "ebc_get_stats: NULL argument");
    ebc::Ctx &c = h->c;
    ebc::DevState s;
    CK(h, cudaMemcpyAsync(&s, c.st, sizeof(s), cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaStreamSynchronize(c.stream));
    out->rounds = s.rounds;
    out->certified_rounds = s.certified;
    out->escalated_rounds = s.escalated_rounds;
    out->escalated_candidates = s.escalated_cands;
    out->max_raw_rel_err = s.max_raw_rel_err;
    out->exact_evaluations = s.exact_evals;
    out->prec = (int32_t)c.prec;
    out->refine_k = c.refine_k;
    out->bulk_candidates = s.bulk_cands;
    out->lazy = c.lazy ? 1 : 0;
    return EBC_OK;
}

ebc_status ebc_last_round_candidates(ebc_t h, int32_t *out_idx, int64_t cap, int64_t *count) {
    if (check_handle(h) || !count || cap < 0 || (cap > 0 && !out_idx))
        return fail(h, EBC_EINVAL, "ebc_last_round_candidates: bad arguments");
    ebc::Ctx &c = h->c;
    ebc::DevState s;
    CK(h, cudaMemcpyAsync(&s, c.st, sizeof(s), cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaStreamSynchronize(c.stream));
    if (s.rounds == 0) {
        *count = 0;
        return EBC_OK;
    }
    const int64_t ntop = std::max(0, s.top_count);
    const int64_t nesc = s.need_esc ? std::min<int64_t>(std::max(0, s.esc_count), c.n) : 0;
    *count = ntop + nesc;
    if (cap < ntop + nesc) return EBC_OK;  // sizing call
    if (ntop > 0) CK(h, cudaMemcpyAsync(out_idx, c.top_idx, sizeof(int32_t) * ntop, cudaMemcpyDeviceToHost, c.stream));
    if (nesc > 0)
        CK(h, cudaMemcpyAsync(out_idx + ntop, c.esc_idx, sizeof(int32_t) * nesc, cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaStreamSynchronize(c.stream));
    return EBC_OK;
}

}  // extern "C"

ebc_status ebc::autotune_handle(ebc_t h, int32_t reps, bool only_if_missing) {
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (c.prec == EBC_FP32) return fail(h, EBC_EINVAL, "ebc_autotune: the FP32 plain kernel has no tuned configuration");
    if (reps < 1 || reps > 100) return fail(h, EBC_EINVAL, "ebc_autotune: reps must be in [1, 100]");
    const int RB = ebc::tc_row_bytes(c);
    if (only_if_missing && ebc::tune_has((int)c.prec, RB, c.n)) return EBC_OK;
    const bool fp8 = c.prec == EBC_FP8E4M3;
    CK(h, cudaStreamSynchronize(c.stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(h, cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    double best = INFINITY;
    ebc::TuneCfg best_cfg, cfg;
    auto bulk = [&]() {
        int nch = 1;
        return fp8 ? ebc::launch_gains_tc8(c, nullptr, c.n, &nch) : ebc::launch_gains_tc(c, nullptr, c.n, true, &nch);
    };
    if (err == cudaSuccess) err = fp8 ? ebc::launch_prep_tc8(c, true) : ebc::launch_prep_tc(c, true);
    // every point-tile width x shape that fits shared memory x chunk
    // policy; the fastest of reps timed launches (after one untimed) counts
    // (at 256 points also: issuer turns on or off, drain split by column
    // halves or by region)
    for (int bn = 256; bn >= 128 && err == cudaSuccess; bn /= 2)
    for (int es = 0; es <= (bn == 256 ? 1 : 0) && err == cudaSuccess; ++es)
    for (int turns = bn == 256 ? 1 : 0; turns >= 0 && err == cudaSuccess; --turns)
    for (int na = 1; na <= 2 && err == cudaSuccess; ++na)
        for (int ns = 2; ns <= 6 && err == cudaSuccess; ++ns) {
            if (!ebc::tc_config_fits(RB, na, ns, bn)) continue;
            for (int chunk = 0; chunk <= 2 && err == cudaSuccess; ++chunk) {
                cfg.na = na;
                cfg.ns = ns;
                cfg.chunk = chunk;
                cfg.bn = bn;
                cfg.turns = turns;
                cfg.es = es;
                c.tune_force = &cfg;
                err = bulk();
                double ms_min = INFINITY;
                for (int r = 0; r < reps && err == cudaSuccess; ++r) {
                    err = cudaEventRecord(e0, c.stream);
                    if (err == cudaSuccess) err = bulk();
                    if (err == cudaSuccess) err = cudaEventRecord(e1, c.stream);
                    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                    if (err == cudaSuccess) ms_min = std::min(ms_min, (double)ms);
                }
                if (err == cudaSuccess && ms_min < best) {
                    best = ms_min;
                    best_cfg = cfg;
                }
            }
        }
    c.tune_force = nullptr;
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(h, err, "ebc_autotune");
    if (!(best < INFINITY)) return ebc_sync(h);  // no resident shape fits: the K-blocked kernel has one shape
    ebc::tune_store((int)c.prec, RB, c.n, best_cfg, best);
    if (h->round_exec) {  // recapture rounds with the tuned configuration
        cudaGraphExecDestroy(h->round_exec);
        h->round_exec = nullptr;
    }
    return ebc_sync(h);
}

extern "C" {

ebc_status ebc_autotune(ebc_t h, int32_t reps) { return ebc::autotune_handle(h, reps, false); }

ebc_status ebc_tune_query(ebc_t h, int32_t cfg[6], double *ms) {
    if (check_handle(h) || !cfg) return fail(h, EBC_EINVAL, "ebc_tune_query: NULL argument");
    ebc::TuneCfg t;
    double tms = 0.0;
    cfg[0] = cfg[1] = cfg[2] = cfg[3] = cfg[4] = cfg[5] = 0;
    if (h->c.prec != EBC_FP32 && ebc::tune_get((int)h->c.prec, ebc::tc_row_bytes(h->c), h->c.n, &t, &tms)) {
        cfg[0] = t.bn;
        cfg[1] = t.na;
        cfg[2] = t.ns;
        cfg[3] = t.chunk;
        cfg[4] = t.turns;
        cfg[5] = t.es;
    } else {
        tms = 0.0;
    }
    if (ms) *ms = tms;
    return EBC_OK;
}

ebc_status ebc_set_lazy(ebc_t h, int32_t on) {
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (on && !c.ub64) CK(h, alloc_lazy(c));
    if (on && !c.lazy) CK(h, ebc::launch_lazy_init(c));  // bounds restart from the current state
    c.lazy = on != 0;
    return EBC_OK;
}

// ---- Greedy state snapshot (for pre-empting and resuming an instance) ----
// Layout: header, then m_v (f64 [n]) and the selection flags (u8 [n]).
namespace {
struct StateHeader {
    uint64_t magic;  // "EBCSTATE"
    int32_t version, d;
    int64_t n, nsel;
    double f;        // f(S)
    int64_t rounds, certified, escalated_rounds, escalated_cands, exact_evals, bulk_cands;
    int32_t round, reserved;
};
constexpr uint64_t kStateMagic = 0x4554415453434245ull;  // "EBCSTATE" little-endian
}  // namespace

ebc_status ebc_state_size(ebc_t h, int64_t *bytes) {
    if (check_handle(h) || !bytes) return fail(h, EBC_EINVAL, "ebc_state_size: NULL argument");
    *bytes = (int64_t)sizeof(StateHeader) + h->c.n * (8 + 1);
    return EBC_OK;
}

ebc_status ebc_state_save(ebc_t h, void *host_buf, int64_t bytes) {
    if (check_handle(h) || !host_buf) return fail(h, EBC_EINVAL, "ebc_state_save: NULL argument");
    ebc::Ctx &c = h->c;
    if (bytes < (int64_t)sizeof(StateHeader) + c.n * 9) return fail(h, EBC_EINVAL, "ebc_state_save: buffer too small");
    ebc_status s0 = ebc_sync(h);  // a pending device error would make the snapshot meaningless
    if (s0 != EBC_OK) return s0;
    ebc::DevState st;
    uint8_t *buf = static_cast<uint8_t *>(host_buf);
    CK(h, cudaMemcpyAsync(&st, c.st, sizeof(st), cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaMemcpyAsync(buf + sizeof(StateHeader), c.m64, sizeof(double) * c.n, cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaMemcpyAsync(buf + sizeof(StateHeader) + 8 * c.n, c.sel, c.n, cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaStreamSynchronize(c.stream));
    StateHeader hd;
    memset(&hd, 0, sizeof hd);
    hd.magic = kStateMagic;
    hd.version = 1;
    hd.d = c.d;
    hd.n = c.n;
    hd.nsel = h->nsel;
    hd.f = st.f;
    hd.rounds = st.rounds;
    hd.certified = st.certified;
    hd.escalated_rounds = st.escalated_rounds;
    hd.escalated_cands = st.escalated_cands;
    hd.exact_evals = st.exact_evals;
    hd.bulk_cands = st.bulk_cands;
    hd.round = st.round;
    memcpy(buf, &hd, sizeof hd);
    return EBC_OK;
}

ebc_status ebc_state_load(ebc_t h, const void *host_buf, int64_t bytes) {
    if (check_handle(h) || !host_buf) return fail(h, EBC_EINVAL, "ebc_state_load: NULL argument");
    ebc::Ctx &c = h->c;
    StateHeader hd;
    if (bytes < (int64_t)sizeof hd) return fail(h, EBC_EINVAL, "ebc_state_load: buffer too small");
    memcpy(&hd, host_buf, sizeof hd);
    if (hd.magic != kStateMagic || hd.version != 1) return fail(h, EBC_EINVAL, "ebc_state_load: not a state snapshot");
    if (hd.n != c.n || hd.d != c.d) return fail(h, EBC_EINVAL, "ebc_state_load: snapshot of an instance of another shape");
    if (bytes < (int64_t)sizeof hd + c.n * 9 || hd.nsel < 0 || hd.nsel > c.n || hd.round < 0)
        return fail(h, EBC_EINVAL, "ebc_state_load: truncated or inconsistent snapshot");
    const uint8_t *buf = static_cast<const uint8_t *>(host_buf);
    int64_t nsel = 0;
    for (int64_t i = 0; i < c.n; ++i) nsel += buf[sizeof hd + 8 * c.n + i] ? 1 : 0;
    if (nsel != hd.nsel) return fail(h, EBC_EINVAL, "ebc_state_load: selection flags do not match the header");
    CK(h, ebc::launch_reset_state(c));  // zero the device scalars (and restart any lazy bounds)
    CK(h, cudaMemcpyAsync(c.m64, buf + sizeof hd, sizeof(double) * c.n, cudaMemcpyHostToDevice, c.stream));
    CK(h, cudaMemcpyAsync(c.sel, buf + sizeof hd + 8 * c.n, c.n, cudaMemcpyHostToDevice, c.stream));
    ebc::DevState st;
    CK(h, cudaMemcpyAsync(&st, c.st, sizeof(st), cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaStreamSynchronize(c.stream));
    st.f = hd.f;
    st.rounds = hd.rounds;
    st.certified = hd.certified;
    st.escalated_rounds = hd.escalated_rounds;
    st.escalated_cands = hd.escalated_cands;
    st.exact_evals = hd.exact_evals;
    st.bulk_cands = hd.bulk_cands;
    st.round = hd.round;
    CK(h, cudaMemcpyAsync(c.st, &st, sizeof(st), cudaMemcpyHostToDevice, c.stream));
    if (c.ub64) CK(h, ebc::launch_lazy_init(c));  // after the flags: selected candidates get -1
    CK(h, cudaStreamSynchronize(c.stream));
    h->nsel = hd.nsel;
    h->sieve_ub.clear();
    return EBC_OK;
}

ebc_status ebc_current_f(ebc_t h, double *out_f) {
    if (check_handle(h) || !out_f) return fail(h, EBC_EINVAL, "ebc_current_f: NULL argument");
    ebc::Ctx &c = h->c;
    CK(h, ebc::launch_current_f(c, h->d_scalar));
    double v = 0;
    CK(h, cudaMemcpyAsync(&v, h->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(h, cudaStreamSynchronize(c.stream));
    *out_f = v;
    return EBC_OK;
}

ebc_status ebc_gains(ebc_t h, const int32_t *cand_idx, int64_t m, double *out_gain) {
    ebc::TraceRange trace_("ebc_gains");
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (m < 0) return fail(h, EBC_EINVAL, "ebc_gains: m < 0");
    if (!cand_idx && m != c.n) return fail(h, EBC_EINVAL, "ebc_gains: cand_idx NULL requires m == n");
    if (m == 0) return EBC_OK;
    if (!out_gain) return fail(h, EBC_EINVAL, "ebc_gains: out_gain is NULL");
    // process in batches of at most n candidates (the partial buffer holds nch x n)
    for (int64_t j0 = 0; j0 < m; j0 += c.n) {
        int64_t mb = std::min<int64_t>(c.n, m - j0);
        k_sanitize<<<(unsigned)((mb + 255) / 256), 256, 0, c.stream>>>(cand_idx ? cand_idx + j0 : nullptr, mb, c.n,
                                                                       c.cand_buf, c.st);
        CK(h, cudaGetLastError());
        h->prof.p.launches += 1;
        int nch = h->nch;
        // all candidates in index order: no gather, the candidate is the row
        const int *cl = cand_idx ? c.cand_buf : nullptr;
        if (c.prec == EBC_FP32) {
            CK(h, launch(h, PK_BULK, 1, [&] { return ebc::launch_gains_fp32(c, c.cand_buf, mb, false, h->ch, h->nch); }));
        } else if (c.prec == EBC_FP8E4M3) {
            CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc8(c, false); }));
            CK(h, launch(h, PK_BULK, 2, [&] { return ebc::launch_gains_tc8(c, cl, mb, &nch); }));
        } else {
            CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc(c, false); }));
            CK(h, launch(h, PK_BULK, 2, [&] { return ebc::launch_gains_tc(c, cl, mb, false, &nch); }));
        }
        h->prof.p.bulk_evals += mb * c.n;
        CK(h, launch(h, -1, 2, [&] {
               return ebc::launch_reduce_select(c, mb, nch, c.cand_buf, false, out_gain + j0, h->nblk);
           }));
        k_zero_masked<<<(unsigned)((mb + 255) / 256), 256, 0, c.stream>>>(c.cand_buf, mb, out_gain + j0);
        CK(h, cudaGetLastError());
    }
    return EBC_OK;
}

ebc_status ebc_gains_host(ebc_t h, const int32_t *cand_idx, int64_t m, double *out_gain) {
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (m < 0 || (!cand_idx && m != c.n) || (m > 0 && !out_gain)) return fail(h, EBC_EINVAL, "ebc_gains_host: bad arguments");
    if (m == 0) return EBC_OK;
    if (cand_idx)
        for (int64_t j = 0; j < m; ++j)
            if (cand_idx[j] < 0 || (int64_t)cand_idx[j] >= c.n) return fail(h, EBC_EINDEX, "ebc_gains_host: index outside [0, n)");
    int32_t *d_c = nullptr;
    double *d_g = nullptr;
    if (cand_idx) CK(h, dalloc(&d_c, m, c));
    cudaError_t e = dalloc(&d_g, m, c);
    if (e != cudaSuccess) {
        ebc::pool_free(d_c, c.stream);
        return cuda_fail(h, e, "ebc_gains_host: allocation");
    }
    ebc_status s = EBC_OK;
    if (cand_idx) e = cudaMemcpyAsync(d_c, cand_idx, sizeof(int32_t) * m, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) s = ebc_gains(h, d_c, m, d_g);
    if (e == cudaSuccess && s == EBC_OK)
        e = cudaMemcpyAsync(out_gain, d_g, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && s == EBC_OK) e = cudaStreamSynchronize(c.stream);
    ebc::pool_free(d_g, c.stream);
    ebc::pool_free(d_c, c.stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "ebc_gains_host");
    if (s != EBC_OK) return s;
    return ebc_sync(h);
}

ebc_status ebc_gain_bounds(ebc_t h, const int32_t *cand_idx, int64_t m, double *out_ub) {
    ebc::TraceRange trace_("ebc_gain_bounds");
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (m < 0) return fail(h, EBC_EINVAL, "ebc_gain_bounds: m < 0");
    if (!cand_idx && m != c.n) return fail(h, EBC_EINVAL, "ebc_gain_bounds: cand_idx NULL requires m == n");
    if (m == 0) return EBC_OK;
    if (!out_ub) return fail(h, EBC_EINVAL, "ebc_gain_bounds: out_ub is NULL");
    const double scale = 1.0 + bulk_eta(c);
    for (int64_t j0 = 0; j0 < m; j0 += c.n) {
        const int64_t mb = std::min<int64_t>(c.n, m - j0);
        k_sanitize<<<(unsigned)((mb + 255) / 256), 256, 0, c.stream>>>(cand_idx ? cand_idx + j0 : nullptr, mb, c.n,
                                                                       c.cand_buf, c.st);
        CK(h, cudaGetLastError());
        h->prof.p.launches += 1;
        int nch = h->nch;
        const int *cl = cand_idx ? c.cand_buf : nullptr;
        if (c.prec == EBC_FP32) {
            CK(h, launch(h, PK_BULK, 1, [&] { return ebc::launch_gains_fp32(c, c.cand_buf, mb, true, h->ch, h->nch); }));
        } else {  // upper-bound mode of the 16-bit kernel (FP8 handles use their BF16 copy)
            CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc(c, true); }));
            CK(h, launch(h, PK_BULK, 2, [&] { return ebc::launch_gains_tc(c, cl, mb, true, &nch); }));
        }
        h->prof.p.bulk_evals += mb * c.n;
        CK(h, launch(h, -1, 2, [&] {
               return ebc::launch_reduce_select(c, mb, nch, c.cand_buf, false, out_ub + j0, h->nblk);
           }));
        k_zero_masked<<<(unsigned)((mb + 255) / 256), 256, 0, c.stream>>>(c.cand_buf, mb, out_ub + j0);
        CK(h, cudaGetLastError());
        k_scale<<<(unsigned)((mb + 255) / 256), 256, 0, c.stream>>>(out_ub + j0, mb, scale);
        CK(h, cudaGetLastError());
        h->prof.p.launches += 2;
    }
    return EBC_OK;
}

ebc_status ebc_gain_bounds_host(ebc_t h, const int32_t *cand_idx, int64_t m, double *out_ub) {
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (m < 0 || (!cand_idx && m != c.n) || (m > 0 && !out_ub)) return fail(h, EBC_EINVAL, "ebc_gain_bounds_host: bad arguments");
    if (m == 0) return EBC_OK;
    if (cand_idx)
        for (int64_t j = 0; j < m; ++j)
            if (cand_idx[j] < 0 || (int64_t)cand_idx[j] >= c.n) return fail(h, EBC_EINDEX, "ebc_gain_bounds_host: index outside [0, n)");
    int32_t *d_c = nullptr;
    double *d_u = nullptr;
    if (cand_idx) CK(h, dalloc(&d_c, m, c));
    cudaError_t e = dalloc(&d_u, m, c);
    if (e != cudaSuccess) {
        ebc::pool_free(d_c, c.stream);
        return cuda_fail(h, e, "ebc_gain_bounds_host: allocation");
    }
    ebc_status st = EBC_OK;
    if (cand_idx) e = cudaMemcpyAsync(d_c, cand_idx, sizeof(int32_t) * m, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) st = ebc_gain_bounds(h, d_c, m, d_u);
    if (e == cudaSuccess && st == EBC_OK)
        e = cudaMemcpyAsync(out_ub, d_u, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && st == EBC_OK) e = cudaStreamSynchronize(c.stream);
    ebc::pool_free(d_u, c.stream);
    ebc::pool_free(d_c, c.stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "ebc_gain_bounds_host");
    if (st != EBC_OK) return st;
    return ebc_sync(h);
}

ebc_status ebc_eval_sets(ebc_t h, const int32_t *csr_idx, const int64_t *csr_off, int64_t l, double *out_f) {
    ebc::TraceRange trace_("ebc_eval_sets");
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (l < 0) return fail(h, EBC_EINVAL, "ebc_eval_sets: l < 0");
    if (l == 0) return EBC_OK;
    if (!csr_off || !out_f) return fail(h, EBC_EINVAL, "ebc_eval_sets: NULL argument");
    if (c.prec != EBC_FP32) {
        // tensor cores, planned on the device.  The member buffers must hold
        // csr_off[l] members: a reservation covering l sets says how many;
        // without one the count is read from the device (8 bytes, one wait).
        int64_t members = c.tc.res_members;
        if (l > c.tc.res_sets || members <= 0) {
            CK(h, cudaMemcpyAsync(c.h_err, csr_off + l, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
            CK(h, cudaStreamSynchronize(c.stream));
            memcpy(&members, c.h_err, sizeof(int64_t));
            if (members < 0) return fail(h, EBC_EINVAL, "ebc_eval_sets: csr_off[l] < 0");
            if (members > 0 && !csr_idx) return fail(h, EBC_EINVAL, "ebc_eval_sets: csr_idx is NULL");
        }
        const int64_t rows = c.tc.n_pad / 256 * 8;  // (point unit, epilogue warp)
        ebc_status s = ensure_set_part(h, rows * std::min<int64_t>(l, std::max<int64_t>(128, ((int64_t)1 << 24) / rows)));
        if (s) return s;
        int64_t nl = 0;
        CK(h, launch(h, PK_EVAL, 0, [&] { return ebc::launch_eval_sets_tc(c, csr_idx, csr_off, l, members, out_f, &nl); }));
        h->prof.p.launches += nl;
        h->prof.p.eval_launches += nl;
        return EBC_OK;
    }
    CK(h, cudaMemsetAsync(h->d_bad, 0, sizeof(int), c.stream));
    k_check_csr<<<(unsigned)((l + 255) / 256), 256, 0, c.stream>>>(csr_off, l, c.st, h->d_bad);
    CK(h, cudaGetLastError());
    int64_t ntiles = (c.n + 127) / 128;
    int64_t want = std::min<int64_t>(ntiles * l, std::max<int64_t>(ntiles * 64, (int64_t)1 << 24));
    ebc_status s = ensure_set_part(h, want);
    if (s) return s;
    h->prof.p.launches += 1;
    CK(h, launch(h, PK_EVAL, 2, [&] { return ebc::launch_eval_sets_fp32(c, csr_idx, csr_off, l, out_f, h->d_bad); }));
    return EBC_OK;
}

ebc_status ebc_reserve_sets(ebc_t h, int64_t max_sets, int64_t max_members) {
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (max_sets < 0 || max_members < 0) return fail(h, EBC_EINVAL, "ebc_reserve_sets: negative size");
    if (c.prec == EBC_FP32 || c.tc.prec < 0)
        return fail(h, EBC_EINVAL, "ebc_reserve_sets: needs a tensor-core precision (ebc_set_precision)");
    if (max_sets > 0) {
        const int64_t rows = c.tc.n_pad / 256 * 8;
        ebc_status s = ensure_set_part(
            h, rows * std::min<int64_t>(max_sets, std::max<int64_t>(128, ((int64_t)1 << 24) / rows)));
        if (s) return s;
        CK(h, ebc::tc_sets_reserve(c, max_sets, max_members));
    }
    c.tc.res_sets = max_sets;
    c.tc.res_members = max_members;
    return EBC_OK;
}

ebc_status ebc_eval_sets_host(ebc_t h, const int32_t *csr_idx, const int64_t *csr_off, int64_t l, double *out_f) {
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (l < 0 || (l > 0 && (!csr_off || !out_f))) return fail(h, EBC_EINVAL, "ebc_eval_sets_host: bad arguments");
    if (l == 0) return EBC_OK;
    if (csr_off[0] != 0) return fail(h, EBC_EINVAL, "ebc_eval_sets_host: csr_off[0] != 0");
    for (int64_t j = 0; j < l; ++j)
        if (csr_off[j + 1] < csr_off[j]) return fail(h, EBC_EINVAL, "ebc_eval_sets_host: offsets decrease");
    int64_t nnz = csr_off[l];
    if (nnz > 0 && !csr_idx) return fail(h, EBC_EINVAL, "ebc_eval_sets_host: csr_idx is NULL");
    for (int64_t p = 0; p < nnz; ++p)
        if (csr_idx[p] < 0 || (int64_t)csr_idx[p] >= c.n) return fail(h, EBC_EINDEX, "ebc_eval_sets_host: index outside [0, n)");
    int32_t *d_i = nullptr;
    int64_t *d_o = nullptr;
    double *d_f = nullptr;
    cudaError_t e = dalloc(&d_i, nnz, c);
    if (e == cudaSuccess) e = dalloc(&d_o, l + 1, c);
    if (e == cudaSuccess) e = dalloc(&d_f, l, c);
    ebc_status s = EBC_OK;
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(d_i, csr_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_o, csr_off, sizeof(int64_t) * (l + 1), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) s = ebc_eval_sets(h, d_i, d_o, l, d_f);
    if (e == cudaSuccess && s == EBC_OK) e = cudaMemcpyAsync(out_f, d_f, sizeof(double) * l, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && s == EBC_OK) e = cudaStreamSynchronize(c.stream);
    ebc::pool_free(d_i, c.stream);
    ebc::pool_free(d_o, c.stream);
    ebc::pool_free(d_f, c.stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "ebc_eval_sets_host");
    if (s != EBC_OK) return s;
    return ebc_sync(h);
}

static ebc_status greedy_round(ebc_t h, int32_t *out_idx_base, double *out_f_base) {
    ebc::Ctx &c = h->c;
    const int K = c.refine_k;
    const double eta = bulk_eta(c);
    int nch = h->nch;
    ebc::Ctx::Sel &S = c.cert;
    const bool fp8 = c.prec == EBC_FP8E4M3;
    const bool lazy = (c.lazy && c.prec != EBC_FP32) || fp8;
    if (fp8) {
        // FP8 bulk upper bounds of every candidate tighten the stale bounds;
        // the lazy round below certifies with BF16 bounds of the candidates
        // that can still win
        int nch8 = 1;
        CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc8(c, true); }));
        CK(h, launch(h, PK_BULK, 1, [&] { return ebc::launch_gains_tc8(c, nullptr, c.n, &nch8); }));
        h->prof.p.bulk_evals += (c.n - h->nsel) * c.n;
        CK(h, launch(h, -1, 2, [&] {
               cudaError_t e = ebc::launch_reduce_select(c, c.n, nch8, nullptr, true, nullptr, h->nblk);
               return e != cudaSuccess ? e : ebc::launch_lazy_from_full(c, eta);
           }));
    }
    if (lazy) {
        // lazy round (k_lazy.cu): certified lower bound from the largest stale
        // bounds, then bulk bounds only for candidates whose stale bound reaches it
        const int KP = 8;  // one pass of the few-candidate bound kernel
        CK(h, launch(h, -1, 2, [&] { return ebc::launch_lazy_preselect(c, h->nblk, KP); }));
        CK(h, launch(h, PK_REFINE, 1, [&] {
               return ebc::launch_bounds_list(c, c.top_idx, &c.st->top_count, KP, S.part_lo, S.part_hi, S.chunk,
                                              S.nchunks);
           }));
        CK(h, launch(h, -1, 3, [&] {
               cudaError_t e = ebc::launch_fold_bounds(c, S.part_lo, S.part_hi, &c.st->top_count, KP, S.top_lo, S.top_hi);
               if (e == cudaSuccess) e = ebc::launch_lazy_threshold(c);
               return e != cudaSuccess ? e : ebc::launch_lazy_build(c);
           }));
        CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc(c, true); }));
        CK(h, launch(h, PK_LIST, 2, [&] { return ebc::launch_gains_tc_list(c, c.lazy_idx, &c.st->list_m, c.n); }));
        CK(h, launch(h, -1, 1, [&] { return ebc::launch_lazy_select(c, eta, h->nblk); }));
    } else {
        if (c.prec == EBC_FP32) {
            CK(h, launch(h, PK_BULK, 1, [&] { return ebc::launch_gains_fp32(c, nullptr, c.n, true, h->ch, h->nch); }));
        } else {
            CK(h, launch(h, -1, 1, [&] { return ebc::launch_prep_tc(c, true); }));
            CK(h, launch(h, PK_BULK, 1, [&] { return ebc::launch_gains_tc(c, nullptr, c.n, true, &nch); }));
        }
        h->prof.p.bulk_evals += (c.n - h->nsel) * c.n;
        CK(h, launch(h, -1, 1, [&] { return ebc::launch_reduce_select(c, c.n, nch, nullptr, true, nullptr, h->nblk); }));
    }
    return ebc::round_certify(h, out_idx_base, out_f_base, lazy);
}

}  // extern "C"

// The certified pick of a round whose bulk bounds are in place (per-block
// top lists from the reduction of the bulk partials, or the lazy list's),
// then the m_v update.
ebc_status ebc::round_certify(ebc_t h, int32_t *out_idx_base, double *out_f_base, bool lazy) {
    ebc::Ctx &c = h->c;
    const int K = c.refine_k;
    const double eta = bulk_eta(c);
    ebc::Ctx::Sel &S = c.cert;
    CK(h, launch(h, -1, 1, [&] { return ebc::launch_merge_top(c, h->nblk, K, eta); }));
    // level 1: bounds for the top list, then for the escalated candidates
    const int64_t esc_off = (int64_t)ebc::kMaxRefineK * S.nchunks;
    CK(h, launch(h, PK_REFINE, 1, [&] {
           return ebc::launch_bounds_list(c, c.top_idx, &c.st->top_count, K, S.part_lo, S.part_hi, S.chunk, S.nchunks);
       }));
    CK(h, launch(h, -1, 3, [&] {
           cudaError_t e = ebc::launch_fold_bounds(c, S.part_lo, S.part_hi, &c.st->top_count, K, S.top_lo, S.top_hi);
           if (e == cudaSuccess) e = ebc::launch_decide_top(c, eta);
           if (e != cudaSuccess) return e;
           return lazy ? ebc::launch_lazy_collect(c, eta) : ebc::launch_collect_escalation(c, eta);
       }));
    CK(h, launch(h, PK_REFINE, 2, [&] {
           cudaError_t e = ebc::launch_bounds_list(c, c.esc_idx, &c.st->esc_count, S.cap, S.part_lo + esc_off,
                                                   S.part_hi + esc_off, S.chunk, S.nchunks);
           return e != cudaSuccess ? e : ebc::launch_refine_overflow(c, c.esc_idx, &c.st->esc_count, S.cap, c.esc_exact);
       }));
    CK(h, launch(h, -1, 2, [&] {
           cudaError_t e = ebc::launch_fold_bounds(c, S.part_lo + esc_off, S.part_hi + esc_off, &c.st->esc_count,
                                                   S.cap, S.esc_lo, S.esc_hi);
           return e != cudaSuccess ? e : ebc::launch_decide_contenders(c);
       }));
    // level 2: exact gains of the contenders only
    CK(h, launch(h, PK_REFINE, 1, [&] {
           return ebc::launch_exact_list(c, S.ctd_idx, &c.st->ctd_count, ebc::kMaxRefineK + S.cap, S.ctd_part,
                                         S.chunk, S.nchunks);
       }));
    CK(h, launch(h, -1, 2, [&] {
           cudaError_t e = ebc::launch_commit_pick(c, out_idx_base, out_f_base);
           return e != cudaSuccess ? e : ebc::launch_update(c);
       }));
    return EBC_OK;
}

extern "C" {

// Capture one Greedy round (outputs into the handle's by-round buffers) as a
// graph.  A capture failure leaves direct launches in use.
static ebc_status capture_round(ebc_t h) {
    ebc::Ctx &c = h->c;
    if (!h->g_idx) {
        cudaError_t e = dalloc(&h->g_idx, c.n, c);
        if (e == cudaSuccess) e = dalloc(&h->g_f, c.n, c);
        if (e != cudaSuccess) {  // both or neither
            ebc::pool_free(h->g_idx, c.stream);
            h->g_idx = nullptr;
            h->g_f = nullptr;
            CK(h, e);
        }
    }
    if (h->round_exec) {
        cudaGraphExecDestroy(h->round_exec);
        h->round_exec = nullptr;
    }
    const int64_t launches0 = h->prof.p.launches;
    const int64_t bulk0 = h->prof.p.bulk_launches, evals0 = h->prof.p.bulk_evals, ref0 = h->prof.p.refine_launches;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        h->graphs = false;
        return EBC_OK;
    }
    ebc_status s = greedy_round(h, h->g_idx, h->g_f);
    cudaError_t e = cudaStreamEndCapture(c.stream, &g);
    h->round_launches = h->prof.p.launches - launches0;
    h->prof.p.launches = launches0;
    h->prof.p.bulk_launches = bulk0;
    h->prof.p.bulk_evals = evals0;
    h->prof.p.refine_launches = ref0;
    if (s != EBC_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        h->graphs = false;  // keep direct launches for this handle
        return EBC_OK;
    }
    e = cudaGraphInstantiate(&h->round_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->round_exec = nullptr;
        h->graphs = false;
        return EBC_OK;
    }
    h->round_stream = c.stream;
    h->prec_at_capture = (int)c.prec;
    h->ctas_at_capture = c.max_ctas;
    h->lazy_at_capture = c.lazy ? 1 : 0;
    h->wait_at_capture = ebc::wait_limit_ns();
    return EBC_OK;
}

ebc_status ebc_greedy(ebc_t h, int32_t k, int32_t *out_idx, double *out_f) {
    ebc::TraceRange trace_("ebc_greedy");
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (k < 0) return fail(h, EBC_EINVAL, "ebc_greedy: k < 0");
    if ((int64_t)k > c.n - h->nsel) return fail(h, EBC_EINVAL, "ebc_greedy: k exceeds the unselected points");
    if (k == 0) return EBC_OK;
    if (!out_idx || !out_f) return fail(h, EBC_EINVAL, "ebc_greedy: NULL output");
    // k_commit writes out[round] with round counted since reset: shift the base
    int32_t *ib = out_idx - h->nsel;
    double *fb = out_f - h->nsel;
    int32_t t = 0;
    // graph replay: only on a capturable stream, without per-launch events,
    // after one direct round has set every kernel attribute
    const bool use_graph = h->graphs && !h->prof.on && c.stream != nullptr;
    if (use_graph && (!h->round_exec || h->round_stream != c.stream || h->prec_at_capture != (int)c.prec ||
                      h->ctas_at_capture != c.max_ctas || h->lazy_at_capture != (c.lazy ? 1 : 0) ||
                      h->wait_at_capture != ebc::wait_limit_ns())) {
        if (!h->attrs_ready) {
            ebc_status s = greedy_round(h, ib, fb);
            if (s) return s;
            h->nsel += 1;
            h->attrs_ready = true;
            t = 1;
        }
        if (t < k) {
            ebc_status s = capture_round(h);
            if (s) return s;
        }
    }
    if (use_graph && h->round_exec) {
        const int64_t first = h->nsel;
        for (; t < k; ++t) {
            h->prof.p.bulk_evals += (c.n - h->nsel) * c.n;
            h->prof.p.launches += h->round_launches;
            h->prof.p.bulk_launches += 1;
            CK(h, cudaGraphLaunch(h->round_exec, c.stream));
            h->nsel += 1;
        }
        const int64_t cnt = h->nsel - first;
        if (cnt > 0) {
            CK(h, cudaMemcpyAsync(ib + first, h->g_idx + first, sizeof(int32_t) * cnt, cudaMemcpyDeviceToDevice,
                                  c.stream));
            CK(h, cudaMemcpyAsync(fb + first, h->g_f + first, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, c.stream));
        }
        return EBC_OK;
    }
    for (; t < k; ++t) {
        ebc_status s = greedy_round(h, ib, fb);
        if (s) return s;
        h->nsel += 1;
        h->attrs_ready = true;
    }
    return EBC_OK;
}

ebc_status ebc_set_max_ctas(ebc_t h, int32_t max_ctas) {
    if (check_handle(h) || max_ctas < 0) return EBC_EINVAL;
    h->c.max_ctas = max_ctas;
    return EBC_OK;
}

ebc_status ebc_set_kblocked(ebc_t h, int32_t on) {
    if (check_handle(h)) return EBC_EINVAL;
    h->c.force_kb = on != 0;
    if (h->round_exec) {  // rounds captured with the other kernel
        cudaGraphExecDestroy(h->round_exec);
        h->round_exec = nullptr;
    }
    h->attrs_ready = false;  // one direct round sets the kernel's attributes before a capture
    return EBC_OK;
}

ebc_status ebc_set_graphs(ebc_t h, int32_t on) {
    if (check_handle(h)) return EBC_EINVAL;
    h->graphs = on != 0;
    return EBC_OK;
}

ebc_status ebc_greedy_host(ebc_t h, int32_t k, int32_t *out_idx, double *out_f) {
    if (check_handle(h)) return EBC_EINVAL;
    ebc::Ctx &c = h->c;
    if (k < 0 || (int64_t)k > c.n - h->nsel) return fail(h, EBC_EINVAL, "ebc_greedy_host: bad k");
    if (k == 0) return EBC_OK;
    if (!out_idx || !out_f) return fail(h, EBC_EINVAL, "ebc_greedy_host: NULL output");
    int32_t *d_i = nullptr;
    double *d_f = nullptr;
    cudaError_t e = dalloc(&d_i, k, c);
    if (e == cudaSuccess) e = dalloc(&d_f, k, c);
    ebc_status s = EBC_OK;
    if (e == cudaSuccess) s = ebc_greedy(h, k, d_i, d_f);
    if (e == cudaSuccess && s == EBC_OK) e = cudaMemcpyAsync(out_idx, d_i, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && s == EBC_OK) e = cudaMemcpyAsync(out_f, d_f, sizeof(double) * k, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && s == EBC_OK) e = cudaStreamSynchronize(c.stream);
    ebc::pool_free(d_i, c.stream);
    ebc::pool_free(d_f, c.stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "ebc_greedy_host");
    if (s != EBC_OK) return s;
    return ebc_sync(h);
}

}  // extern "C"
