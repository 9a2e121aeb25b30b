// ebc_eval_sets_noalloc: multi-set evaluation that allocates nothing.
//
// Some callers may not allocate device memory once they are running: a
// process-control loop with a fixed latency budget (cudaMalloc and cudaFree
// can synchronise the device and take an unbounded time), or a host program
// whose device memory is entirely owned by another allocator.  For them this
// file provides one entry point that needs no handle and no allocation: the
// caller passes V, the CSR sets and the output, all in device memory, and the
// per-tile partial sums live in a file-scope static device array.
//
// The scratch array is 8 MiB per GPU that loads the library and stays
// allocated until the process exits.  Every call shares it and it keeps the
// last call's contents; the error words are cleared at the start of each
// call, the partials are fully overwritten.  Calls whose work overlaps on
// the GPU (on different streams, or from several host threads) race on the
// array and must not be issued.
//
// The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current and caches it; that first
// call should come before any stream capture.
//
// The arithmetic is the FP32 direct-distance evaluation of the handle-based
// ebc_eval_sets (work matrix rows of Sec. 4.2 reduced on the fly), with
// ||v||^2 formed per point inside the kernel instead of read from the
// handle's resident norms.
#include <math.h>
#include <string.h>

#include <mutex>

#include "ebc_internal.cuh"

namespace ebc {
namespace {

constexpr int NA_T = 128;                              // points per block
constexpr int NA_SG = 8;                               // sets per block
constexpr int NA_DC = 256;                             // member stage depth (dims)
constexpr int64_t kScratchDoubles = (int64_t)1 << 20;  // 8 MiB of partials
constexpr int kMaxDevices = 64;

// [0, kScratchDoubles): per-(point tile, set) partial sums; then two error words.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles + 2];

double *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Offsets must start at 0 and never decrease; a NULL member list is only
// valid when every set is empty.  Either failure sets err[1], after which the
// evaluation kernels read no member.
__global__ void k_na_check_csr(const int32_t *__restrict__ idx, const int64_t *__restrict__ off, int64_t l,
                               int *__restrict__ err) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if ((j == 0 && (off[0] != 0 || (idx == nullptr && off[l] != 0))) || (j < l && off[j + 1] < off[j])) {
        atomicCAS(&err[0], 0, (int)EBC_EINVAL);
        atomicExch(&err[1], 1);
    }
}

// One thread per point; ||v||^2 in FP64 (index order) rounded to FP32; for
// each set of the block's group the FP32 direct distance to every member,
// four members at a time from a shared [dim][4] stage; max(0, ||v||^2 - min)
// summed over the block in FP64.
__global__ void __launch_bounds__(NA_T) k_na_eval_sets(const float *__restrict__ V, int64_t n, int d,
                                                       const int32_t *__restrict__ idx,
                                                       const int64_t *__restrict__ off, int64_t l,
                                                       double *__restrict__ part, int *__restrict__ err) {
    if (err[1]) return;  // offsets failed validation: read nothing
    __shared__ __align__(16) float stage[NA_DC * 4];
    __shared__ double red[NA_T / 32];
    const int t = threadIdx.x;
    const int64_t tile = blockIdx.x;
    const int64_t v = tile * NA_T + t;
    const bool vok = v < n;
    float nv = 0.f;
    if (vok) {
        double acc = 0.0;
        for (int i = 0; i < d; ++i) {
            double x = (double)V[v * d + i];
            acc = __dadd_rn(acc, __dmul_rn(x, x));
        }
        nv = (float)acc;
    }
    const int dstage = min(d, NA_DC);
    const int64_t j0 = (int64_t)blockIdx.y * NA_SG;
    for (int64_t j = j0; j < min(j0 + NA_SG, l); ++j) {
        const int64_t mb = off[j], me = off[j + 1];
        float dmin = INFINITY;
        for (int64_t s0 = mb; s0 < me; s0 += 4) {
            int mi[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t p = s0 + u;
                int x = p < me ? idx[p] : -1;
                if (p < me && (x < 0 || (int64_t)x >= n)) {
                    if (t == 0) atomicCAS(&err[0], 0, (int)EBC_EINDEX);
                    x = -1;
                }
                mi[u] = x;
            }
            float dist[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k0 = 0; k0 < d; k0 += dstage) {
                const int kn = min(dstage, d - k0);
                __syncthreads();
                for (int e = t; e < kn * 4; e += NA_T) {
                    int i = e >> 2, u = e & 3;
                    stage[i * 4 + u] = mi[u] >= 0 ? V[(int64_t)mi[u] * d + k0 + i] : 0.f;
                }
                __syncthreads();
                if (vok) {
                    for (int i = 0; i < kn; ++i) {
                        const float x = V[v * d + k0 + i];
                        const float4 s4 = reinterpret_cast<const float4 *>(stage)[i];
                        float d0 = x - s4.x, d1 = x - s4.y, d2 = x - s4.z, d3 = x - s4.w;
                        dist[0] = fmaf(d0, d0, dist[0]);
                        dist[1] = fmaf(d1, d1, dist[1]);
                        dist[2] = fmaf(d2, d2, dist[2]);
                        dist[3] = fmaf(d3, d3, dist[3]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (mi[u] >= 0) dmin = fminf(dmin, dist[u]);
        }
        double val = vok ? (double)fmaxf(0.f, nv - dmin) : 0.0;
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
        __syncthreads();
        if ((t & 31) == 0) red[t >> 5] = val;
        __syncthreads();
        if (t == 0) {
            double s = 0.0;
            for (int w = 0; w < NA_T / 32; ++w) s += red[w];
            part[tile * l + j] = s;
        }
    }
}

__global__ void k_na_finalize(const double *__restrict__ part, int64_t ntiles, int64_t lb, int64_t j0,
                              double inv_n, double *__restrict__ out_f) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= lb) return;
    double s = 0.0;
    for (int64_t q = 0; q < ntiles; ++q) s += part[q * lb + j];
    out_f[j0 + j] = s * inv_n;
}

thread_local char g_na_error[256];

ebc_status na_fail(ebc_status s, const char *msg) {
    strncpy(g_na_error, msg, sizeof g_na_error - 1);
    g_na_error[sizeof g_na_error - 1] = 0;
    return s;
}

}  // namespace
}  // namespace ebc

extern "C" const char *ebc_noalloc_last_error(void) { return ebc::g_na_error; }

extern "C" ebc_status ebc_eval_sets_noalloc(const float *V, int64_t n, int32_t d, const int32_t *csr_idx,
                                            const int64_t *csr_off, int64_t l, double *out_f, void *stream) {
    using namespace ebc;
    g_na_error[0] = 0;
    if (!V || n <= 0 || d <= 0 || d > 4096 || l < 0) return na_fail(EBC_EINVAL, "ebc_eval_sets_noalloc: bad V, n, d or l");
    if (n > (int64_t)INT32_MAX - 1) return na_fail(EBC_EINVAL, "ebc_eval_sets_noalloc: n exceeds int32 indexing");
    if (l == 0) return EBC_OK;
    if (!csr_off || !out_f) return na_fail(EBC_EINVAL, "ebc_eval_sets_noalloc: NULL csr_off or out_f");
    const int64_t ntiles = (n + NA_T - 1) / NA_T;
    if (ntiles > kScratchDoubles)
        return na_fail(EBC_EINVAL,
                       "ebc_eval_sets_noalloc: n exceeds the static scratch (at most 1048576 tiles of 128 points)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return na_fail(EBC_ENODEV, "ebc_eval_sets_noalloc: no usable CUDA device");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            // one-time set-up on this device (it is current): the array's address
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return na_fail(EBC_ECUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int *err = reinterpret_cast<int *>(scratch + kScratchDoubles);
    if (cudaMemsetAsync(err, 0, 2 * sizeof(int), st) != cudaSuccess)
        return na_fail(EBC_ECUDA, "ebc_eval_sets_noalloc: clearing the error words failed");
    k_na_check_csr<<<(unsigned)((l + 255) / 256), 256, 0, st>>>(csr_idx, csr_off, l, err);
    // sets per pass: the partials must fit the array and the set groups the
    // grid's y extent (at most 65,535 blocks)
    const int64_t batch = lmin(kScratchDoubles / ntiles, (int64_t)65535 * NA_SG);
    for (int64_t j0 = 0; j0 < l; j0 += batch) {
        const int64_t lb = lmin(batch, l - j0);
        dim3 grid((unsigned)ntiles, (unsigned)((lb + NA_SG - 1) / NA_SG));
        k_na_eval_sets<<<grid, NA_T, 0, st>>>(V, n, d, csr_idx, csr_off + j0, lb, scratch, err);
        k_na_finalize<<<(unsigned)((lb + 255) / 256), 256, 0, st>>>(scratch, ntiles, lb, j0, 1.0 / (double)n, out_f);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(EBC_ECUDA, cudaGetErrorString(e));
    int herr[2] = {0, 0};
    e = cudaMemcpyAsync(herr, err, sizeof herr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(EBC_ECUDA, cudaGetErrorString(e));
    if (herr[0] == EBC_EINDEX) return na_fail(EBC_EINDEX, "ebc_eval_sets_noalloc: index outside [0, n)");
    if (herr[0] != 0)
        return na_fail((ebc_status)herr[0],
                       "ebc_eval_sets_noalloc: offsets not non-decreasing from 0, or NULL csr_idx with members");
    return EBC_OK;
}
