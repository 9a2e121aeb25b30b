// Device helpers shared by the selection kernels: ordering of (gain, index)
// pairs (gain descending, index ascending) and a block-wide argmax.
#pragma once

#include <float.h>
#include <limits.h>

namespace ebc {

// ---------------------------------------------------------------------------
// Block-wide argmax in the order (value descending, index ascending).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool better(double va, int ia, double vb, int ib) {
    return va > vb || (va == vb && ia < ib);
}

__device__ __forceinline__ void block_best(double &v, int &i) {
    __shared__ double sv[32];
    __shared__ int si[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sv[w] = v;
        si[w] = i;
    }
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        v = lane < nw ? sv[lane] : -DBL_MAX;
        i = lane < nw ? si[lane] : INT_MAX;
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, v, o);
            int oi = __shfl_xor_sync(0xffffffffu, i, o);
            if (better(ov, oi, v, i)) {
                v = ov;
                i = oi;
            }
        }
        if (lane == 0) {
            sv[0] = v;
            si[0] = i;
        }
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
    __syncthreads();
}

// Extract the `cnt` best entries of the thread-strided range [beg, end) of
// (val[], idx[]) in order; entries with value < 0 are never taken.
__device__ __forceinline__ void block_topk(const double *__restrict__ val, const int *__restrict__ idx, int64_t beg, int64_t end,
                           int cnt, double *out_v, int *out_i) {
    double lastv = DBL_MAX;
    int lasti = -1;
    for (int r = 0; r < cnt; ++r) {
        double bv = -DBL_MAX;
        int bi = INT_MAX;
        for (int64_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
            double x = val[j];
            int xi = idx ? idx[j] : (int)j;
            if (x < 0.0) continue;
            if (!better(lastv, lasti, x, xi)) continue;  // already taken
            if (better(x, xi, bv, bi)) {
                bv = x;
                bi = xi;
            }
        }
        block_best(bv, bi);
        if (threadIdx.x == 0) {
            out_v[r] = bi == INT_MAX ? -1.0 : bv;
            out_i[r] = bi == INT_MAX ? -1 : bi;
        }
        lastv = bv;
        lasti = bi;
    }
}

}  // namespace ebc
