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

}  // namespace ebc
