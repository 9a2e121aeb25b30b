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

// Block-wide minimum index (the value travels with it; INT_MAX = none).
__device__ __forceinline__ void block_min_index(double &v, int &i) {
    __shared__ double sv[32];
    __shared__ int si[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (oi < i) {
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
        v = lane < nw ? sv[lane] : -1.0;
        i = lane < nw ? si[lane] : INT_MAX;
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, v, o);
            int oi = __shfl_xor_sync(0xffffffffu, i, o);
            if (oi < i) {
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

// ---------------------------------------------------------------------------
// Top-L selection (L <= 32) in the order above, with per-warp sorted lists:
// lane r of a warp holds the warp's r-th best entry so far.  A batch of 32
// entries is compared with the list's last entry (the threshold); each entry
// that beats it is inserted (ballot gives its rank, the lanes below it shift
// down by one shuffle).  The block's lists are then merged into warp 0's the
// same way.  The result is the exact top L (the order is a strict total
// order on distinct indices), whatever the order of the scan.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool wl_insert(double &lv, int &li, double nv, int ni, int L) {
    const int lane = threadIdx.x & 31;
    const double tv = __shfl_sync(0xffffffffu, lv, L - 1);
    const int ti = __shfl_sync(0xffffffffu, li, L - 1);
    if (!better(nv, ni, tv, ti)) return false;  // warp-uniform
    const bool stays = lane < L && better(lv, li, nv, ni);
    const int p = __popc(__ballot_sync(0xffffffffu, stays));
    const double uv = __shfl_up_sync(0xffffffffu, lv, 1);
    const int ui = __shfl_up_sync(0xffffffffu, li, 1);
    if (lane > p) {
        lv = uv;
        li = ui;
    }
    if (lane == p) {
        lv = nv;
        li = ni;
    }
    return true;
}

// Extract the `cnt` (<= 32) best entries of [beg, end) of (val[], idx[])
// (index = position when idx is null); entries with value < 0 are never
// taken.  out_v / out_i[r] for r < cnt, (-1, -1) where there are fewer.
// blockDim.x must be a multiple of 32 (at most 1024).
__device__ __forceinline__ void block_topk(const double *__restrict__ val, const int *__restrict__ idx, int64_t beg,
                                           int64_t end, int cnt, double *out_v, int *out_i) {
    __shared__ double wv[32][32];
    __shared__ int wi[32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int L = cnt;
    double lv = -DBL_MAX;
    int li = INT_MAX;
    for (int64_t base = beg + (int64_t)warp * 32; base < end; base += (int64_t)nw * 32) {
        const int64_t j = base + lane;
        double x = -1.0;
        int xi = INT_MAX;
        if (j < end) {
            x = val[j];
            xi = idx ? idx[j] : (int)j;
        }
        const double tv = __shfl_sync(0xffffffffu, lv, L - 1);
        const int ti = __shfl_sync(0xffffffffu, li, L - 1);
        unsigned mask = __ballot_sync(0xffffffffu, x >= 0.0 && better(x, xi, tv, ti));
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const double nv = __shfl_sync(0xffffffffu, x, src);
            const int ni = __shfl_sync(0xffffffffu, xi, src);
            wl_insert(lv, li, nv, ni, L);
        }
    }
    __syncthreads();
    wv[warp][lane] = lv;
    wi[warp][lane] = li;
    __syncthreads();
    if (warp == 0) {
        for (int w = 1; w < nw; ++w)
            for (int r = 0; r < L; ++r) {
                const double nv = wv[w][r];
                const int ni = wi[w][r];
                // lists are sorted: once an entry misses, the rest of its list does too
                if (ni == INT_MAX || !wl_insert(lv, li, nv, ni, L)) break;
            }
        if (lane < L) {
            out_v[lane] = li == INT_MAX ? -1.0 : lv;
            out_i[lane] = li == INT_MAX ? -1 : li;
        }
    }
    __syncthreads();
}

}  // namespace ebc
