// acs_reduce.cuh -- compensated FP64 accumulation helpers shared by the
// reduction kernels (energy / maximum norm, adjoint gradient sums).
#pragma once

#include "acs_device.cuh"

namespace acs {

struct CSum {
    double s, c;
};

__device__ __forceinline__ void cadd(CSum& a, double x) {
    const double t = a.s + x;
    if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x; else a.c += (x - t) + a.s;
    a.s = t;
}

// a + b as an unevaluated pair (Knuth's TwoSum) merged with both compensations.
__device__ __forceinline__ CSum cmerge(CSum a, CSum b) {
    const double s = a.s + b.s;
    const double bb = s - a.s;
    const double err = (a.s - (s - bb)) + (b.s - bb);
    return CSum{s, (a.c + b.c) + err};
}

// NaN-sticky maximum.
__device__ __forceinline__ double nmax(double m, double v) {
    if (v != v || m != m) return v != v ? v : m;
    return v > m ? v : m;
}

__device__ __forceinline__ CSum shfl_down(CSum v, int off) {
    return CSum{__shfl_down_sync(0xffffffffu, v.s, off), __shfl_down_sync(0xffffffffu, v.c, off)};
}

// Sum a CSum over a block of blockDim.x threads (<= 1024) in a fixed order; the
// result is valid in thread 0.  `scratch` needs 32 entries.
__device__ __forceinline__ CSum block_csum(CSum v, CSum* scratch) {
    for (int off = 16; off > 0; off >>= 1) v = cmerge(v, shfl_down(v, off));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)((blockDim.x + 31) >> 5); ++w) v = cmerge(v, scratch[w]);
    return v;
}

}  // namespace acs
