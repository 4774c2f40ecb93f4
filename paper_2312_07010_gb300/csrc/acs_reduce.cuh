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

// Sum a CSum over the threads of a block (<= 1024, any shape) in a fixed order; the
// result is valid in thread 0.  `scratch` needs 32 entries.
__device__ __forceinline__ CSum block_csum(CSum v, CSum* scratch) {
    for (int off = 16; off > 0; off >>= 1) v = cmerge(v, shfl_down(v, off));
    // linear thread index, so 2D blocks (32 x k) reduce correctly too
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nwarps = (int)((blockDim.x * blockDim.y + 31) >> 5);
    if ((tid & 31) == 0) scratch[tid >> 5] = v;
    __syncthreads();
    if (tid == 0)
        for (int w = 1; w < nwarps; ++w) v = cmerge(v, scratch[w]);
    return v;
}

// ---------------------------------------------------------------- FP32 states
// FP64 arithmetic runs at 1/57 of the FP32 rate on this GPU, so the FP32 path forms
// every term exactly with error-free FP32 transformations (the build uses
// -fmad=false, so nothing below is contracted): the difference q - p of two floats
// is an exact pair (TwoSum), its square and p^2 are exact pairs up to the
// negligible lo^2 term (TwoProduct via fma), and terms are accumulated into an
// unevaluated float pair (hi, lo).  All terms are non-negative, so the pair keeps
// about 2^-46 relative accuracy; every 32 points it is flushed into the FP64
// compensated sum.

struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return F2{s, (a - (s - bb)) + (b - bb)};
}

// acc += x (x >= 0 given as an unevaluated pair)
__device__ __forceinline__ void f2_acc(F2& acc, float xh, float xl) {
    const F2 t = two_sum(acc.hi, xh);
    acc.hi = t.hi;
    acc.lo = (acc.lo + t.lo) + xl;
}

// the exact square of (q - p), accumulated
__device__ __forceinline__ void link_sq(F2& acc, float q, float p) {
    const F2 d = two_sum(q, -p);
    const float sq = d.hi * d.hi;
    const float sql = __fmaf_rn(d.hi, d.hi, -sq) + 2.0f * d.hi * d.lo;
    f2_acc(acc, sq, sql);
}

__device__ __forceinline__ void flush(F2& acc, CSum& sum) {
    cadd(sum, (double)acc.hi);
    cadd(sum, (double)acc.lo);
    acc = F2{0.0f, 0.0f};
}

// the exact (p^2 - 1)^2 up to 2^-46, accumulated (the 1/4 is applied at the end)
__device__ __forceinline__ void bulk_sq(F2& acc, float p) {
    const float s2 = p * p;
    const float s2l = __fmaf_rn(p, p, -s2);
    const F2 w = two_sum(s2, -1.0f);
    const float wh = w.hi, wl = w.lo + s2l;
    const float q = wh * wh;
    const float ql = __fmaf_rn(wh, wh, -q) + 2.0f * wh * wl;
    f2_acc(acc, q, ql);
}

}  // namespace acs
