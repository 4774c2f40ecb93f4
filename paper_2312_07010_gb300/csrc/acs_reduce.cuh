// acs_reduce.cuh -- accumulation helpers shared by the reduction kernels (energy /
// maximum norm, phase volume, adjoint gradient sums): compensated FP64 sums within a
// thread, exact float-pair terms for FP32 states, and the exact fixed-point
// combination of partial sums across a block.
#pragma once

#include <climits>

#include "acs_device.cuh"
#include "f2ops.cuh"

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

// ---------------------------------------------------------------- exact combination
// FP64 arithmetic on this GPU has a small fraction of the FP32 issue rate and a long
// dependent latency, so trees of compensated FP64 merges (about six dependent
// operations per level) made a block's final combination cost more than its data
// (15 us for 16 K values).  Partial sums are combined exactly in 128-bit two's-
// complement fixed point instead: with E the largest biased exponent among the
// values, the unit is 2^(E - 1122), so every value is below 2^100 units and up to
// 2^26 of them sum without overflow; bits below 2^-99 of the largest value are
// dropped (truncated toward zero).  Integer addition is associative, so the result
// does not depend on the order of the tree, and the tree runs on the integer pipes.
// All block-level helpers below take blocks whose size is a multiple of 32 and must
// be called by every thread of the block.

struct Fix {
    unsigned long long lo;
    long long hi;
};

constexpr int kFixShift = 47;  // the largest value is below 2^(53 + kFixShift) units
constexpr int kFixUnit = 1075 + kFixShift;

__device__ __forceinline__ int dexp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7ff); }

__device__ __forceinline__ Fix fix_neg(Fix x) {
    x.lo = ~x.lo + 1ull;
    x.hi = ~x.hi + (x.lo == 0ull ? 1ll : 0ll);
    return x;
}

// v in units of 2^(E - kFixUnit), truncated toward zero; exact when v is a multiple of
// the unit.  Requires dexp(v) <= E + 27 (|v| below 2^127 units).
__device__ __forceinline__ Fix fix_of(double v, int E) {
    const long long bits = __double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7ff);
    unsigned long long m = (unsigned long long)bits & 0x000fffffffffffffull;
    if (e != 0) m |= 0x0010000000000000ull;
    const int sh = (e == 0 ? 1 : e) - E + kFixShift;  // v = m 2^(e - 1075) = m 2^sh units
    Fix r{0ull, 0ll};
    if (m == 0ull || sh <= -53) return r;
    if (sh < 0) {
        r.lo = m >> (-sh);
    } else if (sh == 0) {
        r.lo = m;
    } else if (sh < 64) {
        r.lo = m << sh;
        r.hi = (long long)(m >> (64 - sh));
    } else {
        r.hi = (long long)(m << (sh - 64));
    }
    return bits < 0 ? fix_neg(r) : r;
}

__device__ __forceinline__ Fix fix_add(Fix a, Fix b) {
    Fix r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ll : 0ll);
    return r;
}

__device__ __forceinline__ Fix fix_shfl_down(Fix a, int off) {
    return Fix{__shfl_down_sync(0xffffffffu, a.lo, off), __shfl_down_sync(0xffffffffu, a.hi, off)};
}

// 2^k as a double, -1074 <= k <= 1023 (below 2^-1022 as an exact product of two)
__device__ __forceinline__ double pow2i(int k) {
    if (k >= -1022) return __longlong_as_double((long long)(k + 1023) << 52);
    return __longlong_as_double((long long)(k + 200 + 1023) << 52) * __longlong_as_double((long long)(823) << 52);
}

// x (in whole units) as a double: the magnitude's two 64-bit halves combined by one
// fused multiply-add (at most two roundings).
__device__ __forceinline__ double fix_units(Fix x) {
    const bool neg = x.hi < 0;
    if (neg) x = fix_neg(x);
    const double d = __fma_rn((double)(unsigned long long)x.hi, 18446744073709551616.0, (double)x.lo);
    return neg ? -d : d;
}

// The unevaluated pair (s, c) of x units of 2^(E - kFixUnit): s = x rounded, c the
// exact integer remainder x - s rounded, so s + c carries about 106 bits.
__device__ __forceinline__ CSum fix_to_csum(Fix x, int E) {
    const double s_units = fix_units(x);
    const Fix rem = fix_add(x, fix_neg(fix_of(s_units, kFixUnit)));  // s_units is an integer
    const double c_units = fix_units(rem);
    const double scale = pow2i(E - kFixUnit);
    return CSum{s_units * scale, c_units * scale};
}

__device__ __forceinline__ int block_tid() { return threadIdx.y * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int block_nwarps() { return (int)((blockDim.x * blockDim.y + 31) >> 5); }

// Block-wide maximum (op 0) or bitwise or (op 1) of an int, returned to every thread.
template <int OP>
__device__ __forceinline__ int block_int_reduce(int v) {
    __shared__ int sw[32];
    __shared__ int res;
    v = OP == 0 ? __reduce_max_sync(0xffffffffu, v) : (int)__reduce_or_sync(0xffffffffu, (unsigned)v);
    const int tid = block_tid();
    if ((tid & 31) == 0) sw[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        int w = tid < block_nwarps() ? sw[tid] : (OP == 0 ? INT_MIN : 0);
        w = OP == 0 ? __reduce_max_sync(0xffffffffu, w) : (int)__reduce_or_sync(0xffffffffu, (unsigned)w);
        if (tid == 0) res = w;
    }
    __syncthreads();
    return res;
}

// Block-wide sum of one Fix per thread (valid in thread 0).
__device__ __forceinline__ Fix block_fix_sum(Fix v) {
    __shared__ Fix sw[32];
    for (int off = 16; off > 0; off >>= 1) v = fix_add(v, fix_shfl_down(v, off));
    const int tid = block_tid();
    if ((tid & 31) == 0) sw[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        Fix w = tid < block_nwarps() ? sw[tid] : Fix{0ull, 0ll};
        for (int off = 16; off > 0; off >>= 1) w = fix_add(w, fix_shfl_down(w, off));
        v = w;
    }
    __syncthreads();
    return v;
}

// non-finite classes of a double: 1 = NaN, 2 = +Inf, 4 = -Inf, 0 = finite
__device__ __forceinline__ int nonfinite_bits(double v) {
    if (v != v) return 1;
    if (dexp(v) != 0x7ff) return 0;
    return v > 0.0 ? 2 : 4;
}
__device__ __forceinline__ CSum nonfinite_sum(int bits) {
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    if ((bits & 1) || (bits & 6) == 6) return CSum{inf - inf, 0.0};
    return CSum{(bits & 2) ? inf : -inf, 0.0};
}

// arithmetic shift right of a two's-complement 128-bit value (truncates toward -inf)
__device__ __forceinline__ Fix fix_shr(Fix x, int k) {
    if (k <= 0) return x;
    if (k >= 127) return Fix{x.hi < 0 ? ~0ull : 0ull, x.hi < 0 ? -1ll : 0ll};
    if (k >= 64) return Fix{(unsigned long long)(x.hi >> (k - 64)), x.hi < 0 ? -1ll : 0ll};
    return Fix{(x.lo >> k) | ((unsigned long long)x.hi << (64 - k)), x.hi >> k};
}

// A running exact sum whose unit follows the largest exponent seen so far: a larger
// exponent rescales the sum (a right shift, dropping bits below the new unit), so one
// pass over the values suffices.  Non-finite values are recorded as classes.
struct FixAcc {
    Fix f{0ull, 0ll};
    int E = 0;
    int bad = 0;
    __device__ __forceinline__ void add(double v) {
        const int e = dexp(v);
        if (e == 0x7ff) {
            bad |= nonfinite_bits(v);
            return;
        }
        if (e > E) {
            f = fix_shr(f, e - E);
            E = e;
        }
        f = fix_add(f, fix_of(v, E));
    }
};

// Combine one FixAcc per thread over the block; the (s, c) result is valid in thread
// 0.  Non-finite inputs give NaN if any is NaN or both infinities occur, else that
// infinity.  At most 2^26 values in all.
__device__ __forceinline__ CSum block_fixacc(const FixAcc& a) {
    const int bad = block_int_reduce<1>(a.bad);
    if (bad) return nonfinite_sum(bad);
    const int E = block_int_reduce<0>(a.E);
    return fix_to_csum(block_fix_sum(fix_shr(a.f, E - a.E)), E);
}

// Exact sum over the block of the pairs get(i), i = tid, tid + nthreads, ... < n
// (n <= 2^25), in one pass; the result is valid in thread 0.
template <typename Get>
__device__ __forceinline__ CSum block_sum_pairs(int n, Get get) {
    const int tid = block_tid(), nt = (int)(blockDim.x * blockDim.y);
    FixAcc a;
#pragma unroll 4
    for (int i = tid; i < n; i += nt) {
        const CSum p = get(i);
        a.add(p.s);
        a.add(p.c);
    }
    return block_fixacc(a);
}

// Exact sum of one CSum per thread over a block (result valid in thread 0).
__device__ __forceinline__ CSum block_csum(CSum v) {
    FixAcc a;
    a.add(v.s);
    a.add(v.c);
    return block_fixacc(a);
}

// maximum of non-negative doubles (NaN wins), on their bit patterns
__device__ __forceinline__ double max_bits(double a, double b) {
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}

// The energy reduction's block step in one pass: the exact sums of two FixAcc (bulk
// and link terms) and the maximum of non-negative doubles, valid in thread 0.  One
// barrier publishes every warp's exponent maxima, which each thread then folds itself,
// and one more publishes the warp sums, so the block pays three barriers instead of
// the fourteen of three separate reductions.
struct Combined2 {
    CSum b, l;
    double m;
};
__device__ __forceinline__ Combined2 block_combine2(const FixAcc& b, const FixAcc& l, double m) {
    struct W1 {
        int bad, eb, el;
    };
    struct W2 {
        Fix fb, fl;
        long long m;
    };
    __shared__ W1 s1[32];
    __shared__ W2 s2[32];
    const int tid = block_tid(), lane = tid & 31, warp = tid >> 5, nw = block_nwarps();
    W1 w{(int)__reduce_or_sync(0xffffffffu, (unsigned)(b.bad | (l.bad << 3))),
         __reduce_max_sync(0xffffffffu, b.E), __reduce_max_sync(0xffffffffu, l.E)};
    if (lane == 0) s1[warp] = w;
    __syncthreads();
    W1 t{0, 0, 0};
    for (int k = 0; k < nw; ++k) {
        const W1 v = s1[k];
        t.bad |= v.bad;
        t.eb = max(t.eb, v.eb);
        t.el = max(t.el, v.el);
    }
    Fix fb = fix_shr(b.f, t.eb - b.E), fl = fix_shr(l.f, t.el - l.E);
    long long mb = __double_as_longlong(m);
    for (int off = 16; off > 0; off >>= 1) {
        fb = fix_add(fb, fix_shfl_down(fb, off));
        fl = fix_add(fl, fix_shfl_down(fl, off));
        mb = max(mb, __shfl_down_sync(0xffffffffu, mb, off));
    }
    if (lane == 0) s2[warp] = W2{fb, fl, mb};
    __syncthreads();
    Combined2 r{CSum{0.0, 0.0}, CSum{0.0, 0.0}, 0.0};
    if (tid == 0) {
        for (int k = 1; k < nw; ++k) {
            fb = fix_add(fb, s2[k].fb);
            fl = fix_add(fl, s2[k].fl);
            mb = max(mb, s2[k].m);
        }
        r.b = (t.bad & 7) ? nonfinite_sum(t.bad & 7) : fix_to_csum(fb, t.eb);
        r.l = (t.bad >> 3) ? nonfinite_sum(t.bad >> 3) : fix_to_csum(fl, t.el);
        r.m = __longlong_as_double(mb);
    }
    __syncthreads();  // s1 / s2 may be reused by a following call
    return r;
}

// Block-wide maximum of non-negative doubles (NaN wins: as integers the bit patterns
// of non-negative values, +Inf and positive NaN are ordered); valid in thread 0.
__device__ __forceinline__ double block_max_nonneg(double v) {
    __shared__ long long sw[32];
    long long b = __double_as_longlong(v);
    for (int off = 16; off > 0; off >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, off));
    const int tid = block_tid();
    if ((tid & 31) == 0) sw[tid >> 5] = b;
    __syncthreads();
    if (tid < 32) {
        long long w = tid < block_nwarps() ? sw[tid] : 0ll;
        for (int off = 16; off > 0; off >>= 1) w = max(w, __shfl_down_sync(0xffffffffu, w, off));
        b = w;
    }
    __syncthreads();
    return __longlong_as_double(b);
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

// The same terms for two points at once (packed lanes; the operations of each lane
// are those of the scalar helpers above, so each lane's terms are those bits).  The
// accumulator holds one unevaluated pair per lane.
struct F2x2 {
    f2 hi, lo;
};
struct EftConst {
    f2 m1, two;  // -1 and 2 in both lanes
};
__device__ __forceinline__ EftConst eft_const() { return EftConst{f2_splat(-1.0f), f2_splat(2.0f)}; }

// two_sum(a, b) per lane
__device__ __forceinline__ F2x2 two_sum2(f2 a, f2 b) {
    const f2 s = f2_add(a, b);
    const f2 bb = f2_sub(s, a);
    return F2x2{s, f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb))};
}
// two_sum(q, -p) per lane: (-p) - bb = -(p + bb), so the error term is
// (q - (s - bb)) - (p + bb) with the same rounding
__device__ __forceinline__ F2x2 two_diff2(f2 q, f2 p) {
    const f2 s = f2_sub(q, p);
    const f2 bb = f2_sub(s, q);
    return F2x2{s, f2_sub(f2_sub(q, f2_sub(s, bb)), f2_add(p, bb))};
}
__device__ __forceinline__ void f2_acc2(F2x2& acc, f2 xh, f2 xl) {
    const F2x2 t = two_sum2(acc.hi, xh);
    acc.hi = t.hi;
    acc.lo = f2_add(f2_add(acc.lo, t.lo), xl);
}
// the exact square of an unevaluated pair (h, l): h^2 as (sq, fma(h, h, -sq) + (2 h) l)
__device__ __forceinline__ void sq_acc2(F2x2& acc, f2 h, f2 l, const EftConst& k) {
    const f2 sq = f2_mul(h, h);
    const f2 sql = f2_add(f2_fma(h, h, f2_mul(sq, k.m1)), f2_mul(f2_mul(k.two, h), l));
    f2_acc2(acc, sq, sql);
}
__device__ __forceinline__ void link_sq2(F2x2& acc, f2 q, f2 p, const EftConst& k) {
    const F2x2 d = two_diff2(q, p);
    sq_acc2(acc, d.hi, d.lo, k);
}
__device__ __forceinline__ void bulk_sq2(F2x2& acc, f2 p, const EftConst& k) {
    const f2 s2 = f2_mul(p, p);
    const f2 s2l = f2_fma(p, p, f2_mul(s2, k.m1));
    const F2x2 w = two_sum2(s2, k.m1);
    sq_acc2(acc, w.hi, f2_add(w.lo, s2l), k);
}

}  // namespace acs
