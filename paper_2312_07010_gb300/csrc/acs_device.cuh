// acs_device.cuh -- per-point arithmetic of the RLB-MIE-FD step, shared by every
// stepping kernel so that all variants (naive, tiled, temporally blocked, batched)
// produce bit-identical states.  The library is built with -fmad=false: every
// fused multiply-add below is an explicit fma(), nothing is contracted behind
// our back, and the order of every sum is fixed here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "acs.h"

namespace acs {

// Cubic-solve modes (a template parameter of every stepping kernel; the host picks
// one per context, so all variants of that context round identically).
enum Solve : int {
    kSolveNewton = 0,  // a seed (three-term series or rational) + `newton` Newton corrections
    kSolveSeries = 1,  // SeriesTerms<T> terms of the Lagrange series, no division
    kSolveFex = 2,     // FEX-FD scheme of Remark 2: no cubic at all
    kSolveSeriesUnit = 3  // kSolveSeries with Theorem 2's condition known to hold (c.clamp): the
                          // series_root_unit() path without a run-time test (temporal kernels)
};
template <typename T>
struct SeriesTerms { static constexpr int value = sizeof(T) == 4 ? 5 : 9; };
template <typename T>
struct NewtonMax { static constexpr int value = sizeof(T) == 4 ? 4 : 6; };

// Coefficients of one step in the state's precision T.
//   lam = eps^2 dt / h^2 (Eq. IE-FD-vector-form), a = dt/2, b = 1 - a.
// Remark 1's explicit part xi = (1 - 2 d lam) phi - (dt/2)(phi^3 - phi) + lam S, with
// S the sum of the 2d neighbours, is evaluated
//   FP64:  xi = c0 phi - a phi^3 + lam S,           c0 = 1 - 2 d lam + a;
//   FP32:  xi = phi + [lam (S - 2 d phi) + (-a) phi (phi^2 - 1)]   (increment form;
//          each operation of it has a packed two-lane FP32 instruction, see f32x2.cuh).
// The FP32 form keeps the rounded coefficients (lam, a) on the small increment only:
// with c0 (and 1/b below) rounded to FP32, every step carries the same relative
// error of up to 4e-8 in phi, which accumulates near a moving interface (2.7e-5
// after 2000 steps of the 4096^2 Dirichlet star run against 5.8e-6 in this form).
// For the FEX-FD scheme of Remark 2 the same expression with a = dt is the new
// state and no cubic is solved.
//
// The root theta of a theta^3 + b theta = xi (Remark 1) as a series in xi
// (Lagrange inversion): with x = xi/b, y = (a/b) x^2,
//   theta = x sum_k (-y)^k C_k,  C_k = binom(3k, k) / (2k + 1)  (1, 1, 3, 12, 55, ...),
// convergent for y < 4/27; so theta = xi sum_k q_k (xi^2)^k with
//   q_k = C_k (-a)^k / b^(3k+1).
// Both precisions evaluate theta = xi + xi R(xi^2) with R = P - 1 (its constant term
// q_0 - 1 = a/b), for the same reason as the increment form, and so that theta = +-1
// comes out exactly at xi = +-1 (see series_root_unit).
template <typename T>
struct IncForm { static constexpr bool value = sizeof(T) == 4; };

template <typename T>
struct Coef {
    T lam, c0, a, b, three_a;
    T m2d;        // -2 d (exact), the increment form's Laplacian weight of phi
    T na;         // -a, the increment form's reaction weight
    T q[10];      // kSolveSeries: theta = xi + xi * sum_k q[k] xi^(2k), q[0] = a/b
    T xi2max;     // kSolveSeries applies while xi^2 <= xi2max
    T fast2max;   // several-points fast path (tiled kernels): xi^2 bound, see roots()
    T rb, t;      // kSolveNewton: 1/b, a/b
    T ymax;       // kSolveNewton applies while y = t (xi/b)^2 <= ymax
    int newton;   // kSolveNewton: corrections after the seed (1..6)
    int seed;     // kSolveNewton: 0 = three-term series in y (y <= ymax), 1 = xi / (b + a xi^2) (xi^2 <= xi2max)
    T clamp_hi;   // 1 + 16 ulp: overshoots up to this are rounding and go back to +-1
    int clamp;    // 1: apply that rounding guard (set only when Theorem 2's condition holds)
    int solve;    // the Solve mode this context uses
    int split;    // FP64 series: 1 = terms k >= kSeriesSplit of R in FP32 (series_eval)
    float qf[4];  // those terms' coefficients q[kSeriesSplit ..] rounded to FP32 (3 used)
};

// FP64 series terms from this index on may be summed in FP32: the host allows it
// (Coef::split) only where their whole contribution to theta, times the FP32 error
// factor, stays below 2^-58 -- a small fraction of theta's own rounding -- and the
// FP64 pipe, which bounds the FP64 step, then runs 2 of the 8 Horner steps fewer.
constexpr int kSeriesSplit = 6;

// 32-bit shared-memory address of a generic pointer into shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <typename T> __device__ __forceinline__ T dfma(T a, T b, T c);
template <> __device__ __forceinline__ float dfma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double dfma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// Approximate reciprocal (relative error about 2^-22): good enough for a Newton
// correction, whose own size is tiny.  FP64 goes through the FP32 unit on purpose.
__device__ __forceinline__ float arcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double arcp(double x) { return (double)arcp((float)x); }

// p(theta) = a theta^3 + b theta - xi, given th2 = theta^2.  FP32 writes it as
// (theta - xi) + a (theta^3 - theta), which does not use the rounded b (a bias in b
// would move the root itself, not only the convergence).
template <typename T>
__device__ __forceinline__ T residual(T th, T th2, T xi, T a, T b) {
    if (IncForm<T>::value) return dfma(a, dfma(th2, th, -th), th - xi);
    return dfma(dfma(a, th2, b), th, -xi);
}

// Robust root of a theta^3 + b theta = xi for any xi (used when the fast path does
// not apply, e.g. when the maximum-principle condition is violated).  p is odd and
// increasing, so solve for |xi| and restore the sign.  Newton from
// min(|xi|/b, cbrt(|xi|/a)), two upper bounds of the root: p is convex on
// theta > 0, so the iterates decrease monotonically to the root; stop when they
// stop decreasing.  NaN propagates.
template <typename T>
__device__ __noinline__ T cubic_robust(T xi, T a, T b) {
    T ax = xi < T(0) ? -xi : xi;
    if (!(ax > T(0))) return xi;  // 0 or NaN
    T th = ax / b;
    T cb = cbrt(ax / a);
    if (cb < th) th = cb;
    for (int it = 0; it < 200; ++it) {
        T th2 = th * th;
        T p = residual(th, th2, ax, a, b);
        T nt = th - p / dfma(T(3) * a, th2, b);
        if (!(nt < th)) break;
        th = nt;
    }
    return xi < T(0) ? -th : th;
}

// Seeds of the Newton solve.  seed3: the Lagrange series in y = (a/b) x^2, x = xi/b,
// cut after three terms.  rational: xi / (b + a xi^2), exact at xi = 0 and xi = +-1
// (a + b = 1) and an upper bound of |theta| in between (|theta| >= |xi| there), so
// the corrections descend monotonically.
template <typename T>
__device__ __forceinline__ T newton_seed3(T x, T y) {
    const T u = -y;
    return x * dfma(u, dfma(T(3), u, T(1)), T(1));
}
template <typename T>
__device__ __forceinline__ T newton_seed_rational(T xi, T x2, const Coef<T>& c) {
    return xi * arcp(dfma(c.a, x2, c.b));
}
// c.newton Newton corrections theta -= p(theta) / p'(theta) with an approximate
// reciprocal (the host counted them from an error bound that includes its error);
// at most NewtonMax<T> of them.
template <typename T>
__device__ __forceinline__ T newton_fix(T th, T xi, const Coef<T>& c) {
#pragma unroll
    for (int k = 0; k < NewtonMax<T>::value; ++k) {
        if (k < c.newton) {
            const T th2 = th * th;
            const T p = residual(th, th2, xi, c.a, c.b);
            const T dp = dfma(c.three_a, th2, c.b);
            th = dfma(-p, arcp(dp), th);
        }
    }
    return th;
}

// The truncated Lagrange series at xi (x2 = xi^2): xi + xi R(x2), R = P - 1.
// x >= 0 (x = xi^2) as a float on the integer units, the mantissa truncated (relative
// error below 2^-23) and values below 2^-126 flushed to +0.  NaN gives some finite
// value; the FP64 operations that also take x then carry the NaN.
__device__ __forceinline__ float nonneg_f64_to_f32(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)(hi >> 20) - 896;                       // 1023 - 127
    const unsigned m = __funnelshift_l(lo, hi, 3) & 0x7fffffu;  // top 23 of the 52 mantissa bits
    return e <= 0 ? 0.0f : __uint_as_float(((unsigned)e << 23) | m);
}
// A normal float as a double on the integer units (exact); zero and subnormals give
// a signed zero.
__device__ __forceinline__ double f32_to_f64_int(float t) {
    const unsigned u = __float_as_uint(t), mag = u & 0x7fffffffu;
    if (mag < 0x00800000u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return __hiloint2double((int)((u & 0x80000000u) | ((mag >> 3) + (896u << 20))), (int)(u << 29));
}

template <typename T, int NT>
__device__ __forceinline__ T series_eval(T xi, T x2, const Coef<T>& c) {
    if constexpr (sizeof(T) == 8 && NT > kSeriesSplit && NT - kSeriesSplit <= 4) {
        if (c.split) {
            // the tail q[6] + q[7] x2 + q[8] x2^2 in FP32, the rest of the Horner scheme in FP64
            const float x2f = nonneg_f64_to_f32(x2);
            float t = c.qf[NT - 1 - kSeriesSplit];
#pragma unroll
            for (int k = NT - 2; k >= kSeriesSplit; --k) t = __fmaf_rn(t, x2f, c.qf[k - kSeriesSplit]);
            T R = f32_to_f64_int(t);
#pragma unroll
            for (int k = kSeriesSplit - 1; k >= 0; --k) R = dfma(R, x2, c.q[k]);
            return dfma(xi, R, xi);
        }
    }
    T R = c.q[NT - 1];
#pragma unroll
    for (int k = NT - 2; k >= 0; --k) R = dfma(R, x2, c.q[k]);
    return dfma(xi, R, xi);
}

// Root of theta + (dt/2) f(theta) = xi (Remark 1), i.e. a theta^3 + b theta = xi.
// The host picks the mode and its limits from a-priori error bounds so that the
// fast paths are accurate to the last bit of T for |xi| <= 1.001 (Theorem 2's
// range plus rounding); larger |xi| take the robust path.
// x limited to [-1, 1]; NaN passes through.  FP32: PTX max.NaN / min.NaN.  FP64: a
// test of the high word on the integer units (it keeps the FP64 pipe, which bounds
// the FP64 step, free): 1 <= |x| < Inf becomes +-1, anything else is kept.
__device__ __forceinline__ float clamp_unit(float x) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(-1.0f));
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(r), "f"(1.0f));
    return r;
}
__device__ __forceinline__ double clamp_unit(double x) {
    const int hi = __double2hiint(x);
    const unsigned ahi = (unsigned)hi & 0x7fffffffu;
    if (ahi >= 0x3ff00000u && ahi < 0x7ff00000u) return __hiloint2double((hi & (int)0x80000000) | 0x3ff00000, 0);
    return x;
}

// Series solve while Theorem 2's condition holds (c.clamp): with |phi| <= 1 the exact
// predictor obeys |xi| <= 1 (its explicit part is a convex combination), so xi is
// limited to [-1, 1] (a no-op in exact arithmetic), and then |theta| <= 1 needs no
// guard: the series' truncation error (<= 2^-26 FP32, 2^-55 FP64, chosen by the host
// for |xi| <= 1.001) and the rounding of R stay below the half-ulp gap above 1
// (2^-24, 2^-53), so xi = +-1 gives +-1 exactly and |xi| < 1 gives |theta| <= 1.
template <typename T>
__device__ __forceinline__ T series_root_unit(T xi, const Coef<T>& c) {
    const T xc = clamp_unit(xi);
    return series_eval<T, SeriesTerms<T>::value>(xc, xc * xc, c);
}

template <typename T, int SOLVE>
__device__ __forceinline__ T cubic_root(T xi, const Coef<T>& c) {
    T th;
    if constexpr (SOLVE == kSolveSeriesUnit) return series_root_unit(xi, c);
    if constexpr (SOLVE == kSolveSeries) {
        if (c.clamp) return series_root_unit(xi, c);
    }
    if (SOLVE == kSolveSeries) {
        constexpr int NT = SeriesTerms<T>::value;
        const T x2 = xi * xi;
        if (x2 <= c.xi2max) {
            th = series_eval<T, NT>(xi, x2, c);
        } else {
            th = cubic_robust(xi, c.a, c.b);
        }
    } else {
        bool ok;
        if (c.seed == 0) {
            const T x = xi * c.rb;
            const T y = (c.t * x) * x;
            ok = y <= c.ymax;
            th = newton_seed3(x, y);
        } else {
            const T x2 = xi * xi;
            ok = x2 <= c.xi2max;
            th = newton_seed_rational(xi, x2, c);
        }
        if (ok) th = newton_fix(th, xi, c);
        else th = cubic_robust(xi, c.a, c.b);
    }
    if (c.clamp) {
        const T ath = th < T(0) ? -th : th;
        if (ath > T(1) && ath <= c.clamp_hi) th = th < T(0) ? T(-1) : T(1);
    }
    return th;
}

// Pieces of update() for kernels that decide the cubic path once for several points:
// the explicit predictor xi, the series root without its range check, the clamp.
template <typename T>
__device__ __forceinline__ T predictor(T p, T s, const Coef<T>& c) {
    if (IncForm<T>::value) {
        const T lap = dfma(c.m2d, p, s);       // S - 2 d phi
        const T cub = p * dfma(p, p, T(-1));   // phi^3 - phi = phi (phi^2 - 1)
        return p + dfma(c.lam, lap, c.na * cub);
    }
    const T p2 = p * p;
    return dfma(c.lam, s, p * dfma(-c.a, p2, c.c0));
}
// The new value of one unknown from its old value p and the sum s of its 2d
// ghost-ruled neighbours.
template <typename T, int SOLVE>
__device__ __forceinline__ T update(T p, T s, const Coef<T>& c) {
    const T xi = predictor(p, s, c);
    if (SOLVE == kSolveFex) return xi;
    return cubic_root<T, SOLVE>(xi, c);
}

// Fixed summation order of the neighbours: z pair, then y pair, then x pair.
template <typename T>
__device__ __forceinline__ T nsum(T xm, T xp) { return xm + xp; }
template <typename T>
__device__ __forceinline__ T nsum(T ym, T yp, T xm, T xp) { return (ym + yp) + (xm + xp); }
template <typename T>
__device__ __forceinline__ T nsum(T zm, T zp, T ym, T yp, T xm, T xp) {
    return ((zm + zp) + (ym + yp)) + (xm + xp);
}

// Geometry: the fastest axis is x (n[dims-1]); then y, then z.  Absent axes have size 1.
struct Geo {
    int64_t nx, ny, nz;  // sizes
    int64_t sy, sz;      // strides of y and z (x stride is 1)
    int64_t total;
};

// Dispatch of the temporal kernels: the series solve under Theorem 2's condition is
// its own case (kSolveSeriesUnit), so the kernels carry no test of c.clamp.
#define ACS_SOLVE_DISPATCH_UNIT(c, S, ...)                      \
    do {                                                        \
        if ((c).solve == ::acs::kSolveSeries && (c).clamp) {    \
            constexpr int S = ::acs::kSolveSeriesUnit;          \
            __VA_ARGS__;                                        \
        } else {                                                \
            ACS_SOLVE_DISPATCH((c).solve, S, __VA_ARGS__);      \
        }                                                       \
    } while (0)

// Dispatch a runtime Solve mode to a template parameter.
#define ACS_SOLVE_DISPATCH(mode, S, ...)                 \
    do {                                                 \
        if ((mode) == ::acs::kSolveSeries) {             \
            constexpr int S = ::acs::kSolveSeries;       \
            __VA_ARGS__;                                 \
        } else if ((mode) == ::acs::kSolveFex) {         \
            constexpr int S = ::acs::kSolveFex;          \
            __VA_ARGS__;                                 \
        } else {                                         \
            constexpr int S = ::acs::kSolveNewton;       \
            __VA_ARGS__;                                 \
        }                                                \
    } while (0)

}  // namespace acs
