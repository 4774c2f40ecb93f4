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
    kSolveFex = 2      // FEX-FD scheme of Remark 2: no cubic at all
};
template <typename T>
struct SeriesTerms { static constexpr int value = sizeof(T) == 4 ? 5 : 9; };
template <typename T>
struct NewtonMax { static constexpr int value = sizeof(T) == 4 ? 4 : 6; };

// Coefficients of one step in the state's precision T.
//   lam = eps^2 dt / h^2 (Eq. IE-FD-vector-form), a = dt/2, b = 1 - a.
//   xi = c0 phi - a phi^3 + lam S, S = sum of the 2d neighbours, c0 = 1 - 2 d lam + a
// (Remark 1's xi = (1 - 2 d lam) phi - (dt/2)(phi^3 - phi) + lam S, regrouped).
// For the FEX-FD scheme of Remark 2 the same expression with a = dt,
// c0 = 1 - 2 d lam + dt is the new state and no cubic is solved.
//
// The root theta of a theta^3 + b theta = xi (Remark 1) as a series in xi
// (Lagrange inversion): with x = xi/b, y = (a/b) x^2,
//   theta = x sum_k (-y)^k C_k,  C_k = binom(3k, k) / (2k + 1)  (1, 1, 3, 12, 55, ...),
// convergent for y < 4/27; so theta = xi sum_k q_k (xi^2)^k with
//   q_k = C_k (-a)^k / b^(3k+1).
template <typename T>
struct Coef {
    T lam, c0, a, b, three_a;
    T q[10];      // kSolveSeries: theta = xi * sum_k q[k] xi^(2k)
    T xi2max;     // kSolveSeries applies while xi^2 <= xi2max
    T fast2max;   // several-points fast path (tiled kernels): xi^2 bound, see roots()
    T rb, t;      // kSolveNewton: 1/b, a/b
    T ymax;       // kSolveNewton applies while y = t (xi/b)^2 <= ymax
    int newton;   // kSolveNewton: corrections after the seed (1..6)
    int seed;     // kSolveNewton: 0 = three-term series in y (y <= ymax), 1 = xi / (b + a xi^2) (xi^2 <= xi2max)
    T clamp_hi;   // 1 + 16 ulp: overshoots up to this are rounding and go back to +-1
    int clamp;    // 1: apply that rounding guard (set only when Theorem 2's condition holds)
    int solve;    // the Solve mode this context uses
};

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
        T p = dfma(dfma(a, th2, b), th, -ax);
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
            const T p = dfma(dfma(c.a, th2, c.b), th, -xi);
            const T dp = dfma(c.three_a, th2, c.b);
            th = dfma(-p, arcp(dp), th);
        }
    }
    return th;
}

// Root of theta + (dt/2) f(theta) = xi (Remark 1), i.e. a theta^3 + b theta = xi.
// The host picks the mode and its limits from a-priori error bounds so that the
// fast paths are accurate to the last bit of T for |xi| <= 1.001 (Theorem 2's
// range plus rounding); larger |xi| take the robust path.
template <typename T, int SOLVE>
__device__ __forceinline__ T cubic_root(T xi, const Coef<T>& c) {
    T th;
    if (SOLVE == kSolveSeries) {
        constexpr int NT = SeriesTerms<T>::value;
        const T x2 = xi * xi;
        if (x2 <= c.xi2max) {
            T P = c.q[NT - 1];
#pragma unroll
            for (int k = NT - 2; k >= 0; --k) P = dfma(P, x2, c.q[k]);
            th = xi * P;
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
    const T p2 = p * p;
    return dfma(c.lam, s, p * dfma(-c.a, p2, c.c0));
}
// The new value of one unknown from its old value p and the sum s of its 2d
// ghost-ruled neighbours.
template <typename T, int SOLVE>
__device__ __forceinline__ T update(T p, T s, const Coef<T>& c) {
    const T p2 = p * p;
    const T xi = dfma(c.lam, s, p * dfma(-c.a, p2, c.c0));
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
