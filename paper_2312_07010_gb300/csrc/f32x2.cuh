// f32x2.cuh -- packed two-lane FP32 arithmetic for the FP32 step (PTX add / mul /
// fma.rn.f32x2).  One instruction performs the two IEEE round-to-nearest FP32
// operations of its lanes, so a pair computes exactly what two scalar operations
// compute, in one issue slot.  The helpers below evaluate the FP32 per-point
// arithmetic of acs_device.cuh (predictor() in its increment form, the series root
// series_eval() with its clamp) on pairs of points, operation for operation, so a
// kernel using them gives the scalar kernels' bits.
#pragma once

#include "f2ops.cuh"
#include "stream_tile.cuh"

namespace acs {


// Coefficients of Coef<float> as pairs (registers: the packed instructions take no
// immediate or constant-bank operands).
struct PackedCoef {
    f2 m2d, lam, na, m1;
    f2 q[SeriesTerms<float>::value];
};
__device__ __forceinline__ PackedCoef packed_coef(const Coef<float>& c) {
    PackedCoef pc;
    pc.m2d = f2_splat(c.m2d);
    pc.lam = f2_splat(c.lam);
    pc.na = f2_splat(c.na);
    pc.m1 = f2_splat(-1.0f);
#pragma unroll
    for (int k = 0; k < SeriesTerms<float>::value; ++k) pc.q[k] = f2_splat(c.q[k]);
    return pc;
}

// predictor() of two points from their values p and neighbour sums s.
__device__ __forceinline__ f2 predictor2(f2 p, f2 s, const PackedCoef& pc) {
    const f2 lap = f2_fma(pc.m2d, p, s);              // S - 2 d phi
    const f2 cub = f2_mul(p, f2_fma(p, p, pc.m1));    // phi (phi^2 - 1)
    return f2_add(p, f2_fma(pc.lam, lap, f2_mul(pc.na, cub)));
}

// The 2D predictor of one lane's four consecutive points z[0..3] (rows m above and p
// below, outer x neighbours left and right): nsum(m, p, xm, xp) = (m + p) + (xm + xp)
// per point, the x pair summed in scalar form (its operands straddle the pairs).
__device__ __forceinline__ void predict4_2d(const float (&m)[4], const float (&z)[4], const float (&p)[4], float left,
                                            float right, const PackedCoef& pc, f2 (&xi)[2]) {
    const f2 sx0 = f2_make(left + z[1], z[0] + z[2]);
    const f2 sx1 = f2_make(z[1] + z[3], z[2] + right);
    const f2 s0 = f2_add(f2_add(f2_make(m[0], m[1]), f2_make(p[0], p[1])), sx0);
    const f2 s1 = f2_add(f2_add(f2_make(m[2], m[3]), f2_make(p[2], p[3])), sx1);
    xi[0] = predictor2(f2_make(z[0], z[1]), s0, pc);
    xi[1] = predictor2(f2_make(z[2], z[3]), s1, pc);
}

// The 3D predictor: nsum(zm, zp, ym, yp, xm, xp) = ((zm + zp) + (ym + yp)) + (xm + xp).
__device__ __forceinline__ void predict4_3d(const float (&zm)[4], const float (&zp)[4], const float (&ym)[4],
                                            const float (&z)[4], const float (&yp)[4], float left, float right,
                                            const PackedCoef& pc, f2 (&xi)[2]) {
    const f2 sx0 = f2_make(left + z[1], z[0] + z[2]);
    const f2 sx1 = f2_make(z[1] + z[3], z[2] + right);
    const f2 a0 = f2_add(f2_make(zm[0], zm[1]), f2_make(zp[0], zp[1]));
    const f2 a1 = f2_add(f2_make(zm[2], zm[3]), f2_make(zp[2], zp[3]));
    const f2 b0 = f2_add(f2_make(ym[0], ym[1]), f2_make(yp[0], yp[1]));
    const f2 b1 = f2_add(f2_make(ym[2], ym[3]), f2_make(yp[2], yp[3]));
    xi[0] = predictor2(f2_make(z[0], z[1]), f2_add(f2_add(a0, b0), sx0), pc);
    xi[1] = predictor2(f2_make(z[2], z[3]), f2_add(f2_add(a1, b1), sx1), pc);
}

// arcp() of both lanes (the approximate reciprocal has no packed form).
__device__ __forceinline__ f2 arcp2(f2 x) { return f2_make(arcp(f2_lo(x)), arcp(f2_hi(x))); }

// roots() for FP32 points held as NP pairs: with the series solve, series_root_unit()
// on pairs while Theorem 2's condition holds, else the fast path (every xi^2 <=
// fast2max) on pairs with the per-point clamp; with the Newton solve, roots()' fast
// path (seed, c.newton corrections, clamp) on pairs; any other case unpacks and takes
// roots()' scalar path, which gives the same values.
template <int SOLVE, int NP>
__device__ __forceinline__ void roots2(const f2 (&xi)[NP], float (&out)[2 * NP], const Coef<float>& c,
                                       const PackedCoef& pc) {
    constexpr int NT = SeriesTerms<float>::value;
    if (SOLVE == kSolveSeriesUnit || (SOLVE == kSolveSeries && c.clamp)) {
        // series_root_unit() on pairs
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const f2 xc = f2_make(clamp_unit(f2_lo(xi[i])), clamp_unit(f2_hi(xi[i])));
            const f2 x2 = f2_mul(xc, xc);
            f2 R = pc.q[NT - 1];
#pragma unroll
            for (int k = NT - 2; k >= 0; --k) R = f2_fma(R, x2, pc.q[k]);
            const f2 th = f2_fma(xc, R, xc);
            out[2 * i] = f2_lo(th);
            out[2 * i + 1] = f2_hi(th);
        }
        return;
    }
    if (SOLVE == kSolveSeries) {
        f2 x2[NP];
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            x2[i] = f2_mul(xi[i], xi[i]);
            m = nanmax(m, nanmax(f2_lo(x2[i]), f2_hi(x2[i])));
        }
        if (m <= c.fast2max) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                f2 R = pc.q[NT - 1];
#pragma unroll
                for (int k = NT - 2; k >= 0; --k) R = f2_fma(R, x2[i], pc.q[k]);
                const f2 th = f2_fma(xi[i], R, xi[i]);
                float lo = f2_lo(th), hi = f2_hi(th);
                if (c.clamp) {
                    lo = fminf(fmaxf(lo, -1.0f), 1.0f);
                    hi = fminf(fmaxf(hi, -1.0f), 1.0f);
                }
                out[2 * i] = lo;
                out[2 * i + 1] = hi;
            }
            return;
        }
    }
    if (SOLVE == kSolveNewton) {
        // the operations of roots()' Newton fast path, two points per instruction:
        // seed, corrections theta -= p / p' (residual() in its FP32 form
        // a (theta^3 - theta) + (theta - xi)), clamp; the same tests decide the path
        const f2 rb = f2_splat(c.rb), t = f2_splat(c.t), a = f2_splat(c.a), b = f2_splat(c.b);
        const f2 three_a = f2_splat(c.three_a), one = f2_splat(1.0f), three = f2_splat(3.0f);
        f2 th[NP];
        bool ok;
        if (c.seed == 0) {
            float my = 0.0f, m2 = 0.0f;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const f2 x = f2_mul(xi[i], rb);
                const f2 y = f2_mul(f2_mul(t, x), x);
                const f2 x2 = f2_mul(xi[i], xi[i]);
                my = nanmax(my, nanmax(f2_lo(y), f2_hi(y)));
                m2 = nanmax(m2, nanmax(f2_lo(x2), f2_hi(x2)));
                const f2 u = f2_mul(y, pc.m1);  // -y
                th[i] = f2_mul(x, f2_fma(u, f2_fma(three, u, one), one));
            }
            ok = my <= c.ymax && m2 <= c.fast2max;
        } else {
            float m2 = 0.0f;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const f2 x2 = f2_mul(xi[i], xi[i]);
                m2 = nanmax(m2, nanmax(f2_lo(x2), f2_hi(x2)));
                th[i] = f2_mul(xi[i], arcp2(f2_fma(a, x2, b)));
            }
            ok = m2 <= c.xi2max && m2 <= c.fast2max;
        }
        if (ok) {
#pragma unroll
            for (int k = 0; k < NewtonMax<float>::value; ++k) {
                if (k < c.newton) {
#pragma unroll
                    for (int i = 0; i < NP; ++i) {
                        const f2 th2 = f2_mul(th[i], th[i]);
                        const f2 p = f2_fma(a, f2_fma(th2, th[i], f2_mul(th[i], pc.m1)), f2_sub(th[i], xi[i]));
                        const f2 dp = f2_fma(three_a, th2, b);
                        th[i] = f2_fma(f2_mul(p, pc.m1), arcp2(dp), th[i]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                float lo = f2_lo(th[i]), hi = f2_hi(th[i]);
                if (c.clamp) {
                    lo = fminf(fmaxf(lo, -1.0f), 1.0f);
                    hi = fminf(fmaxf(hi, -1.0f), 1.0f);
                }
                out[2 * i] = lo;
                out[2 * i + 1] = hi;
            }
            return;
        }
    }
    float x[2 * NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        x[2 * i] = f2_lo(xi[i]);
        x[2 * i + 1] = f2_hi(xi[i]);
    }
    roots<float, SOLVE, 2 * NP>(x, out, c);
}

}  // namespace acs
