// stream_tile.cuh -- tile geometry and vector helpers of the TMA-streamed step
// kernels (3D: xy tiles streamed through z; 2D: x tiles streamed through row blocks).
#pragma once

#include "acs_kernels.cuh"
#include "acs_reduce.cuh"

namespace acs {

// Geometry of a streamed tile: 256 threads = 32 lanes x 8 warps; each thread owns
// one 16-byte vector (VX values) in RPT consecutive rows, so the tile is
// TX = 32 VX wide and TY = 8 RPT high; S ring slots of TMA-loaded boxes.
template <typename T, int RPT_ = 2, int S_ = 4>
struct Tile3 {
    static constexpr int RPT = RPT_;                // rows per thread
    static constexpr int VX = 16 / (int)sizeof(T);  // unknowns per 16-byte vector
    static constexpr int TX = 32 * VX;              // tile width
    static constexpr int TY = 8 * RPT;              // tile height
    static constexpr int BW = TX + 2 * VX;          // box width (16-byte aligned halo)
    static constexpr int BH = TY + 2;               // box height
    static constexpr int S = S_;                    // ring slots
    static constexpr int SLOT = BW * BH;                        // values in one box
    static constexpr uint32_t SLOT_BYTES = SLOT * sizeof(T);    // bytes one TMA load writes
    // TMA tensor copies need a 128-byte aligned shared-memory destination
    static constexpr uint32_t SLOT_STRIDE = (SLOT_BYTES + 127u) / 128u * 128u;
    static constexpr uint32_t BAR_BYTES = 128;                  // S mbarriers, padded
    static constexpr size_t SMEM = 128 + BAR_BYTES + (size_t)S * SLOT_STRIDE;  // + base alignment slack
    static_assert(SLOT_STRIDE % 128 == 0 && S * sizeof(uint64_t) <= BAR_BYTES, "ring layout");
    static_assert((VX * sizeof(T)) % 16 == 0 && (BW * sizeof(T)) % 16 == 0, "16-byte TMA x granularity");
    static_assert(BW <= 256 && BH <= 256, "TMA box dimensions");
};

// max that propagates NaN (so one comparison can screen several values)
__device__ __forceinline__ float nanmax(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) ? b : a; }

// Modes of the streamed kernels: one step, or the energy / max-norm reduction of the
// input state (same pipeline, the step's ghost-ruled forward neighbours).
enum StreamMode : int { kModeStep = 0, kModeEnergy = 1 };

// Per-thread E_h / max-norm accumulation for the streamed kernels.  FP32 states: terms
// are formed exactly with error-free transformations into float pairs (acs_reduce.cuh;
// two points at once on packed lanes) and folded into FP64 every 8 planes (at most 128
// terms per pair: about 2^-41 relative accumulation error); FP64 states: FP64 sums.  The bulk sum is of (p^2 - 1)^2
// (the 1/4 is applied by the finishing kernel), the link sum of squared differences.
template <typename T>
struct EnergyAcc;
template <>
struct EnergyAcc<float> {
    F2 fb{0.0f, 0.0f}, fl{0.0f, 0.0f};
    // the same sums for pairs of points (two lanes each; point_pair / point2_pair)
    F2x2 pb{f2_splat(0.0f), f2_splat(0.0f)}, pl{f2_splat(0.0f), f2_splat(0.0f)};
    EftConst k = eft_const();
    double db = 0.0, dl = 0.0, mx = 0.0;
    float fmx = 0.0f;
    int planes = 0;
    // two neighbouring points (lanes) p with their forward x, y (and z) neighbours
    __device__ __forceinline__ void point_pair(f2 p, f2 xn, f2 yn, f2 zn) {
        bulk_sq2(pb, p, k);
        link_sq2(pl, xn, p, k);
        link_sq2(pl, yn, p, k);
        link_sq2(pl, zn, p, k);
        fmx = nanmax(fmx, nanmax(fabsf(f2_lo(p)), fabsf(f2_hi(p))));
    }
    __device__ __forceinline__ void point2_pair(f2 p, f2 xn, f2 yn) {
        bulk_sq2(pb, p, k);
        link_sq2(pl, xn, p, k);
        link_sq2(pl, yn, p, k);
        fmx = nanmax(fmx, nanmax(fabsf(f2_lo(p)), fabsf(f2_hi(p))));
    }
    __device__ __forceinline__ void point(float p, float xn, float yn, float zn) {
        bulk_sq(fb, p);
        link_sq(fl, xn, p);
        link_sq(fl, yn, p);
        link_sq(fl, zn, p);
        fmx = nanmax(fmx, fabsf(p));
    }
    __device__ __forceinline__ void point2(float p, float xn, float yn) {
        bulk_sq(fb, p);
        link_sq(fl, xn, p);
        link_sq(fl, yn, p);
        fmx = nanmax(fmx, fabsf(p));
    }
    __device__ __forceinline__ void ghost_link(float p) { link_sq(fl, 0.0f, p); }
    // the scalar pair and the two lanes of the packed pair, summed exactly in FP32 (their
    // high parts by TwoSum, their low parts, about 2^-24 of the highs, plainly)
    static __device__ __forceinline__ F2 merge(F2 a, const F2x2& p) {
        const F2 t = two_sum(f2_lo(p.hi), f2_hi(p.hi));
        const F2 u = two_sum(a.hi, t.hi);
        return F2{u.hi, ((a.lo + (f2_lo(p.lo) + f2_hi(p.lo))) + t.lo) + u.lo};
    }
    __device__ __forceinline__ void fold() {
        const F2 b = merge(fb, pb), l = merge(fl, pl);
        db += (double)b.hi + (double)b.lo;
        dl += (double)l.hi + (double)l.lo;
        fb = F2{0.0f, 0.0f};
        fl = F2{0.0f, 0.0f};
        pb = F2x2{f2_splat(0.0f), f2_splat(0.0f)};
        pl = F2x2{f2_splat(0.0f), f2_splat(0.0f)};
    }
    // fold every 8 planes: a lane then holds at most 32 bulk and 96 link terms of the
    // 2 x 2 pairs a thread forms per plane (FP64 operations are scarce on this GPU)
    __device__ __forceinline__ void plane_done() {
        if (++planes == 8) { fold(); planes = 0; }
    }
    __device__ __forceinline__ void finish() {
        fold();
        mx = (double)fmx;
    }
};
template <>
struct EnergyAcc<double> {
    double db = 0.0, dl = 0.0, mx = 0.0;
    __device__ __forceinline__ void point(double p, double xn, double yn, double zn) {
        const double w = fma(p, p, -1.0);
        db = fma(w, w, db);
        const double a = xn - p, b = yn - p, c = zn - p;
        dl = fma(a, a, dl);
        dl = fma(b, b, dl);
        dl = fma(c, c, dl);
        mx = nanmax(mx, fabs(p));
    }
    __device__ __forceinline__ void point2(double p, double xn, double yn) {
        const double w = fma(p, p, -1.0);
        db = fma(w, w, db);
        const double a = xn - p, b = yn - p;
        dl = fma(a, a, dl);
        dl = fma(b, b, dl);
        mx = nanmax(mx, fabs(p));
    }
    __device__ __forceinline__ void ghost_link(double p) { dl = fma(p, p, dl); }
    __device__ __forceinline__ void plane_done() {}
    __device__ __forceinline__ void finish() {}
};

// Block-combine the per-thread sums (thread 0 writes the block's partial).
template <typename T>
__device__ __forceinline__ void energy_block_write(EnergyAcc<T>& acc, RedPartial* out) {
    acc.finish();
    const CSum b = block_csum(CSum{acc.db, 0.0});
    const CSum l = block_csum(CSum{acc.dl, 0.0});
    const double m = block_max_nonneg(acc.mx);
    if (block_tid() == 0) *out = RedPartial{b.s, b.c, l.s, l.c, m, 0.0, 0.0, 0.0};
}

// Tile variants offered to the autotuner: (rows per thread, ring slots).
constexpr int kNumTileVariants = 3;
#define ACS_TILE_VARIANT_DISPATCH(var, RPTV, SV, ...)          \
    do {                                                      \
        if ((var) == 1) {                                     \
            constexpr int RPTV = 2, SV = 6;                   \
            __VA_ARGS__;                                      \
        } else if ((var) == 2) {                              \
            constexpr int RPTV = 4, SV = 4;                   \
            __VA_ARGS__;                                      \
        } else {                                              \
            constexpr int RPTV = 2, SV = 4;                   \
            __VA_ARGS__;                                      \
        }                                                     \
    } while (0)

// Cubic root of the RPT x VX values of one thread.  The series solve under Theorem 2's
// condition: series_root_unit() per point.  Otherwise, with the series
// solve and every xi^2 <= fast2max, the series is evaluated without per-point checks
// and (when the rounding guard is on) clamped with plain min/max: fast2max keeps |xi| <= 1 + 8 ulp,
// where the exact root is within [-1, 1] to rounding, so this gives the same values
// as the per-point path.  The Newton solve does the same once every point is within
// its seed's range.  Otherwise every point takes cubic_root().
template <typename T, int SOLVE, int N>
__device__ __forceinline__ void roots(const T (&xi)[N], T (&out)[N], const Coef<T>& c) {
    if (SOLVE == kSolveFex) {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = xi[i];
        return;
    }
    if constexpr (SOLVE == kSolveSeriesUnit) {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = series_root_unit(xi[i], c);
        return;
    }
    if constexpr (SOLVE == kSolveSeries) {
        if (c.clamp) {
#pragma unroll
            for (int i = 0; i < N; ++i) out[i] = series_root_unit(xi[i], c);
            return;
        }
    }
    if (SOLVE == kSolveSeries) {
        T x2[N];
        T m = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            x2[i] = xi[i] * xi[i];
            m = nanmax(m, x2[i]);
        }
        if (m <= c.fast2max) {
            constexpr int NT = SeriesTerms<T>::value;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T th = series_eval<T, NT>(xi[i], x2[i], c);
                if (c.clamp) th = fmin(fmax(th, T(-1)), T(1));
                out[i] = th;
            }
            return;
        }
    }
    if (SOLVE == kSolveNewton) {
        // the same seed and corrections as cubic_root(), decided once for all N
        // points: every point within its seed's range and, with the rounding guard
        // on, every |xi| <= 1 + 8 ulp (fast2max), where min/max is the guard
        T th[N];
        bool ok;
        if (c.seed == 0) {
            T my = T(0), m2 = T(0);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const T x = xi[i] * c.rb;
                const T y = (c.t * x) * x;
                my = nanmax(my, y);
                m2 = nanmax(m2, xi[i] * xi[i]);
                th[i] = newton_seed3(x, y);
            }
            ok = my <= c.ymax && m2 <= c.fast2max;
        } else {
            T m2 = T(0);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const T x2 = xi[i] * xi[i];
                m2 = nanmax(m2, x2);
                th[i] = newton_seed_rational(xi[i], x2, c);
            }
            ok = m2 <= c.xi2max && m2 <= c.fast2max;
        }
        if (ok) {
#pragma unroll
            for (int k = 0; k < NewtonMax<T>::value; ++k) {
                if (k < c.newton) {
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                        const T th2 = th[i] * th[i];
                        const T p = residual(th[i], th2, xi[i], c.a, c.b);
                        const T dp = dfma(c.three_a, th2, c.b);
                        th[i] = dfma(-p, arcp(dp), th[i]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < N; ++i) out[i] = c.clamp ? fmin(fmax(th[i], T(-1)), T(1)) : th[i];
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = cubic_root<T, SOLVE>(xi[i], c);
}

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using V = float4;
    static __device__ __forceinline__ void get(const float* p, float* o) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void put(float* p, const float* o) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
    static __device__ __forceinline__ void ldg(const float* p, float* o) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <>
struct Vec<double> {
    using V = double2;
    static __device__ __forceinline__ void get(const double* p, double* o) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void put(double* p, const double* o) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
    static __device__ __forceinline__ void ldg(const double* p, double* o) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
};

// z coordinate to load for logical plane p (ghost rule along z).
template <int BC>
__device__ __forceinline__ int zsrc(int p, int nz) {
    if (p >= 0 && p < nz) return p;
    if (BC == ACS_BC_PERIODIC) return p < 0 ? p + nz : p - nz;
    if (BC == ACS_BC_NEUMANN) return p < 0 ? 0 : nz - 1;
    return p;  // outside the tensor: TMA fills zeros
}

}  // namespace acs
