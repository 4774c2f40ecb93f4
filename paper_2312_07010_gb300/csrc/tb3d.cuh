// tb3d.cuh -- K fused RLB-MIE-FD steps (Eq. IE-FD, Remark 1) per pass through HBM on
// a 3D grid (temporal blocking), FP32, rows of an even number of values.
//
// A CTA of 16 warps owns an xy window of 64 x 64 unknowns (a lane holds two values
// of each of four rows; warp w holds rows 4 w .. 4 w + 3) and streams a chunk of z
// planes through it with K time levels in flight.  When level 0 receives plane r,
// level s computes plane r - 2 s from its predecessor's planes r - 2 s - 1, r - 2 s,
// r - 2 s + 1, all computed in earlier iterations, so the K levels of an iteration
// are independent (one group of cubic solves).  A thread keeps, per level, its
// values of the last three planes in registers (the z neighbours); x neighbours come
// from warp shuffles, y neighbours from the thread's own rows or, for its first and
// last row, from the rows the warps above and below published in shared memory
// (three slots, one barrier per plane).  Level s is exact on the window minus s
// cells at each side, so the outer pair of columns and the outer K rows at each side
// are halo: a CTA writes 60 x (64 - 2 K) unknowns per plane, and a chunk streams K
// planes beyond each end.  Per point the arithmetic is the single-step kernels'
// (the same neighbour order, predictor2() / roots2() on pairs), so a pass gives the
// bits of K single steps.
//
// Ghost rules at every level (Eq. Ddeltax), as in the 2D kernel: the window is filled
// from a virtual extension that the scheme maps onto itself (periodic wraps, Neumann
// mirrors about the half cell beyond the face); for Dirichlet the nodes outside the
// grid are loaded as +0 and reset to +0 after every level.
#pragma once

#include <type_traits>

#include "acs_host.h"
#include "f32x2.cuh"
#include "tb2d.cuh"

namespace acs {

constexpr int kTb3Warps = 16;
constexpr int kMaxTemporalDepth3d = 2;

template <int K>
struct Tb3 {
    static constexpr int VX = 2;                     // values per lane and row (one pair)
    static constexpr int RY = 4;                     // rows per thread
    static constexpr int HG = (K + VX - 1) / VX;     // halo pairs per side
    static constexpr int WW = 32 * VX;               // window width
    static constexpr int OW = WW - 2 * HG * VX;      // columns written per window
    static constexpr int WH = kTb3Warps * RY;        // window height
    static constexpr int OH = WH - 2 * K;            // rows written per window
    // published boundary rows: [slot 3][level K][warp][first, last][lane] pairs
    static constexpr size_t PUB_BYTES = (size_t)3 * K * kTb3Warps * 2 * 32 * sizeof(f2);
};

__device__ __forceinline__ f2 ld_pair(const float* p) {
    f2 r;
    r.v = __ldg(reinterpret_cast<const unsigned long long*>(p));
    return r;
}
__device__ __forceinline__ void st_pair(float* p, f2 v) { *reinterpret_cast<unsigned long long*>(p) = v.v; }

template <int BC, int SOLVE, int K>
__global__ void __launch_bounds__(kTb3Warps * 32, 1) k_step3d_tb(const float* __restrict__ src, float* __restrict__ dst,
                                                                  Geo g, Coef<float> c, int ntx, int zch) {
    pdl_wait();
    using TB = Tb3<K>;
    constexpr int VX = TB::VX, RY = TB::RY, HG = TB::HG, WW = TB::WW, OW = TB::OW, WH = TB::WH, OH = TB::OH;
    extern __shared__ __align__(16) unsigned char tb3_smem[];
    f2* pub = reinterpret_cast<f2*>(tb3_smem);
    // pair published by (slot, level, warp, first / last row, lane) at
    // (((slot K + level) 16 + warp) 2 + which) 32 + lane

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz;
    const int64_t sz = g.sz;
    const int strip = blockIdx.x % ntx, trow = blockIdx.x / ntx;
    const int wx = strip * OW - HG * VX;     // first column of the window
    const int cx = wx + lane * VX;           // first column of this lane
    const int wy = trow * OH - K;            // first (virtual) row of the window
    const int ry0 = wy + warp * RY;          // first row of this thread
    const int za = blockIdx.y * zch, zb = min(za + zch, nz);
    const int NI = (zb - za) + 2 * K;        // planes streamed: the chunk plus K each side
    const bool colsin = wx >= 0 && wx + WW <= nx;
    const bool edge = BC == ACS_BC_DIRICHLET && (!colsin || wy < 0 || wy + WH > ny || za - K < 0 || zb + K > nz);
    const bool wlane = lane >= HG && lane < 32 - HG && cx < nx;
    const int wabove = warp > 0 ? warp - 1 : 0, wbelow = warp < kTb3Warps - 1 ? warp + 1 : kTb3Warps - 1;

    // offsets within a plane (which has fewer than 2^31 values) of this thread's stored
    // rows (-1: a Dirichlet row outside the grid), and whether a row is one the window
    // writes
    int rb[RY];
    bool rowout[RY], rowin[RY];
#pragma unroll
    for (int rr = 0; rr < RY; ++rr) {
        const int vy = ry0 + rr;
        const int yu = vmap<BC>(vy, ny);
        rb[rr] = yu < 0 ? -1 : yu * nx;
        rowin[rr] = vy >= 0 && vy < ny;
        rowout[rr] = warp * RY + rr >= K && warp * RY + rr < WH - K && vy < ny;
    }
    // published pairs: this thread's first row, and the rows it reads from the warps
    // above (their last row) and below (their first row), at slot 0, level 0
    const int pw = warp * 64 + lane, pa = wabove * 64 + 32 + lane, pb = wbelow * 64 + lane;
    constexpr int PLEV = kTb3Warps * 64, PSLOT = K * PLEV;
    const int xu0 = vmap<BC>(cx, nx), xu1 = vmap<BC>(cx + 1, nx);
    const bool colin0 = cx >= 0 && cx < nx, colin1 = cx + 1 >= 0 && cx + 1 < nx;

    auto run = [&](auto edge_tag) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        const PackedCoef pc = packed_coef(c);
        // plane i of the stream is virtual plane za - K + i
        auto load_plane = [&](int i, f2 (&o)[RY]) {
            const int zu = vmap<BC>(za - K + i, nz);
            const float* pl = src + (int64_t)zu * sz;
#pragma unroll
            for (int rr = 0; rr < RY; ++rr) {
                if (BC == ACS_BC_DIRICHLET && (zu < 0 || rb[rr] < 0)) {
                    o[rr] = f2_make(0.0f, 0.0f);
                    continue;
                }
                const float* rowp = pl + rb[rr];
                if (colsin) {
                    o[rr] = ld_pair(rowp + cx);
                } else {
                    o[rr] = f2_make(xu0 < 0 ? 0.0f : __ldg(rowp + xu0), xu1 < 0 ? 0.0f : __ldg(rowp + xu1));
                }
            }
        };
        f2 pre[RY];    // the next plane, in flight
        f2 w[K][3][RY];  // level s: this thread's pairs of the planes it computed in the last three iterations
#pragma unroll
        for (int s = 0; s < K; ++s)
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int rr = 0; rr < RY; ++rr) w[s][k][rr] = f2_make(0.0f, 0.0f);
        load_plane(0, pre);

        // Iteration i, PH = i % 3: levels 1..A compute; slot PH of each level's ring
        // holds iteration i - 3 (its z - 1 plane), PH + 1 iteration i - 2 (the centre,
        // whose boundary rows the warps published in shared-memory slot (PH + 1) % 3),
        // PH + 2 iteration i - 1 (z + 1).
        auto iter = [&](auto phc, auto ac, int i) {
            constexpr int PH = decltype(phc)::value;
            constexpr int A = decltype(ac)::value;
            constexpr int PC = (PH + 1) % 3, PN = (PH + 2) % 3;
            if constexpr (A > 0) {
                f2 xi[A * RY];
#pragma unroll
                for (int s = A; s >= 1; --s) {
                    const f2(&zm)[RY] = w[s - 1][PH];
                    const f2(&zc)[RY] = w[s - 1][PC];
                    const f2(&zp)[RY] = w[s - 1][PN];
                    const f2 above = pub[PC * PSLOT + (s - 1) * PLEV + pa];
                    const f2 below = pub[PC * PSLOT + (s - 1) * PLEV + pb];
#pragma unroll
                    for (int rr = 0; rr < RY; ++rr) {
                        const f2 ym = rr == 0 ? above : zc[rr - 1];
                        const f2 yp = rr == RY - 1 ? below : zc[rr + 1];
                        const float z0 = f2_lo(zc[rr]), z1 = f2_hi(zc[rr]);
                        const float left = __shfl_up_sync(0xffffffffu, z1, 1);
                        const float right = __shfl_down_sync(0xffffffffu, z0, 1);
                        // ((zm + zp) + (ym + yp)) + (xm + xp), the neighbour order of nsum()
                        const f2 sx = f2_make(left + z1, z0 + right);
                        const f2 sum = f2_add(f2_add(f2_add(zm[rr], zp[rr]), f2_add(ym, yp)), sx);
                        xi[(s - 1) * RY + rr] = predictor2(zc[rr], sum, pc);
                    }
                }
                float out[2 * A * RY];
                roots2<SOLVE, A * RY>(xi, out, c, pc);
#pragma unroll
                for (int s = A; s >= 1; --s) {
                    const int vz = za - K + i - 2 * s;  // virtual plane of level s's new plane
                    f2 o[RY];
#pragma unroll
                    for (int rr = 0; rr < RY; ++rr) {
                        float lo = out[2 * ((s - 1) * RY + rr)], hi = out[2 * ((s - 1) * RY + rr) + 1];
                        if (EDGE) {
                            const bool pin = vz >= 0 && vz < nz && rowin[rr];
                            lo = (pin && colin0) ? lo : 0.0f;
                            hi = (pin && colin1) ? hi : 0.0f;
                        }
                        o[rr] = f2_make(lo, hi);
                    }
                    if (s < K) {
#pragma unroll
                        for (int rr = 0; rr < RY; ++rr) w[s][PH][rr] = o[rr];
                        pub[PH * PSLOT + s * PLEV + pw] = o[0];
                        pub[PH * PSLOT + s * PLEV + pw + 32] = o[RY - 1];
                    } else if (wlane && vz >= za && vz < zb) {
                        float* op = dst + (int64_t)vz * sz + (ry0 * nx + cx);
#pragma unroll
                        for (int rr = 0; rr < RY; ++rr)
                            if (rowout[rr]) st_pair(op + rr * nx, o[rr]);
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < RY; ++rr) w[0][PH][rr] = pre[rr];
            pub[PH * PSLOT + pw] = pre[0];
            pub[PH * PSLOT + pw + 32] = pre[RY - 1];
            if (i + 1 < NI) load_plane(i + 1, pre);
            __syncthreads();
        };
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        using I2 = std::integral_constant<int, 2>;
        // the first 3 K iterations run only the levels with exact input (as in 2D)
        tb_prologue<0, K>([&](auto ac, int i) {
            iter(I0(), ac, i);
            iter(I1(), ac, i + 1);
            iter(I2(), ac, i + 2);
        });
        using IK = std::integral_constant<int, K>;
        const int NL = NI + K;
        for (int i0 = 3 * K; i0 < NL; i0 += 3) {
            iter(I0(), IK(), i0);
            iter(I1(), IK(), i0 + 1);
            iter(I2(), IK(), i0 + 2);
        }
    };
    if (edge) run(std::true_type());
    else run(std::false_type());
    pdl_trigger();
}

}  // namespace acs
