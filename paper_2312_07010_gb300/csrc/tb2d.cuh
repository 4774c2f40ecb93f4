// tb2d.cuh -- K fused RLB-MIE-FD steps (Eq. IE-FD, Remark 1) per pass through
// HBM on a 2D grid (temporal blocking), rows a multiple of 16 bytes.
//
// Each warp owns a column strip and a chunk of rows and streams down the rows with
// K time levels in flight.  A lane holds one 16-byte vector (VX values) of every
// row; for each level it keeps the last three rows it computed in registers.  When
// level 0 receives row r, level s computes row r - 2 s from its predecessor's rows
// r - 2 s - 1, r - 2 s, r - 2 s + 1 (x neighbours by warp shuffles), all computed in
// earlier iterations, so the K levels of an iteration are independent; a row is
// read from HBM once and written once for K steps.  The strip's window is 32 VX columns wide and every
// level is computed over all of it; level s is exact on the window minus s columns
// at each side, so the outer HG = ceil(K / VX) vectors of each side are halo and
// the inner 32 VX - 2 HG VX columns are written.  Along y the chunk is extended by
// K rows at each end the same way.  Per point the arithmetic is the single-step
// kernels' (predictor(), roots(), the same neighbour order), so the state after a
// pass is bit-identical to K single steps.
//
// Ghost rules at every intermediate level (Eq. Ddeltax): the window is filled from
// a virtual extension of the grid that the scheme maps onto itself -- periodic
// wraps, Neumann mirrors about the half-cell beyond the edge (phi_{-1-v} = phi_v,
// so the mirrored node carries the edge node's own value at every level, and the
// two neighbours of an edge node are summed in the commuted order, which IEEE
// addition does not distinguish).  For Dirichlet the nodes outside the grid are
// loaded as +0 and reset to +0 after every level.
#pragma once

#include <type_traits>

#include "acs_host.h"
#include "f32x2.cuh"

namespace acs {

constexpr int kTbWarps = 4;  // warps per CTA (the warps are independent; small CTAs spread evenly)

// Stored index of virtual coordinate v on an axis of n nodes: periodic wraps,
// Neumann reflects about -1/2 and n - 1/2; Dirichlet gives -1 outside [0, n)
// (the value there is +0).
template <int BC>
__device__ __forceinline__ int vmap(int v, int n) {
    if (v >= 0 && v < n) return v;
    if (BC == ACS_BC_PERIODIC) {
        int u = v % n;
        return u < 0 ? u + n : u;
    }
    if (BC == ACS_BC_NEUMANN) {
        const int m = 2 * n;
        int u = v % m;
        if (u < 0) u += m;
        return u < n ? u : m - 1 - u;
    }
    return -1;
}

// Groups g = G..K-1 of three iterations (3 g, 3 g + 1, 3 g + 2) of the fill, each
// running levels 1..g: f(std::integral_constant<int, g>, 3 g).
template <int G, int K, typename F>
__device__ __forceinline__ void tb_prologue(F&& f) {
    if constexpr (G < K) {
        f(std::integral_constant<int, G>(), 3 * G);
        tb_prologue<G + 1, K>(f);
    }
}

template <typename T, int K>
struct Tb2 {
    static constexpr int VX = 16 / (int)sizeof(T);  // values per lane and row
    static constexpr int HG = (K + VX - 1) / VX;    // halo vectors per side
    static constexpr int WW = 32 * VX;              // window width
    static constexpr int OW = WW - 2 * HG * VX;     // columns written per strip
};

// CTAs per SM the register budget is aimed at: FP32 16, 20, 24 warps for K = 4, 3, 2;
// FP64 (bound by its arithmetic pipe) no tighter than the default.
template <typename T, int K>
struct TbMinBlocks { static constexpr int value = sizeof(T) == 8 ? 1 : (K <= 2 ? 6 : (K == 3 ? 5 : 4)); };

template <typename T, int BC, int SOLVE, int K>
__global__ void __launch_bounds__(kTbWarps * 32, TbMinBlocks<T, K>::value) k_step2d_tb(const T* __restrict__ src, T* __restrict__ dst, Geo g,
                                                             Coef<T> c, int nstrips, int ych, int nwarps) {
    pdl_wait();
    using TB = Tb2<T, K>;
    constexpr int VX = TB::VX, HG = TB::HG, WW = TB::WW, OW = TB::OW;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * kTbWarps + (threadIdx.x >> 5);
    if (wid < nwarps) {
        const int nx = (int)g.nx, ny = (int)g.ny;
        const int strip = wid % nstrips, chunk = wid / nstrips;
        const int wx = strip * OW - HG * VX;  // first column of the window
        const int cx = wx + lane * VX;        // first column of this lane
        const int ya = chunk * ych, yb = min(ya + ych, ny);
        const int NI = (yb - ya) + 2 * K;     // rows streamed: the chunk plus K each side
        const bool wlane = lane >= HG && lane < 32 - HG && cx < nx;
        // the window's columns lie inside the grid: 16-byte vector loads
        const bool colsin = wx >= 0 && wx + WW <= nx;
        // the Dirichlet zero fix-ups are compiled only into the copy of the loop that
        // warps touching the boundary run (Neumann and periodic need none)
        const bool edge = BC == ACS_BC_DIRICHLET && (!colsin || ya - K < 0 || yb + K > ny);

        auto run = [&](auto edge_tag) {
            constexpr bool EDGE = decltype(edge_tag)::value;
            PackedCoef pc;
            if constexpr (std::is_same<T, float>::value) pc = packed_coef(c);
            // Dirichlet: columns of this lane outside the grid hold +0 at every level
            bool colin[VX];
#pragma unroll
            for (int v = 0; v < VX; ++v) colin[v] = cx + v >= 0 && cx + v < nx;
            // row i of the stream is virtual row ya - K + i
            auto load_row = [&](int i, T (&o)[VX]) {
                const int u = vmap<BC>(ya - K + i, ny);
                if (u < 0) {
#pragma unroll
                    for (int v = 0; v < VX; ++v) o[v] = T(0);
                    return;
                }
                const T* rowp = src + (int64_t)u * nx;
                if (colsin) {
                    Vec<T>::ldg(rowp + cx, o);
                } else {
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        const int xu = vmap<BC>(cx + v, nx);
                        o[v] = xu < 0 ? T(0) : __ldg(rowp + xu);
                    }
                }
            };

            T pre[3][VX];  // stream rows i, i + 1, i + 2 in flight
            T w[K][3][VX]; // level s: the rows it computed in the last three iterations, iteration i' in slot i' % 3
#pragma unroll
            for (int s = 0; s < K; ++s)
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int v = 0; v < VX; ++v) w[s][k][v] = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) load_row(k, pre[k]);

            // Iteration i: level 0 takes stream row i; level s >= 1 computes stream row
            // i - 2 s from the rows its predecessor computed in iterations i - 3, i - 2,
            // i - 1, so the K levels of one iteration are independent of each other (the
            // solve of all their K VX points is one group).  Level s is exact on stream
            // rows [s, NI - s), which it computes in iterations [3 s, NI + s); level K's
            // rows [K, NI - K) are the chunk.  The first 3 K iterations (unrolled) run
            // only the levels that have exact input, the rest run all K levels (the last
            // K iterations compute a few rows past the exact range, never stored).
            //   A: levels 1..A computed in this iteration; PH = i % 3.
            auto iter = [&](auto phc, auto ac, int i) {
                constexpr int PH = decltype(phc)::value;
                constexpr int A = decltype(ac)::value;
                if constexpr (A > 0) {
                    T out[A * VX];
                    if constexpr (std::is_same<T, float>::value) {
                        // FP32: the same operations on pairs of points
                        f2 xi[2 * A];
#pragma unroll
                        for (int s = A; s >= 1; --s) {
                            const T(&m)[VX] = w[s - 1][PH];            // iteration i - 3
                            const T(&z)[VX] = w[s - 1][(PH + 1) % 3];  // iteration i - 2
                            const T(&p)[VX] = w[s - 1][(PH + 2) % 3];  // iteration i - 1
                            const T left = __shfl_up_sync(0xffffffffu, z[VX - 1], 1);
                            const T right = __shfl_down_sync(0xffffffffu, z[0], 1);
                            f2 x2p[2];
                            predict4_2d(m, z, p, left, right, pc, x2p);
                            xi[2 * (s - 1)] = x2p[0];
                            xi[2 * (s - 1) + 1] = x2p[1];
                        }
                        roots2<SOLVE, 2 * A>(xi, out, c, pc);
                    } else {
                        T xi[A * VX];
#pragma unroll
                        for (int s = A; s >= 1; --s) {
                            const T(&m)[VX] = w[s - 1][PH];
                            const T(&z)[VX] = w[s - 1][(PH + 1) % 3];
                            const T(&p)[VX] = w[s - 1][(PH + 2) % 3];
                            const T left = __shfl_up_sync(0xffffffffu, z[VX - 1], 1);
                            const T right = __shfl_down_sync(0xffffffffu, z[0], 1);
#pragma unroll
                            for (int v = 0; v < VX; ++v) {
                                const T xm = v == 0 ? left : z[v - 1];
                                const T xp = v == VX - 1 ? right : z[v + 1];
                                xi[(s - 1) * VX + v] = predictor(z[v], nsum(m[v], p[v], xm, xp), c);
                            }
                        }
                        roots<T, SOLVE, A * VX>(xi, out, c);
                    }
#pragma unroll
                    for (int s = A; s >= 1; --s) {
                        const int q = ya - K + i - 2 * s;  // grid row of level s's new row
                        T* o = &out[(s - 1) * VX];
                        if (EDGE) {
                            const bool rowin = q >= 0 && q < ny;
#pragma unroll
                            for (int v = 0; v < VX; ++v) o[v] = (rowin && colin[v]) ? o[v] : T(0);
                        }
                        if (s < K) {
#pragma unroll
                            for (int v = 0; v < VX; ++v) w[s][PH][v] = o[v];
                        } else if (wlane && q >= ya && q < yb) {
                            Vec<T>::put(dst + (int64_t)q * nx + cx, o);
                        }
                    }
                }
#pragma unroll
                for (int v = 0; v < VX; ++v) w[0][PH][v] = pre[PH][v];
                if (i + 3 < NI) load_row(i + 3, pre[PH]);
            };
            using I0 = std::integral_constant<int, 0>;
            using I1 = std::integral_constant<int, 1>;
            using I2 = std::integral_constant<int, 2>;
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
    }
    pdl_trigger();
}

bool step2d_tb_supported(int dtype, int depth, const Geo& g);

// Rows per chunk: about one wave of resident warps, but chunks of at least 8 K rows
// (a chunk streams 3 K rows beyond its own).
inline int choose_ych(int64_t nstrips, int64_t ny, int K, int resident_warps) {
    const int64_t minrows = 8 * K;
    int64_t chunks = std::max<int64_t>(1, resident_warps / std::max<int64_t>(1, nstrips));
    int64_t ych = (ny + chunks - 1) / chunks;
    if (ych < minrows) ych = std::min<int64_t>(ny, minrows);
    return (int)std::max<int64_t>(1, ych);
}

template <typename T, int K>
static cudaError_t launch_tb2d_k(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int ych,
                                 cudaStream_t st) {
    using TB = Tb2<T, K>;
    const int64_t nstrips = (g.nx + TB::OW - 1) / TB::OW;
    cudaError_t e = cudaSuccess;
    ACS_SOLVE_DISPATCH_UNIT(c, SV, {
        auto kern = bc == 0 ? k_step2d_tb<T, 0, SV, K> : (bc == 1 ? k_step2d_tb<T, 1, SV, K> : k_step2d_tb<T, 2, SV, K>);
        if (ych <= 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTbWarps * 32, 0);
            ych = choose_ych(nstrips, g.ny, K, std::max(1, sms * std::max(1, per_sm) * kTbWarps));
        }
        const int64_t nchunks = (g.ny + ych - 1) / ych;
        const int64_t nwarps = nstrips * nchunks;
        if (nwarps > 0x7fffffff / 2) return cudaErrorNotSupported;
        const unsigned blocks = (unsigned)((nwarps + kTbWarps - 1) / kTbWarps);
        e = launch_pdl(kern, dim3(blocks), dim3(kTbWarps * 32), 0, st, src, dst, g, c, (int)nstrips, ych,
                       (int)nwarps);
    });
    return e;
}

template <typename T>
cudaError_t launch_step2d_tb(int bc, int depth, const T* src, T* dst, const Geo& g, const Coef<T>& c, int ych,
                             cudaStream_t st) {
    switch (depth) {
        case 2: return launch_tb2d_k<T, 2>(bc, src, dst, g, c, ych, st);
        case 3: return launch_tb2d_k<T, 3>(bc, src, dst, g, c, ych, st);
        case 4: return launch_tb2d_k<T, 4>(bc, src, dst, g, c, ych, st);
        default: return cudaErrorNotSupported;
    }
}
}  // namespace acs
