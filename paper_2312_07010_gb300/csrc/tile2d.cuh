// tile2d.cuh -- shared-memory tiles for 2D steps: the tile plus a one-cell halo is
// staged with cp.async (ghost rules of Eq. Ddeltax applied while loading, so the
// compute is the same for every point), then each thread updates its points.
// Used by the single-problem 2D kernel and the batched persistent kernel.
#pragma once

#include "acs_device.cuh"

namespace acs {

template <typename T>
struct Tile2 {
    static constexpr int TX = 128;        // tile width
    static constexpr int TY = 16;         // tile height
    static constexpr int BW = TX + 2;     // staged width (one-cell halo)
    static constexpr int BH = TY + 2;     // staged height
    static constexpr int N = BW * BH;     // staged values
    static constexpr int THREADS = 256;
    static constexpr int PTS = TX * TY / THREADS;  // points per thread (8)
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Source index of staged position (gy, gx) in a ny x nx grid, or -1 for "zero":
// the box itself, the ghost ring by the boundary rule (wrap / mirror / zero), and
// zero for positions beyond the ghost ring (never read by a stored point).
__device__ __forceinline__ int64_t ghost_index(int gy, int gx, int ny, int nx, int bc) {
    if (gy < -1 || gy > ny || gx < -1 || gx > nx) return -1;
    const bool oy = gy < 0 || gy >= ny, ox = gx < 0 || gx >= nx;
    if (oy && ox) return -1;  // corner: the 5-point stencil never reads it
    if (oy || ox) {
        if (bc == ACS_BC_DIRICHLET) return -1;
        if (bc == ACS_BC_NEUMANN) {
            gy = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
            gx = gx < 0 ? 0 : (gx >= nx ? nx - 1 : gx);
        } else {
            gy = gy < 0 ? ny - 1 : (gy >= ny ? 0 : gy);
            gx = gx < 0 ? nx - 1 : (gx >= nx ? 0 : gx);
        }
    }
    return (int64_t)gy * nx + gx;
}

// Stage the tile at (x0, y0) of a ny x nx grid (halo included) into `buf`.
template <typename T>
__device__ __forceinline__ void stage_tile(T* buf, const T* __restrict__ src, int ny, int nx, int bc, int x0,
                                           int y0) {
    using TT = Tile2<T>;
    for (int i = threadIdx.x; i < TT::N; i += TT::THREADS) {
        const int r = i / TT::BW, cc = i - r * TT::BW;
        const int64_t j = ghost_index(y0 - 1 + r, x0 - 1 + cc, ny, nx, bc);
        const T* s = src + (j < 0 ? 0 : j);
        if (sizeof(T) == 4) cp_async4(buf + i, s, j >= 0);
        else cp_async8(buf + i, s, j >= 0);
    }
}

// Update the tile staged in `buf`: thread t owns rows (t / 32) * 2 + {0, 1} and
// columns lane + 32 k, k = 0..3; the five-point sum is read from shared memory.
template <typename T, int SOLVE>
__device__ __forceinline__ void update_tile(const T* buf, T* __restrict__ dst, int ny, int nx, int x0, int y0,
                                            const Coef<T>& c) {
    using TT = Tile2<T>;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int r = 2 * w + rr;  // tile row
        const int gy = y0 + r;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int cx = lane + 32 * k;  // tile column
            const int gx = x0 + cx;
            const T* q = buf + (r + 1) * TT::BW + (cx + 1);
            const T p = q[0];
            const T s = nsum(q[-TT::BW], q[TT::BW], q[-1], q[1]);
            const T v = update<T, SOLVE>(p, s, c);
            if (gy < ny && gx < nx) dst[(int64_t)gy * nx + gx] = v;
        }
    }
}

}  // namespace acs
