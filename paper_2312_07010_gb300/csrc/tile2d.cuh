// tile2d.cuh -- shared-memory tiles for 2D steps of any shape: the tile plus a
// one-cell halo is staged with cp.async (ghost rules of Eq. Ddeltax applied while
// loading, so the compute is the same for every point), then each thread updates
// its points.  Used by the single-problem 2D kernel for rows that are not a multiple
// of 16 bytes and by the 2D adjoint for such rows.
//
// Layout of a staged tile: TY + 2 rows of BW values; the tile's interior starts at
// column VX (one 16-byte vector) so each thread can read its VX values as one
// aligned vector; the x halo sits at columns VX - 1 and VX + TX.
#pragma once

#include "acs_device.cuh"

namespace acs {

template <typename T>
struct Tile2 {
    static constexpr int VX = 16 / (int)sizeof(T);  // values per 16-byte vector
    static constexpr int TX = 32 * VX;              // tile width: one vector per lane
    static constexpr int TY = 16;                   // tile height: 8 warps x 2 rows
    static constexpr int BW = TX + 2 * VX;          // staged row (interior at column VX)
    static constexpr int BH = TY + 2;               // staged rows (one-cell halo)
    static constexpr int N = BW * BH;               // staged values (halo columns beyond one cell unused)
    static constexpr int THREADS = 256;
    static constexpr int DEPTH = 3;                 // staged tiles in flight (ring of buffers)
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

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
    if (sizeof(T) == 4) cp_async4(dst, src, valid);
    else cp_async8(dst, src, valid);
}

// Stage the tile at (x0, y0) of a ny x nx grid (one-cell halo included) into `buf`:
// staged column c holds grid column x0 - VX + c; only columns VX - 1 .. VX + TX are used.
// Warps take staged rows in turn and lanes walk a row, so addresses are a base plus the
// lane; the ghost rule applies to whole ghost rows and to the two ends of a row.
template <typename T>
__device__ __forceinline__ void stage_tile(T* buf, const T* __restrict__ src, int ny, int nx, int bc, int x0,
                                           int y0) {
    using TT = Tile2<T>;
    constexpr int W = TT::TX + 2;  // used columns per staged row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < TT::BH; r += TT::THREADS / 32) {
        int gy = y0 - 1 + r;
        bool rowok = true;
        if (gy < 0 || gy >= ny) {
            if (bc == ACS_BC_DIRICHLET || gy < -1 || gy > ny) rowok = false;
            else if (bc == ACS_BC_NEUMANN) gy = gy < 0 ? 0 : ny - 1;
            else gy = gy < 0 ? ny - 1 : 0;
        }
        const T* row = src + (int64_t)(rowok ? gy : 0) * nx;
        T* out = buf + r * TT::BW + (TT::VX - 1);
        for (int cc = lane; cc < W; cc += 32) {
            int gx = x0 - 1 + cc;
            bool ok = rowok;
            if (gx < 0 || gx >= nx) {
                if (bc == ACS_BC_DIRICHLET || gx < -1 || gx > nx) ok = false;
                else if (bc == ACS_BC_NEUMANN) gx = gx < 0 ? 0 : nx - 1;
                else gx = gx < 0 ? nx - 1 : 0;
            }
            cp_async_elem(out + cc, row + (ok ? gx : 0), ok);
        }
    }
}

template <typename T>
struct TileVec;
template <>
struct TileVec<float> {
    static __device__ __forceinline__ void get(const float* p, float* o) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <>
struct TileVec<double> {
    static __device__ __forceinline__ void get(const double* p, double* o) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        o[0] = v.x; o[1] = v.y;
    }
};

// Update the tile staged in `buf` (ghost values already in its halo): warp w owns
// tile rows 2w and 2w + 1, lane l the VX columns VX l .. VX l + VX - 1; x neighbours
// come from registers and shuffles, y neighbours as aligned vectors.
template <typename T, int SOLVE>
__device__ __forceinline__ void update_tile(const T* buf, T* __restrict__ dst, int ny, int nx, int x0, int y0,
                                            const Coef<T>& c) {
    using TT = Tile2<T>;
    constexpr int VX = TT::VX, BW = TT::BW;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = 2 * w;
    const int cx = VX * lane;  // first tile column of this thread
    T cz[2][VX], below[VX], above[VX];
    TileVec<T>::get(buf + (r0 + 1) * BW + VX + cx, cz[0]);
    TileVec<T>::get(buf + (r0 + 2) * BW + VX + cx, cz[1]);
    TileVec<T>::get(buf + r0 * BW + VX + cx, below);
    TileVec<T>::get(buf + (r0 + 3) * BW + VX + cx, above);
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int gy = y0 + r0 + rr;
        T left = __shfl_up_sync(0xffffffffu, cz[rr][VX - 1], 1);
        T right = __shfl_down_sync(0xffffffffu, cz[rr][0], 1);
        if (lane == 0) left = buf[(r0 + rr + 1) * BW + VX - 1];
        if (lane == 31) right = buf[(r0 + rr + 1) * BW + VX + TT::TX];
        T out[VX];
#pragma unroll
        for (int v = 0; v < VX; ++v) {
            const T ym = rr == 0 ? below[v] : cz[0][v];
            const T yp = rr == 1 ? above[v] : cz[1][v];
            const T xm = v == 0 ? left : cz[rr][v - 1];
            const T xp = v == VX - 1 ? right : cz[rr][v + 1];
            out[v] = update<T, SOLVE>(cz[rr][v], nsum(ym, yp, xm, xp), c);
        }
        if (gy < ny) {
            T* o = dst + (int64_t)gy * nx + x0 + cx;
#pragma unroll
            for (int v = 0; v < VX; ++v)
                if (x0 + cx + v < nx) o[v] = out[v];
        }
    }
}

}  // namespace acs
