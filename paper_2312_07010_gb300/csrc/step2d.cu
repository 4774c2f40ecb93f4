// step2d.cu -- one RLB-MIE-FD step (Eq. IE-FD, Remark 1) on a 2D grid from
// shared-memory tiles.
//
// Each CTA walks a run of 128 x 16 tiles down a vertical strip.  The next tile plus
// its one-cell halo is staged with cp.async (ghost rules applied while loading)
// while the current one is updated, so loads and arithmetic overlap; every unknown
// is read from HBM once per step (halo rows come back from L2) and written once.
// Any grid shape works: no alignment condition on the row length.
#include "acs_host.h"
#include "tile2d.cuh"

namespace acs {

template <typename T, int BC, int SOLVE>
__global__ void __launch_bounds__(256) k_step2d(const T* __restrict__ src, T* __restrict__ dst, Geo g, Coef<T> c,
                                                int ntx, int nty, int per_cta) {
    using TT = Tile2<T>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* const base = reinterpret_cast<T*>(sm_raw);
    const int ny = (int)g.ny, nx = (int)g.nx;
    const int ntiles = ntx * nty;
    const int t0 = blockIdx.x * per_cta;
    const int t1 = min(t0 + per_cta, ntiles);
    if (t0 >= t1) return;
    // tiles are numbered down each vertical strip: t -> (x tile t / nty, y tile t % nty)
    auto origin = [&](int t, int& x0, int& y0) {
        x0 = (t / nty) * TT::TX;
        y0 = (t % nty) * TT::TY;
    };
    // ring of DEPTH staged tiles: tile t lives in buffer (t - t0) % DEPTH
#pragma unroll
    for (int k = 0; k < TT::DEPTH - 1; ++k) {
        if (t0 + k < t1) {
            int x0, y0;
            origin(t0 + k, x0, y0);
            stage_tile<T>(base + k * TT::N, src, ny, nx, BC, x0, y0);
        }
        cp_async_commit();
    }
    for (int t = t0; t < t1; ++t) {
        if (t + TT::DEPTH - 1 < t1) {
            int x0, y0;
            origin(t + TT::DEPTH - 1, x0, y0);
            stage_tile<T>(base + ((t + TT::DEPTH - 1 - t0) % TT::DEPTH) * TT::N, src, ny, nx, BC, x0, y0);
        }
        cp_async_commit();
        cp_async_wait<TT::DEPTH - 1>();
        __syncthreads();
        int x0, y0;
        origin(t, x0, y0);
        update_tile<T, SOLVE>(base + ((t - t0) % TT::DEPTH) * TT::N, dst, ny, nx, x0, y0, c);
        __syncthreads();
    }
}

bool step2d_supported(const Geo& g) { return g.nz == 1 && g.nx < (1 << 30) && g.ny < (1 << 30); }

template <typename T>
cudaError_t launch_step2d(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int per_cta,
                          cudaStream_t st) {
    using TT = Tile2<T>;
    const int ntx = (int)((g.nx + TT::TX - 1) / TT::TX);
    const int nty = (int)((g.ny + TT::TY - 1) / TT::TY);
    const int64_t ntiles = (int64_t)ntx * nty;
    if (ntiles > 0x7fffffff) return cudaErrorNotSupported;
    if (per_cta <= 0) per_cta = (int)std::max<int64_t>(1, std::min<int64_t>(16, ntiles / (152 * 6)));
    const int grid = (int)((ntiles + per_cta - 1) / per_cta);
    const size_t smem = TT::DEPTH * TT::N * sizeof(T);
    cudaError_t e = cudaSuccess;
#define ACS_2D_CASE(B)                                                                               \
    if (bc == B) {                                                                                   \
        ACS_SOLVE_DISPATCH(c.solve, SV, {                                                            \
            auto kern = k_step2d<T, B, SV>;                                                          \
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
            if (e == cudaSuccess) kern<<<grid, TT::THREADS, smem, st>>>(src, dst, g, c, ntx, nty, per_cta); \
        });                                                                                          \
    }
    ACS_2D_CASE(0) ACS_2D_CASE(1) ACS_2D_CASE(2)
#undef ACS_2D_CASE
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template cudaError_t launch_step2d<float>(int, const float*, float*, const Geo&, const Coef<float>&, int,
                                          cudaStream_t);
template cudaError_t launch_step2d<double>(int, const double*, double*, const Geo&, const Coef<double>&, int,
                                           cudaStream_t);

}  // namespace acs
