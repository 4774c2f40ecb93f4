// step_naive.cu -- one RLB-MIE-FD step (Eq. IE-FD, Remark 1), one thread per unknown.
//
// Every thread reads its own value and its 2d neighbours straight from global
// memory (the L1/L2 caches supply the reuse) and writes one value.  It is the
// reference variant for the optimized kernels and the fallback for shapes they do
// not cover; its per-point arithmetic is acs::update(), shared by all variants.
#include "acs_kernels.cuh"

namespace acs {

// Neighbour one step down / up an axis of size n and stride s, with the ghost
// rule of Eq. (Ddeltax): periodic wraps, Neumann mirrors onto the node itself,
// Dirichlet reads 0.
template <int BC, typename T>
__device__ __forceinline__ T nb_lo(const T* __restrict__ p, int64_t i, int64_t c, int64_t n, int64_t s) {
    if (c > 0) return p[i - s];
    if (BC == ACS_BC_PERIODIC) return p[i + (n - 1) * s];
    if (BC == ACS_BC_NEUMANN) return p[i];
    return T(0);
}
template <int BC, typename T>
__device__ __forceinline__ T nb_hi(const T* __restrict__ p, int64_t i, int64_t c, int64_t n, int64_t s) {
    if (c < n - 1) return p[i + s];
    if (BC == ACS_BC_PERIODIC) return p[i - (n - 1) * s];
    if (BC == ACS_BC_NEUMANN) return p[i];
    return T(0);
}

template <typename T, int D, int BC, int SOLVE>
__global__ void __launch_bounds__(256) k_step_naive(const T* __restrict__ src, T* __restrict__ dst,
                                                    Geo g, Coef<T> c) {
    pdl_wait();
    for (int64_t z = blockIdx.z; z < g.nz; z += gridDim.z) {
        for (int64_t y = blockIdx.y; y < g.ny; y += gridDim.y) {
            const int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < g.nx;
                 x += (int64_t)gridDim.x * blockDim.x) {
                const int64_t i = row + x;
                const T p = src[i];
                T s;
                const T xm = nb_lo<BC>(src, i, x, g.nx, 1), xp = nb_hi<BC>(src, i, x, g.nx, 1);
                if (D == 1) {
                    s = nsum(xm, xp);
                } else if (D == 2) {
                    const T ym = nb_lo<BC>(src, i, y, g.ny, g.sy), yp = nb_hi<BC>(src, i, y, g.ny, g.sy);
                    s = nsum(ym, yp, xm, xp);
                } else {
                    const T ym = nb_lo<BC>(src, i, y, g.ny, g.sy), yp = nb_hi<BC>(src, i, y, g.ny, g.sy);
                    const T zm = nb_lo<BC>(src, i, z, g.nz, g.sz), zp = nb_hi<BC>(src, i, z, g.nz, g.sz);
                    s = nsum(zm, zp, ym, yp, xm, xp);
                }
                dst[i] = update<T, SOLVE>(p, s, c);
            }
        }
    }
    pdl_trigger();
}

static dim3 naive_grid(const Geo& g) {
    const int64_t bx = (g.nx + 255) / 256;
    dim3 grid((unsigned)std::min<int64_t>(bx, 1 << 20), (unsigned)std::min<int64_t>(g.ny, 65535),
              (unsigned)std::min<int64_t>(g.nz, 65535));
    return grid;
}

template <typename T>
cudaError_t launch_step_naive(int dims, int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c,
                              cudaStream_t st) {
    dim3 grid = naive_grid(g), block(256);
#define ACS_NAIVE_CASE(D, B)                                                                 \
    if (dims == D && bc == B) {                                                              \
        cudaError_t e = cudaSuccess;                                                         \
        ACS_SOLVE_DISPATCH(c.solve, S, (e = launch_pdl(k_step_naive<T, D, B, S>, grid, block, 0, st, src, dst, g, c))); \
        return e;                                                                            \
    }
    ACS_NAIVE_CASE(1, 0) ACS_NAIVE_CASE(1, 1) ACS_NAIVE_CASE(1, 2)
    ACS_NAIVE_CASE(2, 0) ACS_NAIVE_CASE(2, 1) ACS_NAIVE_CASE(2, 2)
    ACS_NAIVE_CASE(3, 0) ACS_NAIVE_CASE(3, 1) ACS_NAIVE_CASE(3, 2)
#undef ACS_NAIVE_CASE
    return cudaErrorInvalidValue;
}

template cudaError_t launch_step_naive<float>(int, int, const float*, float*, const Geo&, const Coef<float>&, cudaStream_t);
template cudaError_t launch_step_naive<double>(int, int, const double*, double*, const Geo&, const Coef<double>&, cudaStream_t);

}  // namespace acs
