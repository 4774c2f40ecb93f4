// step_lb.cu -- the time step in its collide-and-stream (population) form (Sec. II):
// the lattice Boltzmann form the scheme is derived from, kept for comparison with
// the macroscopic form (Eq. IE-FD) that the other kernels implement.
//
// A DdQ(2d+1) lattice stores 2d+1 populations per node.  Per step:
//   collide  g_k(y) = f_k^eq(y) + s_A w_k c_k . Pi^ne(y)                (Eqs. fieq-Fi, fneq)
//            f_k^eq = w_k phi,  c_k . Pi^ne = -dt c_s^2 (c_k . grad phi) / s,  s_A = (1 - s) / c_s^2,
//            c_k . grad phi (y) = (phi(y + c_k dt) - phi(y)) / dt      (Eq. pine, per link)
//            so g_k(y) = w_k phi(y) - kappa (phi(y + c_k dt) - phi(y)),  kappa = (1 - s) w_1 / s,
//            and g_0 = w_0 phi;
//   stream   every node pulls g_k(x - c_k dt) and sums over k; with the source terms of
//            Eq. (RLB), sum_k F_k = -f(phi):  theta + (dt/2) f(theta) = sum_k g_k(x - c_k dt) - (dt/2) f(phi(x));
//   solve    the cubic for theta (Remark 1).
// Boundaries: a ghost node outside the box holds the boundary value of Eq. (Ddeltax)
// (wrap, mirror onto the boundary node, zero) and its populations collide like any
// other; the stream kernel forms the one population a ghost sends inward from the
// boundary node's own value (periodic: the wrapped node's stored population).
//
// The populations live in a caller buffer, one array of n^d values per direction
// (k = 0; +x, +y, +z; -x, -y, -z), n^d + kLbGap values apart.  Summed, the form equals Eq. (IE-FD) up to
// rounding; it moves (2d+1) values out and back in per node where Eq. (IE-FD) moves
// none, which is the memory and traffic cost the macroscopic form removes.
#include "acs_kernels.cuh"
#include "stream_tile.cuh"

namespace acs {

template <typename T>
struct LbCoef {
    T w0, w1, kappa;  // rest weight, link weight, (1 - s) w1 / s
};

// phi one step along +/-axis (stride s, coordinate c of n) with the ghost rule.
template <int BC, typename T>
__device__ __forceinline__ T lb_nbr(const T* src, int64_t i, int64_t c, int64_t n, int64_t s, int dir) {
    if (dir > 0) {
        if (c < n - 1) return src[i + s];
        if (BC == ACS_BC_PERIODIC) return src[i - (n - 1) * s];
    } else {
        if (c > 0) return src[i - s];
        if (BC == ACS_BC_PERIODIC) return src[i + (n - 1) * s];
    }
    return BC == ACS_BC_NEUMANN ? src[i] : T(0);
}

template <typename T, int D, int BC>
__global__ void __launch_bounds__(256) k_lb_collide(const T* __restrict__ src, T* __restrict__ pop, Geo g,
                                                    LbCoef<T> lc) {
    const int64_t tot = g.total + kLbGap;  // stride between population arrays
    for (int64_t z = blockIdx.z; z < g.nz; z += gridDim.z)
        for (int64_t y = blockIdx.y; y < g.ny; y += gridDim.y) {
            const int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < g.nx;
                 x += (int64_t)gridDim.x * blockDim.x) {
                const int64_t i = row + x;
                const T p = src[i];
                pop[i] = lc.w0 * p;
                const int64_t c[3] = {x, y, z}, n[3] = {g.nx, g.ny, g.nz}, s[3] = {1, g.sy, g.sz};
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T up = lb_nbr<BC>(src, i, c[k], n[k], s[k], +1);
                    const T dn = lb_nbr<BC>(src, i, c[k], n[k], s[k], -1);
                    pop[(1 + k) * tot + i] = lc.w1 * p - lc.kappa * (up - p);
                    pop[(1 + D + k) * tot + i] = lc.w1 * p - lc.kappa * (dn - p);
                }
            }
        }
}

template <typename T, int D, int BC, int SOLVE>
__global__ void __launch_bounds__(256) k_lb_stream(const T* __restrict__ src, const T* __restrict__ pop,
                                                   T* __restrict__ dst, Geo g, LbCoef<T> lc, Coef<T> cf) {
    const int64_t tot = g.total + kLbGap;  // stride between population arrays
    for (int64_t z = blockIdx.z; z < g.nz; z += gridDim.z)
        for (int64_t y = blockIdx.y; y < g.ny; y += gridDim.y) {
            const int64_t row = z * g.sz + y * g.sy;
            for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < g.nx;
                 x += (int64_t)gridDim.x * blockDim.x) {
                const int64_t i = row + x;
                const T p = src[i];
                // population a boundary ghost sends into this node: w1 * phi_ghost - kappa * (p - phi_ghost)
                const T ghost = BC == ACS_BC_NEUMANN ? lc.w1 * p : -(lc.kappa * p);
                T sum = pop[i];
                const int64_t c[3] = {x, y, z}, n[3] = {g.nx, g.ny, g.nz}, s[3] = {1, g.sy, g.sz};
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T* gp = pop + (1 + k) * tot;      // +e_k population, sent from x - e_k
                    const T* gm = pop + (1 + D + k) * tot;  // -e_k population, sent from x + e_k
                    T from_lo, from_hi;
                    if (c[k] > 0) from_lo = gp[i - s[k]];
                    else from_lo = BC == ACS_BC_PERIODIC ? gp[i + (n[k] - 1) * s[k]] : ghost;
                    if (c[k] < n[k] - 1) from_hi = gm[i + s[k]];
                    else from_hi = BC == ACS_BC_PERIODIC ? gm[i - (n[k] - 1) * s[k]] : ghost;
                    sum = sum + from_lo;
                    sum = sum + from_hi;
                }
                const T xi = sum - cf.a * (p * p * p - p);
                dst[i] = cubic_root<T, SOLVE>(xi, cf);
            }
        }
}

// Vectorised forms for rows of a multiple of VX values (one 16-byte vector per
// thread; the same operations in the same order as the scalar kernels above, so the
// results are identical).  Blocks are 32 vectors of 8 rows; the neighbours of a vector
// along x are its own values plus one scalar load at each end.
template <typename T, int BC>
__device__ __forceinline__ void lb_row_nbr(const T* src, int64_t i, int64_t c, int64_t n, int64_t s, int dir,
                                           const T (&p)[16 / sizeof(T)], T (&o)[16 / sizeof(T)]) {
    constexpr int VX = 16 / sizeof(T);
    if (dir > 0 ? c < n - 1 : c > 0) {
        Vec<T>::ldg(src + i + dir * s, o);
    } else if (BC == ACS_BC_PERIODIC) {
        Vec<T>::ldg(src + i - dir * (n - 1) * s, o);
    } else {
#pragma unroll
        for (int v = 0; v < VX; ++v) o[v] = BC == ACS_BC_NEUMANN ? p[v] : T(0);
    }
}

template <typename T, int D, int BC>
__global__ void __launch_bounds__(256) k_lb_collide_v(const T* __restrict__ src, T* __restrict__ pop, Geo g,
                                                      LbCoef<T> lc) {
    constexpr int VX = 16 / sizeof(T);
    const int64_t tot = g.total + kLbGap, nxv = g.nx / VX;  // tot: array stride
    for (int64_t z = blockIdx.z; z < g.nz; z += gridDim.z)
        for (int64_t y = blockIdx.y * (int64_t)blockDim.y + threadIdx.y; y < g.ny; y += (int64_t)gridDim.y * blockDim.y) {
            const int64_t row = z * g.sz + y * g.sy;
            for (int64_t xv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; xv < nxv;
                 xv += (int64_t)gridDim.x * blockDim.x) {
                const int64_t x = xv * VX, i = row + x;
                T p[VX], o[VX], up[VX], dn[VX];
                Vec<T>::ldg(src + i, p);
#pragma unroll
                for (int v = 0; v < VX; ++v) o[v] = lc.w0 * p[v];
                Vec<T>::put(pop + i, o);
                // x: the vector's own values and one neighbour at each end
                const T xl = x > 0 ? src[i - 1]
                                   : (BC == ACS_BC_PERIODIC ? src[row + g.nx - 1] : (BC == ACS_BC_NEUMANN ? p[0] : T(0)));
                const T xr = x + VX < g.nx ? src[i + VX]
                                           : (BC == ACS_BC_PERIODIC ? src[row] : (BC == ACS_BC_NEUMANN ? p[VX - 1] : T(0)));
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    up[v] = v < VX - 1 ? p[v + 1] : xr;
                    dn[v] = v > 0 ? p[v - 1] : xl;
                }
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    if (k == 1) {
                        lb_row_nbr<T, BC>(src, i, y, g.ny, g.sy, +1, p, up);
                        lb_row_nbr<T, BC>(src, i, y, g.ny, g.sy, -1, p, dn);
                    } else if (k == 2) {
                        lb_row_nbr<T, BC>(src, i, z, g.nz, g.sz, +1, p, up);
                        lb_row_nbr<T, BC>(src, i, z, g.nz, g.sz, -1, p, dn);
                    }
                    T a[VX], b[VX];
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        a[v] = lc.w1 * p[v] - lc.kappa * (up[v] - p[v]);
                        b[v] = lc.w1 * p[v] - lc.kappa * (dn[v] - p[v]);
                    }
                    Vec<T>::put(pop + (1 + k) * tot + i, a);
                    Vec<T>::put(pop + (1 + D + k) * tot + i, b);
                }
            }
        }
}

template <typename T, int D, int BC, int SOLVE>
__global__ void __launch_bounds__(256) k_lb_stream_v(const T* __restrict__ src, const T* __restrict__ pop,
                                                     T* __restrict__ dst, Geo g, LbCoef<T> lc, Coef<T> cf) {
    constexpr int VX = 16 / sizeof(T);
    const int64_t tot = g.total + kLbGap, nxv = g.nx / VX;  // tot: array stride
    for (int64_t z = blockIdx.z; z < g.nz; z += gridDim.z)
        for (int64_t y = blockIdx.y * (int64_t)blockDim.y + threadIdx.y; y < g.ny; y += (int64_t)gridDim.y * blockDim.y) {
            const int64_t row = z * g.sz + y * g.sy;
            for (int64_t xv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; xv < nxv;
                 xv += (int64_t)gridDim.x * blockDim.x) {
                const int64_t x = xv * VX, i = row + x;
                T p[VX], sum[VX], ghost[VX], lo[VX], hi[VX], w[VX];
                Vec<T>::ldg(src + i, p);
                Vec<T>::ldg(pop + i, sum);
#pragma unroll
                for (int v = 0; v < VX; ++v) ghost[v] = BC == ACS_BC_NEUMANN ? lc.w1 * p[v] : -(lc.kappa * p[v]);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T* gp = pop + (1 + k) * tot;      // +e_k population, sent from x - e_k
                    const T* gm = pop + (1 + D + k) * tot;  // -e_k population, sent from x + e_k
                    if (k == 0) {
                        Vec<T>::ldg(gp + i, w);
                        const T l = x > 0 ? gp[i - 1] : (BC == ACS_BC_PERIODIC ? gp[row + g.nx - 1] : ghost[0]);
#pragma unroll
                        for (int v = 0; v < VX; ++v) lo[v] = v > 0 ? w[v - 1] : l;
                        Vec<T>::ldg(gm + i, w);
                        const T r = x + VX < g.nx ? gm[i + VX] : (BC == ACS_BC_PERIODIC ? gm[row] : ghost[VX - 1]);
#pragma unroll
                        for (int v = 0; v < VX; ++v) hi[v] = v < VX - 1 ? w[v + 1] : r;
                    } else {
                        const int64_t c = k == 1 ? y : z, n = k == 1 ? g.ny : g.nz, s = k == 1 ? g.sy : g.sz;
                        if (c > 0) Vec<T>::ldg(gp + i - s, lo);
                        else if (BC == ACS_BC_PERIODIC) Vec<T>::ldg(gp + i + (n - 1) * s, lo);
                        else {
#pragma unroll
                            for (int v = 0; v < VX; ++v) lo[v] = ghost[v];
                        }
                        if (c < n - 1) Vec<T>::ldg(gm + i + s, hi);
                        else if (BC == ACS_BC_PERIODIC) Vec<T>::ldg(gm + i - (n - 1) * s, hi);
                        else {
#pragma unroll
                            for (int v = 0; v < VX; ++v) hi[v] = ghost[v];
                        }
                    }
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        sum[v] = sum[v] + lo[v];
                        sum[v] = sum[v] + hi[v];
                    }
                }
                T out[VX];
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    const T xi = sum[v] - cf.a * (p[v] * p[v] * p[v] - p[v]);
                    out[v] = cubic_root<T, SOLVE>(xi, cf);
                }
                Vec<T>::put(dst + i, out);
            }
        }
}

template <typename T>
static dim3 lb_grid(const Geo& g) {
    return dim3((unsigned)std::min<int64_t>((g.nx + 255) / 256, 1 << 20), (unsigned)std::min<int64_t>(g.ny, 65535),
                (unsigned)std::min<int64_t>(g.nz, 65535));
}

// One step src -> dst through the population buffer pop ((2 dims + 1) * total values).
template <typename T>
cudaError_t launch_step_lb(int dims, int bc, const T* src, T* pop, T* dst, const Geo& g, double omega1,
                           double lam, const Coef<T>& cf, cudaStream_t st) {
    LbCoef<T> lc;
    // s = w1 / lambda (Sec. II); the lambda = 0 limit of (1 - s) w1 / s is -w1
    const double s = omega1 / lam;
    lc.w0 = (T)(1.0 - 2.0 * dims * omega1);
    lc.w1 = (T)omega1;
    lc.kappa = (T)(lam > 0.0 ? (1.0 - s) * omega1 / s : -omega1);
    constexpr int VX = 16 / (int)sizeof(T);
    // vector kernels: rows of a multiple of VX values and 16-byte aligned buffers
    const bool vec = g.nx % VX == 0 && ((uintptr_t)src | (uintptr_t)pop | (uintptr_t)dst) % 16 == 0;
    const dim3 grid = lb_grid<T>(g), block(256);
    const dim3 vblock(32, 8);
    const dim3 vgrid((unsigned)std::min<int64_t>((g.nx / VX + 31) / 32, 1 << 20),
                     (unsigned)std::min<int64_t>((g.ny + 7) / 8, 65535), (unsigned)std::min<int64_t>(g.nz, 65535));
#define ACS_LB_CASE(D, B)                                                                                \
    if (dims == D && bc == B) {                                                                          \
        if (vec) {                                                                                       \
            k_lb_collide_v<T, D, B><<<vgrid, vblock, 0, st>>>(src, pop, g, lc);                          \
            ACS_SOLVE_DISPATCH(cf.solve, SV,                                                             \
                               (k_lb_stream_v<T, D, B, SV><<<vgrid, vblock, 0, st>>>(src, pop, dst, g, lc, cf))); \
        } else {                                                                                         \
            k_lb_collide<T, D, B><<<grid, block, 0, st>>>(src, pop, g, lc);                              \
            ACS_SOLVE_DISPATCH(cf.solve, SV, (k_lb_stream<T, D, B, SV><<<grid, block, 0, st>>>(src, pop, dst, g, lc, cf))); \
        }                                                                                                \
        return cudaGetLastError();                                                                       \
    }
    ACS_LB_CASE(1, 0) ACS_LB_CASE(1, 1) ACS_LB_CASE(1, 2)
    ACS_LB_CASE(2, 0) ACS_LB_CASE(2, 1) ACS_LB_CASE(2, 2)
    ACS_LB_CASE(3, 0) ACS_LB_CASE(3, 1) ACS_LB_CASE(3, 2)
#undef ACS_LB_CASE
    return cudaErrorInvalidValue;
}

template cudaError_t launch_step_lb<float>(int, int, const float*, float*, float*, const Geo&, double, double,
                                           const Coef<float>&, cudaStream_t);
template cudaError_t launch_step_lb<double>(int, int, const double*, double*, double*, const Geo&, double, double,
                                            const Coef<double>&, cudaStream_t);

}  // namespace acs
