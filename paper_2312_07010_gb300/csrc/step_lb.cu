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
// (k = 0; +x, +y, +z; -x, -y, -z).  Summed, the form equals Eq. (IE-FD) up to
// rounding; it moves (2d+1) values out and back in per node where Eq. (IE-FD) moves
// none, which is the memory and traffic cost the macroscopic form removes.
#include "acs_kernels.cuh"

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
    const int64_t tot = g.total;
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
    const int64_t tot = g.total;
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
    const dim3 grid = lb_grid<T>(g), block(256);
#define ACS_LB_CASE(D, B)                                                                                \
    if (dims == D && bc == B) {                                                                          \
        k_lb_collide<T, D, B><<<grid, block, 0, st>>>(src, pop, g, lc);                                  \
        ACS_SOLVE_DISPATCH(cf.solve, SV, (k_lb_stream<T, D, B, SV><<<grid, block, 0, st>>>(src, pop, dst, g, lc, cf))); \
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
