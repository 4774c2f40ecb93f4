// adjoint.cu -- the hand-written adjoint of the discrete RLB-MIE-FD stepper.
//
// One step (Eq. IE-FD, Remark 1) maps phi^n to phi^{n+1} pointwise through
//   xi_i = c0 phi_i - a phi_i^3 + lambda sum_nbr phi,   a theta^3 + b theta = xi_i,
// (a = dt/2, b = 1 - a, c0 = 1 - 2 d lambda + a).  Implicit differentiation of the
// cubic gives d theta / d xi = 1 / (3 a theta^2 + b), so for a terminal loss with
// adjoint state adj^{n+1} = dL/dphi^{n+1}:
//   mu_i    = adj^{n+1}_i / (3 a (phi^{n+1}_i)^2 + b)
//   adj^n_j = mu_j (c0 - 3 a (phi^n_j)^2) + lambda sum_nbr(j) mu
// (the ghost-rule stencil is symmetric -- the matrices D of Eq. Ddeltax are -- so
// its transpose is the same stencil applied to mu), and since lambda = eps^2 dt/h^2
// with dt, h fixed,
//   dL/d(eps^2) += (dt/h^2) sum_i mu_i (sum_nbr(i) phi^n - 2 d phi^n_i).
// The eps^2 sums are accumulated in FP64 with compensation, per step in a fixed
// order (deterministic).  Forward states are checkpointed every `every` steps and
// each segment is recomputed (with the forward kernel's arithmetic, so bit for bit
// the same states) before its backward sweep.
#include <cmath>
#include <cstring>

#include "acs_host.h"
#include "acs_reduce.cuh"
#include "stream_tile.cuh"
#include "tile2d.cuh"
#include "tma.cuh"

namespace acs {

template <int BC, typename T>
__device__ __forceinline__ T gnb(const T* __restrict__ p, int64_t i, int64_t c, int64_t n, int64_t s, int dir) {
    if (dir < 0) {
        if (c > 0) return p[i - s];
        if (BC == ACS_BC_PERIODIC) return p[i + (n - 1) * s];
        if (BC == ACS_BC_NEUMANN) return p[i];
        return T(0);
    }
    if (c < n - 1) return p[i + s];
    if (BC == ACS_BC_PERIODIC) return p[i - (n - 1) * s];
    if (BC == ACS_BC_NEUMANN) return p[i];
    return T(0);
}

// mu at the (ghost-ruled) neighbour: the ghost of mu follows the same rule as phi.
template <int BC, typename T>
__device__ __forceinline__ T mu_nb(const T* __restrict__ adj1, const T* __restrict__ th1, int64_t i, int64_t c,
                                   int64_t n, int64_t s, int dir, const Coef<T>& cf) {
    int64_t j;
    if (dir < 0) {
        if (c > 0) j = i - s;
        else if (BC == ACS_BC_PERIODIC) j = i + (n - 1) * s;
        else if (BC == ACS_BC_NEUMANN) j = i;
        else return T(0);
    } else {
        if (c < n - 1) j = i + s;
        else if (BC == ACS_BC_PERIODIC) j = i - (n - 1) * s;
        else if (BC == ACS_BC_NEUMANN) j = i;
        else return T(0);
    }
    const T t = th1[j];
    return adj1[j] / dfma(cf.three_a, t * t, cf.b);
}

template <typename T, int D, int BC>
__global__ void __launch_bounds__(256) k_adjoint(const T* __restrict__ phin, const T* __restrict__ phin1,
                                                 const T* __restrict__ adj1, T* __restrict__ adj0, Geo g,
                                                 Coef<T> cf, CSum* part) {
    CSum ge{0.0, 0.0};
    const int64_t rows = g.ny * g.nz;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int64_t z = r / g.ny, y = r - z * g.ny;
        const int64_t row = z * g.sz + y * g.sy;
        for (int64_t x = threadIdx.x; x < g.nx; x += blockDim.x) {
            const int64_t i = row + x;
            const T t = phin1[i];
            const T mu = adj1[i] / dfma(cf.three_a, t * t, cf.b);
            const T p = phin[i];
            T smu, sphi;
            {
                const T mxm = mu_nb<BC>(adj1, phin1, i, x, g.nx, 1, -1, cf);
                const T mxp = mu_nb<BC>(adj1, phin1, i, x, g.nx, 1, +1, cf);
                const T pxm = gnb<BC>(phin, i, x, g.nx, 1, -1), pxp = gnb<BC>(phin, i, x, g.nx, 1, +1);
                if (D == 1) {
                    smu = nsum(mxm, mxp);
                    sphi = nsum(pxm, pxp);
                } else {
                    const T mym = mu_nb<BC>(adj1, phin1, i, y, g.ny, g.sy, -1, cf);
                    const T myp = mu_nb<BC>(adj1, phin1, i, y, g.ny, g.sy, +1, cf);
                    const T pym = gnb<BC>(phin, i, y, g.ny, g.sy, -1), pyp = gnb<BC>(phin, i, y, g.ny, g.sy, +1);
                    if (D == 2) {
                        smu = nsum(mym, myp, mxm, mxp);
                        sphi = nsum(pym, pyp, pxm, pxp);
                    } else {
                        const T mzm = mu_nb<BC>(adj1, phin1, i, z, g.nz, g.sz, -1, cf);
                        const T mzp = mu_nb<BC>(adj1, phin1, i, z, g.nz, g.sz, +1, cf);
                        const T pzm = gnb<BC>(phin, i, z, g.nz, g.sz, -1), pzp = gnb<BC>(phin, i, z, g.nz, g.sz, +1);
                        smu = nsum(mzm, mzp, mym, myp, mxm, mxp);
                        sphi = nsum(pzm, pzp, pym, pyp, pxm, pxp);
                    }
                }
            }
            adj0[i] = dfma(cf.lam, smu, mu * dfma(-cf.three_a, p * p, cf.c0));
            cadd(ge, (double)mu * ((double)sphi - 2.0 * D * (double)p));
        }
    }
    ge = block_csum(ge);
    if (threadIdx.x == 0) part[blockIdx.x] = cmerge(part[blockIdx.x], ge);
}

// acc += the partials of a segment: steps x nparts entries, in a fixed order.
__global__ void k_adjoint_finish(const CSum* part, int steps, int stride, int nparts, CSum* acc) {
    const CSum s = block_sum_pairs(steps * nparts, [&](int i) {
        const int st = i / nparts, b = i - st * nparts;
        return part[(size_t)st * stride + b];
    });
    if (threadIdx.x == 0) acc[0] = cmerge(acc[0], s);
}

__global__ void k_zero_acc(CSum* acc) { acc[0] = CSum{0.0, 0.0}; }

// 2D adjoint step from shared-memory tiles: phi^n, phi^{n+1} and adj^{n+1} are staged
// with the ghost rule (cp.async), mu = adj^{n+1} / (3 a (phi^{n+1})^2 + b) is formed
// once per staged point in place, then each thread updates its 8 points.  The ghost of
// mu follows the same rule as phi (the stencil is symmetric).
template <typename T, int BC>
__global__ void __launch_bounds__(256) k_adjoint2d(const T* __restrict__ phin, const T* __restrict__ phin1,
                                                   const T* __restrict__ adj1, T* __restrict__ adj0, Geo g,
                                                   Coef<T> cf, int ntx, int nty, int per_cta, CSum* part) {
    using TT = Tile2<T>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* P = reinterpret_cast<T*>(sm_raw);
    const int ny = (int)g.ny, nx = (int)g.nx;
    const int ntiles = ntx * nty;
    const int t0 = blockIdx.x * per_cta, t1 = min(t0 + per_cta, ntiles);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    CSum ge{0.0, 0.0};
    // two sets of (phi^n, phi^{n+1}, adj^{n+1}) tiles: the next tile is staged while
    // the current one is processed
    auto stage = [&](int t, int set) {
        const int x0 = (t / nty) * TT::TX, y0 = (t % nty) * TT::TY;
        T* base = P + set * 3 * TT::N;
        stage_tile<T>(base, phin, ny, nx, BC, x0, y0);
        stage_tile<T>(base + TT::N, phin1, ny, nx, BC, x0, y0);
        stage_tile<T>(base + 2 * TT::N, adj1, ny, nx, BC, x0, y0);
    };
    if (t0 < t1) stage(t0, 0);
    cp_async_commit();
    for (int t = t0; t < t1; ++t) {
        const int set = (t - t0) & 1;
        if (t + 1 < t1) stage(t + 1, set ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const int x0 = (t / nty) * TT::TX, y0 = (t % nty) * TT::TY;
        T* Pc = P + set * 3 * TT::N;
        T* Qc = Pc + TT::N;
        T* Mc = Qc + TT::N;
        for (int i = threadIdx.x; i < TT::N; i += TT::THREADS) {
            const T q = Qc[i];
            Mc[i] = Mc[i] / dfma(cf.three_a, q * q, cf.b);
        }
        __syncthreads();
        T tile_sum = T(0);
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int r = 2 * w + rr;
            const int gy = y0 + r;
#pragma unroll
            for (int k = 0; k < TT::VX; ++k) {
                const int cx = lane + 32 * k;  // tile column (staged column VX + cx)
                const int gx = x0 + cx;
                const int i = (r + 1) * TT::BW + TT::VX + cx;
                const T mu = Mc[i], p = Pc[i];
                const T smu = nsum(Mc[i - TT::BW], Mc[i + TT::BW], Mc[i - 1], Mc[i + 1]);
                const T sphi = nsum(Pc[i - TT::BW], Pc[i + TT::BW], Pc[i - 1], Pc[i + 1]);
                if (gy < ny && gx < nx) {
                    adj0[(int64_t)gy * nx + gx] = dfma(cf.lam, smu, mu * dfma(-cf.three_a, p * p, cf.c0));
                    tile_sum = dfma(mu, sphi - T(4) * p, tile_sum);
                }
            }
        }
        cadd(ge, (double)tile_sum);
        __syncthreads();
    }
    ge = block_csum(ge);
    if (threadIdx.x == 0) part[blockIdx.x] = cmerge(part[blockIdx.x], ge);
}

// mu = adj / (3 a theta^2 + b) of the streamed kernel: the denominator lies in
// [b, 1 + 2a], well away from 0, so a reciprocal suffices -- FP32: the fast
// division (2 ulp); FP64: the FP32 reciprocal refined by two Newton steps.
__device__ __forceinline__ float adj_mu(float l, float q, const Coef<float>& cf) {
    return __fdividef(l, __fmaf_rn(cf.three_a, q * q, cf.b));
}
__device__ __forceinline__ double adj_mu(double l, double q, const Coef<double>& cf) {
    const double d = __fma_rn(cf.three_a, q * q, cf.b);
    double r = (double)__frcp_rn((float)d);
    r = r * __fma_rn(-d, r, 2.0);
    r = r * __fma_rn(-d, r, 2.0);
    return l * r;
}

// Sum of one value per thread over a block of 32 x 8 threads, valid in thread (0, 0).
// FP32: unevaluated float pairs (TwoSum) through the warp shuffles and the eight warp
// sums, about 2^-44 relative, returned as an exact double pair -- no FP64 arithmetic,
// whose dependent latency on this GPU would dominate the step's tail.  FP64: the
// exact fixed-point block sum.
__device__ __forceinline__ CSum cta_sum(float v) {
    F2 a{v, 0.0f};
    for (int off = 16; off > 0; off >>= 1) {
        const float bh = __shfl_down_sync(0xffffffffu, a.hi, off);
        const float bl = __shfl_down_sync(0xffffffffu, a.lo, off);
        const F2 t = two_sum(a.hi, bh);
        a = F2{t.hi, (a.lo + bl) + t.lo};
    }
    __shared__ F2 ws[8];
    if (threadIdx.x == 0) ws[threadIdx.y] = a;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        for (int w = 1; w < 8; ++w) {
            const F2 t = two_sum(a.hi, ws[w].hi);
            a = F2{t.hi, (a.lo + ws[w].lo) + t.lo};
        }
    }
    return CSum{(double)a.hi, (double)a.lo};
}
__device__ __forceinline__ CSum cta_sum(double v) { return block_csum(CSum{v, 0.0}); }

// 2D adjoint step streamed through TMA (rows a multiple of 16 bytes).  A CTA owns a
// column of TX unknowns and a run of 16-row blocks; per block one thread loads the
// halo boxes of phi^n, phi^{n+1} and adj^{n+1} into a ring slot.  mu is formed in
// place over the adj^{n+1} box (zero outside the grid, which is the Dirichlet
// ghost), then each thread updates its RPT x VX points with mu and phi^n neighbours
// from registers, shuffles and shared memory; at a Neumann face the ghost is the
// point itself, at a periodic face the wrapped value, read from global memory.
template <typename T, int BC, bool EDGE>
__device__ __forceinline__ void adjoint_block(const T* P, const T* M, const T* __restrict__ phin,
                                              const T* __restrict__ phin1, const T* __restrict__ adj1,
                                              T* __restrict__ adj0, const Geo& g, const Coef<T>& cf, int x0, int y0,
                                              T& tile_sum) {
    using TT = Tile3<T, 2, 2>;
    constexpr int VX = TT::VX, TX = TT::TX, BW = TT::BW, RPT = TT::RPT;
    const int nx = (int)g.nx, ny = (int)g.ny;
    const int64_t sy = g.sy;
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int xl = lx * VX, gx = x0 + xl, r0 = RPT * ly, gy0 = y0 + r0;
    auto mu_at = [&](int64_t j) { return adj_mu(adj1[j], phin1[j], cf); };
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
        const int br = r0 + rr + 1;  // box row of grid row gyr
        const int gyr = gy0 + rr;
        T mu[VX], p[VX], mb[VX], ma[VX], pb[VX], pa[VX];
        Vec<T>::get(M + br * BW + VX + xl, mu);
        Vec<T>::get(P + br * BW + VX + xl, p);
        Vec<T>::get(M + (br - 1) * BW + VX + xl, mb);
        Vec<T>::get(M + (br + 1) * BW + VX + xl, ma);
        Vec<T>::get(P + (br - 1) * BW + VX + xl, pb);
        Vec<T>::get(P + (br + 1) * BW + VX + xl, pa);
        // the tile's outer two x neighbours from the halo group (a broadcast read)
        const T mhl = M[br * BW + VX - 1], mhr = M[br * BW + VX + TX];
        const T phl = P[br * BW + VX - 1], phr = P[br * BW + VX + TX];
        const T msu = __shfl_up_sync(0xffffffffu, mu[VX - 1], 1), msd = __shfl_down_sync(0xffffffffu, mu[0], 1);
        const T psu = __shfl_up_sync(0xffffffffu, p[VX - 1], 1), psd = __shfl_down_sync(0xffffffffu, p[0], 1);
        T ml = lx == 0 ? mhl : msu, mr = lx == 31 ? mhr : msd;
        T pl = lx == 0 ? phl : psu, pr = lx == 31 ? phr : psd;
        if (EDGE && gyr < ny && gx < nx) {
            if (gyr == 0) {
                if (BC == ACS_BC_NEUMANN) {
#pragma unroll
                    for (int v = 0; v < VX; ++v) { mb[v] = mu[v]; pb[v] = p[v]; }
                } else if (BC == ACS_BC_PERIODIC) {
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        const int64_t j = (int64_t)(ny - 1) * sy + gx + v;
                        mb[v] = mu_at(j);
                        pb[v] = phin[j];
                    }
                }
            }
            if (gyr == ny - 1) {
                if (BC == ACS_BC_NEUMANN) {
#pragma unroll
                    for (int v = 0; v < VX; ++v) { ma[v] = mu[v]; pa[v] = p[v]; }
                } else if (BC == ACS_BC_PERIODIC) {
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        const int64_t j = gx + v;
                        ma[v] = mu_at(j);
                        pa[v] = phin[j];
                    }
                }
            }
            if (gx == 0) {
                if (BC == ACS_BC_NEUMANN) {
                    ml = mu[0];
                    pl = p[0];
                } else if (BC == ACS_BC_PERIODIC) {
                    const int64_t j = (int64_t)gyr * sy + nx - 1;
                    ml = mu_at(j);
                    pl = phin[j];
                }
            }
            if (gx + VX == nx) {
                if (BC == ACS_BC_NEUMANN) {
                    mr = mu[VX - 1];
                    pr = p[VX - 1];
                } else if (BC == ACS_BC_PERIODIC) {
                    const int64_t j = (int64_t)gyr * sy;
                    mr = mu_at(j);
                    pr = phin[j];
                }
            }
        }
        T out[VX];
#pragma unroll
        for (int v = 0; v < VX; ++v) {
            const T mxm = v == 0 ? ml : mu[v - 1], mxp = v == VX - 1 ? mr : mu[v + 1];
            const T pxm = v == 0 ? pl : p[v - 1], pxp = v == VX - 1 ? pr : p[v + 1];
            const T smu = nsum(mb[v], ma[v], mxm, mxp);
            const T sphi = nsum(pb[v], pa[v], pxm, pxp);
            out[v] = dfma(cf.lam, smu, mu[v] * dfma(-cf.three_a, p[v] * p[v], cf.c0));
            if (gyr < ny && gx + v < nx) tile_sum = dfma(mu[v], sphi - T(4) * p[v], tile_sum);
        }
        if (gyr < ny && gx < nx) Vec<T>::put(adj0 + (int64_t)gyr * sy + gx, out);
    }
}

template <typename T, int BC, int SS>
__global__ void __launch_bounds__(256) k_adjoint2d_tma(const __grid_constant__ CUtensorMap map_p,
                                                       const __grid_constant__ CUtensorMap map_q,
                                                       const __grid_constant__ CUtensorMap map_l,
                                                       const T* __restrict__ phin, const T* __restrict__ phin1,
                                                       const T* __restrict__ adj1, T* __restrict__ adj0, Geo g,
                                                       Coef<T> cf, int ybchunk, int* err, CSum* part) {
    pdl_wait();  // the previous launch's stores (states, adjoint, partials) are visible from here on
    using TT = Tile3<T, 2, SS>;
    constexpr int VX = TT::VX, TX = TT::TX, TY = TT::TY, S = TT::S;
    constexpr int BOX = TT::SLOT_STRIDE / sizeof(T);  // elements per box (128-byte aligned)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(base);
    T* ring = reinterpret_cast<T*>(base + TT::BAR_BYTES);  // S slots of 3 boxes: phi^n, phi^{n+1}, adj^{n+1}
    const int nx = (int)g.nx, ny = (int)g.ny;
    const int nyb = (ny + TY - 1) / TY;
    const int x0 = blockIdx.x * TX;
    const int b0 = blockIdx.y * ybchunk, b1 = min(b0 + ybchunk, nyb);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int b, int slot) {
        T* d = ring + (size_t)slot * 3 * BOX;
        if ((smem_u32(d) & 127u) != 0u || (((x0 - VX) * (int)sizeof(T)) & 15) != 0) {
            atomicExch(err, 2);
            return;
        }
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[slot], 3u * TT::SLOT_BYTES);
        tma_load_2d(d, &map_p, &full[slot], x0 - VX, b * TY - 1);
        tma_load_2d(d + BOX, &map_q, &full[slot], x0 - VX, b * TY - 1);
        tma_load_2d(d + 2 * BOX, &map_l, &full[slot], x0 - VX, b * TY - 1);
    };
    int last_issued = min(b0 + S, b1) - 1;
    if (tid == 0)
        for (int b = b0; b <= last_issued; ++b) issue(b, b - b0);
    const bool edge = BC != ACS_BC_DIRICHLET && (x0 == 0 || x0 + TX >= nx || b0 == 0 || b1 * TY >= ny);
    T tile_sum = T(0);  // this thread's eps^2 terms of the launch
    bool failed = false;
    int sc = 0;
    uint32_t pc = 0u;
    for (int b = b0; b < b1 && !failed; ++b) {
        const bool ok = mbar_wait(&full[sc], pc);
        T* P = ring + (size_t)sc * 3 * BOX;
        const T* Q = P + BOX;
        T* M = P + 2 * BOX;
        // mu over the whole box, in place of adj^{n+1}
        for (int i = tid; i < TT::SLOT; i += 256) M[i] = adj_mu(M[i], Q[i], cf);
        __syncthreads();
        if (edge && (x0 == 0 || x0 + TX >= nx || b == 0 || (b + 1) * TY >= ny))
            adjoint_block<T, BC, true>(P, M, phin, phin1, adj1, adj0, g, cf, x0, b * TY, tile_sum);
        else
            adjoint_block<T, BC, false>(P, M, phin, phin1, adj1, adj0, g, cf, x0, b * TY, tile_sum);
        failed = __syncthreads_or(!ok);
        // block b + S reuses block b's slot, free now that every thread is past it
        if (!failed && tid == 0 && b + S < b1) {
            issue(b + S, sc);
            last_issued = b + S;
        }
        if (++sc == S) {
            sc = 0;
            pc ^= 1u;
        }
    }
    if (failed && tid == 0) {
        atomicExch(err, 1);
        for (int b = max(b0, last_issued - S + 1); b <= last_issued; ++b) {
            const int k = b - b0;
            mbar_wait(&full[k % S], (uint32_t)((k / S) & 1));
        }
    }
    // the CTA's share of this step, added to its running sum over the sweep
    const CSum t = cta_sum(tile_sum);
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid == 0) part[cta] = cmerge(part[cta], t);
    pdl_trigger();
}

// One adjoint step adding its per-block eps^2 partials into `part` (kMaxRedBlocks
// entries, the same CTA -> entry map every step); returns their number in *nparts.
template <typename T>
static cudaError_t launch_adjoint(int dims, int bc, const T* phin, const T* phin1, const T* adj1, T* adj0,
                                  const Geo& g, const Coef<T>& cf, CSum* part, int* nparts, int* err,
                                  cudaStream_t st) {
    if (dims == 2 && (g.nx * (int64_t)sizeof(T)) % 16 == 0 && g.nx < (1 << 30) && g.ny < (1 << 30) && err) {
        using TT = Tile3<T, 2, 2>;
        const int ntx = (int)((g.nx + TT::TX - 1) / TT::TX), nyb = (int)((g.ny + TT::TY - 1) / TT::TY);
        // about three CTAs per SM, at most kMaxRedBlocks partials
        // one block per CTA while the partials fit, else about three CTAs per SM
        const int want = (int64_t)ntx * nyb <= kMaxRedBlocks ? nyb : std::max(1, (152 * 3) / ntx);
        const int chunks = std::max(1, std::min(nyb, want));
        const int ybchunk = (nyb + chunks - 1) / chunks;
        const int nchunks = (nyb + ybchunk - 1) / ybchunk;
        if ((int64_t)ntx * nchunks <= kMaxRedBlocks && nchunks <= 65535) {
            CUtensorMap mp, mq, ml;
            const uint64_t dims2[2] = {(uint64_t)g.nx, (uint64_t)g.ny};
            const uint32_t box[2] = {(uint32_t)TT::BW, (uint32_t)TT::BH};
            if (encode_tensor_map(&mp, sizeof(T), 2, phin, dims2, box) &&
                encode_tensor_map(&mq, sizeof(T), 2, phin1, dims2, box) &&
                encode_tensor_map(&ml, sizeof(T), 2, adj1, dims2, box)) {
                // one block per CTA needs one ring slot: more CTAs fit on an SM
                const int S = ybchunk == 1 ? 1 : 2;
                const size_t smem = 128 + TT::BAR_BYTES + (size_t)S * 3 * TT::SLOT_STRIDE;
                auto kern = S == 1 ? (bc == 0 ? k_adjoint2d_tma<T, 0, 1>
                                              : (bc == 1 ? k_adjoint2d_tma<T, 1, 1> : k_adjoint2d_tma<T, 2, 1>))
                                   : (bc == 0 ? k_adjoint2d_tma<T, 0, 2>
                                              : (bc == 1 ? k_adjoint2d_tma<T, 1, 2> : k_adjoint2d_tma<T, 2, 2>));
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                e = launch_pdl(kern, dim3((unsigned)ntx, (unsigned)nchunks), dim3(32, 8), smem, st, mp, mq, ml, phin,
                               phin1, adj1, adj0, g, cf, ybchunk, err, part);
                *nparts = ntx * nchunks;
                return e;
            }
        }
    }
    if (dims == 2 && g.nx < (1 << 30) && g.ny < (1 << 30)) {
        using TT = Tile2<T>;
        const int ntx = (int)((g.nx + TT::TX - 1) / TT::TX), nty = (int)((g.ny + TT::TY - 1) / TT::TY);
        const int64_t ntiles = (int64_t)ntx * nty;
        const int per = (int)std::max<int64_t>(1, (ntiles + kMaxRedBlocks - 1) / kMaxRedBlocks);
        const int grid = (int)((ntiles + per - 1) / per);
        const size_t smem = 6 * TT::N * sizeof(T);
        cudaError_t e = cudaSuccess;
        auto kern = bc == 0 ? k_adjoint2d<T, 0> : (bc == 1 ? k_adjoint2d<T, 1> : k_adjoint2d<T, 2>);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, TT::THREADS, smem, st>>>(phin, phin1, adj1, adj0, g, cf, ntx, nty, per, part);
        *nparts = grid;
        return cudaGetLastError();
    }
    const int nb = reduce_blocks(g);
#define ACS_ADJ_CASE(D, B) \
    if (dims == D && bc == B) k_adjoint<T, D, B><<<nb, 256, 0, st>>>(phin, phin1, adj1, adj0, g, cf, part); else
    ACS_ADJ_CASE(1, 0) ACS_ADJ_CASE(1, 1) ACS_ADJ_CASE(1, 2)
    ACS_ADJ_CASE(2, 0) ACS_ADJ_CASE(2, 1) ACS_ADJ_CASE(2, 2)
    ACS_ADJ_CASE(3, 0) ACS_ADJ_CASE(3, 1) ACS_ADJ_CASE(3, 2)
    return cudaErrorInvalidValue;
#undef ACS_ADJ_CASE
    *nparts = nb;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- recording layout

namespace {
constexpr size_t kA = 256;
size_t al(size_t x) { return (x + kA - 1) / kA * kA; }

struct GradLayout {
    size_t sb;        // aligned state bytes
    int64_t nckpt;    // checkpoint slots
    size_t ckpt, seg, adjA, adjB, part, acc, total;
};

GradLayout layout(const CtxView& v, int64_t max_steps, int64_t every) {
    GradLayout L;
    L.sb = al((size_t)v.g.total * v.esize);
    L.nckpt = max_steps / every + 1;
    L.ckpt = 0;
    L.seg = L.ckpt + L.sb * (size_t)L.nckpt;
    L.adjA = L.seg + L.sb * (size_t)every;
    L.adjB = L.adjA + L.sb;
    L.part = L.adjB + L.sb;
    L.acc = L.part + al(sizeof(CSum) * kMaxRedBlocks * (size_t)every);
    L.total = L.acc + kA;
    return L;
}
}  // namespace

int grad_on_set_state(acs_ctx* c) {
    CtxView v = ctx_view(c);
    GradState& G = *v.grad;
    if (!G.active) return ACS_OK;
    GradLayout L = layout(v, G.max_steps, G.every);
    if (cudaMemcpyAsync(G.buf + L.ckpt, v.phi, (size_t)v.g.total * v.esize, cudaMemcpyDeviceToDevice, v.stream) !=
        cudaSuccess)
        return ACS_E_CUDA;
    G.recorded = 0;
    G.started = true;
    return ACS_OK;
}

void grad_drop_graphs(GradState& G) {
    for (auto& g : G.graphs) cudaGraphExecDestroy(g.exec);
    G.graphs.clear();
}

// Record one graph of `enqueue(stream)` on the capture stream and cache it under
// (kind, a, b); null if the stream cannot be captured (the caller then runs directly).
template <typename F>
static cudaGraphExec_t grad_graph(const CtxView& v, int kind, int64_t a, int64_t b, F&& enqueue) {
    GradState& G = *v.grad;
    for (auto& g : G.graphs)
        if (g.kind == kind && g.a == a && g.b == b) return g.exec;
    if (!v.cap) return nullptr;
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(v.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return nullptr;
    const bool ok = enqueue(v.cap);
    const cudaError_t e2 = cudaStreamEndCapture(v.cap, &graph);
    cudaGraphExec_t exec = nullptr;
    if (!ok || e2 != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
    if (e2 == cudaSuccess) cudaGraphDestroy(graph);
    if (!exec) {
        cudaGetLastError();
        return nullptr;
    }
    if (G.graphs.size() >= 8) {
        cudaGraphExecDestroy(G.graphs.front().exec);
        G.graphs.erase(G.graphs.begin());
    }
    G.graphs.push_back(GradGraph{kind, a, b, exec});
    return exec;
}

// n steps from the current state with a checkpoint copy at every multiple of `every`
// (one recorded graph per (first step, n)).
int grad_record_steps(acs_ctx* c, int64_t n) {
    CtxView v = ctx_view(c);
    GradState& G = *v.grad;
    if (!G.started) return ACS_E_STATE;
    if (G.recorded + n > G.max_steps) return ACS_E_NOMEM;
    const GradLayout L = layout(v, G.max_steps, G.every);
    const int64_t start = G.recorded;
    auto enqueue = [&](cudaStream_t st) -> bool {
        if (G.every == 1) {
            // every state is a checkpoint: each step writes straight into the next slot
            // (no copies, and the backward sweep recomputes nothing); the context's
            // state is then the last slot
            for (int64_t j = 0; j < n; ++j) {
                const char* src = G.buf + L.ckpt + L.sb * (size_t)(start + j);
                char* dst = G.buf + L.ckpt + L.sb * (size_t)(start + j + 1);
                if (ctx_launch_one(c, src, dst, st) != cudaSuccess) return false;
            }
            return cudaMemcpyAsync(v.phi, G.buf + L.ckpt + L.sb * (size_t)(start + n), (size_t)v.g.total * v.esize,
                                   cudaMemcpyDeviceToDevice, st) == cudaSuccess;
        }
        int64_t rec = start, left = n;
        while (left > 0) {
            const int64_t k = std::min(left, G.every - (rec % G.every));
            if (ctx_enqueue_steps(c, k, st) != cudaSuccess) return false;
            rec += k;
            left -= k;
            if (rec % G.every == 0) {
                char* slot = G.buf + L.ckpt + L.sb * (size_t)(rec / G.every);
                if (cudaMemcpyAsync(slot, v.phi, (size_t)v.g.total * v.esize, cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess)
                    return false;
            }
        }
        return true;
    };
    cudaGraphExec_t exec = n >= 4 ? grad_graph(v, 0, start, n, enqueue) : nullptr;
    if (exec) {
        if (cudaGraphLaunch(exec, v.stream) != cudaSuccess) return ACS_E_CUDA;
    } else if (!enqueue(v.stream)) {
        return ACS_E_CUDA;
    }
    G.recorded += n;
    return ACS_OK;
}

}  // namespace acs

using namespace acs;

extern "C" {

ACS_API size_t acs_grad_work_bytes(const acs_ctx* c, int64_t max_steps, int64_t every) {
    if (!c || max_steps < 1 || every < 1) return 0;
    CtxView v = ctx_view(const_cast<acs_ctx*>(c));
    return layout(v, max_steps, every).total;
}

ACS_API int acs_grad_bind(acs_ctx* c, void* d_grad_work, size_t bytes, int64_t max_steps, int64_t every) {
    if (!c || !d_grad_work || max_steps < 1 || every < 1 || ((uintptr_t)d_grad_work % 256)) return ACS_E_INVAL;
    CtxView v = ctx_view(c);
    if (!v.phi) return ACS_E_STATE;
    GradLayout L = layout(v, max_steps, every);
    if (bytes < L.total) return ACS_E_NOMEM;
    GradState& G = *v.grad;
    grad_drop_graphs(G);
    G.active = true;
    G.buf = (char*)d_grad_work;
    G.bytes = bytes;
    G.max_steps = max_steps;
    G.every = every;
    G.recorded = 0;
    G.started = false;
    // record from the current state
    return grad_on_set_state(c);
}

ACS_API int acs_grad(acs_ctx* c, const void* d_dL_dphiT, void* d_dL_dphi0, double* dL_deps2_host) {
    if (!c || !d_dL_dphiT || !d_dL_dphi0 || !dL_deps2_host) return ACS_E_INVAL;
    CtxView v = ctx_view(c);
    GradState& G = *v.grad;
    if (!G.active || !G.started) return ACS_E_STATE;
    if (v.cf.solve == kSolveFex) return ACS_E_UNSUPPORTED;
    const GradLayout L = layout(v, G.max_steps, G.every);
    const size_t bytes = (size_t)v.g.total * v.esize;
    cudaStream_t st = v.stream;
    char* A = G.buf + L.adjA;
    char* B = G.buf + L.adjB;
    CSum* part = (CSum*)(G.buf + L.part);
    CSum* acc = (CSum*)(G.buf + L.acc);
    if (cudaMemcpyAsync(A, d_dL_dphiT, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return ACS_E_CUDA;
    const int64_t N = G.recorded;
    // The whole sweep, recorded once per (N, every): per segment (last first)
    // recompute its states from the checkpoint, then step the adjoint back through
    // them.  Each adjoint launch adds its per-CTA eps^2 partials into part[cta]
    // (always the same CTA order), combined exactly once at the end: deterministic.
    auto sweep = [&](cudaStream_t s) -> bool {
        char* a = A;
        char* b = B;
        k_zero_acc<<<1, 1, 0, s>>>(acc);
        if (cudaMemsetAsync(part, 0, sizeof(CSum) * kMaxRedBlocks, s) != cudaSuccess) return false;
        int nparts = 0;
        for (int64_t seg = N > 0 ? (N - 1) / G.every : -1; seg >= 0; --seg) {
            const int64_t s0 = seg * G.every;
            const int64_t m = std::min(G.every, N - s0);
            char* ck = G.buf + L.ckpt + L.sb * (size_t)seg;
            const char* prev = ck;
            // with a checkpoint after every step the segment's end state is stored
            const bool stored = G.every == 1;
            for (int64_t j = 0; j < m && !stored; ++j) {
                char* dst = G.buf + L.seg + L.sb * (size_t)j;
                if (ctx_launch_one(c, prev, dst, s) != cudaSuccess) return false;
                prev = dst;
            }
            for (int64_t k = m - 1; k >= 0; --k) {
                const char* pk = k == 0 ? ck : G.buf + L.seg + L.sb * (size_t)(k - 1);
                const char* pk1 = stored ? ck + L.sb : G.buf + L.seg + L.sb * (size_t)k;
                cudaError_t e;
                CSum* row = part;
                if (v.dtype == ACS_F32)
                    e = launch_adjoint<float>(v.dims, v.bc, (const float*)pk, (const float*)pk1, (const float*)a,
                                              (float*)b, v.g, v.cf, row, &nparts, v.err, s);
                else
                    e = launch_adjoint<double>(v.dims, v.bc, (const double*)pk, (const double*)pk1,
                                               (const double*)a, (double*)b, v.g, v.cd, row, &nparts, v.err, s);
                if (e != cudaSuccess) return false;
                std::swap(a, b);
            }
        }
        if (nparts > 0) {
            k_adjoint_finish<<<1, 256, 0, s>>>(part, 1, kMaxRedBlocks, nparts, acc);
            if (cudaGetLastError() != cudaSuccess) return false;
        }
        return true;
    };
    cudaGraphExec_t exec = N >= 4 ? grad_graph(v, 1, N, G.every, sweep) : nullptr;
    if (exec) {
        if (cudaGraphLaunch(exec, st) != cudaSuccess) return ACS_E_CUDA;
    } else if (!sweep(st)) {
        return ACS_E_CUDA;
    }
    // after N adjoint steps the result is in A for even N, in B for odd N
    if (N & 1) std::swap(A, B);
    if (cudaMemcpyAsync(d_dL_dphi0, A, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return ACS_E_CUDA;
    CSum h;
    if (cudaMemcpyAsync(&h, acc, sizeof(CSum), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ACS_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACS_E_CUDA;
    int flag = 0;
    if (v.err && cudaMemcpy(&flag, v.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_E_CUDA;
    if (flag) {
        cudaMemset(v.err, 0, sizeof(int));
        return ACS_E_TIMEOUT;
    }
    *dL_deps2_host = (h.s + h.c) * (v.dt / (v.h * v.h));
    return std::isfinite(*dL_deps2_host) ? ACS_OK : ACS_E_NONFINITE;
}

}  // extern "C"
