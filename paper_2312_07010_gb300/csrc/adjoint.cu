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
#include "tile2d.cuh"

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
    __shared__ CSum scratch[32];
    ge = block_csum(ge, scratch);
    if (threadIdx.x == 0) part[blockIdx.x] = ge;
}

// acc += the partials of a segment: steps x nparts entries, in a fixed order.
__global__ void k_adjoint_finish(const CSum* part, int steps, int stride, int nparts, CSum* acc) {
    CSum s{0.0, 0.0};
    const int total = steps * nparts;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int st = i / nparts, b = i - st * nparts;
        s = cmerge(s, part[(size_t)st * stride + b]);
    }
    __shared__ CSum scratch[32];
    s = block_csum(s, scratch);
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
    __shared__ CSum scratch[32];
    ge = block_csum(ge, scratch);
    if (threadIdx.x == 0) part[blockIdx.x] = ge;
}

// One adjoint step writing its per-block eps^2 partials to `part` (kMaxRedBlocks
// entries); returns the number of partials used in *nparts.
template <typename T>
static cudaError_t launch_adjoint(int dims, int bc, const T* phin, const T* phin1, const T* adj1, T* adj0,
                                  const Geo& g, const Coef<T>& cf, CSum* part, int* nparts, cudaStream_t st) {
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

int grad_record_steps(acs_ctx* c, int64_t n) {
    CtxView v = ctx_view(c);
    GradState& G = *v.grad;
    if (!G.started) return ACS_E_STATE;
    if (G.recorded + n > G.max_steps) return ACS_E_NOMEM;
    GradLayout L = layout(v, G.max_steps, G.every);
    while (n > 0) {
        const int64_t room = G.every - (G.recorded % G.every);
        const int64_t k = std::min(n, room);
        if (ctx_enqueue_steps(c, k, v.stream) != cudaSuccess) return ACS_E_CUDA;
        G.recorded += k;
        n -= k;
        if (G.recorded % G.every == 0) {
            char* slot = G.buf + L.ckpt + L.sb * (size_t)(G.recorded / G.every);
            if (cudaMemcpyAsync(slot, v.phi, (size_t)v.g.total * v.esize, cudaMemcpyDeviceToDevice, v.stream) !=
                cudaSuccess)
                return ACS_E_CUDA;
        }
    }
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
    k_zero_acc<<<1, 1, 0, st>>>(acc);
    const int64_t N = G.recorded;
    if (N > 0) {
        for (int64_t seg = (N - 1) / G.every; seg >= 0; --seg) {
            const int64_t s0 = seg * G.every;
            const int64_t m = std::min(G.every, N - s0);
            char* ck = G.buf + L.ckpt + L.sb * (size_t)seg;
            // recompute phi^{s0+1} .. phi^{s0+m} into the segment buffer
            const char* prev = ck;
            for (int64_t j = 0; j < m; ++j) {
                char* dst = G.buf + L.seg + L.sb * (size_t)j;
                if (ctx_launch_one(c, prev, dst, st) != cudaSuccess) return ACS_E_CUDA;
                prev = dst;
            }
            int nparts = 0;
            for (int64_t k = m - 1; k >= 0; --k) {
                const char* pk = k == 0 ? ck : G.buf + L.seg + L.sb * (size_t)(k - 1);
                const char* pk1 = G.buf + L.seg + L.sb * (size_t)k;
                CSum* pst = part + (size_t)(m - 1 - k) * kMaxRedBlocks;
                cudaError_t e;
                if (v.dtype == ACS_F32)
                    e = launch_adjoint<float>(v.dims, v.bc, (const float*)pk, (const float*)pk1, (const float*)A,
                                              (float*)B, v.g, v.cf, pst, &nparts, st);
                else
                    e = launch_adjoint<double>(v.dims, v.bc, (const double*)pk, (const double*)pk1,
                                               (const double*)A, (double*)B, v.g, v.cd, pst, &nparts, st);
                if (e != cudaSuccess) return ACS_E_CUDA;
                std::swap(A, B);
            }
            // the segment's eps^2 partials, in a fixed order
            k_adjoint_finish<<<1, 256, 0, st>>>(part, (int)m, kMaxRedBlocks, nparts, acc);
            if (cudaGetLastError() != cudaSuccess) return ACS_E_CUDA;
        }
    }
    if (cudaMemcpyAsync(d_dL_dphi0, A, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return ACS_E_CUDA;
    CSum h;
    if (cudaMemcpyAsync(&h, acc, sizeof(CSum), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ACS_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACS_E_CUDA;
    *dL_deps2_host = (h.s + h.c) * (v.dt / (v.h * v.h));
    return std::isfinite(*dL_deps2_host) ? ACS_OK : ACS_E_NONFINITE;
}

}  // extern "C"
