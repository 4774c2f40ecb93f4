// reduce.cu -- the discrete free energy E_h (Theorem 3, Eq. proof2-eq0) and the
// maximum norm (Theorem 2) of a state, in FP64 with compensated sums.
//
// E_h = h^d [ 1/4 sum_i (phi_i^2 - 1)^2 - eps^2/2 Phi^T Lambda_{dx} Phi ], and
// -Phi^T Lambda_{dx} Phi = h^-2 sum over lattice links of the squared difference
// (the matrices D of Eq. Ddeltax are symmetric, so the quadratic form is a sum of
// squares): interior links along every axis; periodic adds the wrap-around link
// of every line; Dirichlet adds the links from the first and last unknown of
// every line to the zero boundary value; Neumann adds nothing.  The sum of squares
// has no cancellation, unlike the phi . (Lambda phi) form.
//
// Two stages, deterministic: a fixed grid (depending only on the shape) writes one
// partial per block; one block combines them.  Each thread sums with Neumaier's
// compensation (FP32 states: exact float-pair terms first); the threads' and the
// blocks' sums are combined exactly in 128-bit fixed point (acs_reduce.cuh), so the
// result does not depend on the order of the combination.
#include "acs_kernels.cuh"
#include "acs_reduce.cuh"

namespace acs {

template <int BC>
__device__ __forceinline__ void axis_links_f(F2& acc, float p, float up, int64_t c, int64_t n) {
    if (c < n - 1 || BC == ACS_BC_PERIODIC) link_sq(acc, up, p);  // `up` is the wrap neighbour at the end
    else if (BC == ACS_BC_DIRICHLET) link_sq(acc, 0.0f, p);
    if (BC == ACS_BC_DIRICHLET && c == 0) link_sq(acc, 0.0f, p);
}

// ---------------------------------------------------------------- FP64 states
template <int BC>
__device__ __forceinline__ void axis_links_d(double& acc, double p, double up, int64_t c, int64_t n) {
    if (c < n - 1 || BC == ACS_BC_PERIODIC) {
        const double d = up - p;
        acc = fma(d, d, acc);
    } else if (BC == ACS_BC_DIRICHLET) {
        acc = fma(p, p, acc);
    }
    if (BC == ACS_BC_DIRICHLET && c == 0) acc = fma(p, p, acc);
}

template <typename T, int D, int BC>
__global__ void __launch_bounds__(256) k_reduce(const T* __restrict__ src, Geo g, RedPartial* part) {
    pdl_wait();
    CSum bulk{0.0, 0.0}, link{0.0, 0.0};
    float mx = 0.0f;
    double mxd = 0.0;
    F2 fb{0.0f, 0.0f}, fl{0.0f, 0.0f};
    double db = 0.0, dl = 0.0;
    int pending = 0;
    const int64_t rows = g.ny * g.nz;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int64_t z = r / g.ny, y = r - z * g.ny;
        const int64_t row = z * g.sz + y * g.sy;
        for (int64_t x = threadIdx.x; x < g.nx; x += blockDim.x) {
            const int64_t i = row + x;
            const T p = src[i];
            const T ux = src[x < g.nx - 1 ? i + 1 : row];
            const T uy = D >= 2 ? src[y < g.ny - 1 ? i + g.sy : z * g.sz + x] : T(0);
            const T uz = D >= 3 ? src[z < g.nz - 1 ? i + g.sz : y * g.sy + x] : T(0);
            if (sizeof(T) == 4) {
                const float pf = (float)p;
                bulk_sq(fb, pf);  // (p^2 - 1)^2 exactly up to 2^-46
                const float ap = fabsf(pf);
                mx = (ap > mx || ap != ap) ? ap : mx;
                axis_links_f<BC>(fl, pf, (float)ux, x, g.nx);
                if (D >= 2) axis_links_f<BC>(fl, pf, (float)uy, y, g.ny);
                if (D >= 3) axis_links_f<BC>(fl, pf, (float)uz, z, g.nz);
                if (++pending == 32) {
                    flush(fb, bulk);
                    flush(fl, link);
                    pending = 0;
                }
            } else {
                const double pd = (double)p;
                const double w = fma(pd, pd, -1.0);
                db = fma(w, w, db);
                mxd = nmax(mxd, fabs(pd));
                axis_links_d<BC>(dl, pd, (double)ux, x, g.nx);
                if (D >= 2) axis_links_d<BC>(dl, pd, (double)uy, y, g.ny);
                if (D >= 3) axis_links_d<BC>(dl, pd, (double)uz, z, g.nz);
                if (++pending == 32) {
                    cadd(bulk, db);
                    cadd(link, dl);
                    db = dl = 0.0;
                    pending = 0;
                }
            }
        }
    }
    if (sizeof(T) == 4) {
        flush(fb, bulk);
        flush(fl, link);
        mxd = (double)mx;
    } else {
        cadd(bulk, db);
        cadd(link, dl);
    }
    // the bulk terms above are (p^2 - 1)^2; the 1/4 is applied at the end (exact)
    FixAcc ab, al;
    ab.add(bulk.s);
    ab.add(bulk.c);
    al.add(link.s);
    al.add(link.c);
    const Combined2 r = block_combine2(ab, al, mxd);
    if (threadIdx.x == 0) part[blockIdx.x] = RedPartial{r.b.s, r.b.c, r.l.s, r.l.c, r.m, 0.0, 0.0, 0.0};
    pdl_trigger();
}

__global__ void k_reduce_finish(const RedPartial* part, int nparts, double hd, double link_scale,
                                double* out2) {
    pdl_wait();
    FixAcc b, l;
    double m = 0.0;
#pragma unroll 4
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const RedPartial p = part[i];
        b.add(p.bulk_s);
        b.add(p.bulk_c);
        l.add(p.link_s);
        l.add(p.link_c);
        m = max_bits(m, p.mx);
    }
    const Combined2 r = block_combine2(b, l, m);
    if (threadIdx.x == 0) {
        const double bulk = r.b.s + r.b.c;
        const double links = r.l.s + r.l.c;
        out2[0] = hd * (0.25 * bulk + link_scale * links);
        out2[1] = r.m;
    }
    pdl_trigger();
}

int reduce_blocks(const Geo& g) {
    const int64_t rows = g.ny * g.nz;
    return (int)std::max<int64_t>(1, std::min<int64_t>(rows, kMaxRedBlocks));
}

template <typename T>
cudaError_t launch_reduce(int dims, int bc, const T* src, const Geo& g, double eps2, double h,
                          RedPartial* partials, double* out2, cudaStream_t st) {
    const int nb = reduce_blocks(g);
    cudaError_t e = cudaSuccess;
#define ACS_RED_CASE(D, B) \
    if (dims == D && bc == B) e = launch_pdl(k_reduce<T, D, B>, dim3(nb), dim3(256), 0, st, src, g, partials); else
    ACS_RED_CASE(1, 0) ACS_RED_CASE(1, 1) ACS_RED_CASE(1, 2)
    ACS_RED_CASE(2, 0) ACS_RED_CASE(2, 1) ACS_RED_CASE(2, 2)
    ACS_RED_CASE(3, 0) ACS_RED_CASE(3, 1) ACS_RED_CASE(3, 2)
    return cudaErrorInvalidValue;
#undef ACS_RED_CASE
    if (e != cudaSuccess) return e;
    const double hd = std::pow(h, (double)dims);
    return launch_pdl(k_reduce_finish, dim3(1), dim3(256), 0, st, (const RedPartial*)partials, nb, hd,
                      0.5 * eps2 / (h * h), out2);
}

template cudaError_t launch_reduce<float>(int, int, const float*, const Geo&, double, double, RedPartial*, double*, cudaStream_t);
template cudaError_t launch_reduce<double>(int, int, const double*, const Geo&, double, double, RedPartial*, double*, cudaStream_t);

cudaError_t launch_reduce_finish(const RedPartial* part, int nparts, int dims, double eps2, double h, double* out2,
                                 cudaStream_t st) {
    return launch_pdl(k_reduce_finish, dim3(1), dim3(256), 0, st, part, nparts, std::pow(h, (double)dims),
                      0.5 * eps2 / (h * h), out2);
}

// ---------------------------------------------------------------- phase volume
// sum_i phi_i over the unknowns (the volume is h^d (N + sum phi) / 2).  FP32 states:
// exact float-pair accumulation (TwoSum) folded into FP64 every 64 values; FP64
// states: plain FP64 per thread.  Partials are compensated and combined in a fixed
// order.
template <typename T>
__global__ void __launch_bounds__(256) k_phase_sum(const T* __restrict__ src, int64_t n, CSum* part) {
    CSum sum{0.0, 0.0};
    F2 f{0.0f, 0.0f};
    double d = 0.0;
    int pending = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (sizeof(T) == 4) {
            const F2 t = two_sum(f.hi, (float)src[i]);
            f.hi = t.hi;
            f.lo += t.lo;
            if (++pending == 64) {
                cadd(sum, (double)f.hi);
                cadd(sum, (double)f.lo);
                f = F2{0.0f, 0.0f};
                pending = 0;
            }
        } else {
            d += (double)src[i];
        }
    }
    if (sizeof(T) == 4) {
        cadd(sum, (double)f.hi);
        cadd(sum, (double)f.lo);
    } else {
        cadd(sum, d);
    }
    sum = block_csum(sum);
    if (threadIdx.x == 0) part[blockIdx.x] = sum;
}

__global__ void k_phase_finish(const CSum* part, int nparts, int64_t n, double hd, double* out) {
    const CSum s = block_sum_pairs(nparts, [&](int i) { return part[i]; });
    if (threadIdx.x == 0) out[0] = hd * 0.5 * ((double)n + (s.s + s.c));
}

template <typename T>
cudaError_t launch_phase_volume(const T* src, int64_t n, int dims, double h, void* scratch, double* out,
                                cudaStream_t st) {
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxRedBlocks, (n + 255) / 256));
    CSum* part = reinterpret_cast<CSum*>(scratch);
    k_phase_sum<T><<<nb, 256, 0, st>>>(src, n, part);
    k_phase_finish<<<1, 256, 0, st>>>(part, nb, n, std::pow(h, (double)dims), out);
    return cudaGetLastError();
}
template cudaError_t launch_phase_volume<float>(const float*, int64_t, int, double, void*, double*, cudaStream_t);
template cudaError_t launch_phase_volume<double>(const double*, int64_t, int, double, void*, double*, cudaStream_t);

}  // namespace acs
