// acs_api.cu -- host side of the C ABI declared in include/acs.h: validation,
// step-size conditions, coefficient set-up, launch planning, CUDA-graph replay,
// reductions and state transfer for single problems.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "acs_host.h"
#include "stream_tile.cuh"

namespace acs {

// ---------------------------------------------------------------- coefficients

// Relative error bound of the fast cubic path after `newton` corrections, for
// y = (a/b) x^2 (see cubic_root in acs_device.cuh).  The three-term series seed
// leaves rho0 <= 12 y^3 / (1 - 27y/4); a Newton correction with a reciprocal of
// relative error eta maps rho to 3 y rho^2 + eta rho.
static double cubic_bound(double y, int newton) {
    if (y >= 4.0 / 27.0) return 1.0;
    const double eta = 2.5e-7;
    double rho = 12.0 * y * y * y / (1.0 - 6.75 * y);
    for (int k = 0; k < newton; ++k) rho = 3.0 * y * rho * rho + eta * rho;
    return rho;
}

static void pick_newton(double t, double rb, double tol, int* newton, double* ymax) {
    const double xneed = 1.001 * rb;  // |xi| <= 1.001 under Theorem 2 (plus rounding)
    const double yneed = t * xneed * xneed;
    int n = 3;
    for (int k = 1; k <= 3; ++k)
        if (cubic_bound(yneed, k) <= tol) { n = k; break; }
    // largest y (below the series' radius 4/27) where the bound holds with n
    // corrections; it is at least yneed whenever the bound holds there
    double lo = 0.0, hi = 0.999 * 4.0 / 27.0;
    if (cubic_bound(hi, n) <= tol) lo = hi;
    else
        for (int it = 0; it < 80; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (cubic_bound(mid, n) <= tol) lo = mid; else hi = mid;
        }
    *newton = n;
    *ymax = lo;
}

// Corrections after the rational seed xi / (b + a xi^2) so that the root is accurate to
// tol for every |xi| <= 1.001, or 0 if kmax do not suffice.  The seed's relative error
// e0 and the contraction K = max 3 a theta^2 / (3 a theta^2 + b) of the relative error
// (e -> K e^2 for exact Newton) are sampled on a fine grid; the approximate
// reciprocal adds eta e per correction.
static int pick_rational(double a, double b, double tol, int kmax) {
    const int N = 4096;
    double e0 = 0.0, K = 0.0;
    for (int i = 1; i <= N; ++i) {
        const double xi = 1.001 * i / N;
        const double seed = xi / (b + a * xi * xi);
        double th = seed;  // an upper bound: Newton descends monotonically to the root
        for (int it = 0; it < 200; ++it) {
            const double nt = th - (a * th * th * th + b * th - xi) / (3.0 * a * th * th + b);
            if (!(nt < th)) break;
            th = nt;
        }
        e0 = std::max(e0, std::fabs(seed / th - 1.0));
        K = std::max(K, 3.0 * a * th * th / (3.0 * a * th * th + b));
    }
    const double eta = 2.5e-7;
    double e = e0 * 1.05 + eta;  // sampling margin; the seed's own approximate reciprocal
    for (int k = 1; k <= kmax; ++k) {
        e = K * e * e + eta * e;
        if (e <= tol) return k;
    }
    return 0;
}

// Lagrange-inversion coefficients C_k = binom(3k, k) / (2k + 1).
static const double kLagrangeC[11] = {1, 1, 3, 12, 55, 273, 1428, 7752, 43263, 246675, 1430715};

// Bound on the relative error of the series truncated after nt terms: the terms
// alternate and shrink (ratio < 27y/4 < 1), so the first omitted term bounds it.
static double series_bound(double y, int nt) {
    if (y >= 4.0 / 27.0) return 1.0;
    return kLagrangeC[nt] * std::pow(y, nt) / (1.0 - 6.75 * y);
}

template <typename T>
Coef<T> make_coef(int dims, double lam, double dt, int scheme, bool mp_ok) {
    Coef<T> c;
    std::memset(&c, 0, sizeof(c));
    const double a = 0.5 * dt, b = 1.0 - a;
    const double tol = sizeof(T) == 4 ? std::ldexp(1.0, -26) : std::ldexp(1.0, -55);
    c.lam = (T)lam;
    c.b = (T)b;
    c.rb = (T)(1.0 / b);
    c.t = (T)(a / b);
    c.three_a = (T)(3.0 * a);
    c.m2d = (T)(-2.0 * dims);
    if (scheme == ACS_SCHEME_FEX_FD) {
        c.a = (T)dt;
        c.na = (T)(-dt);
        c.c0 = (T)(1.0 - 2.0 * dims * lam + dt);
        c.solve = kSolveFex;
    } else {
        c.a = (T)a;
        c.na = (T)(-a);
        c.c0 = (T)(1.0 - 2.0 * dims * lam + a);
        const int nt = SeriesTerms<T>::value;
        const double t = a / b, rb = 1.0 / b;
        const double yneed = t * (1.001 * rb) * (1.001 * rb);
        if (series_bound(yneed, nt) <= tol) {
            c.solve = kSolveSeries;
            double lo = yneed, hi = 0.1;
            if (series_bound(hi, nt) <= tol) lo = hi;
            else
                for (int it = 0; it < 80; ++it) {
                    const double mid = 0.5 * (lo + hi);
                    if (series_bound(mid, nt) <= tol) lo = mid; else hi = mid;
                }
            const double x2max = lo / (t * rb * rb);
            c.xi2max = (T)std::min(x2max, 1e30);
            double ak = 1.0;  // (-a)^k
            for (int k = 0; k < nt; ++k) {
                c.q[k] = (T)(kLagrangeC[k] * ak / std::pow(b, 3.0 * k + 1.0));
                ak *= -a;
            }
            // the kernels sum R = P - 1 and form theta = xi + xi R: its constant term
            // is 1/b - 1 = a/b, computed without cancellation
            c.q[0] = (T)(a / b);
        } else {
            c.solve = kSolveNewton;
        }
        double ymax;
        pick_newton(t, rb, tol, &c.newton, &ymax);
        c.ymax = (T)ymax;
        c.seed = 0;
        if (c.solve == kSolveNewton && (cubic_bound(yneed, c.newton) > tol || ymax < yneed)) {
            // the three-term seed does not cover |xi| <= 1.001: the rational seed does
            const int k = pick_rational(a, b, tol, NewtonMax<T>::value);
            c.seed = 1;
            c.newton = k;
            c.xi2max = (T)(k > 0 ? 1.001 * 1.001 : -1.0);
        }
    }
    const double ulp1 = sizeof(T) == 4 ? std::ldexp(1.0, -23) : std::ldexp(1.0, -52);
    c.clamp_hi = (T)(1.0 + 16.0 * ulp1);
    c.clamp = mp_ok ? 1 : 0;
    // FP64 series: the terms k >= kSeriesSplit of R in FP32 when that moves theta by at
    // most 2^-58 for every xi the series takes (|xi| <= 1 under Theorem 2's clamp, else
    // xi^2 <= xi2max).  theta = xi + xi x2^5 T with T the tail; per term the truncated
    // x2 (2^-23 per power), the FP32 coefficient and the Horner roundings (2^-24 each)
    // stay below (NT - kSeriesSplit + 2) 2^-23 of the term's size.
    if (sizeof(T) == 8 && c.solve == kSolveSeries) {
        const int nt = SeriesTerms<T>::value;
        const double xm2 = c.clamp ? 1.0 : (double)c.xi2max;
        double bound = 0.0;
        for (int k = kSeriesSplit; k < nt; ++k)
            bound += std::fabs((double)c.q[k]) * std::pow(xm2, k + 0.5);
        bound *= (nt - kSeriesSplit + 2) * std::ldexp(1.0, -23);
        if (nt - kSeriesSplit <= 4 && std::isfinite(bound) && bound <= std::ldexp(1.0, -58)) {
            c.split = 1;
            for (int k = kSeriesSplit; k < nt; ++k) c.qf[k - kSeriesSplit] = (float)c.q[k];
        }
    }
    // fast path of the tiled kernels: the series range, and with the rounding guard
    // on, |xi| <= 1 + 8 ulp (exact root within [-1, 1] up to rounding)
    if (c.solve == kSolveSeries) {
        double f2 = (double)c.xi2max;
        if (c.clamp) f2 = std::min(f2, (1.0 + 8.0 * ulp1) * (1.0 + 8.0 * ulp1));
        c.fast2max = (T)f2;
    } else if (c.solve == kSolveNewton) {
        c.fast2max = (T)(c.clamp ? (1.0 + 8.0 * ulp1) * (1.0 + 8.0 * ulp1) : 1e30);
    }
    return c;
}
template Coef<float> make_coef<float>(int, double, double, int, bool);
template Coef<double> make_coef<double>(int, double, double, int, bool);

Geo make_geo(int dims, const int64_t* n) {
    Geo g;
    g.nx = g.ny = g.nz = 1;
    if (dims == 1) g.nx = n[0];
    if (dims == 2) { g.ny = n[0]; g.nx = n[1]; }
    if (dims == 3) { g.nz = n[0]; g.ny = n[1]; g.nx = n[2]; }
    g.sy = g.nx;
    g.sz = g.nx * g.ny;
    g.total = g.nx * g.ny * g.nz;
    return g;
}

}  // namespace acs

using namespace acs;

struct GraphEntry {
    int64_t nsteps, every;
    int kernel, depth, scheme;
    cudaGraphExec_t exec;
};

struct acs_ctx {
    int dims;
    int64_t n[3];
    double eps, dt, h;
    int bc, dtype;
    double lam;
    bool mp_ok, energy_ok;
    Geo g;
    size_t esize;
    int scheme;
    int kernel_req, depth_req;  // as requested
    int kernel, depth;          // resolved
    Coef<float> cf;
    Coef<double> cd;
    // bound resources
    bool bound;
    void* phi;
    char* work;
    size_t work_bytes;
    cudaStream_t stream;
    cudaStream_t cap;
    void* other;
    RedPartial* partials;
    double* result;
    double* log;
    int* err;          // set by kernels whose bounded waits gave up
    int zchunk;        // z planes (3D) / row blocks (2D) per CTA of the tiled kernels (0: default)
    int variant;       // tile shape of the tiled kernels
    bool tuned;        // the autotuner has run (or the cache answered) for this context
    int64_t steps_done;
    void* pop;         // population buffer of ACS_KERNEL_LB (caller-owned), or null
    size_t pop_bytes;
    double omega1;     // lattice weight w_1 of ACS_KERNEL_LB
    std::vector<GraphEntry> graphs;
    // adjoint recording
    GradState grad;
};

namespace {

constexpr size_t kAlign = 256;
constexpr int kLogCap = 4096;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

size_t state_bytes(const acs_ctx* c) { return (size_t)c->g.total * c->esize; }

size_t off_partials(const acs_ctx* c) { return align_up(state_bytes(c)); }
size_t off_result(const acs_ctx* c) { return off_partials(c) + align_up(sizeof(RedPartial) * kMaxStreamParts); }
size_t off_log(const acs_ctx* c) { return off_result(c) + kAlign; }
size_t off_flags(const acs_ctx* c) { return off_log(c) + align_up(sizeof(double) * 2 * kLogCap); }
size_t work_total(const acs_ctx* c) { return off_flags(c) + kAlign; }

void drop_graphs(acs_ctx* c) {
    for (auto& e : c->graphs) cudaGraphExecDestroy(e.exec);
    c->graphs.clear();
    grad_drop_graphs(c->grad);
}

void refresh_coef(acs_ctx* c) {
    c->cf = make_coef<float>(c->dims, c->lam, c->dt, c->scheme, c->mp_ok);
    c->cd = make_coef<double>(c->dims, c->lam, c->dt, c->scheme, c->mp_ok);
}

}  // namespace

// Launch `k` fused steps (k == 1 for non-temporal variants) from src to dst.
static cudaError_t launch_k(acs_ctx* c, int k, const void* src, void* dst, cudaStream_t st) {
    if (c->dtype == ACS_F32) {
        const float* s = (const float*)src;
        float* d = (float*)dst;
        if (c->kernel == ACS_KERNEL_LB)
            return launch_step_lb<float>(c->dims, c->bc, s, (float*)c->pop, d, c->g, c->omega1, c->lam, c->cf, st);
        if (c->kernel == ACS_KERNEL_TEMPORAL)
            return launch_step_temporal<float>(c->dims, c->bc, k, s, d, c->g, c->cf, c->variant, c->zchunk, c->err, st);
        if (c->kernel == ACS_KERNEL_TILED)
            return launch_step_tiled<float>(c->dims, c->bc, s, d, c->g, c->cf, c->variant, c->zchunk, c->err, st);
        return launch_step_naive<float>(c->dims, c->bc, s, d, c->g, c->cf, st);
    }
    const double* s = (const double*)src;
    double* d = (double*)dst;
    if (c->kernel == ACS_KERNEL_LB)
        return launch_step_lb<double>(c->dims, c->bc, s, (double*)c->pop, d, c->g, c->omega1, c->lam, c->cd, st);
    if (c->kernel == ACS_KERNEL_TEMPORAL)
        return launch_step_temporal<double>(c->dims, c->bc, k, s, d, c->g, c->cd, c->variant, c->zchunk, c->err, st);
    if (c->kernel == ACS_KERNEL_TILED)
        return launch_step_tiled<double>(c->dims, c->bc, s, d, c->g, c->cd, c->variant, c->zchunk, c->err, st);
    return launch_step_naive<double>(c->dims, c->bc, s, d, c->g, c->cd, st);
}

// Enqueue n steps; the state starts and ends in c->phi.  The launches are split
// so that their number is even (ping-pong ends where it started); only n == 1
// without temporal blocking, or an odd count of single steps, needs a final copy.
static cudaError_t enqueue_steps(acs_ctx* c, int64_t n, cudaStream_t st) {
    const int K = c->kernel == ACS_KERNEL_TEMPORAL ? c->depth : 1;
    std::vector<int> sizes;
    for (int64_t r = n; r > 0;) {
        const int k = (int)std::min<int64_t>(K, r);
        sizes.push_back(k);
        r -= k;
    }
    if (sizes.size() % 2 == 1) {
        for (size_t i = 0; i < sizes.size(); ++i)
            if (sizes[i] >= 2) {
                const int k = sizes[i];
                sizes[i] = k / 2;
                sizes.insert(sizes.begin() + i + 1, k - k / 2);
                break;
            }
    }
    const void* src = c->phi;
    void* dst = c->other;
    for (int k : sizes) {
        cudaError_t e = launch_k(c, k, src, dst, st);
        if (e != cudaSuccess) return e;
        const void* t = src;
        src = dst;
        dst = const_cast<void*>(t);
    }
    if (src != c->phi) return cudaMemcpyAsync(c->phi, src, state_bytes(c), cudaMemcpyDeviceToDevice, st);
    return cudaSuccess;
}

static int maybe_autotune(acs_ctx* c);

static cudaError_t enqueue_reduce(acs_ctx* c, const void* state, double* out2, cudaStream_t st);

// `count` single steps from `src` (phi or other), alternating buffers, ending in phi.
static cudaError_t enqueue_steps_from(acs_ctx* c, int64_t count, void* src, cudaStream_t st) {
    void* a = src;
    void* b = src == c->phi ? c->other : c->phi;
    for (int64_t j = 0; j < count; ++j) {
        cudaError_t e = launch_k(c, 1, a, b, st);
        if (e != cudaSuccess) return e;
        std::swap(a, b);
    }
    if (a != c->phi) return cudaMemcpyAsync(c->phi, a, state_bytes(c), cudaMemcpyDeviceToDevice, st);
    return cudaSuccess;
}

// A logged 3D run on the streamed kernels: the first step of every logged interval also
// reduces its input state (the fused mode of the 3D kernel), so those energies cost no
// pass of their own; the last logged state is reduced on its own.  cudaErrorNotSupported
// (before anything is enqueued) where the fused mode does not apply.
static cudaError_t enqueue_run_fused(acs_ctx* c, int64_t n, int64_t every, cudaStream_t st) {
    const bool rows16 = (c->g.nx * (int64_t)c->esize) % 16 == 0;
    if (c->dims != 3 || c->kernel != ACS_KERNEL_TILED || !rows16 || !tiled_supported(c->dims, c->dtype, c->g) ||
        every < 1)
        return cudaErrorNotSupported;
    const int64_t m = n / every + 1;
    for (int64_t k = 0; k + 1 < m; ++k) {
        int np = 0;
        cudaError_t e =
            c->dtype == ACS_F32
                ? launch_step_energy3d<float>(c->bc, (const float*)c->phi, (float*)c->other, c->g, c->cf, c->err,
                                              c->partials, &np, st)
                : launch_step_energy3d<double>(c->bc, (const double*)c->phi, (double*)c->other, c->g, c->cd, c->err,
                                               c->partials, &np, st);
        if (e != cudaSuccess) return e;  // NotSupported can only come at k = 0 (same shape every time)
        e = launch_reduce_finish(c->partials, np, c->dims, c->eps * c->eps, c->h, c->log + 2 * k, st);
        if (e == cudaSuccess) e = enqueue_steps_from(c, every - 1, c->other, st);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = enqueue_reduce(c, c->phi, c->log + 2 * (m - 1), st);
    const int64_t rest = n - (m - 1) * every;
    if (e == cudaSuccess && rest > 0) e = enqueue_steps(c, rest, st);
    return e;
}

// n steps with {E_h, max|phi|} of the states 0, every, 2 every, ... written to the
// context's log (every = 0: the steps alone).
static cudaError_t enqueue_run(acs_ctx* c, int64_t n, int64_t every, cudaStream_t st) {
    if (every <= 0) return enqueue_steps(c, n, st);
    if (n >= every) {
        const cudaError_t e = enqueue_run_fused(c, n, every, st);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();
    }
    const int64_t m = n / every + 1;
    cudaError_t e = enqueue_reduce(c, c->phi, c->log, st);
    for (int64_t k = 1; k < m && e == cudaSuccess; ++k) {
        e = enqueue_steps(c, every, st);
        if (e == cudaSuccess) e = enqueue_reduce(c, c->phi, c->log + 2 * k, st);
    }
    const int64_t rest = n - (m - 1) * every;
    if (e == cudaSuccess && rest > 0) e = enqueue_steps(c, rest, st);
    return e;
}

// Replay (recording on first use) the graph of exactly n steps (logged every `every`
// steps when every > 0), so a whole run costs one launch on the host.
static int launch_graph(acs_ctx* c, int64_t n, int64_t every = 0) {
    if (n < 4 && every <= 0) return enqueue_steps(c, n, c->stream) == cudaSuccess ? ACS_OK : ACS_E_CUDA;
    GraphEntry* hit = nullptr;
    for (auto& e : c->graphs)
        if (e.nsteps == n && e.every == every && e.kernel == c->kernel && e.depth == c->depth &&
            e.scheme == c->scheme)
            hit = &e;
    if (!hit) {
        if (c->graphs.size() >= 8) {
            cudaGraphExecDestroy(c->graphs.front().exec);
            c->graphs.erase(c->graphs.begin());
        }
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ACS_E_CUDA;
        cudaError_t e1 = enqueue_run(c, n, every, c->cap);
        cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            if (e2 == cudaSuccess) cudaGraphDestroy(graph);
            cudaGetLastError();
            return ACS_E_CUDA;
        }
        cudaGraphExec_t exec;
        cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) return ACS_E_CUDA;
        c->graphs.push_back(GraphEntry{n, every, c->kernel, c->depth, c->scheme, exec});
        hit = &c->graphs.back();
    }
    return cudaGraphLaunch(hit->exec, c->stream) == cudaSuccess ? ACS_OK : ACS_E_CUDA;
}

// Long runs replay a graph of kGraphSteps steps (each ends with the state back in
// phi) as often as needed plus one of the remainder, so graphs stay small.
constexpr int64_t kGraphSteps = 1024;

static int run_steps(acs_ctx* c, int64_t n) {
    if (n <= 0) return ACS_OK;
    if (int rc = maybe_autotune(c)) return rc;
    if (c->grad.active) {
        int rc = grad_record_steps(c, n);
        if (rc) return rc;
        c->steps_done += n;
        return ACS_OK;
    }
    for (int64_t left = n; left > 0;) {
        const int64_t k = left > kGraphSteps ? kGraphSteps : left;
        if (int rc = launch_graph(c, k)) return rc;
        left -= k;
    }
    c->steps_done += n;
    return ACS_OK;
}

// After a stream synchronization: report (and clear) a timeout recorded by a kernel.
static int check_err_flag(acs_ctx* c) {
    int h = 0;
    if (cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_E_CUDA;
    if (!h) return ACS_OK;
    cudaMemset(c->err, 0, sizeof(int));
    return ACS_E_TIMEOUT;
}

static cudaError_t enqueue_reduce(acs_ctx* c, const void* state, double* out2, cudaStream_t st) {
    const bool rows16 = (c->g.nx * (int64_t)c->esize) % 16 == 0;
    // the reduction follows the step's kernel family: the streamed (tile-per-CTA) pass
    // with the tiled kernels, the row-per-block one with the one-thread-per-unknown
    // kernel, which small grids take because it spreads them over more SMs
    if (c->kernel == ACS_KERNEL_TILED && (c->dims == 3 || c->dims == 2) && rows16 &&
        tiled_supported(c->dims, c->dtype, c->g)) {
        // the TMA-streamed pipeline: vector loads, neighbours from registers and shuffles
        int np = 0;
        cudaError_t e;
        if (c->dims == 3)
            e = c->dtype == ACS_F32
                    ? launch_energy3d<float>(c->bc, (const float*)state, c->g, c->cf, c->err, c->partials, &np, st)
                    : launch_energy3d<double>(c->bc, (const double*)state, c->g, c->cd, c->err, c->partials, &np, st);
        else
            e = c->dtype == ACS_F32
                    ? launch_energy2d<float>(c->bc, (const float*)state, c->g, c->cf, c->err, c->partials, &np, st)
                    : launch_energy2d<double>(c->bc, (const double*)state, c->g, c->cd, c->err, c->partials, &np, st);
        if (e == cudaSuccess) return launch_reduce_finish(c->partials, np, c->dims, c->eps * c->eps, c->h, out2, st);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();
    }
    if (c->dtype == ACS_F32)
        return launch_reduce<float>(c->dims, c->bc, (const float*)state, c->g, c->eps * c->eps, c->h,
                                    c->partials, out2, st);
    return launch_reduce<double>(c->dims, c->bc, (const double*)state, c->g, c->eps * c->eps, c->h,
                                 c->partials, out2, st);
}

// ---------------------------------------------------------------- helpers for other units

namespace acs {
cudaError_t ctx_enqueue_steps(acs_ctx* c, int64_t n, cudaStream_t st) { return enqueue_steps(c, n, st); }
cudaError_t ctx_launch_one(acs_ctx* c, const void* src, void* dst, cudaStream_t st) {
    // one step; every FD variant gives identical bits, so use the context's tiled
    // kernel when it has one; the population form recomputes with itself
    if (c->kernel == ACS_KERNEL_TILED || c->kernel == ACS_KERNEL_LB) return launch_k(c, 1, src, dst, st);
    if (c->dtype == ACS_F32)
        return launch_step_naive<float>(c->dims, c->bc, (const float*)src, (float*)dst, c->g, c->cf, st);
    return launch_step_naive<double>(c->dims, c->bc, (const double*)src, (double*)dst, c->g, c->cd, st);
}
// Enqueue n_steps steps with {E_h, max|phi|} of the states 0, every, 2 every, ...
// written to the context's device log (2 doubles per entry); nothing synchronizes.
int ctx_enqueue_logged(acs_ctx* c, int64_t n_steps, int64_t every, double** d_log, int64_t* entries) {
    if (!c->bound) return ACS_E_STATE;
    const int64_t m = every > 0 ? n_steps / every + 1 : 0;
    if (m > kLogCap) return ACS_E_INVAL;
    *d_log = c->log;
    *entries = m;
    if (m == 0) return run_steps(c, n_steps);
    if (int rc = maybe_autotune(c)) return rc;
    if (!c->grad.active && n_steps <= kGraphSteps) {
        // the whole logged run as one recorded graph
        if (int rc = launch_graph(c, n_steps, every)) return rc;
        c->steps_done += n_steps;
        return ACS_OK;
    }
    if (enqueue_reduce(c, c->phi, c->log, c->stream) != cudaSuccess) return ACS_E_CUDA;
    int64_t done = 0;
    for (int64_t k = 1; k < m; ++k) {
        if (int rc = run_steps(c, every)) return rc;
        done += every;
        if (enqueue_reduce(c, c->phi, c->log + 2 * k, c->stream) != cudaSuccess) return ACS_E_CUDA;
    }
    return run_steps(c, n_steps - done);
}
int ctx_check_err(acs_ctx* c) { return check_err_flag(c); }
CtxView ctx_view(acs_ctx* c) {
    CtxView v;
    v.dims = c->dims; v.bc = c->bc; v.dtype = c->dtype; v.g = c->g; v.esize = c->esize;
    v.lam = c->lam; v.dt = c->dt; v.h = c->h; v.eps = c->eps;
    v.phi = c->phi; v.other = c->other; v.stream = c->stream; v.cap = c->cap; v.err = c->err; v.partials = c->partials;
    v.result = c->result; v.steps_done = c->steps_done; v.cf = c->cf; v.cd = c->cd; v.grad = &c->grad;
    return v;
}
}  // namespace acs

// ---------------------------------------------------------------- C ABI

extern "C" {

ACS_API const char* acs_version(void) { return "0.1.0"; }

ACS_API const char* acs_strerror(int s) {
    switch (s) {
        case ACS_OK: return "ok";
        case ACS_WARN_MP_CONDITION: return "warning: dt > 1 - 2 d lambda, the maximum principle (Theorem 2) is not guaranteed";
        case ACS_WARN_ENERGY_CONDITION: return "warning: dt > 4 (1 - 2 d lambda), energy decay (Theorem 3) is not guaranteed";
        case ACS_E_INVAL: return "invalid argument";
        case ACS_E_CUDA: return "CUDA runtime error";
        case ACS_E_NOMEM: return "work buffer too small or host allocation failed";
        case ACS_E_TIMEOUT: return "a bounded device-side wait gave up";
        case ACS_E_NONFINITE: return "state is not finite (NaN or Inf)";
        case ACS_E_STATE: return "call out of order (bind/set_state/record first)";
        case ACS_E_UNSUPPORTED: return "kernel variant not available for this problem";
        default: return "unknown status";
    }
}

ACS_API int acs_dt_max(int dims, double eps, double h, double* dt_mp, double* dt_energy) {
    if (dims < 1 || dims > 3 || !(eps >= 0) || !(h > 0) || !std::isfinite(eps) || !std::isfinite(h))
        return ACS_E_INVAL;
    const double r = eps * eps / (h * h);
    // Theorem 2: dt <= 1 - 2 d lambda, lambda = r dt  =>  dt <= 1 / (1 + 2 d r)
    if (dt_mp) *dt_mp = 1.0 / (1.0 + 2.0 * dims * r);
    // Theorem 3: dt <= 4 (1 - 2 d lambda)  =>  dt <= 4 / (1 + 8 d r)
    if (dt_energy) *dt_energy = 4.0 / (1.0 + 8.0 * dims * r);
    return ACS_OK;
}

ACS_API int acs_create(int dims, const int64_t n[3], double eps, double dt, double h, int bc, int dtype,
                       acs_ctx** out) {
    if (!out || !n || dims < 1 || dims > 3) return ACS_E_INVAL;
    if (!std::isfinite(eps) || !std::isfinite(dt) || !std::isfinite(h)) return ACS_E_INVAL;
    if (eps < 0 || !(h > 0) || !(dt > 0) || !(dt < 2)) return ACS_E_INVAL;
    if (bc < 0 || bc > 2 || (dtype != ACS_F32 && dtype != ACS_F64)) return ACS_E_INVAL;
    if (!shape_ok(dims, n)) return ACS_E_INVAL;
    acs_ctx* c = new (std::nothrow) acs_ctx();
    if (!c) return ACS_E_NOMEM;
    c->dims = dims;
    for (int k = 0; k < 3; ++k) c->n[k] = k < dims ? n[k] : 1;
    c->eps = eps; c->dt = dt; c->h = h; c->bc = bc; c->dtype = dtype;
    c->lam = eps * eps * dt / (h * h);
    double dmp, den;
    acs_dt_max(dims, eps, h, &dmp, &den);
    c->mp_ok = dt <= dmp * (1.0 + 1e-12);
    c->energy_ok = dt <= den * (1.0 + 1e-12);
    c->g = make_geo(dims, c->n);
    c->esize = dtype == ACS_F32 ? 4 : 8;
    c->scheme = ACS_SCHEME_RLB_MIE_FD;
    c->kernel_req = ACS_KERNEL_AUTO;
    c->depth_req = 1;
    c->kernel = ACS_KERNEL_NAIVE;
    c->depth = 1;
    refresh_coef(c);
    c->bound = false;
    c->phi = nullptr; c->work = nullptr; c->work_bytes = 0;
    c->stream = nullptr; c->cap = nullptr;
    c->steps_done = 0;
    c->err = nullptr;
    c->zchunk = 0;
    c->variant = 0;
    c->tuned = false;
    c->pop = nullptr;
    c->pop_bytes = 0;
    c->omega1 = 0.0;
    c->grad = GradState();
    resolve_auto_kernel(c->dims, c->dtype, c->bc, c->g, &c->kernel, &c->depth);
    *out = c;
    if (!c->energy_ok) return ACS_WARN_ENERGY_CONDITION;
    if (!c->mp_ok) return ACS_WARN_MP_CONDITION;
    return ACS_OK;
}

ACS_API size_t acs_work_bytes(const acs_ctx* c) { return c ? work_total(c) : 0; }

ACS_API int acs_bind(acs_ctx* c, void* d_phi, void* d_work, size_t work_bytes, void* stream) {
    if (!c || !d_phi || !d_work) return ACS_E_INVAL;
    if (((uintptr_t)d_phi % 16) || ((uintptr_t)d_work % kAlign)) return ACS_E_INVAL;
    if (work_bytes < work_total(c)) return ACS_E_NOMEM;
    if (!c->cap) {
        if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) return ACS_E_CUDA;
    }
    drop_graphs(c);
    c->phi = d_phi;
    c->work = (char*)d_work;
    c->work_bytes = work_bytes;
    c->stream = (cudaStream_t)stream;
    c->other = c->work;
    c->partials = (RedPartial*)(c->work + off_partials(c));
    c->result = (double*)(c->work + off_result(c));
    c->log = (double*)(c->work + off_log(c));
    c->err = (int*)(c->work + off_flags(c));
    if (cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) != cudaSuccess) return ACS_E_CUDA;
    c->steps_done = 0;
    c->bound = true;
    return ACS_OK;
}

ACS_API int acs_set_scheme(acs_ctx* c, int scheme) {
    if (!c || (scheme != ACS_SCHEME_RLB_MIE_FD && scheme != ACS_SCHEME_FEX_FD)) return ACS_E_INVAL;
    if (c->kernel == ACS_KERNEL_LB && scheme != ACS_SCHEME_RLB_MIE_FD) return ACS_E_UNSUPPORTED;
    c->scheme = scheme;
    refresh_coef(c);
    drop_graphs(c);
    return ACS_OK;
}

ACS_API int acs_set_kernel(acs_ctx* c, int kernel, int depth) {
    if (!c) return ACS_E_INVAL;
    if (kernel == ACS_KERNEL_AUTO) {
        c->kernel_req = kernel;
        resolve_auto_kernel(c->dims, c->dtype, c->bc, c->g, &c->kernel, &c->depth);
        drop_graphs(c);
        return ACS_OK;
    }
    if (kernel == ACS_KERNEL_NAIVE) {
        c->kernel_req = c->kernel = kernel;
        c->depth = 1;
        drop_graphs(c);
        return ACS_OK;
    }
    if (kernel == ACS_KERNEL_TILED) {
        if (!tiled_supported(c->dims, c->dtype, c->g)) return ACS_E_UNSUPPORTED;
        c->kernel_req = c->kernel = kernel;
        c->depth = 1;
        drop_graphs(c);
        return ACS_OK;
    }
    if (kernel == ACS_KERNEL_LB) {
        if (!c->pop) return ACS_E_STATE;
        if (c->scheme != ACS_SCHEME_RLB_MIE_FD) return ACS_E_UNSUPPORTED;
        c->kernel_req = c->kernel = kernel;
        c->depth = 1;
        drop_graphs(c);
        return ACS_OK;
    }
    if (kernel == ACS_KERNEL_TEMPORAL) {
        if (depth < 1 || depth > 8) return ACS_E_INVAL;
        if (!temporal_supported(c->dims, c->dtype, depth, c->g)) return ACS_E_UNSUPPORTED;
        c->kernel_req = c->kernel = kernel;
        c->depth = depth;
        drop_graphs(c);
        return ACS_OK;
    }
    return ACS_E_INVAL;
}

ACS_API int acs_get_kernel(const acs_ctx* c, int* kernel, int* depth) {
    if (!c) return ACS_E_INVAL;
    if (kernel) *kernel = c->kernel;
    if (depth) *depth = c->depth;
    return ACS_OK;
}

ACS_API int acs_get_root(const acs_ctx* c, int* mode, int* split) {
    if (!c) return ACS_E_INVAL;
    static_assert(kSolveNewton == ACS_ROOT_NEWTON && kSolveSeries == ACS_ROOT_SERIES && kSolveFex == ACS_ROOT_NONE,
                  "root modes");
    if (mode) *mode = c->dtype == ACS_F32 ? c->cf.solve : c->cd.solve;
    if (split) *split = c->dtype == ACS_F32 ? c->cf.split : c->cd.split;
    return ACS_OK;
}

ACS_API size_t acs_lb_bytes(const acs_ctx* c) {
    return c ? (size_t)(2 * c->dims + 1) * (state_bytes(c) + (size_t)kLbGap * c->esize) : 0;
}

ACS_API int acs_lb_bind(acs_ctx* c, void* d_pop, size_t bytes, double omega1) {
    if (!c || !d_pop || ((uintptr_t)d_pop % 16)) return ACS_E_INVAL;
    if (!std::isfinite(omega1) || omega1 > 1.0 / (2.0 * c->dims) * (1.0 + 1e-15)) return ACS_E_INVAL;
    if (bytes < acs_lb_bytes(c)) return ACS_E_NOMEM;
    // the paper's weights: w_1 = 1/3, 1/5, 1/6 for d = 1, 2, 3 (Sec. IV)
    static const double kDefaultW1[4] = {0.0, 1.0 / 3.0, 1.0 / 5.0, 1.0 / 6.0};
    c->omega1 = omega1 > 0.0 ? omega1 : kDefaultW1[c->dims];
    c->pop = d_pop;
    c->pop_bytes = bytes;
    drop_graphs(c);
    return ACS_OK;
}

ACS_API int acs_set_state(acs_ctx* c, const void* d_phi0) {
    if (!c || !d_phi0) return ACS_E_INVAL;
    if (!c->bound) return ACS_E_STATE;
    if (d_phi0 != c->phi &&
        cudaMemcpyAsync(c->phi, d_phi0, state_bytes(c), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return ACS_E_CUDA;
    c->steps_done = 0;
    return grad_on_set_state(c);
}

ACS_API int acs_set_state_host(acs_ctx* c, const void* h_phi0) {
    if (!c || !h_phi0) return ACS_E_INVAL;
    if (!c->bound) return ACS_E_STATE;
    if (cudaMemcpyAsync(c->phi, h_phi0, state_bytes(c), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return ACS_E_CUDA;
    c->steps_done = 0;
    return grad_on_set_state(c);
}

ACS_API int acs_get_state_host(acs_ctx* c, void* h_phi) {
    if (!c || !h_phi) return ACS_E_INVAL;
    if (!c->bound) return ACS_E_STATE;
    if (cudaMemcpyAsync(h_phi, c->phi, state_bytes(c), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return ACS_E_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ACS_E_CUDA;
    return check_err_flag(c);
}

ACS_API int acs_step(acs_ctx* c, int64_t n_steps) {
    if (!c || n_steps < 0) return ACS_E_INVAL;
    if (!c->bound) return ACS_E_STATE;
    return run_steps(c, n_steps);
}

ACS_API int64_t acs_steps_done(const acs_ctx* c) { return c ? c->steps_done : -1; }

ACS_API int acs_observe_async(acs_ctx* c, double* d_out2) {
    if (!c || !d_out2) return ACS_E_INVAL;
    if (!c->bound) return ACS_E_STATE;
    return enqueue_reduce(c, c->phi, d_out2, c->stream) == cudaSuccess ? ACS_OK : ACS_E_CUDA;
}

static int observe_host(acs_ctx* c, double* e, double* m) {
    if (!c->bound) return ACS_E_STATE;
    if (enqueue_reduce(c, c->phi, c->result, c->stream) != cudaSuccess) return ACS_E_CUDA;
    double hbuf[2];
    if (cudaMemcpyAsync(hbuf, c->result, sizeof(hbuf), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return ACS_E_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ACS_E_CUDA;
    if (int rc = check_err_flag(c)) return rc;
    if (e) *e = hbuf[0];
    if (m) *m = hbuf[1];
    const double v = e ? hbuf[0] : hbuf[1];
    return std::isfinite(v) && std::isfinite(hbuf[1]) ? ACS_OK : ACS_E_NONFINITE;
}

ACS_API int acs_energy(acs_ctx* c, double* out_host) {
    if (!c || !out_host) return ACS_E_INVAL;
    return observe_host(c, out_host, nullptr);
}

ACS_API int acs_maxnorm(acs_ctx* c, double* out_host) {
    if (!c || !out_host) return ACS_E_INVAL;
    double m = 0.0;
    int rc = observe_host(c, nullptr, &m);
    *out_host = m;
    return rc;
}

ACS_API int acs_phase_volume(acs_ctx* c, double* out_host) {
    if (!c || !out_host) return ACS_E_INVAL;
    if (!c->bound) return ACS_E_STATE;
    cudaError_t e = c->dtype == ACS_F32
                        ? launch_phase_volume<float>((const float*)c->phi, c->g.total, c->dims, c->h, c->partials,
                                                     c->result, c->stream)
                        : launch_phase_volume<double>((const double*)c->phi, c->g.total, c->dims, c->h, c->partials,
                                                      c->result, c->stream);
    if (e != cudaSuccess) return ACS_E_CUDA;
    double v = 0.0;
    if (cudaMemcpyAsync(&v, c->result, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return ACS_E_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ACS_E_CUDA;
    if (int rc = check_err_flag(c)) return rc;
    *out_host = v;
    return std::isfinite(v) ? ACS_OK : ACS_E_NONFINITE;
}

ACS_API int acs_run_logged(acs_ctx* c, int64_t n_steps, int64_t every, double* h_energy, double* h_maxnorm) {
    if (!c || n_steps < 0 || every < 1 || !h_energy || !h_maxnorm) return ACS_E_INVAL;
    double* d_log = nullptr;
    int64_t entries = 0;
    if (int rc = ctx_enqueue_logged(c, n_steps, every, &d_log, &entries)) return rc;
    std::vector<double> buf(2 * entries);
    if (cudaMemcpyAsync(buf.data(), d_log, sizeof(double) * 2 * entries, cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
        return ACS_E_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ACS_E_CUDA;
    if (int rc = check_err_flag(c)) return rc;
    bool finite = true;
    for (int64_t k = 0; k < entries; ++k) {
        h_energy[k] = buf[2 * k];
        h_maxnorm[k] = buf[2 * k + 1];
        finite = finite && std::isfinite(buf[2 * k]) && std::isfinite(buf[2 * k + 1]);
    }
    return finite ? ACS_OK : ACS_E_NONFINITE;
}

ACS_API int acs_num_variants(void) { return kNumTileVariants; }

ACS_API int acs_set_variant(acs_ctx* c, int variant, int chunk) {
    if (!c || variant < 0 || variant >= kNumTileVariants || chunk < 0) return ACS_E_INVAL;
    c->variant = variant;
    c->zchunk = chunk;
    drop_graphs(c);
    return ACS_OK;
}

ACS_API int acs_get_variant(const acs_ctx* c, int* variant, int* chunk) {
    if (!c) return ACS_E_INVAL;
    if (variant) *variant = c->variant;
    if (chunk) *chunk = c->zchunk;
    return ACS_OK;
}

ACS_API int acs_autotune(acs_ctx* c, double* us_per_step) {
    if (!c) return ACS_E_INVAL;
    if (!c->bound) return ACS_E_STATE;
    if (c->grad.active) return ACS_E_STATE;
    struct Cand { int kernel, depth, variant, chunk; };
    std::vector<Cand> cands;
    cands.push_back({ACS_KERNEL_NAIVE, 1, 0, 0});
    if (tiled_supported(c->dims, c->dtype, c->g)) {
        for (int v = 0; v < kNumTileVariants; ++v) {
            cands.push_back({ACS_KERNEL_TILED, 1, v, 0});
            if (c->dims == 3 && c->g.nz >= 64) {
                cands.push_back({ACS_KERNEL_TILED, 1, v, 16});
                cands.push_back({ACS_KERNEL_TILED, 1, v, 32});
            }
            if (c->dims == 2) {
                // 16-row blocks per CTA
                cands.push_back({ACS_KERNEL_TILED, 1, v, 1});
                cands.push_back({ACS_KERNEL_TILED, 1, v, 2});
            }
        }
    }
    for (int k = 2; k <= 8; ++k)
        if (temporal_supported(c->dims, c->dtype, k, c->g)) cands.push_back({ACS_KERNEL_TEMPORAL, k, 0, 0});
    const Cand saved = {c->kernel, c->depth, c->variant, c->zchunk};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ACS_E_CUDA;
    double best = 1e300;
    Cand win = saved;
    const double per_launch_units = (double)c->g.total;
    for (const Cand& k : cands) {
        c->kernel = k.kernel;
        c->depth = k.depth;
        c->variant = k.variant;
        c->zchunk = k.chunk;
        const int steps = k.kernel == ACS_KERNEL_TEMPORAL ? k.depth : 1;
        // warm up, then time launches phi -> work (the state is only read)
        if (launch_k(c, steps, c->phi, c->other, c->stream) != cudaSuccess) { cudaGetLastError(); continue; }
        int reps = 3;
        for (int round = 0; round < 2; ++round) {
            cudaEventRecord(e0, c->stream);
            for (int r = 0; r < reps; ++r) launch_k(c, steps, c->phi, c->other, c->stream);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return ACS_E_CUDA; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double us = 1e3 * ms / reps / steps;
            if (round == 1 && us < best) { best = us; win = k; }
            // second round: enough launches for about 2 ms
            reps = (int)std::min<double>(200.0, std::max(3.0, 2000.0 / std::max(1e-3, 1e3 * ms / reps)));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)per_launch_units;
    c->kernel = win.kernel;
    c->depth = win.depth;
    c->variant = win.variant;
    c->zchunk = win.chunk;
    c->tuned = true;
    drop_graphs(c);
    if (int rc = check_err_flag(c)) return rc;
    tune_cache_store(c->dims, c->n, c->bc, c->dtype, c->scheme, win.kernel, win.depth, win.variant, win.chunk, best);
    if (us_per_step) *us_per_step = best;
    return ACS_OK;
}

ACS_API int acs_sync(acs_ctx* c) {
    if (!c) return ACS_E_INVAL;
    if (!c->bound) return ACS_OK;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ACS_E_CUDA;
    return check_err_flag(c);
}

ACS_API void acs_destroy(acs_ctx* c) {
    if (!c) return;
    if (c->bound) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

}  // extern "C"

// ACS_KERNEL_AUTO: on the first step of a large enough problem, take the cached
// choice for this problem or run the autotuner.
static int maybe_autotune(acs_ctx* c) {
    if (c->tuned || c->kernel_req != ACS_KERNEL_AUTO || c->grad.active) return ACS_OK;
    c->tuned = true;
    const char* env = std::getenv("ACS_AUTOTUNE");
    int k, d, v, ch;
    if (tune_cache_lookup(c->dims, c->n, c->bc, c->dtype, c->scheme, &k, &d, &v, &ch)) {
        const bool ok = (k == ACS_KERNEL_NAIVE) || (k == ACS_KERNEL_TILED && tiled_supported(c->dims, c->dtype, c->g)) ||
                        (k == ACS_KERNEL_TEMPORAL && temporal_supported(c->dims, c->dtype, d, c->g));
        if (ok && v >= 0 && v < kNumTileVariants) {
            c->kernel = k; c->depth = d; c->variant = v; c->zchunk = ch;
            drop_graphs(c);
            return ACS_OK;
        }
    }
    if (c->g.total < (int64_t(1) << 20) || (env && std::strcmp(env, "0") == 0)) return ACS_OK;
    return acs_autotune(c, nullptr);
}
