// lines.cu -- many independent 1D problems (lines), each held on chip for all the
// time steps of a call: the 1D path at scale.
//
// A line of n <= 32 R points (R in {1, 2, 4, ..., 32}; FP64 up to 16) belongs to one
// warp: lane l keeps points l R .. l R + R - 1 in registers, takes its two outer
// neighbours from the adjacent lanes by shuffles and updates its R points together, so
// no memory is touched between the first load and the last store.  A longer line (up
// to LineSmemMax<T> points) belongs to one CTA that ping-pongs it in shared memory.
// Either way each point's new value is the predictor and root of the same operands in
// the same order as the single-problem 1D kernel (Eq. IE-FD with d = 1, the ghost rule
// of Eq. Ddeltax at both ends, Remark 1's cubic), so every line is bit-identical to its
// standalone run.  Lines are independent: one launch per size class, the classes on
// concurrent streams, no grid synchronization.
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "acs_host.h"
#include "f32x2.cuh"
#include "stream_tile.cuh"

namespace acs {

template <typename T>
struct LineRec {
    int64_t off;  // first value of the line in the packed state
    int n;        // points
    int bc;
    Coef<T> c;
};

// longest line a CTA keeps in shared memory (two buffers plus the two ghosts)
template <typename T>
struct LineSmemMax {
    static constexpr int value = sizeof(T) == 4 ? 28672 : 14336;
};

// One warp per line, R points per lane in registers.
template <typename T, int R, int SOLVE>
__device__ __forceinline__ void line_warp(T* __restrict__ phi, const LineRec<T>& L, int64_t nsteps) {
    const int lane = threadIdx.x & 31;
    const int n = L.n, bc = L.bc;
    const Coef<T> c = L.c;
    PackedCoef pc;
    if constexpr (std::is_same<T, float>::value) pc = packed_coef(c);
    T* p = phi + L.off;
    T x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gi = lane * R + r;
        x[r] = gi < n ? p[gi] : T(0);
    }
    const int ln = (n - 1) / R, rn = (n - 1) % R;  // lane and slot of point n - 1
    for (int64_t s = 0; s < nsteps; ++s) {
        const T up = __shfl_up_sync(0xffffffffu, x[R - 1], 1);
        const T dn = __shfl_down_sync(0xffffffffu, x[0], 1);
        // the end values, for the periodic wrap
        T mine_last = x[0];
#pragma unroll
        for (int r = 1; r < R; ++r)
            if (r == rn) mine_last = x[r];
        const T last = __shfl_sync(0xffffffffu, mine_last, ln);
        const T first = __shfl_sync(0xffffffffu, x[0], 0);
        // ghosts of point 0 (left) and point n - 1 (right)
        const T gl = bc == ACS_BC_PERIODIC ? last : (bc == ACS_BC_NEUMANN ? first : T(0));
        const T gr = bc == ACS_BC_PERIODIC ? first : (bc == ACS_BC_NEUMANN ? last : T(0));
        // xi of the R points, then their roots together (the multi-point solve gives
        // the per-point cubic_root() values)
        T xi[R], out[R];
        T sn[R];  // neighbour sums
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int gi = lane * R + r;
            const T xm = r == 0 ? (lane == 0 ? gl : up) : x[r - 1];
            T xp = r < R - 1 ? x[r + 1] : dn;
            if (gi == n - 1) xp = gr;
            sn[r] = nsum(xm, xp);
        }
        if constexpr (std::is_same<T, float>::value && R % 2 == 0) {
            // FP32: the same operations on pairs of points
            f2 xp2[R / 2];
#pragma unroll
            for (int r = 0; r < R; r += 2)
                xp2[r / 2] = predictor2(f2_make(x[r], x[r + 1]), f2_make(sn[r], sn[r + 1]), pc);
            roots2<SOLVE, R / 2>(xp2, out, c, pc);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) xi[r] = predictor(x[r], sn[r], c);
            roots<T, SOLVE, R>(xi, out, c);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (lane * R + r < n) x[r] = out[r];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gi = lane * R + r;
        if (gi < n) p[gi] = x[r];
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(64) k_lines_warp(T* phi, const LineRec<T>* __restrict__ lines,
                                                    const int* __restrict__ ids, int nlines, int64_t nsteps) {
    const int w = blockIdx.x * 2 + (threadIdx.x >> 5);
    if (w >= nlines) return;  // whole warps leave together
    const LineRec<T>& L = lines[ids[w]];
    ACS_SOLVE_DISPATCH_UNIT(L.c, SV, line_warp<T, R, SV>(phi, L, nsteps));
}

// One CTA per line in shared memory: buffers of n + 2 values (ghosts at both ends),
// padded to a multiple of 4 with zeros.  Each thread updates groups of 4 consecutive
// points with the multi-point root solve (the per-point values, see roots()).
template <typename T, int SOLVE>
__device__ __forceinline__ void line_cta(T* __restrict__ phi, const LineRec<T>& L, int64_t nsteps, T* A, T* B) {
    constexpr int G = 4;
    const int n = L.n, bc = L.bc;
    const int npad = (n + G - 1) / G * G;
    const Coef<T> c = L.c;
    PackedCoef pc;
    if constexpr (std::is_same<T, float>::value) pc = packed_coef(c);
    T* p = phi + L.off;
    for (int i = threadIdx.x; i < npad + 2; i += blockDim.x) {
        A[i] = i >= 1 && i <= n ? p[i - 1] : T(0);
        B[i] = T(0);
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        __syncthreads();
        if (threadIdx.x == 0) {
            A[0] = bc == ACS_BC_PERIODIC ? A[n] : (bc == ACS_BC_NEUMANN ? A[1] : T(0));
            A[n + 1] = bc == ACS_BC_PERIODIC ? A[1] : (bc == ACS_BC_NEUMANN ? A[n] : T(0));
        }
        __syncthreads();
        for (int g0 = threadIdx.x * G; g0 < n; g0 += blockDim.x * G) {
            T v[G + 2], xi[G], out[G];
#pragma unroll
            for (int k = 0; k < G + 2; ++k) v[k] = A[g0 + k];  // points g0 - 1 .. g0 + G
            // points past n read the ghost and the zero padding; their results are unused
            if constexpr (std::is_same<T, float>::value) {
                f2 xp2[G / 2];
#pragma unroll
                for (int k = 0; k < G; k += 2)
                    xp2[k / 2] = predictor2(f2_make(v[k + 1], v[k + 2]),
                                            f2_make(nsum(v[k], v[k + 2]), nsum(v[k + 1], v[k + 3])), pc);
                roots2<SOLVE, G / 2>(xp2, out, c, pc);
            } else {
#pragma unroll
                for (int k = 0; k < G; ++k) xi[k] = predictor(v[k + 1], nsum(v[k], v[k + 2]), c);
                roots<T, SOLVE, G>(xi, out, c);
            }
#pragma unroll
            for (int k = 0; k < G; ++k)
                if (g0 + k < n) B[g0 + k + 1] = out[k];
        }
        T* t = A;
        A = B;
        B = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = A[i + 1];
}

template <typename T>
__global__ void __launch_bounds__(256) k_lines_cta(T* phi, const LineRec<T>* __restrict__ lines,
                                                   const int* __restrict__ ids, int64_t nsteps, int maxn) {
    extern __shared__ __align__(16) unsigned char sm[];
    T* A = reinterpret_cast<T*>(sm);
    T* B = A + ((maxn + 3) / 4 * 4 + 2);
    const LineRec<T>& L = lines[ids[blockIdx.x]];
    ACS_SOLVE_DISPATCH_UNIT(L.c, SV, line_cta<T, SV>(phi, L, nsteps, A, B));
}

}  // namespace acs

using namespace acs;

// size classes: R = 1, 2, 4, ..., 32 (warp-resident), then the shared-memory class
static constexpr int kLineClasses = 7;

struct acs_lines {
    int count, dtype;
    size_t esize;
    std::vector<int64_t> n, off;
    std::vector<double> eps, dt, h;
    std::vector<int> bc;
    std::vector<LineRec<float>> recf;
    std::vector<LineRec<double>> recd;
    std::vector<int> ids;          // line indices grouped by class
    int cls_begin[kLineClasses + 1];
    int maxn_cta;                  // longest line of the shared-memory class
    int64_t numel;
    bool bound;
    char* phi;
    char* work;
    cudaStream_t stream;
    void* drec;
    int* dids;
    RedPartial* partials;
    double* results;
    cudaStream_t aux[kLineClasses];  // one stream per size class
    cudaEvent_t fork, join[kLineClasses];
    bool have_streams;
};

namespace {
constexpr size_t kLA = 256;
size_t lal(size_t x) { return (x + kLA - 1) / kLA * kLA; }
size_t rec_bytes(const acs_lines* L) {
    return lal((size_t)L->count * (L->dtype == ACS_F32 ? sizeof(LineRec<float>) : sizeof(LineRec<double>)));
}
size_t off_ids(const acs_lines* L) { return rec_bytes(L); }
size_t off_part(const acs_lines* L) { return off_ids(L) + lal(sizeof(int) * (size_t)L->count); }
size_t off_res(const acs_lines* L) { return off_part(L) + lal(sizeof(RedPartial) * kMaxRedBlocks); }
size_t lines_total(const acs_lines* L) { return off_res(L) + lal(sizeof(double) * 2 * (size_t)L->count); }

// class k < 6: warp-resident with R = 2^k points per lane (up to R = 32, FP64 16, where
// the values still leave registers for several warps per SM); class 6: one CTA in
// shared memory
int line_class(int64_t n, int dtype) {
    const int kmax = dtype == ACS_F32 ? 6 : 5;  // FP64: R <= 16
    for (int k = 0; k < kmax; ++k)
        if (n <= 32LL << k) return k;
    return 6;
}

template <typename T>
void fill_recs(acs_lines* L, std::vector<LineRec<T>>& v) {
    v.resize(L->count);
    for (int i = 0; i < L->count; ++i) {
        LineRec<T>& r = v[i];
        std::memset(&r, 0, sizeof(r));
        r.off = L->off[i];
        r.n = (int)L->n[i];
        r.bc = L->bc[i];
        const double lam = L->eps[i] * L->eps[i] * L->dt[i] / (L->h[i] * L->h[i]);
        double dmp, den;
        acs_dt_max(1, L->eps[i], L->h[i], &dmp, &den);
        r.c = make_coef<T>(1, lam, L->dt[i], ACS_SCHEME_RLB_MIE_FD, L->dt[i] <= dmp * (1.0 + 1e-12));
    }
}

template <typename T>
cudaError_t launch_class(acs_lines* L, int k, int64_t nsteps, cudaStream_t st) {
    T* phi = (T*)L->phi;
    const LineRec<T>* rec = (const LineRec<T>*)L->drec;
    const int b = L->cls_begin[k], cnt = L->cls_begin[k + 1] - b;
    const int* ids = L->dids + b;
    if (k < kLineClasses - 1) {
        const dim3 grid((unsigned)((cnt + 1) / 2));  // two warps (lines) per CTA
        switch (k) {
            case 0: k_lines_warp<T, 1><<<grid, 64, 0, st>>>(phi, rec, ids, cnt, nsteps); break;
            case 1: k_lines_warp<T, 2><<<grid, 64, 0, st>>>(phi, rec, ids, cnt, nsteps); break;
            case 2: k_lines_warp<T, 4><<<grid, 64, 0, st>>>(phi, rec, ids, cnt, nsteps); break;
            case 3: k_lines_warp<T, 8><<<grid, 64, 0, st>>>(phi, rec, ids, cnt, nsteps); break;
            case 4: k_lines_warp<T, 16><<<grid, 64, 0, st>>>(phi, rec, ids, cnt, nsteps); break;
            default:  // FP32 only
                k_lines_warp<T, sizeof(T) == 4 ? 32 : 16><<<grid, 64, 0, st>>>(phi, rec, ids, cnt, nsteps);
                break;
        }
    } else {
        const size_t smem = 2 * (size_t)((L->maxn_cta + 3) / 4 * 4 + 2) * sizeof(T);
        cudaError_t e = cudaFuncSetAttribute(k_lines_cta<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_lines_cta<T><<<cnt, 256, smem, st>>>(phi, rec, ids, nsteps, L->maxn_cta);
    }
    return cudaGetLastError();
}

// The size classes run concurrently: each on its own stream, forked from and joined
// back into the bound stream with events.
template <typename T>
cudaError_t launch_lines(acs_lines* L, int64_t nsteps, cudaStream_t st) {
    if (cudaEventRecord(L->fork, st) != cudaSuccess) return cudaErrorUnknown;
    for (int k = 0; k < kLineClasses; ++k) {
        if (L->cls_begin[k + 1] <= L->cls_begin[k]) continue;
        cudaStream_t s = L->aux[k];
        if (cudaStreamWaitEvent(s, L->fork, 0) != cudaSuccess) return cudaErrorUnknown;
        cudaError_t e = launch_class<T>(L, k, nsteps, s);
        if (e != cudaSuccess) return e;
        if (cudaEventRecord(L->join[k], s) != cudaSuccess || cudaStreamWaitEvent(st, L->join[k], 0) != cudaSuccess)
            return cudaErrorUnknown;
    }
    return cudaSuccess;
}
}  // namespace

extern "C" {

ACS_API int acs_lines_create(int count, const int64_t* n, const double* eps, const double* dt, const double* h,
                             const int* bc, int dtype, acs_lines** out) {
    if (!out || count < 1 || !n || !eps || !dt || !h || !bc) return ACS_E_INVAL;
    if (dtype != ACS_F32 && dtype != ACS_F64) return ACS_E_INVAL;
    const int64_t vx = dtype == ACS_F32 ? 4 : 2;
    const int64_t maxn = dtype == ACS_F32 ? LineSmemMax<float>::value : LineSmemMax<double>::value;
    int64_t numel = 0;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || n[i] > maxn) return ACS_E_INVAL;
        if (!std::isfinite(eps[i]) || !std::isfinite(dt[i]) || !std::isfinite(h[i])) return ACS_E_INVAL;
        if (eps[i] < 0 || !(h[i] > 0) || !(dt[i] > 0) || !(dt[i] < 2) || bc[i] < 0 || bc[i] > 2) return ACS_E_INVAL;
        numel += (n[i] + vx - 1) / vx * vx;
        if (numel > (int64_t(1) << 40)) return ACS_E_INVAL;
    }
    acs_lines* L = new (std::nothrow) acs_lines();
    if (!L) return ACS_E_NOMEM;
    L->count = count;
    L->dtype = dtype;
    L->esize = dtype == ACS_F32 ? 4 : 8;
    L->numel = 0;
    L->maxn_cta = 0;
    int warn = ACS_OK;
    std::vector<std::vector<int>> cls(kLineClasses);
    for (int i = 0; i < count; ++i) {
        L->n.push_back(n[i]);
        L->eps.push_back(eps[i]);
        L->dt.push_back(dt[i]);
        L->h.push_back(h[i]);
        L->bc.push_back(bc[i]);
        L->off.push_back(L->numel);  // lines start on 16-byte boundaries
        L->numel += (n[i] + vx - 1) / vx * vx;
        const int k = line_class(n[i], dtype);
        cls[k].push_back(i);
        if (k == kLineClasses - 1) L->maxn_cta = std::max<int>(L->maxn_cta, (int)n[i]);
        double dmp, den;
        acs_dt_max(1, eps[i], h[i], &dmp, &den);
        if (dt[i] > den * (1.0 + 1e-12)) warn = ACS_WARN_ENERGY_CONDITION;
        else if (dt[i] > dmp * (1.0 + 1e-12) && warn == ACS_OK) warn = ACS_WARN_MP_CONDITION;
    }
    L->cls_begin[0] = 0;
    for (int k = 0; k < kLineClasses; ++k) {
        L->ids.insert(L->ids.end(), cls[k].begin(), cls[k].end());
        L->cls_begin[k + 1] = (int)L->ids.size();
    }
    if (dtype == ACS_F32) fill_recs<float>(L, L->recf);
    else fill_recs<double>(L, L->recd);
    L->bound = false;
    L->have_streams = false;
    L->phi = L->work = nullptr;
    L->stream = nullptr;
    *out = L;
    return warn;
}

ACS_API size_t acs_lines_numel(const acs_lines* L) { return L ? (size_t)L->numel : 0; }

ACS_API int acs_lines_offsets(const acs_lines* L, int64_t* offsets) {
    if (!L || !offsets) return ACS_E_INVAL;
    for (int i = 0; i < L->count; ++i) offsets[i] = L->off[i];
    return ACS_OK;
}

ACS_API size_t acs_lines_work_bytes(const acs_lines* L) { return L ? lines_total(L) : 0; }

ACS_API int acs_lines_bind(acs_lines* L, void* d_phi, void* d_work, size_t work_bytes, void* stream) {
    if (!L || !d_phi || !d_work || ((uintptr_t)d_phi % 16) || ((uintptr_t)d_work % kLA)) return ACS_E_INVAL;
    if (work_bytes < lines_total(L)) return ACS_E_NOMEM;
    L->bound = false;
    if (!L->have_streams) {
        if (cudaEventCreateWithFlags(&L->fork, cudaEventDisableTiming) != cudaSuccess) return ACS_E_CUDA;
        for (int k = 0; k < kLineClasses; ++k)
            if (cudaStreamCreateWithFlags(&L->aux[k], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&L->join[k], cudaEventDisableTiming) != cudaSuccess)
                return ACS_E_CUDA;
        L->have_streams = true;
    }
    L->phi = (char*)d_phi;
    L->work = (char*)d_work;
    L->stream = (cudaStream_t)stream;
    L->drec = L->work;
    L->dids = (int*)(L->work + off_ids(L));
    L->partials = (RedPartial*)(L->work + off_part(L));
    L->results = (double*)(L->work + off_res(L));
    const void* host = L->dtype == ACS_F32 ? (const void*)L->recf.data() : (const void*)L->recd.data();
    const size_t rb = (size_t)L->count * (L->dtype == ACS_F32 ? sizeof(LineRec<float>) : sizeof(LineRec<double>));
    if (cudaMemcpyAsync(L->drec, host, rb, cudaMemcpyHostToDevice, L->stream) != cudaSuccess ||
        cudaMemcpyAsync(L->dids, L->ids.data(), sizeof(int) * L->ids.size(), cudaMemcpyHostToDevice, L->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(L->stream) != cudaSuccess)
        return ACS_E_CUDA;
    L->bound = true;
    return ACS_OK;
}

ACS_API int acs_lines_step(acs_lines* L, int64_t n_steps) {
    if (!L || n_steps < 0) return ACS_E_INVAL;
    if (!L->bound) return ACS_E_STATE;
    if (n_steps == 0) return ACS_OK;
    const cudaError_t e = L->dtype == ACS_F32 ? launch_lines<float>(L, n_steps, L->stream)
                                              : launch_lines<double>(L, n_steps, L->stream);
    return e == cudaSuccess ? ACS_OK : ACS_E_CUDA;
}

ACS_API int acs_lines_observe(acs_lines* L, double* h_energy, double* h_maxnorm) {
    if (!L || !h_energy || !h_maxnorm) return ACS_E_INVAL;
    if (!L->bound) return ACS_E_STATE;
    for (int i = 0; i < L->count; ++i) {
        const int64_t nn[1] = {L->n[i]};
        const Geo g = make_geo(1, nn);
        cudaError_t e;
        if (L->dtype == ACS_F32)
            e = launch_reduce<float>(1, L->bc[i], (const float*)L->phi + L->off[i], g, L->eps[i] * L->eps[i], L->h[i],
                                     L->partials, L->results + 2 * i, L->stream);
        else
            e = launch_reduce<double>(1, L->bc[i], (const double*)L->phi + L->off[i], g, L->eps[i] * L->eps[i],
                                      L->h[i], L->partials, L->results + 2 * i, L->stream);
        if (e != cudaSuccess) return ACS_E_CUDA;
    }
    std::vector<double> buf(2 * (size_t)L->count);
    if (cudaMemcpyAsync(buf.data(), L->results, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost, L->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(L->stream) != cudaSuccess)
        return ACS_E_CUDA;
    bool finite = true;
    for (int i = 0; i < L->count; ++i) {
        h_energy[i] = buf[2 * i];
        h_maxnorm[i] = buf[2 * i + 1];
        finite = finite && std::isfinite(buf[2 * i]) && std::isfinite(buf[2 * i + 1]);
    }
    return finite ? ACS_OK : ACS_E_NONFINITE;
}

ACS_API void acs_lines_destroy(acs_lines* L) {
    if (!L) return;
    if (L->bound) cudaStreamSynchronize(L->stream);
    if (L->have_streams) {
        for (int k = 0; k < kLineClasses; ++k) {
            cudaStreamSynchronize(L->aux[k]);
            cudaStreamDestroy(L->aux[k]);
            cudaEventDestroy(L->join[k]);
        }
        cudaEventDestroy(L->fork);
    }
    delete L;
}

}  // extern "C"
