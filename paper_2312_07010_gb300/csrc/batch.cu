// batch.cu -- many independent 2D problems advanced together in one persistent,
// cooperative launch per acs_batch_step() call (recorded once into a CUDA graph).
//
// Every instance is cut into 128 x 16 tiles; the tiles of all instances form one
// list, and each CTA owns a contiguous run of it (so its tiles mostly belong to one
// instance).  Per time step a CTA stages and updates its tiles exactly as the
// single-problem 2D kernel does (same ghost rules, same per-point arithmetic, same
// coefficients), then all CTAs meet at a software grid barrier before the next
// step.  Each instance is therefore bit-identical to its standalone run.
//
// The barrier spins with a one-second bound (%globaltimer); a CTA that gives up
// records ACS_E_TIMEOUT and raises an abort flag that releases every other waiter,
// so a broken launch ends in about a second instead of hanging the GPU.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "acs_host.h"
#include "tile2d.cuh"
#include "tma.cuh"

namespace acs {

template <typename T>
struct DevInst {
    int64_t off;    // first element of the instance in the packed state
    int nx, ny;     // sides (x fastest)
    int bc;
    int nty;        // tiles along y
    int tile0;      // index of its first tile in the global tile list
    int ntiles;
    Coef<T> c;
};

struct BarrierState {
    unsigned count;  // arrivals in the current phase
    unsigned gen;    // phase counter
    int abort;       // set by a waiter that gave up: everyone leaves
    int inject;      // testing aid: 1 = the last CTA skips one arrival
};

// Returns false (and the CTA must leave) if the barrier was aborted or timed out.
__device__ __forceinline__ bool grid_barrier(BarrierState* bs, unsigned nblocks, int* err, bool skip_arrival) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vgen = &bs->gen;
        volatile int* vabort = &bs->abort;
        const unsigned g = *vgen;
        __threadfence();
        if (!skip_arrival) {
            const unsigned arrived = atomicAdd(&bs->count, 1u);
            if (arrived == nblocks - 1) {
                atomicExch(&bs->count, 0u);
                __threadfence();
                atomicAdd(&bs->gen, 1u);
            }
        }
        const uint64_t t0 = global_ns();
        uint32_t i = 0;
        while (*vgen == g) {
            if (*vabort) { ok = 0; break; }
            if ((++i & 63u) == 0u && global_ns() - t0 > kWaitNs) {
                atomicExch(err, 1);
                atomicExch(&bs->abort, 1);
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    __threadfence();  // every thread: acquire side of the barrier before reading other CTAs' results
    return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ void batch_update_tile(const T* buf, T* dst, const DevInst<T>& in, int x0, int y0,
                                                  const Coef<T>& c) {
    if (c.solve == kSolveSeries) update_tile<T, kSolveSeries>(buf, dst, in.ny, in.nx, x0, y0, c);
    else if (c.solve == kSolveFex) update_tile<T, kSolveFex>(buf, dst, in.ny, in.nx, x0, y0, c);
    else update_tile<T, kSolveNewton>(buf, dst, in.ny, in.nx, x0, y0, c);
}

template <typename T>
__global__ void __launch_bounds__(256) k_batch2d(T* A, T* B, const DevInst<T>* __restrict__ inst, int count,
                                                 int total_tiles, int nsteps, BarrierState* bs, int* err) {
    using TT = Tile2<T>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* const base = reinterpret_cast<T*>(sm_raw);
    const int per = (total_tiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per;
    const int t1 = min(t0 + per, total_tiles);
    // instance of the first tile (binary search over tile0)
    int i0 = 0;
    if (t0 < t1) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst[mid].tile0 <= t0) lo = mid; else hi = mid - 1;
        }
        i0 = lo;
    }
    const bool injector = bs->inject != 0 && blockIdx.x == gridDim.x - 1;
    for (int step = 0; step < nsteps; ++step) {
        const T* src = (step & 1) ? B : A;
        T* dst = (step & 1) ? A : B;
        if (t0 < t1) {
            int ii = i0;
            auto locate = [&](int t, int& which, int& x0, int& y0) {
                while (ii + 1 < count && inst[ii + 1].tile0 <= t) ++ii;
                which = ii;
                const int lt = t - inst[ii].tile0;
                x0 = (lt / inst[ii].nty) * TT::TX;
                y0 = (lt % inst[ii].nty) * TT::TY;
            };
            int w, x0, y0;
            locate(t0, w, x0, y0);
            stage_tile<T>(base, src + inst[w].off, inst[w].ny, inst[w].nx, inst[w].bc, x0, y0);
            cp_async_commit();
            for (int t = t0; t < t1; ++t) {
                const int cur = (t - t0) & 1;
                const int cw = w, cx0 = x0, cy0 = y0;
                if (t + 1 < t1) {
                    locate(t + 1, w, x0, y0);
                    stage_tile<T>(base + (cur ^ 1) * TT::N, src + inst[w].off, inst[w].ny, inst[w].nx, inst[w].bc,
                                  x0, y0);
                }
                cp_async_commit();
                cp_async_wait<1>();
                __syncthreads();
                const Coef<T> c = inst[cw].c;
                batch_update_tile<T>(base + cur * TT::N, dst + inst[cw].off, inst[cw], cx0, cy0, c);
                __syncthreads();
            }
        }
        if (step + 1 < nsteps) {
            if (!grid_barrier(bs, gridDim.x, err, injector && step == 0)) return;
        }
    }
}

}  // namespace acs

using namespace acs;

struct acs_batch {
    int count, dtype;
    size_t esize;
    std::vector<int64_t> n, off;
    std::vector<double> eps, dt, h;
    std::vector<int> bc;
    std::vector<DevInst<float>> inf;
    std::vector<DevInst<double>> ind;
    int total_tiles;
    int64_t numel;
    // bound
    bool bound;
    char* phi;
    char* work;
    cudaStream_t stream, cap;
    char* other;
    void* dinst;
    BarrierState* bs;
    int* err;
    RedPartial* partials;
    double* results;
    int grid;
    std::vector<std::pair<int64_t, cudaGraphExec_t>> graphs;
};

namespace {
constexpr size_t kA = 256;
size_t al(size_t x) { return (x + kA - 1) / kA * kA; }
size_t inst_bytes(const acs_batch* b) {
    return al((size_t)b->count * (b->dtype == ACS_F32 ? sizeof(DevInst<float>) : sizeof(DevInst<double>)));
}
size_t off_inst(const acs_batch* b) { return al((size_t)b->numel * b->esize); }
size_t off_bar(const acs_batch* b) { return off_inst(b) + inst_bytes(b); }
size_t off_part(const acs_batch* b) { return off_bar(b) + kA; }
size_t off_res(const acs_batch* b) { return off_part(b) + al(sizeof(RedPartial) * kMaxRedBlocks); }
size_t total_bytes(const acs_batch* b) { return off_res(b) + al(sizeof(double) * 2 * (size_t)b->count); }

void drop_graphs(acs_batch* b) {
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
}

template <typename T>
cudaError_t launch_batch(acs_batch* b, int64_t nsteps, cudaStream_t st) {
    using TT = Tile2<T>;
    auto kern = k_batch2d<T>;
    const size_t smem = 2 * TT::N * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    T* A = (T*)b->phi;
    T* B = (T*)b->other;
    const DevInst<T>* in = (const DevInst<T>*)b->dinst;
    int count = b->count, tiles = b->total_tiles, ns = (int)nsteps;
    void* args[] = {&A, &B, &in, &count, &tiles, &ns, &b->bs, &b->err};
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3(TT::THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)kern, args);
}

// One launch advances nsteps; the packed state starts in phi and, after an even
// number of steps, ends there (an odd count ends with one device copy back).
cudaError_t enqueue_batch(acs_batch* b, int64_t nsteps, cudaStream_t st) {
    const int64_t chunk_max = 1 << 20;
    for (int64_t done = 0; done < nsteps;) {
        const int64_t k = std::min(chunk_max, nsteps - done);
        cudaError_t e = b->dtype == ACS_F32 ? launch_batch<float>(b, k, st) : launch_batch<double>(b, k, st);
        if (e != cudaSuccess) return e;
        if (k & 1) {
            e = cudaMemcpyAsync(b->phi, b->other, (size_t)b->numel * b->esize, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
        done += k;
    }
    return cudaSuccess;
}

template <typename T>
void fill_inst(acs_batch* b, std::vector<DevInst<T>>& v) {
    using TT = Tile2<T>;
    v.resize(b->count);
    int tile0 = 0;
    for (int i = 0; i < b->count; ++i) {
        DevInst<T>& d = v[i];
        std::memset(&d, 0, sizeof(d));
        d.off = b->off[i];
        d.nx = (int)b->n[i];
        d.ny = (int)b->n[i];
        d.bc = b->bc[i];
        const int ntx = (d.nx + TT::TX - 1) / TT::TX;
        d.nty = (d.ny + TT::TY - 1) / TT::TY;
        d.ntiles = ntx * d.nty;
        d.tile0 = tile0;
        tile0 += d.ntiles;
        const double lam = b->eps[i] * b->eps[i] * b->dt[i] / (b->h[i] * b->h[i]);
        double dmp, den;
        acs_dt_max(2, b->eps[i], b->h[i], &dmp, &den);
        const bool mp_ok = b->dt[i] <= dmp * (1.0 + 1e-12);
        d.c = make_coef<T>(2, lam, b->dt[i], ACS_SCHEME_RLB_MIE_FD, mp_ok);
    }
    b->total_tiles = tile0;
}

}  // namespace

extern "C" {

ACS_API int acs_batch_create(int count, const int64_t* n, const double* eps, const double* dt, const double* h,
                             const int* bc, int dtype, acs_batch** out) {
    if (!out || count < 1 || !n || !eps || !dt || !h || !bc) return ACS_E_INVAL;
    if (dtype != ACS_F32 && dtype != ACS_F64) return ACS_E_INVAL;
    int64_t numel = 0, tiles = 0;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || n[i] > (1 << 20)) return ACS_E_INVAL;
        if (!std::isfinite(eps[i]) || !std::isfinite(dt[i]) || !std::isfinite(h[i])) return ACS_E_INVAL;
        if (eps[i] < 0 || !(h[i] > 0) || !(dt[i] > 0) || !(dt[i] < 2) || bc[i] < 0 || bc[i] > 2) return ACS_E_INVAL;
        numel += n[i] * n[i];
        tiles += ((n[i] + 63) / 64) * ((n[i] + 15) / 16);  // the FP64 tile (64 x 16) bounds both
        if (numel > (int64_t(1) << 40) || tiles > 0x7fffffff) return ACS_E_INVAL;
    }
    acs_batch* b = new (std::nothrow) acs_batch();
    if (!b) return ACS_E_NOMEM;
    b->count = count;
    b->dtype = dtype;
    b->esize = dtype == ACS_F32 ? 4 : 8;
    b->numel = 0;
    int warn = ACS_OK;
    for (int i = 0; i < count; ++i) {
        b->n.push_back(n[i]);
        b->eps.push_back(eps[i]);
        b->dt.push_back(dt[i]);
        b->h.push_back(h[i]);
        b->bc.push_back(bc[i]);
        b->off.push_back(b->numel);
        // instances start on 16-byte boundaries
        b->numel += (n[i] * n[i] + 3) / 4 * 4;
        double dmp, den;
        acs_dt_max(2, eps[i], h[i], &dmp, &den);
        if (dt[i] > den * (1.0 + 1e-12)) warn = ACS_WARN_ENERGY_CONDITION;
        else if (dt[i] > dmp * (1.0 + 1e-12) && warn == ACS_OK) warn = ACS_WARN_MP_CONDITION;
    }
    if (dtype == ACS_F32) fill_inst<float>(b, b->inf);
    else fill_inst<double>(b, b->ind);
    b->bound = false;
    b->phi = b->work = b->other = nullptr;
    b->stream = b->cap = nullptr;
    b->grid = 0;
    *out = b;
    return warn;
}

ACS_API size_t acs_batch_numel(const acs_batch* b) { return b ? (size_t)b->numel : 0; }

ACS_API int acs_batch_offsets(const acs_batch* b, int64_t* offsets) {
    if (!b || !offsets) return ACS_E_INVAL;
    for (int i = 0; i < b->count; ++i) offsets[i] = b->off[i];
    return ACS_OK;
}

ACS_API size_t acs_batch_work_bytes(const acs_batch* b) { return b ? total_bytes(b) : 0; }

ACS_API int acs_batch_bind(acs_batch* b, void* d_phi, void* d_work, size_t work_bytes, void* stream) {
    if (!b || !d_phi || !d_work || ((uintptr_t)d_phi % 16) || ((uintptr_t)d_work % kA)) return ACS_E_INVAL;
    if (work_bytes < total_bytes(b)) return ACS_E_NOMEM;
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return ACS_E_CUDA;
    drop_graphs(b);
    b->phi = (char*)d_phi;
    b->work = (char*)d_work;
    b->other = b->work;
    b->stream = (cudaStream_t)stream;
    b->dinst = b->work + off_inst(b);
    b->bs = (BarrierState*)(b->work + off_bar(b));
    b->err = (int*)((char*)b->bs + 64);
    b->partials = (RedPartial*)(b->work + off_part(b));
    b->results = (double*)(b->work + off_res(b));
    const void* host = b->dtype == ACS_F32 ? (const void*)b->inf.data() : (const void*)b->ind.data();
    const size_t ib = (size_t)b->count * (b->dtype == ACS_F32 ? sizeof(DevInst<float>) : sizeof(DevInst<double>));
    if (cudaMemcpyAsync(b->dinst, host, ib, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) return ACS_E_CUDA;
    if (cudaMemsetAsync(b->bs, 0, kA, b->stream) != cudaSuccess) return ACS_E_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ACS_E_CUDA;
    // persistent grid: every SM's resident CTAs, never more than the tiles
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    if (b->dtype == ACS_F32) {
        const size_t smem = 2 * Tile2<float>::N * sizeof(float);
        cudaFuncSetAttribute(k_batch2d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch2d<float>, Tile2<float>::THREADS, smem);
    } else {
        const size_t smem = 2 * Tile2<double>::N * sizeof(double);
        cudaFuncSetAttribute(k_batch2d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch2d<double>, Tile2<double>::THREADS, smem);
    }
    if (e != cudaSuccess || per_sm < 1) return ACS_E_CUDA;
    b->grid = (int)std::min<int64_t>((int64_t)sms * per_sm, b->total_tiles);
    b->bound = true;
    return ACS_OK;
}

ACS_API int acs_batch_step(acs_batch* b, int64_t n_steps) {
    if (!b || n_steps < 0) return ACS_E_INVAL;
    if (!b->bound) return ACS_E_STATE;
    if (n_steps == 0) return ACS_OK;
    cudaGraphExec_t exec = nullptr;
    for (auto& g : b->graphs)
        if (g.first == n_steps) exec = g.second;
    if (!exec) {
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ACS_E_CUDA;
        cudaError_t e1 = enqueue_batch(b, n_steps, b->cap);
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
        cudaError_t e3 = cudaErrorUnknown;
        if (e1 == cudaSuccess && e2 == cudaSuccess) e3 = cudaGraphInstantiate(&exec, graph, 0);
        if (e2 == cudaSuccess) cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) {
            // this driver cannot record the cooperative launch: launch it directly
            cudaGetLastError();
            return enqueue_batch(b, n_steps, b->stream) == cudaSuccess ? ACS_OK : ACS_E_CUDA;
        }
        if (b->graphs.size() >= 8) {
            cudaGraphExecDestroy(b->graphs.front().second);
            b->graphs.erase(b->graphs.begin());
        }
        b->graphs.push_back({n_steps, exec});
    }
    return cudaGraphLaunch(exec, b->stream) == cudaSuccess ? ACS_OK : ACS_E_CUDA;
}

ACS_API int acs_batch_observe(acs_batch* b, double* h_energy, double* h_maxnorm) {
    if (!b || !h_energy || !h_maxnorm) return ACS_E_INVAL;
    if (!b->bound) return ACS_E_STATE;
    for (int i = 0; i < b->count; ++i) {
        const int64_t nn[2] = {b->n[i], b->n[i]};
        const Geo g = make_geo(2, nn);
        cudaError_t e;
        if (b->dtype == ACS_F32)
            e = launch_reduce<float>(2, b->bc[i], (const float*)b->phi + b->off[i], g, b->eps[i] * b->eps[i], b->h[i],
                                     b->partials, b->results + 2 * i, b->stream);
        else
            e = launch_reduce<double>(2, b->bc[i], (const double*)b->phi + b->off[i], g, b->eps[i] * b->eps[i],
                                      b->h[i], b->partials, b->results + 2 * i, b->stream);
        if (e != cudaSuccess) return ACS_E_CUDA;
    }
    std::vector<double> buf(2 * (size_t)b->count);
    if (cudaMemcpyAsync(buf.data(), b->results, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost, b->stream) !=
        cudaSuccess)
        return ACS_E_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ACS_E_CUDA;
    int flag = 0;
    if (cudaMemcpy(&flag, b->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_E_CUDA;
    if (flag) {
        cudaMemset(b->bs, 0, kA);
        return ACS_E_TIMEOUT;
    }
    bool finite = true;
    for (int i = 0; i < b->count; ++i) {
        h_energy[i] = buf[2 * i];
        h_maxnorm[i] = buf[2 * i + 1];
        finite = finite && std::isfinite(buf[2 * i]) && std::isfinite(buf[2 * i + 1]);
    }
    return finite ? ACS_OK : ACS_E_NONFINITE;
}

ACS_API int acs_batch_inject_fault(acs_batch* b, int mode) {
    if (!b || mode < 0 || mode > 1) return ACS_E_INVAL;
    if (!b->bound) return ACS_E_STATE;
    const int v = mode;
    if (cudaMemcpyAsync(&b->bs->inject, &v, sizeof(int), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return ACS_E_CUDA;
    return cudaStreamSynchronize(b->stream) == cudaSuccess ? ACS_OK : ACS_E_CUDA;
}

ACS_API void acs_batch_destroy(acs_batch* b) {
    if (!b) return;
    if (b->bound) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // extern "C"
