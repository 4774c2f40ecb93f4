// batch_tb.cu -- the batched form with temporal blocking: many independent 2D FP32
// problems advanced K steps (Eq. IE-FD, Remark 1) per pass through HBM in one
// persistent, cooperative launch.
//
// Work: every instance is cut into units of one column strip (the window of the 2D
// temporal kernel, 32 lanes x 4 values wide, its inner 120 columns written) by a
// chunk of rows.  Warps draw units from one ticket counter in pass-major order and
// stream each through the register pipeline of the single-problem temporal kernel
// (the same skewed schedule of the K levels, the same virtual extension for the
// ghost rules of Eq. Ddeltax, the same per-point arithmetic), so after every pass an
// instance holds the bits of K single steps.
//
// There is no grid barrier between passes.  Instance i keeps a counter of its
// completed units; a unit of pass p waits until the counter reaches p times the
// instance's unit count (all of its pass p - 1 done: their reads of the buffer this
// pass writes and their writes of the buffer it reads).  Passes thus overlap across
// instances, and the small instances, listed last, fill the end of each pass.  Tickets
// are drawn in order and every CTA is resident (cooperative launch), so the unit with
// the lowest unfinished ticket never waits and every wait ends; each is bounded all
// the same by about one second of %globaltimer, after which the warp records
// ACS_E_TIMEOUT and raises the abort flag that sends every other warp home.
//
// The state is read with ld.global.cg (L2, not the SM's L1): a buffer is written by
// other SMs between the passes of one launch.
#include <type_traits>

#include "batch.cuh"
#include "f32x2.cuh"
#include "tb2d.cuh"
#include "tma.cuh"

namespace acs {

namespace {

// vmap() with the boundary rule known at run time, for coordinates a few periods
// outside [0, n) at most: periodic folds by n, Neumann reflects about -1/2 and
// n - 1/2 (the same index as the period-2n fold), Dirichlet gives -1 (the value +0).
// Compact loops, not divisions: the call sites sit in the unit's streaming loop.
__device__ __forceinline__ int vmap_rt(int v, int n, int bc) {
    if (v >= 0 && v < n) return v;
    if (bc == ACS_BC_DIRICHLET) return -1;
    if (bc == ACS_BC_PERIODIC) {
        while (v < 0) v += n;
        while (v >= n) v -= n;
        return v;
    }
    while (v < 0 || v >= n) v = v < 0 ? -1 - v : 2 * n - 1 - v;
    return v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *p >= need; false if the abort flag was raised or the bound ran out.
__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned need, const int* abort) {
    if (ld_acquire(p) >= need) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        __nanosleep(64);
        if (ld_acquire(p) >= need) return true;
        if (*(volatile const int*)abort) return false;
        if ((i & 15u) == 15u && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

// One unit: rows [ya, yb) of the strip's output columns advanced K steps, src -> dst
// (both already offset to the instance).  The schedule is the single-problem temporal
// kernel's, with every level run from the first iteration (rows computed before a
// level has exact input lie outside the rows the next levels take exactly, so they
// are never stored).  The series root under Theorem 2 runs the loop unrolled three
// times (the ring of the last three rows of every level in fixed registers); the
// other roots run it once with the rings rotated by register moves, which keeps
// their much larger code small enough for the instruction caches.
template <int K, int SOLVE>
__device__ __forceinline__ void tb_unit(const float* __restrict__ src, float* __restrict__ dst, int n, int ld, int bc,
                                        const Coef<float>& c, int strip, int ya, int yb, int lane) {
    using TB = Tb2<float, K>;
    constexpr int VX = TB::VX, HG = TB::HG, WW = TB::WW, OW = TB::OW;
    constexpr bool ROT = SOLVE != kSolveSeriesUnit;
    static_assert(VX == 4 && OW == kBatchTbCols, "unit geometry");
    const int wx = strip * OW - HG * VX;  // first column of the window
    const int cx = wx + lane * VX;        // first column of this lane
    const int NI = (yb - ya) + 2 * K;     // rows streamed: the chunk plus K each side
    const bool wlane = lane >= HG && lane < 32 - HG && cx < n;
    const int nvalid = min(VX, n - cx);   // values of the lane's vector inside the row (ragged last vector)
    const bool colsin = wx >= 0 && wx + WW <= n;
    // Dirichlet: nodes outside the grid are reset to +0 after every level (a
    // warp-uniform branch, taken only by units touching the boundary)
    const bool edge = bc == ACS_BC_DIRICHLET && (!colsin || ya - K < 0 || yb + K > n);
    const PackedCoef pc = packed_coef(c);
    // stored columns of the lane's values (-1: +0), for windows that leave the grid
    int xu[VX];
    bool colin[VX];
#pragma unroll
    for (int v = 0; v < VX; ++v) {
        xu[v] = vmap_rt(cx + v, n, bc);
        colin[v] = cx + v >= 0 && cx + v < n;
    }
    // row i of the stream is virtual row ya - K + i
    auto load_row = [&](int i, float (&o)[VX]) {
        const int u = vmap_rt(ya - K + i, n, bc);
        if (u < 0) {
#pragma unroll
            for (int v = 0; v < VX; ++v) o[v] = 0.0f;
            return;
        }
        const float* rowp = src + (int64_t)u * ld;
        if (colsin) {
            const float4 q = __ldcg(reinterpret_cast<const float4*>(rowp + cx));
            o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
        } else {
#pragma unroll
            for (int v = 0; v < VX; ++v) o[v] = xu[v] < 0 ? 0.0f : __ldcg(rowp + xu[v]);
        }
    };

    float pre[3][VX];  // stream rows i, i + 1, i + 2 in flight
    float w[K][3][VX]; // level s: the rows it computed in the last three iterations
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int v = 0; v < VX; ++v) w[s][k][v] = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) load_row(k, pre[k]);

    // Iteration i: level 0 takes stream row i, level s >= 1 computes stream row i - 2 s
    // from its predecessor's rows of iterations i - 3, i - 2, i - 1, held in ring slots
    // PH, PH + 1, PH + 2 (mod 3); the new rows replace slot PH.  With ROT, PH is 0 and
    // the rings shift by one slot after every iteration.
    auto iter = [&](auto phc, int i) {
        constexpr int PH = decltype(phc)::value;
        float out[K * VX];
        f2 xi[2 * K];
#pragma unroll
        for (int s = K; s >= 1; --s) {
            const float(&m)[VX] = w[s - 1][PH];
            const float(&z)[VX] = w[s - 1][(PH + 1) % 3];
            const float(&p)[VX] = w[s - 1][(PH + 2) % 3];
            const float left = __shfl_up_sync(0xffffffffu, z[VX - 1], 1);
            const float right = __shfl_down_sync(0xffffffffu, z[0], 1);
            f2 x2p[2];
            predict4_2d(m, z, p, left, right, pc, x2p);
            xi[2 * (s - 1)] = x2p[0];
            xi[2 * (s - 1) + 1] = x2p[1];
        }
        roots2<SOLVE, 2 * K>(xi, out, c, pc);
#pragma unroll
        for (int s = K; s >= 1; --s) {
            const int q = ya - K + i - 2 * s;  // grid row of level s's new row
            float* o = &out[(s - 1) * VX];
            if (edge) {
                const bool rowin = q >= 0 && q < n;
#pragma unroll
                for (int v = 0; v < VX; ++v) o[v] = (rowin && colin[v]) ? o[v] : 0.0f;
            }
            if (s == K && wlane && q >= ya && q < yb) {
                float* op = dst + (int64_t)q * ld + cx;
                if (nvalid == VX) {
                    Vec<float>::put(op, o);
                } else {
#pragma unroll
                    for (int v = 0; v < VX; ++v)
                        if (v < nvalid) op[v] = o[v];
                }
            }
        }
        if constexpr (ROT) {
#pragma unroll
            for (int s = 0; s < K; ++s)
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    w[s][0][v] = w[s][1][v];
                    w[s][1][v] = w[s][2][v];
                    w[s][2][v] = s == 0 ? pre[0][v] : out[(s - 1) * VX + v];
                }
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                pre[0][v] = pre[1][v];
                pre[1][v] = pre[2][v];
            }
            if (i + 3 < NI) load_row(i + 3, pre[2]);
        } else {
#pragma unroll
            for (int s = 1; s < K; ++s)
#pragma unroll
                for (int v = 0; v < VX; ++v) w[s][PH][v] = out[(s - 1) * VX + v];
#pragma unroll
            for (int v = 0; v < VX; ++v) w[0][PH][v] = pre[PH][v];
            if (i + 3 < NI) load_row(i + 3, pre[PH]);
        }
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    const int NL = NI + K;  // the last stored row is computed in iteration NL - 1
    if constexpr (ROT) {
        for (int i = 0; i < NL; ++i) iter(I0(), i);
    } else {
        for (int i0 = 0; i0 < NL; i0 += 3) {
            iter(I0(), i0);
            iter(I1(), i0 + 1);
            iter(I2(), i0 + 2);
        }
    }
}

// 4 CTAs of 4 warps per SM at every depth: the per-unit dispatch holds the Newton
// root's copy of the loop too, which does not fit the tighter budgets of the
// single-problem kernel's depths 2 and 3.
constexpr int kBatchTbMinBlocks = 4;

template <int K>
__global__ void __launch_bounds__(kTbWarps * 32, kBatchTbMinBlocks)
    k_batch2d_tb(float* A, float* B, const DevInst<float>* __restrict__ inst, const TbUnit* __restrict__ units,
                 int nunits, int npasses, int fixed, BarrierState* bs, unsigned* done, int* err) {
    const int lane = threadIdx.x & 31;
    // testing aid: the completion of ticket 0 is not counted, so the next pass of its
    // instance waits until the bound runs out
    const bool inject = bs->inject != 0;
    const unsigned total = (unsigned)npasses * (unsigned)nunits;
    for (;;) {
        unsigned t = 0;
        int stop = 0;
        if (lane == 0) {
            stop = *(volatile const int*)&bs->abort;
            if (!stop) t = atomicAdd(&bs->ctr[0], 1u);
        }
        stop = __shfl_sync(0xffffffffu, stop, 0);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (stop || t >= total) break;
        const int pass = (int)(t / (unsigned)nunits);
        const TbUnit u = units[t - (unsigned)pass * (unsigned)nunits];
        const int64_t off = inst[u.inst].off;
        const int n = inst[u.inst].n, ld = inst[u.inst].ld, bc = inst[u.inst].bc;
        const unsigned per = (unsigned)inst[u.inst].tbunits;
        const bool odd = (pass & 1) && !fixed;
        const float* src = (odd ? B : A) + off;
        float* dst = (odd ? A : B) + off;
        // all units of the instance's previous pass have completed
        int ok = 1;
        if (lane == 0 && pass > 0) ok = wait_count(&done[u.inst], (unsigned)pass * per, &bs->abort);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0) {
                atomicExch(err, 1);
                atomicExch(&bs->abort, 1);
            }
            break;
        }
        __threadfence();  // every lane: acquire side of the wait before reading the state
        const Coef<float> c = inst[u.inst].c;
        // the instance's root (Remark 1): the series under Theorem 2's condition, the
        // series with its run-time tests, or the seeded Newton iteration
        if (c.solve == kSolveSeries && c.clamp)
            tb_unit<K, kSolveSeriesUnit>(src, dst, n, ld, bc, c, u.strip, u.ya, u.yb, lane);
        else if (c.solve == kSolveSeries)
            tb_unit<K, kSolveSeries>(src, dst, n, ld, bc, c, u.strip, u.ya, u.yb, lane);
        else
            tb_unit<K, kSolveNewton>(src, dst, n, ld, bc, c, u.strip, u.ya, u.yb, lane);
        __threadfence();  // every lane: its stores before the completion count
        __syncwarp();
        if (lane == 0 && !(inject && t == 0u)) atomicAdd(&done[u.inst], 1u);
    }
}

template <int K>
cudaError_t launch_k(float* A, float* B, const DevInst<float>* inst, const TbUnit* units, int nunits, int npasses,
                     int fixed, BarrierState* bs, unsigned* done, int* err, int grid, cudaStream_t st) {
    auto kern = k_batch2d_tb<K>;
    void* args[] = {&A, &B, &inst, &units, &nunits, &npasses, &fixed, &bs, &done, &err};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kTbWarps * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)kern, args);
}

template <int K>
int per_sm_k() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch2d_tb<K>, kTbWarps * 32, 0) != cudaSuccess)
        return 0;
    return per_sm;
}

}  // namespace

int batch_tb_threads() { return kTbWarps * 32; }

int batch_tb_per_sm(int K) {
    switch (K) {
        case 2: return per_sm_k<2>();
        case 3: return per_sm_k<3>();
        case 4: return per_sm_k<4>();
        default: return 0;
    }
}

cudaError_t launch_batch_tb(int K, float* A, float* B, const DevInst<float>* inst, const TbUnit* units, int nunits,
                            int npasses, int fixed, BarrierState* bs, unsigned* done, int* err, int grid,
                            cudaStream_t st) {
    if (nunits < 1 || npasses < 1 || grid < 1) return cudaErrorInvalidValue;
    switch (K) {
        case 2: return launch_k<2>(A, B, inst, units, nunits, npasses, fixed, bs, done, err, grid, st);
        case 3: return launch_k<3>(A, B, inst, units, nunits, npasses, fixed, bs, done, err, grid, st);
        case 4: return launch_k<4>(A, B, inst, units, nunits, npasses, fixed, bs, done, err, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace acs
