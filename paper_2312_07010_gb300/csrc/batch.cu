// batch.cu -- many independent 2D problems advanced together in one persistent,
// cooperative launch per acs_batch_step() call (recorded once into a CUDA graph).
//
// Layout: the states are packed one after the other; the rows of instance i are
// ld_i = n_i rounded up to a 16-byte multiple apart (acs_batch_row_strides), so
// every instance has its own TMA tensor maps, one per ping-pong buffer.
//
// Work: every instance is cut into blocks of TX columns x TY rows (FP32 128 x 32,
// FP64 64 x 16), listed instance after instance, down each column strip.  Per step,
// CTAs draw blocks from a ticket counter and stream them through one ring of
// TMA-loaded boxes, each block as the single-problem 2D kernel computes it (same halo
// boxes, same ghost rules, same per-point arithmetic and coefficients), so each
// instance is bit-identical to its standalone run.  The ring runs on across block and
// instance boundaries; when the tickets run out a CTA meets the others at a software
// grid barrier before the next step's loads are issued.
//
// The barrier spins with a one-second bound (%globaltimer); a CTA that gives up
// records ACS_E_TIMEOUT and raises an abort flag that releases every other waiter,
// so a broken launch ends in about a second instead of hanging the GPU.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <new>
#include <string>
#include <vector>

#include "acs_host.h"
#include "batch.cuh"
#include "f32x2.cuh"
#include "stream_tile.cuh"
#include "tma.cuh"

namespace acs {

// One block of one instance.  colx / rowy: where a periodic instance's wrapped
// column / row for this block is fetched from when the main box does not hold it
// (the TMA x coordinate of a VX-wide column box, the y of a one-row box), else -1.
struct BlockRef {
    int inst, x0, y0, colx, rowy, pad0, pad1, pad2;
};

// Tile geometry of the batched kernel.  FP32: 4 rows per thread (128 x 32 blocks), 3
// ring slots, 3 CTAs per SM; FP64: 2 rows (64 x 16 blocks), 4 slots, 2 CTAs per SM
// (4 rows spill there).  Blocks are handed out kch at a time (1 unless the batched
// autotuner chose more).  Each instance has one tensor-map set: main box, column box,
// row box, for each of the two state buffers.  Measured on the 256-instance workload
// (FP32, GLUPS): 2 rows / 4 slots / chunks of 4: 592; 4 rows / 3 slots / chunks of 2:
// 651; chunks of 1: 673; 4 rows / 4 slots: 615; 3 rows: 644.
template <typename T>
using BatchTile = Tile3<T, sizeof(T) == 4 ? 4 : 2, sizeof(T) == 4 ? 3 : 4>;
constexpr int kMapsPerInst = 6;
constexpr int kMaxBatchChunk = 16;  // largest blocks-per-ticket setting
constexpr int kTuneSteps = 16;      // steps per timed launch of acs_batch_autotune (about as many in passes)
constexpr int kFenceWords = 64;  // instances whose maps a CTA remembers as acquired

template <typename T>
struct BatchSmem {
    using TT = BatchTile<T>;
    static constexpr uint32_t COL_BYTES = TT::VX * TT::BH * sizeof(T);  // VX x BH column box
    static constexpr uint32_t ROW_BYTES = TT::BW * sizeof(T);           // BW x 1 row box
    static constexpr uint32_t COL_STRIDE = (COL_BYTES + 127u) / 128u * 128u;
    static constexpr uint32_t ROW_STRIDE = (ROW_BYTES + 127u) / 128u * 128u;
    static constexpr uint32_t OFF_RING = TT::BAR_BYTES;
    static constexpr uint32_t OFF_COL = OFF_RING + TT::S * TT::SLOT_STRIDE;
    static constexpr uint32_t OFF_ROW = OFF_COL + TT::S * COL_STRIDE;
    static constexpr uint32_t INST_BYTES = sizeof(DevInst<T>);
    static constexpr uint32_t INST_STRIDE = (INST_BYTES + 127u) / 128u * 128u;
    static constexpr uint32_t OFF_INST = OFF_ROW + TT::S * ROW_STRIDE;
    static constexpr uint32_t OFF_META = OFF_INST + TT::S * INST_STRIDE;
    static constexpr size_t BYTES = 128 + OFF_META + TT::S * sizeof(BlockRef);
};

// Returns false (and the CTA must leave) if the barrier was aborted or timed out.
// The last arrival after step `step` zeroes the ticket counter of step + 2 (last used
// at step - 2, two barriers ago).  Thread (0, 0), which also issues the TMA loads,
// orders the other CTAs' stores before its next loads through the async proxy.
__device__ __forceinline__ bool grid_barrier(BarrierState* bs, unsigned nblocks, int step, int* err,
                                             bool skip_arrival) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int ok = 1;
        volatile unsigned* vgen = &bs->gen;
        volatile int* vabort = &bs->abort;
        const unsigned g = *vgen;
        __threadfence();
        if (!skip_arrival) {
            const unsigned arrived = atomicAdd(&bs->count, 1u);
            if (arrived == nblocks - 1) {
                atomicExch(&bs->count, 0u);
                atomicExch(&bs->ctr[(step + 2) & 3], 0u);
                __threadfence();
                atomicAdd(&bs->gen, 1u);
            }
        }
        const uint64_t t0 = global_ns();
        uint32_t i = 0;
        while (*vgen == g) {
            if (*vabort) { ok = 0; break; }
            // about one second of %globaltimer, or kSpinLimit polls if the timer stalls
            if (((++i & 63u) == 0u && global_ns() - t0 > kWaitNs) || i >= kSpinLimit) {
                atomicExch(err, 1);
                atomicExch(&bs->abort, 1);
                ok = 0;
                break;
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        s_ok = ok;
    }
    __syncthreads();
    __threadfence();  // every thread: acquire side of the barrier before reading other CTAs' results
    return s_ok != 0;
}

// One block of one instance from its TMA box `cur` (rows y0 - 1 .. y0 + 16, columns
// x0 - VX .. x0 + TX + VX - 1, zero outside the instance): the body of the
// single-problem 2D kernel with the boundary taken at run time.  EDGE blocks touch a
// periodic or Neumann boundary and fix the ghost values there: the first and last
// rows, the first column, and the last column n - 1 (which need not end a vector:
// rows are padded).  Periodic wrap values come from the main box when it holds them,
// else from the column box `colb` (VX x BH) or the row box `rowb` (BW x 1) loaded
// with the block, so no block reads global memory.
template <typename T, int SOLVE, bool EDGE>
__device__ __forceinline__ void batch_block(const T* cur, const T* colb, const T* rowb, T* dst, int n, int bc,
                                            int64_t sy, const Coef<T>& c, const BlockRef& br) {
    using TT = BatchTile<T>;
    constexpr int VX = TT::VX, TX = TT::TX, TY = TT::TY, BW = TT::BW, RPT = TT::RPT, NP = RPT * VX;
    const int x0 = br.x0, y0 = br.y0;
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int xl = lx * VX, gx = x0 + xl, r0 = RPT * ly, gy0 = y0 + r0;
    const bool neu = bc == ACS_BC_NEUMANN;
    const int lastv = n - 1 - gx;  // vector lane of column n - 1 (if in 0 .. VX - 1)
    constexpr bool PACKED = std::is_same<T, float>::value && !EDGE;
    T cz[RPT][VX], below[VX], above[VX], xi[NP];
    f2 xip[2 * RPT];
    PackedCoef pc;
    if constexpr (PACKED) pc = packed_coef(c);
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) Vec<T>::get(cur + (r0 + rr + 1) * BW + VX + xl, cz[rr]);
    Vec<T>::get(cur + r0 * BW + VX + xl, below);
    Vec<T>::get(cur + (r0 + RPT + 1) * BW + VX + xl, above);
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
        const int gyr = gy0 + rr;
        const int br_row = r0 + rr + 1;  // box row of gyr
        T ym[VX], yp[VX];
#pragma unroll
        for (int v = 0; v < VX; ++v) {
            ym[v] = rr == 0 ? below[v] : cz[rr - 1][v];
            yp[v] = rr == RPT - 1 ? above[v] : cz[rr + 1][v];
        }
        T left = __shfl_up_sync(0xffffffffu, cz[rr][VX - 1], 1);
        T right = __shfl_down_sync(0xffffffffu, cz[rr][0], 1);
        if (lx == 0) left = cur[br_row * BW + VX - 1];
        if (lx == 31) right = cur[br_row * BW + VX + TX];
        T wrapx = T(0);  // periodic: right neighbour of column n - 1
        if (EDGE && gyr < n) {
            if (gyr == 0) {
                if (neu) {
#pragma unroll
                    for (int v = 0; v < VX; ++v) ym[v] = cz[rr][v];
                } else {
                    // row n - 1: box row n when it is in the box (n <= TY + 1), else the row box
                    Vec<T>::get(br.rowy >= 0 ? rowb + VX + xl : cur + n * BW + VX + xl, ym);
                }
            }
            if (gyr == n - 1) {
                if (neu) {
#pragma unroll
                    for (int v = 0; v < VX; ++v) yp[v] = cz[rr][v];
                } else {
                    // row 0: box row 1 of the first block row, else the row box
                    Vec<T>::get(br.rowy >= 0 ? rowb + VX + xl : cur + BW + VX + xl, yp);
                }
            }
            if (!neu) {
                // column n - 1 (left of column 0) and column 0 (right of column n - 1)
                if (gx == 0) left = br.colx >= 0 ? colb[br_row * VX + (n - 1) % VX] : cur[br_row * BW + VX + n - 1];
                if (lastv >= 0 && lastv < VX) wrapx = br.colx >= 0 ? colb[br_row * VX] : cur[br_row * BW + VX];
            } else if (gx == 0) {
                left = cz[rr][0];
            }
        }
        if constexpr (PACKED) {
            // FP32 off the boundary: the same operations on pairs of points
            f2 x2p[2];
            predict4_2d(ym, cz[rr], yp, left, right, pc, x2p);
            xip[2 * rr] = x2p[0];
            xip[2 * rr + 1] = x2p[1];
        } else {
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                const T xm = v == 0 ? left : cz[rr][v - 1];
                T xp = v == VX - 1 ? right : cz[rr][v + 1];
                if (EDGE && v == lastv) xp = neu ? cz[rr][v] : wrapx;
                xi[rr * VX + v] = predictor(cz[rr][v], nsum(ym[v], yp[v], xm, xp), c);
            }
        }
    }
    (void)TY;
    T out[NP];
    if constexpr (PACKED) roots2<SOLVE, 2 * RPT>(xip, out, c, pc);
    else roots<T, SOLVE, NP>(xi, out, c);
    T* o = dst + (int64_t)gy0 * sy + gx;
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
        if (gy0 + rr >= n) continue;
        if (gx + VX <= n) {
            Vec<T>::put(o + rr * sy, &out[rr * VX]);
        } else {
#pragma unroll
            for (int v = 0; v < VX; ++v)
                if (gx + v < n) o[rr * sy + v] = out[rr * VX + v];
        }
    }
}

template <typename T>
__device__ __forceinline__ void batch_block_any(const T* cur, const T* colb, const T* rowb, T* dst, int n, int bc,
                                                int64_t sy, const Coef<T>& c, const BlockRef& br) {
    constexpr int TX = BatchTile<T>::TX, TY = BatchTile<T>::TY;
    const bool edge = bc != ACS_BC_DIRICHLET && (br.x0 == 0 || br.x0 + TX >= n || br.y0 == 0 || br.y0 + TY >= n);
    ACS_SOLVE_DISPATCH_UNIT(c, SV, {
        if (edge) batch_block<T, SV, true>(cur, colb, rowb, dst, n, bc, sy, c, br);
        else batch_block<T, SV, false>(cur, colb, rowb, dst, n, bc, sy, c, br);
    });
}

// Persistent cooperative kernel: nsteps steps of every instance (with `fixed`, every
// step reads A and writes B: the same work and barriers, for timing without changing A).  Per step, CTAs take
// chunks of kch consecutive blocks from the step's ticket counter (so instances of
// different cost balance out), stream them through the TMA ring, and meet at the grid
// barrier.  Lane 0 of a ninth warp is the producer: it draws tickets one chunk ahead,
// issues each block's loads into the next free slot with the block's description in
// `meta`, and closes the step with an end marker (a slot whose mbarrier completes
// without data).  The eight compute warps consume slots
// independently: `full[s]` says a slot has landed, `empty[s]` (one arrival per compute
// warp) that every warp is done with it, so no compute warp waits for another and
// only the producer waits, before it refills a slot.
template <typename T>
__global__ void __launch_bounds__(288, sizeof(T) == 4 ? 3 : 2) k_batch2d(T* A, T* B, const DevInst<T>* __restrict__ inst,
                                                 const CUtensorMap* __restrict__ maps, int count,
                                                 const BlockRef* __restrict__ blocks, int nblocks, int kch,
                                                 int nsteps, int fixed, BarrierState* bs, int* err) {
    using TT = BatchTile<T>;
    using SM = BatchSmem<T>;
    constexpr int VX = TT::VX, S = TT::S, WARPS = 8;
    constexpr int SLOT_ELEMS = TT::SLOT_STRIDE / sizeof(T);
    static_assert(2 * S * sizeof(uint64_t) <= TT::BAR_BYTES, "full and empty barriers");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(base);
    uint64_t* empty = full + S;
    T* ring = reinterpret_cast<T*>(base + SM::OFF_RING);
    unsigned char* colbase = base + SM::OFF_COL;
    unsigned char* rowbase = base + SM::OFF_ROW;
    BlockRef* meta = reinterpret_cast<BlockRef*>(base + SM::OFF_META);
    unsigned char* instbase = base + SM::OFF_INST;
    __shared__ unsigned fenced[kFenceWords];
    __shared__ volatile int s_fail;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int lane = threadIdx.x;
    const bool producer = threadIdx.y == WARPS && lane == 0;
    const unsigned nchunks = (unsigned)((nblocks + kch - 1) / kch);
    if (tid < kFenceWords) fenced[tid] = 0u;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], WARPS);
        }
        fence_mbar_init();
        s_fail = 0;
    }
    __syncthreads();
    const bool injector = bs->inject != 0 && blockIdx.x == gridDim.x - 1;
    auto fail = [&]() {
        s_fail = 1;
        atomicExch(err, 1);
    };

    // producer state (the producer thread only)
    int64_t qi = 0;               // next sequence number to fill (slot qi % S, phase (qi / S) & 1)
    unsigned cur = 0, pf = 0;     // current chunk and the next one (drawn ahead)
    int j = 0;                    // next block within the current chunk
    bool closed = false;          // the step's end marker has been issued (or the CTA failed)
    int step = 0;
    auto draw = [&]() -> unsigned { return atomicAdd(&bs->ctr[step & 3], 1u); };
    auto acquire_maps = [&](int i) {
        if (i < kFenceWords * 32) {
            if (fenced[i >> 5] & (1u << (i & 31))) return;
            fenced[i >> 5] |= 1u << (i & 31);
        }
        for (int m = 0; m < kMapsPerInst; ++m) fence_tensormap_acquire(&maps[(size_t)i * kMapsPerInst + m]);
    };
    auto produce = [&]() {
        const int s = (int)(qi % S);
        // every warp must be done with the slot's previous block
        if (qi >= S && !mbar_wait(&empty[s], (uint32_t)(((qi / S) - 1) & 1))) {
            fail();
            closed = true;
            return;
        }
        if (cur >= nchunks) {
            meta[s].inst = -1;
            mbar_arrive(&full[s]);
            closed = true;
            ++qi;
            return;
        }
        const BlockRef br = blocks[(size_t)cur * kch + j];
        meta[s] = br;
        T* dstp = ring + (size_t)s * SLOT_ELEMS;
        unsigned char* colp = colbase + (size_t)s * SM::COL_STRIDE;
        unsigned char* rowp = rowbase + (size_t)s * SM::ROW_STRIDE;
        const int xb = br.x0 - VX;
        if ((smem_u32(dstp) & 127u) != 0u || ((xb * (int)sizeof(T)) & 15) != 0 ||
            (br.colx >= 0 && ((br.colx * (int)sizeof(T)) & 15) != 0)) {
            atomicExch(err, 2);
        } else {
            acquire_maps(br.inst);
            const CUtensorMap* m = &maps[(size_t)br.inst * kMapsPerInst + 3 * (fixed ? 0 : (step & 1))];
            const uint32_t bytes = TT::SLOT_BYTES + SM::INST_BYTES + (br.colx >= 0 ? SM::COL_BYTES : 0u) +
                                   (br.rowy >= 0 ? SM::ROW_BYTES : 0u);
            fence_proxy_async();
            mbar_arrive_expect_tx(&full[s], bytes);
            bulk_load(instbase + (size_t)s * SM::INST_STRIDE, &inst[br.inst], SM::INST_BYTES, &full[s]);
            tma_load_2d(dstp, &m[0], &full[s], xb, br.y0 - 1);
            if (br.colx >= 0) tma_load_2d(colp, &m[1], &full[s], br.colx, br.y0 - 1);
            if (br.rowy >= 0) tma_load_2d(rowp, &m[2], &full[s], xb, br.rowy);
        }
        ++qi;
        if (++j == kch || (size_t)cur * kch + j >= (size_t)nblocks) {
            cur = pf;
            j = 0;
            if (cur < nchunks) {
                pf = draw();
                // the next chunk's descriptors, one block ahead of their first use
                asm volatile("prefetch.L1 [%0];" ::"l"(blocks + (size_t)cur * kch));
            }
        }
    };

    int64_t q = 0;  // next sequence number to consume (the same in every consumer warp)
    bool failed = false;
    for (step = 0; step < nsteps && !failed; ++step) {
        T* dst = (step & 1) && !fixed ? A : B;
        if (producer) {
            // other CTAs' stores of the previous step (ordered by the grid barrier)
            // before this thread's async-proxy reads of them
            asm volatile("fence.proxy.async.global;" ::: "memory");
            cur = draw();
            pf = cur < nchunks ? draw() : cur;
            j = 0;
            closed = false;
            while (!closed) produce();
        } else if (threadIdx.y < WARPS) {
            for (;;) {
                if (s_fail) break;
                const int s = (int)(q % S);
                const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)((q / S) & 1)));
                if (!ok) {
                    if (lane == 0) fail();
                    break;
                }
                ++q;
                const BlockRef br = meta[s];
                if (br.inst >= 0) {
                    // the instance (copied in with the block) and its coefficients in
                    // registers: stores to dst cannot then force them to be read again
                    const DevInst<T>* in =
                        reinterpret_cast<const DevInst<T>*>(instbase + (size_t)s * SM::INST_STRIDE);
                    const Coef<T> c = in->c;
                    batch_block_any<T>(ring + (size_t)s * SLOT_ELEMS,
                                       reinterpret_cast<const T*>(colbase + (size_t)s * SM::COL_STRIDE),
                                       reinterpret_cast<const T*>(rowbase + (size_t)s * SM::ROW_STRIDE),
                                       dst + in->off, in->n, in->bc, in->ld, c, br);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                if (br.inst < 0) break;
            }
        }
        __syncthreads();
        failed = s_fail != 0;
        if (!failed && step + 1 < nsteps && !grid_barrier(bs, gridDim.x, step, err, injector && step == 0))
            failed = true;
    }
    if (failed && producer) {
        atomicExch(err, 1);
        // let the newest fill of every slot land (bounded wait) before the CTA exits
        for (int64_t k = qi > S ? qi - S : 0; k < qi; ++k) mbar_wait(&full[(int)(k % S)], (uint32_t)((k / S) & 1));
    }
    __syncthreads();
}

}  // namespace acs

using namespace acs;

struct acs_batch {
    int count, dtype;
    size_t esize;
    std::vector<int64_t> n, off, ld;
    std::vector<double> eps, dt, h;
    std::vector<int> bc;
    std::vector<DevInst<float>> inf;
    std::vector<DevInst<double>> ind;
    std::vector<BlockRef> blocks;
    int64_t numel;
    // bound
    bool bound;
    char* phi;
    char* work;
    cudaStream_t stream, cap;
    char* other;
    void* dinst;
    CUtensorMap* maps;
    BlockRef* dblocks;
    BarrierState* bs;
    int* err;
    RedPartial* partials;
    double* results;
    int grid;
    // launch configuration (acs_batch_set_config / acs_batch_autotune): CTAs per SM of
    // the persistent grid (0 = all that fit), blocks per ticket, block order
    int ctas, chunk, order;
    int sms, per_sm;                  // SM count and resident CTAs per SM of the kernel
    std::vector<BlockRef> blocks0;    // the blocks in instance order
    // temporal blocking (acs_batch_set_temporal): depth (1 = the single-step kernel
    // only), rows per unit (0 = kDefaultTbRows), whether the batch can use the
    // temporally blocked kernel (FP32), its unit list and persistent grid
    int tdepth, trows, torder;  // torder: unit order, as `order` for the blocks
    bool tok;
    int64_t tcap;                     // units the work buffer has room for
    std::vector<TbUnit> tunits;
    TbUnit* dunits;
    unsigned* ddone;
    int tgrid;
    std::vector<std::pair<int64_t, cudaGraphExec_t>> graphs;
};

namespace {
constexpr size_t kA = 256;
size_t al(size_t x) { return (x + kA - 1) / kA * kA; }
size_t inst_bytes(const acs_batch* b) {
    return al((size_t)b->count * (b->dtype == ACS_F32 ? sizeof(DevInst<float>) : sizeof(DevInst<double>)));
}
// work buffer: the second state buffer, instances, tensor maps (six per instance),
// block list, barrier + error flag, reduction partials, per-instance results
size_t off_inst(const acs_batch* b) { return al((size_t)b->numel * b->esize); }
size_t off_maps(const acs_batch* b) { return off_inst(b) + inst_bytes(b); }
size_t off_blocks(const acs_batch* b) {
    return off_maps(b) + al(sizeof(CUtensorMap) * kMapsPerInst * (size_t)b->count);
}
size_t off_bar(const acs_batch* b) { return off_blocks(b) + al(sizeof(BlockRef) * b->blocks.size()); }
size_t off_part(const acs_batch* b) { return off_bar(b) + kA; }
size_t off_res(const acs_batch* b) { return off_part(b) + al(sizeof(RedPartial) * kMaxRedBlocks); }
size_t off_units(const acs_batch* b) { return off_res(b) + al(sizeof(double) * 2 * (size_t)b->count); }
size_t off_done(const acs_batch* b) { return off_units(b) + al(sizeof(TbUnit) * (size_t)b->tcap); }
size_t total_bytes(const acs_batch* b) { return off_done(b) + al(sizeof(unsigned) * (size_t)b->count); }

constexpr int kDefaultTbRows = 64;         // rows per unit of the temporally blocked kernel by default
constexpr int64_t kMaxTbUnits = 1 << 22;   // room reserved for units at most

void drop_graphs(acs_batch* b) {
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
}

template <typename T>
cudaError_t launch_batch(acs_batch* b, int64_t nsteps, cudaStream_t st, int fixed = 0) {
    auto kern = k_batch2d<T>;
    const size_t smem = BatchSmem<T>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    T* A = (T*)b->phi;
    T* B = (T*)b->other;
    const DevInst<T>* in = (const DevInst<T>*)b->dinst;
    const CUtensorMap* maps = b->maps;
    const BlockRef* blocks = b->dblocks;
    int count = b->count, nblocks = (int)b->blocks.size(), kch = b->chunk, ns = (int)nsteps;
    void* args[] = {&A, &B, &in, &maps, &count, &blocks, &nblocks, &kch, &ns, &fixed, &b->bs, &b->err};
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3(32, 9);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)kern, args);
}

// npasses passes of the temporally blocked kernel (fixed: every pass reads phi and
// writes the second buffer), with fresh ticket and completion counters.
cudaError_t launch_tb(acs_batch* b, int64_t npasses, cudaStream_t st, int fixed = 0) {
    cudaError_t e = cudaMemsetAsync(b->bs->ctr, 0, sizeof(b->bs->ctr), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ddone, 0, sizeof(unsigned) * (size_t)b->count, st);
    if (e != cudaSuccess) return e;
    return launch_batch_tb(b->tdepth, (float*)b->phi, (float*)b->other, (const DevInst<float>*)b->dinst,
                           b->dunits, (int)b->tunits.size(), (int)npasses, fixed, b->bs, b->ddone, b->err, b->tgrid,
                           st);
}

// Launches that advance nsteps; the packed state starts in phi and ends there (a
// launch that leaves it in the second buffer is followed by one device copy back).
// With temporal blocking, nsteps / K passes of K steps run first (one launch, unless
// the ticket count needs more), then the remaining nsteps % K single steps.
cudaError_t enqueue_batch(acs_batch* b, int64_t nsteps, cudaStream_t st) {
    if (b->tdepth >= 2 && nsteps >= b->tdepth) {
        const int64_t K = b->tdepth;
        const int64_t max_passes = std::max<int64_t>(1, ((int64_t)1 << 30) / (int64_t)b->tunits.size());
        for (int64_t left = nsteps / K; left > 0;) {
            const int64_t p = std::min(left, max_passes);
            cudaError_t e = launch_tb(b, p, st);
            if (e != cudaSuccess) return e;
            if (p & 1) {
                e = cudaMemcpyAsync(b->phi, b->other, (size_t)b->numel * b->esize, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return e;
            }
            left -= p;
        }
        nsteps %= K;
    }
    const int64_t chunk_max = 1 << 20;
    for (int64_t done = 0; done < nsteps;) {
        const int64_t k = std::min(chunk_max, nsteps - done);
        // fresh ticket counters for the launch's first steps
        cudaError_t e = cudaMemsetAsync(b->bs->ctr, 0, sizeof(b->bs->ctr), st);
        if (e != cudaSuccess) return e;
        e = b->dtype == ACS_F32 ? launch_batch<float>(b, k, st) : launch_batch<double>(b, k, st);
        if (e != cudaSuccess) return e;
        if (k & 1) {
            e = cudaMemcpyAsync(b->phi, b->other, (size_t)b->numel * b->esize, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
        done += k;
    }
    return cudaSuccess;
}

// The block list in the configured order (0: instance after instance; 1: the largest
// instances first, so their blocks are drawn first and the small ones fill the end of
// every step), each instance's blocks in their own order.
void order_blocks(acs_batch* b) {
    b->blocks = b->blocks0;
    if (b->order == 1)
        std::stable_sort(b->blocks.begin(), b->blocks.end(),
                         [b](const BlockRef& x, const BlockRef& y) { return b->n[x.inst] > b->n[y.inst]; });
}

// Unit list of the temporally blocked kernel: instances in its own configured order (0:
// as given; 1: the largest first), each strip after strip, a strip's chunks of rows down
// it (balanced chunks of at most the configured rows); sets DevInst::tbunits.
void build_tb_units(acs_batch* b) {
    b->tunits.clear();
    const int rows = b->trows > 0 ? b->trows : kDefaultTbRows;
    std::vector<int> idx(b->count);
    for (int i = 0; i < b->count; ++i) idx[i] = i;
    if (b->torder == 1) std::stable_sort(idx.begin(), idx.end(), [b](int x, int y) { return b->n[x] > b->n[y]; });
    for (int i : idx) {
        const int n = (int)b->n[i];
        const int strips = (n + kBatchTbCols - 1) / kBatchTbCols;
        const int chunks0 = (n + rows - 1) / rows;
        const int ych = (n + chunks0 - 1) / chunks0;
        const int chunks = (n + ych - 1) / ych;
        for (int st = 0; st < strips; ++st)
            for (int ck = 0; ck < chunks; ++ck)
                b->tunits.push_back(TbUnit{i, st, ck * ych, std::min(n, (ck + 1) * ych)});
        b->inf[i].tbunits = strips * chunks;
    }
}

// Upload the block list (and with temporal blocking the unit list and the instances'
// unit counts) and size the persistent grids for the configuration.
cudaError_t apply_config(acs_batch* b) {
    order_blocks(b);
    cudaError_t e = cudaMemcpyAsync(b->dblocks, b->blocks.data(), sizeof(BlockRef) * b->blocks.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return e;
    const int ctas = b->ctas > 0 ? std::min(b->ctas, b->per_sm) : b->per_sm;
    const int64_t chunks = ((int64_t)b->blocks.size() + b->chunk - 1) / b->chunk;
    b->grid = (int)std::min<int64_t>((int64_t)b->sms * ctas, chunks);
    if (b->tdepth >= 2) {
        build_tb_units(b);
        if ((int64_t)b->tunits.size() > b->tcap) return cudaErrorInvalidValue;
        const int per = batch_tb_per_sm(b->tdepth);
        if (per < 1) return cudaErrorInvalidConfiguration;
        b->tgrid = b->sms * per;
        e = cudaMemcpyAsync(b->dunits, b->tunits.data(), sizeof(TbUnit) * b->tunits.size(), cudaMemcpyHostToDevice,
                            b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->dinst, b->inf.data(), sizeof(DevInst<float>) * (size_t)b->count,
                                cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return e;
    }
    drop_graphs(b);
    return cudaStreamSynchronize(b->stream);
}

// Workload class of a batch for the tuning cache: dtype, count, total unknowns, a
// histogram of sides in octaves (log2 bins) and the boundary mix.
std::string batch_class(const acs_batch* b) {
    int64_t total = 0;
    int hist[32] = {0}, bcs[3] = {0, 0, 0};
    for (int i = 0; i < b->count; ++i) {
        total += b->n[i] * b->n[i];
        int k = 0;
        while ((int64_t(2) << k) <= b->n[i] && k < 31) ++k;
        ++hist[k];
        ++bcs[b->bc[i]];
    }
    std::string key = "batch/t" + std::to_string(b->dtype) + "/c" + std::to_string(b->count) + "/u" +
                      std::to_string(total) + "/bc" + std::to_string(bcs[0]) + "-" + std::to_string(bcs[1]) + "-" +
                      std::to_string(bcs[2]) + "/h";
    for (int k = 0; k < 32; ++k)
        if (hist[k]) key += std::to_string(k) + ":" + std::to_string(hist[k]) + ",";
    return key;
}

template <typename T>
void fill_inst(acs_batch* b, std::vector<DevInst<T>>& v) {
    using TT = BatchTile<T>;
    v.resize(b->count);
    b->blocks.clear();
    for (int i = 0; i < b->count; ++i) {
        DevInst<T>& d = v[i];
        std::memset(&d, 0, sizeof(d));
        d.off = b->off[i];
        d.n = (int)b->n[i];
        d.ld = (int)b->ld[i];
        d.bc = b->bc[i];
        const double lam = b->eps[i] * b->eps[i] * b->dt[i] / (b->h[i] * b->h[i]);
        double dmp, den;
        acs_dt_max(2, b->eps[i], b->h[i], &dmp, &den);
        const bool mp_ok = b->dt[i] <= dmp * (1.0 + 1e-12);
        d.c = make_coef<T>(2, lam, b->dt[i], ACS_SCHEME_RLB_MIE_FD, mp_ok);
        // down each column strip, strip after strip (consecutive blocks share halo rows)
        const int n = d.n;
        for (int x0 = 0; x0 < n; x0 += TT::TX)
            for (int y0 = 0; y0 < n; y0 += TT::TY) {
                BlockRef r{i, x0, y0, -1, -1, 0, 0, 0};
                if (d.bc == ACS_BC_PERIODIC) {
                    // wrapped column / row from a side box unless the main box holds it
                    if (x0 == 0 && n > TT::TX + TT::VX) r.colx = (n - 1) / TT::VX * TT::VX;
                    if (x0 > 0 && n - 1 < x0 + TT::TX) r.colx = 0;
                    if (y0 == 0 && n - 1 > TT::TY) r.rowy = n - 1;
                    if (y0 > 0 && n - 1 < y0 + TT::TY) r.rowy = 0;
                }
                b->blocks.push_back(r);
            }
    }
}

// Six tensor maps per instance, three per state buffer (phi, then the other one):
// the main halo box (BW x BH), the column box (VX x BH) and the row box (BW x 1) of
// periodic wraps; n x n values, rows ld apart.
template <typename T>
bool encode_maps(acs_batch* b, std::vector<CUtensorMap>& maps) {
    using TT = BatchTile<T>;
    maps.resize((size_t)kMapsPerInst * b->count);
    const uint32_t boxes[3][2] = {{(uint32_t)TT::BW, (uint32_t)TT::BH}, {(uint32_t)TT::VX, (uint32_t)TT::BH},
                                  {(uint32_t)TT::BW, 1u}};
    for (int i = 0; i < b->count; ++i)
        for (int buf = 0; buf < 2; ++buf)
            for (int k = 0; k < 3; ++k) {
                const char* basep = (buf == 0 ? b->phi : b->other) + b->off[i] * (int64_t)b->esize;
                const uint64_t dims[2] = {(uint64_t)b->n[i], (uint64_t)b->n[i]};
                if (!encode_tensor_map(&maps[(size_t)i * kMapsPerInst + 3 * buf + k], (int)sizeof(T), 2, basep, dims,
                                       boxes[k], (uint64_t)b->ld[i] * sizeof(T)))
                    return false;
            }
    return true;
}

}  // namespace

extern "C" {

ACS_API int acs_batch_create(int count, const int64_t* n, const double* eps, const double* dt, const double* h,
                             const int* bc, int dtype, acs_batch** out) {
    if (!out || count < 1 || !n || !eps || !dt || !h || !bc) return ACS_E_INVAL;
    if (dtype != ACS_F32 && dtype != ACS_F64) return ACS_E_INVAL;
    const int64_t vx = dtype == ACS_F32 ? 4 : 2;  // values per 16 bytes
    int64_t numel = 0, blocks = 0;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || n[i] > (1 << 20)) return ACS_E_INVAL;
        if (!std::isfinite(eps[i]) || !std::isfinite(dt[i]) || !std::isfinite(h[i])) return ACS_E_INVAL;
        if (eps[i] < 0 || !(h[i] > 0) || !(dt[i] > 0) || !(dt[i] < 2) || bc[i] < 0 || bc[i] > 2) return ACS_E_INVAL;
        numel += (n[i] + vx - 1) / vx * vx * n[i];
        blocks += ((n[i] + 32 * vx - 1) / (32 * vx)) * ((n[i] + 15) / 16);
        if (numel > (int64_t(1) << 40) || blocks > 0x7fffffff) return ACS_E_INVAL;
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
        // rows padded to a 16-byte multiple, so every instance starts 16-byte aligned
        const int64_t ldi = (n[i] + vx - 1) / vx * vx;
        b->ld.push_back(ldi);
        b->off.push_back(b->numel);
        b->numel += ldi * n[i];
        double dmp, den;
        acs_dt_max(2, eps[i], h[i], &dmp, &den);
        if (dt[i] > den * (1.0 + 1e-12)) warn = ACS_WARN_ENERGY_CONDITION;
        else if (dt[i] > dmp * (1.0 + 1e-12) && warn == ACS_OK) warn = ACS_WARN_MP_CONDITION;
    }
    if (dtype == ACS_F32) fill_inst<float>(b, b->inf);
    else fill_inst<double>(b, b->ind);
    b->blocks0 = b->blocks;
    b->ctas = 0;
    b->chunk = 1;
    b->order = 0;
    b->sms = b->per_sm = 0;
    // temporal blocking: FP32 batches whose instances all use the series root
    b->tdepth = 1;
    b->trows = 0;
    b->torder = 0;
    b->tok = false;
    b->tcap = 0;
    b->tgrid = 0;
    b->dunits = nullptr;
    b->ddone = nullptr;
    if (dtype == ACS_F32) {
        // room for the units of the shortest chunks
        int64_t cap = 0;
        for (int i = 0; i < count; ++i)
            cap += (n[i] + kBatchTbCols - 1) / kBatchTbCols * ((n[i] + kMinBatchRows - 1) / kMinBatchRows);
        if (cap <= kMaxTbUnits) {
            b->tok = true;
            b->tcap = cap;
        }
    }
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

ACS_API int acs_batch_row_strides(const acs_batch* b, int64_t* row_strides) {
    if (!b || !row_strides) return ACS_E_INVAL;
    for (int i = 0; i < b->count; ++i) row_strides[i] = b->ld[i];
    return ACS_OK;
}

ACS_API size_t acs_batch_work_bytes(const acs_batch* b) { return b ? total_bytes(b) : 0; }

ACS_API int acs_batch_bind(acs_batch* b, void* d_phi, void* d_work, size_t work_bytes, void* stream) {
    if (!b || !d_phi || !d_work || ((uintptr_t)d_phi % 16) || ((uintptr_t)d_work % kA)) return ACS_E_INVAL;
    if (work_bytes < total_bytes(b)) return ACS_E_NOMEM;
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return ACS_E_CUDA;
    drop_graphs(b);
    b->bound = false;
    b->phi = (char*)d_phi;
    b->work = (char*)d_work;
    b->other = b->work;
    b->stream = (cudaStream_t)stream;
    b->dinst = b->work + off_inst(b);
    b->maps = (CUtensorMap*)(b->work + off_maps(b));
    b->dblocks = (BlockRef*)(b->work + off_blocks(b));
    b->bs = (BarrierState*)(b->work + off_bar(b));
    b->err = (int*)((char*)b->bs + 64);
    b->partials = (RedPartial*)(b->work + off_part(b));
    b->results = (double*)(b->work + off_res(b));
    b->dunits = (TbUnit*)(b->work + off_units(b));
    b->ddone = (unsigned*)(b->work + off_done(b));
    std::vector<CUtensorMap> maps;
    const bool enc = b->dtype == ACS_F32 ? encode_maps<float>(b, maps) : encode_maps<double>(b, maps);
    if (!enc) return ACS_E_UNSUPPORTED;
    const void* host = b->dtype == ACS_F32 ? (const void*)b->inf.data() : (const void*)b->ind.data();
    const size_t ib = (size_t)b->count * (b->dtype == ACS_F32 ? sizeof(DevInst<float>) : sizeof(DevInst<double>));
    if (cudaMemcpyAsync(b->dinst, host, ib, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->dblocks, b->blocks.data(), sizeof(BlockRef) * b->blocks.size(), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->bs, 0, kA, b->stream) != cudaSuccess)
        return ACS_E_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ACS_E_CUDA;
    // persistent grid: every SM's resident CTAs, never more than the chunks of blocks
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    if (b->dtype == ACS_F32) {
        cudaFuncSetAttribute(k_batch2d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BatchSmem<float>::BYTES);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch2d<float>, 288, BatchSmem<float>::BYTES);
    } else {
        cudaFuncSetAttribute(k_batch2d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BatchSmem<double>::BYTES);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch2d<double>, 288,
                                                          BatchSmem<double>::BYTES);
    }
    if (e != cudaSuccess || per_sm < 1) return ACS_E_CUDA;
    b->sms = sms;
    b->per_sm = per_sm;
    // a configuration the autotuner chose for this workload class earlier
    int v[4];
    if (tune_cache_lookup_class(batch_class(b), v) && v[0] >= 0 && v[1] >= 1 && v[1] <= kMaxBatchChunk &&
        (v[2] == 0 || v[2] == 1) && v[3] >= 0) {
        b->ctas = v[0];
        b->chunk = v[1];
        b->order = v[2];
        // fourth field: depth | unit order << 3 | rows << 4 (0: single steps)
        const int depth = v[3] & 7, torder = (v[3] >> 3) & 1, rows = v[3] >> 4;
        if (depth >= 2 && depth <= kMaxBatchDepth && b->tok && rows >= kMinBatchRows && rows <= (1 << 20)) {
            b->tdepth = depth;
            b->trows = rows;
            b->torder = torder;
        }
    }
    if (apply_config(b) != cudaSuccess) return ACS_E_CUDA;
    b->bound = true;
    return ACS_OK;
}

ACS_API int acs_batch_set_config(acs_batch* b, int ctas_per_sm, int blocks_per_ticket, int order) {
    if (!b || ctas_per_sm < 0 || blocks_per_ticket < 1 || blocks_per_ticket > kMaxBatchChunk ||
        (order != 0 && order != 1))
        return ACS_E_INVAL;
    b->ctas = ctas_per_sm;
    b->chunk = blocks_per_ticket;
    b->order = order;
    if (!b->bound) return ACS_OK;
    return apply_config(b) == cudaSuccess ? ACS_OK : ACS_E_CUDA;
}

ACS_API int acs_batch_set_temporal(acs_batch* b, int depth, int rows_per_unit, int order) {
    if (!b || depth < 1 || depth > kMaxBatchDepth || rows_per_unit < 0 ||
        (rows_per_unit > 0 && rows_per_unit < kMinBatchRows) || rows_per_unit > (1 << 20) ||
        (order != 0 && order != 1))
        return ACS_E_INVAL;
    if (depth >= 2 && !b->tok) return ACS_E_UNSUPPORTED;
    b->tdepth = depth;
    b->trows = rows_per_unit;
    b->torder = order;
    if (!b->bound) return ACS_OK;
    return apply_config(b) == cudaSuccess ? ACS_OK : ACS_E_CUDA;
}

ACS_API int acs_batch_get_temporal(const acs_batch* b, int* depth, int* rows_per_unit, int* order) {
    if (!b) return ACS_E_INVAL;
    if (depth) *depth = b->tdepth;
    if (rows_per_unit) *rows_per_unit = b->trows > 0 ? b->trows : kDefaultTbRows;
    if (order) *order = b->torder;
    return ACS_OK;
}

ACS_API int acs_batch_get_config(const acs_batch* b, int* ctas_per_sm, int* blocks_per_ticket, int* order) {
    if (!b) return ACS_E_INVAL;
    if (ctas_per_sm) *ctas_per_sm = b->bound && b->ctas == 0 ? b->per_sm : b->ctas;
    if (blocks_per_ticket) *blocks_per_ticket = b->chunk;
    if (order) *order = b->order;
    return ACS_OK;
}

ACS_API int acs_batch_autotune(acs_batch* b, double* us_per_step) {
    if (!b) return ACS_E_INVAL;
    if (!b->bound) return ACS_E_STATE;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ACS_E_CUDA;
    int rc = ACS_OK;
    // Microseconds per step of the current configuration: the best of two launches
    // (after one untimed) that each read phi and write the second buffer (the state is
    // only read), kTuneSteps single steps with their grid barriers, or the passes of
    // the temporally blocked kernel that cover about as many steps.
    auto time_config = [&]() -> double {
        if (apply_config(b) != cudaSuccess) {
            rc = ACS_E_CUDA;
            return 1e300;
        }
        const int64_t passes = b->tdepth >= 2 ? std::max(1, kTuneSteps / b->tdepth) : 0;
        const int64_t steps = b->tdepth >= 2 ? passes * b->tdepth : kTuneSteps;
        double best_ms = 1e300;
        for (int round = 0; round < 3; ++round) {
            cudaError_t e = cudaSuccess;
            if (b->tdepth < 2) e = cudaMemsetAsync(b->bs->ctr, 0, sizeof(b->bs->ctr), b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) {
                if (b->tdepth >= 2) e = launch_tb(b, passes, b->stream, 1);
                else if (b->dtype == ACS_F32) e = launch_batch<float>(b, kTuneSteps, b->stream, 1);
                else e = launch_batch<double>(b, kTuneSteps, b->stream, 1);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = ACS_E_CUDA;
                return 1e300;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (round > 0) best_ms = std::min(best_ms, (double)ms / (double)steps);
        }
        return best_ms;
    };
    // the single-step kernel: order x CTAs per SM x blocks per ticket
    int ss[3] = {b->ctas, b->chunk, b->order};
    double ss_best = 1e300;
    static const int kChunks[3] = {1, 2, 4};
    b->tdepth = 1;
    for (int order = 0; order <= 1 && rc == ACS_OK; ++order)
        for (int ctas = 1; ctas <= b->per_sm && rc == ACS_OK; ++ctas)
            for (int ci = 0; ci < 3 && rc == ACS_OK; ++ci) {
                b->ctas = ctas;
                b->chunk = kChunks[ci];
                b->order = order;
                const double ms = time_config();
                if (rc == ACS_OK && ms < ss_best) {
                    ss_best = ms;
                    ss[0] = ctas; ss[1] = kChunks[ci]; ss[2] = order;
                }
            }
    // the temporally blocked kernel: depth x rows per unit x order
    int tb[3] = {1, 0, 0};
    double tb_best = 1e300;
    static const int kRows[3] = {32, 64, 128};
    if (b->tok)
        for (int depth = 2; depth <= kMaxBatchDepth && rc == ACS_OK; ++depth)
            for (int ri = 0; ri < 3 && rc == ACS_OK; ++ri)
                for (int order = 0; order <= 1 && rc == ACS_OK; ++order) {
                    b->tdepth = depth;
                    b->trows = kRows[ri];
                    b->torder = order;
                    const double ms = time_config();
                    if (rc == ACS_OK && ms < tb_best) {
                        tb_best = ms;
                        tb[0] = depth; tb[1] = kRows[ri]; tb[2] = order;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the single-step configuration stays for the steps a temporal block leaves over
    b->ctas = ss[0];
    b->chunk = ss[1];
    b->order = ss[2];
    const bool use_tb = tb_best < ss_best;
    b->tdepth = use_tb ? tb[0] : 1;
    b->trows = use_tb ? tb[1] : 0;
    b->torder = use_tb ? tb[2] : 0;
    if (apply_config(b) != cudaSuccess) rc = ACS_E_CUDA;
    if (rc != ACS_OK) return rc;
    int herr = 0;
    if (cudaMemcpy(&herr, b->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_E_CUDA;
    if (herr) {
        cudaMemset(b->err, 0, sizeof(int));
        return ACS_E_TIMEOUT;
    }
    const double best = use_tb ? tb_best : ss_best;
    const int v[4] = {b->ctas, b->chunk, b->order, use_tb ? b->tdepth | b->torder << 3 | b->trows << 4 : 0};
    tune_cache_store_class(batch_class(b), v, 1e3 * best);
    if (us_per_step) *us_per_step = 1e3 * best;
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
        // rows ld apart: the reduction walks the first n values of each row
        const int64_t nn[2] = {b->n[i], b->n[i]};
        Geo g = make_geo(2, nn);
        g.sy = b->ld[i];
        g.sz = b->ld[i] * b->n[i];
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
