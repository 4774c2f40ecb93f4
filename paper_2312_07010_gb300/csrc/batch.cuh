// batch.cuh -- what the two batched kernels share: the instance record, the barrier /
// ticket state in device memory, and the launch entry of the temporally blocked
// batched kernel (batch_tb.cu).
#pragma once

#include <cstdint>

#include "acs_host.h"
#include "acs_kernels.cuh"

namespace acs {

// One instance as the kernels see it (the single-step kernel copies it into shared
// memory with each block).
template <typename T>
struct alignas(16) DevInst {
    int64_t off;  // first element of the instance in the packed state
    int n;        // side (x fastest)
    int ld;       // row stride in elements (a 16-byte multiple)
    int bc;
    int tbunits;  // units of the instance in the temporally blocked kernel's list (0: none)
    Coef<T> c;
};
static_assert(sizeof(DevInst<float>) % 16 == 0 && sizeof(DevInst<double>) % 16 == 0, "bulk-copy size");

struct BarrierState {
    unsigned count;   // arrivals in the current phase
    unsigned gen;     // phase counter
    int abort;        // set by a waiter that gave up: everyone leaves
    int inject;       // testing aid: 1 = the last CTA skips one arrival / one completion
    unsigned ctr[4];  // chunk tickets of step s in ctr[s & 3] (zeroed before each launch)
};

// One unit of the temporally blocked batched kernel: column strip `strip` of instance
// `inst` (window columns strip * OW - HG * VX .. + 32 VX - 1) over rows [ya, yb).
struct TbUnit {
    int inst, strip, ya, yb;
};

constexpr int kMaxBatchDepth = 4;  // deepest temporal block of the batched form
constexpr int kMinBatchRows = 16;  // smallest chunk of rows of a unit

// Columns a unit writes (the window's inner columns): the same for every depth 2..4.
constexpr int kBatchTbCols = 120;

// Resident CTAs per SM of the temporally blocked batched kernel of depth K (0: none).
int batch_tb_per_sm(int K);
int batch_tb_threads();

// npasses passes of K steps over the unit list; pass p reads A and writes B when p is
// even (B and A when odd), or always A -> B when `fixed`.  `done` holds one zeroed
// counter per instance and bs->ctr[0] the zeroed ticket counter.  grid CTAs, all
// resident (cooperative launch).
cudaError_t launch_batch_tb(int K, float* A, float* B, const DevInst<float>* inst, const TbUnit* units, int nunits,
                            int npasses, int fixed, BarrierState* bs, unsigned* done, int* err, int grid,
                            cudaStream_t st);

}  // namespace acs
