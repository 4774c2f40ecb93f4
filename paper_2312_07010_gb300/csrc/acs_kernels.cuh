// acs_kernels.cuh -- launchers of the device kernels, called by the host API.
#pragma once

#include <algorithm>
#include <utility>

#include "acs_device.cuh"

namespace acs {

// Programmatic dependent launch.  A kernel launched by launch_pdl() may be scheduled
// while the kernel before it in the stream is still draining, which hides the launch
// gap of a chain of short dependent kernels (small grids, one step per launch).  Every
// such kernel calls pdl_wait() before it reads anything its predecessor wrote: the
// wait returns once that predecessor has completed and its memory is visible (at once
// when there is none).  pdl_trigger(), called by each CTA after its last store, lets
// the successor be scheduled as this kernel's CTAs retire.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Reduction partial of one block: compensated FP64 sums of the bulk term
// sum (phi^2 - 1)^2 / 4 and of the squared link differences, and max |phi|.
struct RedPartial {
    double bulk_s, bulk_c, link_s, link_c, mx, pad0, pad1, pad2;
};
constexpr int kMaxRedBlocks = 1024;
constexpr int kMaxStreamParts = 16384;  // partials of the streamed energy kernels

template <typename T>
cudaError_t launch_step_naive(int dims, int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c,
                              cudaStream_t st);

// Tiled variants: return cudaErrorNotSupported when the shape is not covered.
// err: device int set to 1 when a bounded wait inside the kernel gives up.
// variant: tile shape index (0 .. kNumTileVariants - 1); chunk: z planes (3D) or
// 16-row blocks (2D) per CTA, 0 = chosen from the occupancy.
template <typename T>
cudaError_t launch_step_tiled(int dims, int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int variant,
                              int chunk, int* err, cudaStream_t st);
// Temporal blocking: `depth` fused steps per pass (1 = the tiled kernel); chunk:
// 16-row blocks per warp (2D), 0 = chosen from the occupancy.
constexpr int kMaxTemporalDepth2d = 4;
template <typename T>
cudaError_t launch_step_temporal(int dims, int bc, int depth, const T* src, T* dst, const Geo& g,
                                 const Coef<T>& c, int variant, int chunk, int* err, cudaStream_t st);
bool tiled_supported(int dims, int dtype, const Geo& g);

// Collide-and-stream (population) form of the step: pop holds 2 dims + 1 arrays of
// total values, kLbGap values apart; omega1 is the lattice weight w_1 and
// lam = eps^2 dt / h^2 (s = w_1 / lam).  The gap keeps the arrays, whose size is
// often a power of two, from starting on a common alignment: with all seven on one
// alignment the gathering kernel ran 9 % slower at 512^3.
constexpr int64_t kLbGap = 8192;
template <typename T>
cudaError_t launch_step_lb(int dims, int bc, const T* src, T* pop, T* dst, const Geo& g, double omega1,
                           double lam, const Coef<T>& cf, cudaStream_t st);
bool temporal_supported(int dims, int dtype, int depth, const Geo& g);

// E_h and max |phi| with the TMA-streamed pipeline (3D, rows a multiple of 16 bytes);
// cudaErrorNotSupported when it does not apply.
template <typename T>
cudaError_t launch_energy3d(int bc, const T* src, const Geo& g, const Coef<T>& c, int* err, RedPartial* part,
                            int* nparts, cudaStream_t st);
// One 3D step src -> dst with the E_h / max-norm partials of src into part (the
// energy pass fused into the step; same conditions as launch_energy3d).
template <typename T>
cudaError_t launch_step_energy3d(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int* err,
                                 RedPartial* part, int* nparts, cudaStream_t st);
template <typename T>
cudaError_t launch_energy2d(int bc, const T* src, const Geo& g, const Coef<T>& c, int* err, RedPartial* part,
                            int* nparts, cudaStream_t st);
cudaError_t launch_reduce_finish(const RedPartial* part, int nparts, int dims, double eps2, double h, double* out2,
                                 cudaStream_t st);

// h^d sum (1 + phi)/2 into out (scratch: kMaxRedBlocks * 16 bytes).
template <typename T>
cudaError_t launch_phase_volume(const T* src, int64_t n, int dims, double h, void* scratch, double* out,
                                cudaStream_t st);

// E_h and max |phi|: partials then a one-block finish writing {E_h, max} to out2.
int reduce_blocks(const Geo& g);
template <typename T>
cudaError_t launch_reduce(int dims, int bc, const T* src, const Geo& g, double eps2, double h,
                          RedPartial* partials, double* out2, cudaStream_t st);

}  // namespace acs
