// step_tiled.cu -- selection and dispatch of the tiled / temporally blocked step
// kernels, and tensor-map encoding for their TMA loads.
#include <mutex>

#include "acs_host.h"
#include "tma.cuh"

namespace acs {

bool step3d_supported(int dtype, const Geo& g);
template <typename T>
cudaError_t launch_step3d(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int variant, int zchunk,
                          int* err, cudaStream_t st);

bool step2d_supported(const Geo& g);
template <typename T>
cudaError_t launch_step2d(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int per_cta,
                          cudaStream_t st);

bool step2d_tma_supported(int dtype, const Geo& g);
template <typename T>
cudaError_t launch_step2d_tma(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int variant,
                              int ybchunk, int* err, cudaStream_t st);

bool encode_tensor_map(CUtensorMap* map, int esize, int rank, const void* base, const uint64_t* dims,
                       const uint32_t* box, uint64_t row_pitch) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    if (!fn || rank < 1 || rank > 5) return false;
    cuuint64_t gd[5], gs[4];
    cuuint32_t bx[5], es[5];
    uint64_t stride = (uint64_t)esize;
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i > 0) gs[i - 1] = stride;
        stride = (i == 0 && row_pitch) ? row_pitch : stride * dims[i];
    }
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void*>(base), gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool tiled_supported(int dims, int dtype, const Geo& g) {
    if (dims == 3) return step3d_supported(dtype, g);
    if (dims == 2) return step2d_supported(g);
    return false;
}

bool step2d_tb_supported(int dtype, int depth, const Geo& g);
template <typename T>
cudaError_t launch_step2d_tb(int bc, int depth, const T* src, T* dst, const Geo& g, const Coef<T>& c, int ych,
                             cudaStream_t st);

bool step3d_tb_supported(int dtype, int depth, const Geo& g);
template <typename T>
cudaError_t launch_step3d_tb(int bc, int depth, const T* src, T* dst, const Geo& g, const Coef<T>& c, int zch,
                             cudaStream_t st);

// Temporal blocking: 2D grids whose rows are a multiple of 16 bytes, depth 2..4; 3D
// FP32 grids with an even row length, depth 2 (FP64 is bound by its arithmetic pipe,
// where fusing steps saves nothing).
bool temporal_supported(int dims, int dtype, int depth, const Geo& g) {
    if (dims == 2) return step2d_tb_supported(dtype, depth, g);
    if (dims == 3) return step3d_tb_supported(dtype, depth, g);
    return false;
}

template <typename T>
cudaError_t launch_step_tiled(int dims, int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int variant,
                              int chunk, int* err, cudaStream_t st) {
    if (dims == 3) return launch_step3d<T>(bc, src, dst, g, c, variant, chunk, err, st);
    if (dims == 2) {
        if (step2d_tma_supported(sizeof(T) == 4 ? ACS_F32 : ACS_F64, g))
            return launch_step2d_tma<T>(bc, src, dst, g, c, variant, chunk, err, st);
        return launch_step2d<T>(bc, src, dst, g, c, chunk, st);
    }
    return cudaErrorNotSupported;
}
// `depth` fused steps src -> dst; a depth of 1 (the remainder of a run) is the
// single-step tiled kernel, or the one-thread kernel where the tiled one does not
// cover the shape (3D rows that are not a multiple of 16 bytes); all round identically.  chunk: 16-row blocks per warp
// (2D) or z planes per CTA (3D); 0 = chosen from the occupancy.
template <typename T>
cudaError_t launch_step_temporal(int dims, int bc, int depth, const T* src, T* dst, const Geo& g, const Coef<T>& c,
                                 int variant, int chunk, int* err, cudaStream_t st) {
    if (depth == 1) {
        if (tiled_supported(dims, sizeof(T) == 4 ? ACS_F32 : ACS_F64, g))
            return launch_step_tiled<T>(dims, bc, src, dst, g, c, variant, 0, err, st);
        return launch_step_naive<T>(dims, bc, src, dst, g, c, st);
    }
    if (dims == 2) return launch_step2d_tb<T>(bc, depth, src, dst, g, c, 16 * chunk, st);
    if (dims == 3) return launch_step3d_tb<T>(bc, depth, src, dst, g, c, chunk, st);
    return cudaErrorNotSupported;
}
template cudaError_t launch_step_tiled<float>(int, int, const float*, float*, const Geo&, const Coef<float>&, int,
                                              int, int*, cudaStream_t);
template cudaError_t launch_step_tiled<double>(int, int, const double*, double*, const Geo&, const Coef<double>&,
                                               int, int, int*, cudaStream_t);
template cudaError_t launch_step_temporal<float>(int, int, int, const float*, float*, const Geo&,
                                                 const Coef<float>&, int, int, int*, cudaStream_t);
template cudaError_t launch_step_temporal<double>(int, int, int, const double*, double*, const Geo&,
                                                  const Coef<double>&, int, int, int*, cudaStream_t);

// Static choice for problems the autotuner does not time (below 2^20 unknowns).  The
// tiled kernels give a CTA a whole tile (16 rows of 64 FP64 / 128 FP32 values, times
// a run of planes in 3D), so a small grid makes few CTAs: FP64, bound by the FP64
// pipe (1/64 of the FP32 rate), then runs on a fraction of the SMs, and a small FP32
// grid pays the tile pipeline's fill for little work.  One thread per unknown spreads
// those grids over every SM (measured per step, one-thread kernel against tiled:
// 128^2 FP64 2.5 us / 11.8 us, 96^3 FP64 76 / 103 us, 256^2 FP32 1.5 / 2.2 us,
// 384^2 FP32 2.3 / 2.4 us; from 512^2 and 96^3 FP32 the tiled kernels win).
constexpr int64_t kSmallFp64 = int64_t(1) << 20;
constexpr int64_t kSmallFp32 = int64_t(1) << 18;

void resolve_auto_kernel(int dims, int dtype, int bc, const Geo& g, int* kernel, int* depth) {
    (void)bc;
    *depth = 1;
    const bool small = g.total < (dtype == ACS_F64 ? kSmallFp64 : kSmallFp32);
    *kernel = tiled_supported(dims, dtype, g) && !small ? ACS_KERNEL_TILED : ACS_KERNEL_NAIVE;
}

}  // namespace acs
