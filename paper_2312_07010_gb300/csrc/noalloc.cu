// noalloc.cu -- E_h and max|phi| for callers that cannot allocate device memory.
//
// The usual reduction (acs_energy / acs_observe_async) keeps its per-block partial
// sums in the work buffer the caller allocated for acs_bind().  Some callers have
// no such buffer and cannot make one: code that must not call cudaMalloc because
// it can synchronize the whole device (latency-critical loops), plugins whose host
// application owns every byte of device memory through its own pool, and tools
// that only hold a device pointer to someone else's state.  For them,
// acs_observe_noalloc() runs the same two reduction kernels with their scratch
// in the file-scope array below, which the CUDA module provides on every device
// that loads this library (it stays allocated until the process exits).
#include <cmath>
#include <mutex>

#include "acs_host.h"

namespace acs {
namespace {

// Scratch of the no-allocation reduction: one RedPartial (64 bytes) per block of
// the first stage.  The first stage never launches more than kMaxRedBlocks
// blocks, so 64 KiB covers every shape acs_create() accepts.
constexpr int kNoAllocParts = kMaxRedBlocks;
__device__ __align__(256) RedPartial g_noalloc_partials[kNoAllocParts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {nullptr};

// Device address of g_noalloc_partials on the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in, so it is
// never passed to a kernel directly.  The cached address belongs to the device's
// primary context: a process that resets a device (cudaDeviceReset) must not call
// acs_observe_noalloc on it again.
cudaError_t scratch_for_current_device(RedPartial** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = p;
    }
    *out = (RedPartial*)g_scratch[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace acs

using namespace acs;

extern "C" ACS_API int acs_observe_noalloc(int dims, const int64_t n[3], double eps, double h, int bc,
                                           int dtype, const void* d_phi, double* d_out2, void* stream) {
    if (!n || !d_phi || !d_out2 || dims < 1 || dims > 3) return ACS_E_INVAL;
    if (!std::isfinite(eps) || !std::isfinite(h) || eps < 0 || !(h > 0)) return ACS_E_INVAL;
    if (bc < 0 || bc > 2 || (dtype != ACS_F32 && dtype != ACS_F64)) return ACS_E_INVAL;
    const size_t esize = dtype == ACS_F32 ? 4 : 8;
    if (((uintptr_t)d_phi % esize) || ((uintptr_t)d_out2 % 8)) return ACS_E_INVAL;
    // the same shape limit as acs_create: at most 2^40 elements
    if (!shape_ok(dims, n)) return ACS_E_INVAL;
    int64_t nn[3] = {1, 1, 1};
    for (int k = 0; k < dims; ++k) nn[k] = n[k];
    const Geo g = make_geo(dims, nn);
    if (reduce_blocks(g) > kNoAllocParts) return ACS_E_INVAL;  // would not fit the static scratch
    RedPartial* parts = nullptr;
    if (scratch_for_current_device(&parts) != cudaSuccess) return ACS_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (dtype == ACS_F32)
        e = launch_reduce<float>(dims, bc, (const float*)d_phi, g, eps * eps, h, parts, d_out2, st);
    else
        e = launch_reduce<double>(dims, bc, (const double*)d_phi, g, eps * eps, h, parts, d_out2, st);
    return e == cudaSuccess ? ACS_OK : ACS_E_CUDA;
}
