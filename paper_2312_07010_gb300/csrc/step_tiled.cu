// step_tiled.cu -- shared-memory tiled and temporally blocked step kernels.
#include "acs_host.h"

namespace acs {

bool tiled_supported(int dims, int dtype, const Geo& g) { (void)dims; (void)dtype; (void)g; return false; }
bool temporal_supported(int dims, int dtype, int depth, const Geo& g) {
    (void)dims; (void)dtype; (void)depth; (void)g;
    return false;
}

template <typename T>
cudaError_t launch_step_tiled(int, int, const T*, T*, const Geo&, const Coef<T>&, cudaStream_t) {
    return cudaErrorNotSupported;
}
template <typename T>
cudaError_t launch_step_temporal(int, int, int, const T*, T*, const Geo&, const Coef<T>&, cudaStream_t) {
    return cudaErrorNotSupported;
}
template cudaError_t launch_step_tiled<float>(int, int, const float*, float*, const Geo&, const Coef<float>&, cudaStream_t);
template cudaError_t launch_step_tiled<double>(int, int, const double*, double*, const Geo&, const Coef<double>&, cudaStream_t);
template cudaError_t launch_step_temporal<float>(int, int, int, const float*, float*, const Geo&, const Coef<float>&, cudaStream_t);
template cudaError_t launch_step_temporal<double>(int, int, int, const double*, double*, const Geo&, const Coef<double>&, cudaStream_t);

void resolve_auto_kernel(int dims, int dtype, int bc, const Geo& g, int* kernel, int* depth) {
    (void)dims; (void)dtype; (void)bc; (void)g;
    *kernel = ACS_KERNEL_NAIVE;
    *depth = 1;
}

}  // namespace acs
