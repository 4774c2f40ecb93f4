// step2d_tb.cu -- the FP32 instances of the temporally blocked 2D step (tb2d.cuh).
#include "tb2d.cuh"

namespace acs {

bool step2d_tb_supported(int dtype, int depth, const Geo& g) {
    const int esize = dtype == ACS_F32 ? 4 : 8;
    return g.nz == 1 && depth >= 2 && depth <= kMaxTemporalDepth2d && (g.nx * esize) % 16 == 0 &&
           g.nx < (1 << 29) && g.ny < (1 << 29);
}

template cudaError_t launch_step2d_tb<float>(int, int, const float*, float*, const Geo&, const Coef<float>&, int,
                                              cudaStream_t);

}  // namespace acs
