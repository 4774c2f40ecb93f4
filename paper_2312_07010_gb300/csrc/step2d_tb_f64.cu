// step2d_tb_f64.cu -- the FP64 instances of the temporally blocked 2D step (tb2d.cuh).
#include "tb2d.cuh"

namespace acs {

template cudaError_t launch_step2d_tb<double>(int, int, const double*, double*, const Geo&, const Coef<double>&, int,
                                              cudaStream_t);

}  // namespace acs
