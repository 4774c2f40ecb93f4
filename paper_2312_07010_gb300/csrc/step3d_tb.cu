// step3d_tb.cu -- launch of the temporally blocked 3D step (tb3d.cuh), FP32.
#include "tb3d.cuh"

namespace acs {

bool step3d_tb_supported(int dtype, int depth, const Geo& g) {
    return dtype == ACS_F32 && depth >= 2 && depth <= kMaxTemporalDepth3d && g.nz > 1 && g.nx % 2 == 0 &&
           g.nx * g.ny < (int64_t(1) << 31) - 64 * g.nx && g.nz < (1 << 29);
}

// z planes per CTA: minimize (waves of resident CTAs) x (planes streamed per CTA).
static int choose_zchunk_tb(int64_t tiles, int64_t nz, int K, int resident) {
    int best = (int)nz;
    double best_cost = 1e300;
    for (int64_t zc = std::min<int64_t>(nz, 4 * K); zc <= nz; ++zc) {
        const int64_t chunks = (nz + zc - 1) / zc;
        if (chunks > 65535) continue;
        const int64_t waves = (tiles * chunks + resident - 1) / resident;
        const double cost = (double)waves * (double)(zc + 3 * K);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = (int)zc;
        }
    }
    return best;
}

template <int K>
static cudaError_t launch_tb3d_k(int bc, const float* src, float* dst, const Geo& g, const Coef<float>& c, int zch,
                                 cudaStream_t st) {
    using TB = Tb3<K>;
    const int64_t ntx = (g.nx + TB::OW - 1) / TB::OW;
    const int64_t nty = (g.ny + TB::OH - 1) / TB::OH;
    const int64_t tiles = ntx * nty;
    if (tiles > 0x7fffffff) return cudaErrorNotSupported;
    cudaError_t e = cudaSuccess;
    ACS_SOLVE_DISPATCH_UNIT(c, SV, {
        auto kern = bc == 0 ? k_step3d_tb<0, SV, K> : (bc == 1 ? k_step3d_tb<1, SV, K> : k_step3d_tb<2, SV, K>);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TB::PUB_BYTES);
        if (e == cudaSuccess && zch <= 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTb3Warps * 32, TB::PUB_BYTES);
            zch = choose_zchunk_tb(tiles, g.nz, K, std::max(1, sms * std::max(1, per_sm)));
        }
        const int64_t nzc = (g.nz + zch - 1) / zch;
        if (e == cudaSuccess && nzc > 65535) e = cudaErrorNotSupported;
        if (e == cudaSuccess)
            e = launch_pdl(kern, dim3((unsigned)tiles, (unsigned)nzc), dim3(kTb3Warps * 32), TB::PUB_BYTES, st, src,
                           dst, g, c, (int)ntx, zch);
    });
    return e;
}

template <typename T>
cudaError_t launch_step3d_tb(int bc, int depth, const T* src, T* dst, const Geo& g, const Coef<T>& c, int zch,
                             cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (depth == 2) return launch_tb3d_k<2>(bc, src, dst, g, c, zch, st);
    }
    return cudaErrorNotSupported;
}
template cudaError_t launch_step3d_tb<float>(int, int, const float*, float*, const Geo&, const Coef<float>&, int,
                                             cudaStream_t);
template cudaError_t launch_step3d_tb<double>(int, int, const double*, double*, const Geo&, const Coef<double>&, int,
                                              cudaStream_t);

}  // namespace acs
