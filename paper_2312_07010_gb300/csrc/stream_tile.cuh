// stream_tile.cuh -- tile geometry and vector helpers of the TMA-streamed step
// kernels (3D: xy tiles streamed through z; 2D: x tiles streamed through row blocks).
#pragma once

#include "acs_device.cuh"

namespace acs {

template <typename T>
struct Tile3 {
    static constexpr int VX = 16 / (int)sizeof(T);  // unknowns per 16-byte vector
    static constexpr int TX = 32 * VX;              // tile width
    static constexpr int TY = 16;                   // tile height: 8 warps x 2 rows
    static constexpr int BW = TX + 2 * VX;          // box width (16-byte aligned halo)
    static constexpr int BH = TY + 2;               // box height
    static constexpr int S = 4;                     // ring slots
    static constexpr int SLOT = BW * BH;                        // values in one box
    static constexpr uint32_t SLOT_BYTES = SLOT * sizeof(T);    // bytes one TMA load writes
    // TMA tensor copies need a 128-byte aligned shared-memory destination
    static constexpr uint32_t SLOT_STRIDE = (SLOT_BYTES + 127u) / 128u * 128u;
    static constexpr uint32_t BAR_BYTES = 128;                  // S mbarriers, padded
    static constexpr size_t SMEM = 128 + BAR_BYTES + (size_t)S * SLOT_STRIDE;  // + base alignment slack
    static_assert(SLOT_STRIDE % 128 == 0 && S * sizeof(uint64_t) <= BAR_BYTES, "ring layout");
    static_assert((VX * sizeof(T)) % 16 == 0 && (BW * sizeof(T)) % 16 == 0, "16-byte TMA x granularity");
};

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using V = float4;
    static __device__ __forceinline__ void get(const float* p, float* o) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void put(float* p, const float* o) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
    static __device__ __forceinline__ void ldg(const float* p, float* o) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <>
struct Vec<double> {
    using V = double2;
    static __device__ __forceinline__ void get(const double* p, double* o) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void put(double* p, const double* o) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
    static __device__ __forceinline__ void ldg(const double* p, double* o) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
};

// z coordinate to load for logical plane p (ghost rule along z).
template <int BC>
__device__ __forceinline__ int zsrc(int p, int nz) {
    if (p >= 0 && p < nz) return p;
    if (BC == ACS_BC_PERIODIC) return p < 0 ? p + nz : p - nz;
    if (BC == ACS_BC_NEUMANN) return p < 0 ? 0 : nz - 1;
    return p;  // outside the tensor: TMA fills zeros
}

}  // namespace acs
