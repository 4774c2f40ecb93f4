// step2d_tma.cu -- one RLB-MIE-FD step (Eq. IE-FD, Remark 1) on a 2D grid whose rows
// are a multiple of 16 bytes, streaming TMA-staged blocks of 8 RPT rows.
//
// A CTA owns a column of TX unknowns (128 FP32 / 64 FP64) and a run of row blocks.
// One thread issues a TMA load of each block plus a one-cell halo (the x halo widened
// to a 16-byte group) into a ring of S slots (RPT and S are the tile variant), S blocks
// ahead; each of the 256 threads owns one 16-byte vector in RPT rows and takes its x
// neighbours from its registers and warp shuffles, its y neighbours from shared
// memory.  Boundaries as in the 3D kernel: TMA zero fill for Dirichlet, per-row
// fix-ups (own value / wrapped global read) for Neumann and periodic.
#include <type_traits>

#include "acs_host.h"
#include "stream_tile.cuh"
#include "tma.cuh"

namespace acs {

template <typename T, int BC, int SOLVE, int RPT, int SS, int MODE>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && RPT == 2) ? 3 : 2)
    k_step2d_tma(const __grid_constant__ CUtensorMap tmap, const T* __restrict__ src, T* __restrict__ dst, Geo g,
                 Coef<T> c, int ybchunk, int* err, RedPartial* part) {
    pdl_wait();  // the previous step's stores are visible from here on
    using TT = Tile3<T, RPT, SS>;
    constexpr int VX = TT::VX, TX = TT::TX, TY = TT::TY, BW = TT::BW, S = TT::S;
    constexpr int SLOT_ELEMS = TT::SLOT_STRIDE / sizeof(T);
    constexpr int NP = RPT * VX;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(base);
    T* ring = reinterpret_cast<T*>(base + TT::BAR_BYTES);

    const int nx = (int)g.nx, ny = (int)g.ny;
    const int nyb = (ny + TY - 1) / TY;
    const int x0 = blockIdx.x * TX;
    const int b0 = blockIdx.y * ybchunk;
    const int b1 = min(b0 + ybchunk, nyb);
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int tid = ly * 32 + lx;
    const int xl = lx * VX;
    const int gx = x0 + xl;
    const int r0 = RPT * ly;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // block b lives in ring slot (b - b0) % S; the loop tracks the slot and the
    // mbarrier phase incrementally
    auto issue = [&](int b, int slot) {
        T* dstp = ring + (size_t)slot * SLOT_ELEMS;
        if ((smem_u32(dstp) & 127u) != 0u || (((x0 - VX) * (int)sizeof(T)) & 15) != 0) {
            atomicExch(err, 2);
            return;
        }
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[slot], TT::SLOT_BYTES);
        tma_load_2d(dstp, &tmap, &full[slot], x0 - VX, b * TY - 1);
    };
    int last_issued = min(b0 + S, b1) - 1;
    if (tid == 0)
        for (int b = b0; b <= last_issued; ++b) issue(b, b - b0);

    const int64_t sy = g.sy;
    // rows are a multiple of VX, so a thread stores its whole vector or nothing
    const bool xlo = gx == 0, xhi = gx + VX == nx;
    const bool colok = gx < nx;
    bool failed = false;
    EnergyAcc<T> eacc;
    int sc = 0;        // slot of the current block
    uint32_t pc = 0u;  // its mbarrier phase parity
    const bool edge = BC != ACS_BC_DIRICHLET && (x0 == 0 || x0 + TX >= nx || b0 * TY == 0 || b1 * TY >= ny);
    auto run = [&](auto edge_tag) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        for (int b = b0; b < b1 && !failed; ++b) {
            const bool ok = mbar_wait(&full[sc], pc);
            const T* cur = ring + (size_t)sc * SLOT_ELEMS;
            const int gy0 = b * TY + r0;
            T cz[RPT][VX], below[VX], above[VX], xi[NP];
#pragma unroll
            for (int rr = 0; rr < RPT; ++rr) Vec<T>::get(cur + (r0 + rr + 1) * BW + VX + xl, cz[rr]);
            Vec<T>::get(cur + r0 * BW + VX + xl, below);
            Vec<T>::get(cur + (r0 + RPT + 1) * BW + VX + xl, above);
            const bool bedge = EDGE && (x0 == 0 || x0 + TX >= nx || b * TY == 0 || (b + 1) * TY >= ny);
#pragma unroll
            for (int rr = 0; rr < RPT; ++rr) {
                const int gyr = gy0 + rr;
                T ym[VX], yp[VX];
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    ym[v] = rr == 0 ? below[v] : cz[rr - 1][v];
                    yp[v] = rr == RPT - 1 ? above[v] : cz[rr + 1][v];
                }
                // the tile's outer two x neighbours come from the halo group (every lane
                // reads the same word: a broadcast, no branch)
                const T hl = cur[(r0 + rr + 1) * BW + VX - 1];
                const T hr = cur[(r0 + rr + 1) * BW + VX + TX];
                const T su = __shfl_up_sync(0xffffffffu, cz[rr][VX - 1], 1);
                const T sd = __shfl_down_sync(0xffffffffu, cz[rr][0], 1);
                T left = lx == 0 ? hl : su;
                T right = lx == 31 ? hr : sd;
                if (bedge && gyr < ny) {
                    if (gyr == 0) {
                        if (BC == ACS_BC_NEUMANN) {
#pragma unroll
                            for (int v = 0; v < VX; ++v) ym[v] = cz[rr][v];
                        } else if (gx < nx) {
                            Vec<T>::ldg(src + (int64_t)(ny - 1) * sy + gx, ym);
                        }
                    }
                    if (gyr == ny - 1) {
                        if (BC == ACS_BC_NEUMANN) {
#pragma unroll
                            for (int v = 0; v < VX; ++v) yp[v] = cz[rr][v];
                        } else if (gx < nx) {
                            Vec<T>::ldg(src + gx, yp);
                        }
                    }
                    if (xlo) left = BC == ACS_BC_NEUMANN ? cz[rr][0] : src[(int64_t)gyr * sy + nx - 1];
                    if (xhi) right = BC == ACS_BC_NEUMANN ? cz[rr][VX - 1] : src[(int64_t)gyr * sy];
                }
                if (MODE == kModeEnergy) {
                    // forward links along x and y (ghost-ruled as for the step) and the
                    // links of the first unknowns to the zero Dirichlet boundary
                    if (gyr < ny && colok) {  // rows are a multiple of VX: the whole vector
                        if constexpr (std::is_same<T, float>::value) {
                            // FP32: the four points as two packed pairs
                            eacc.point2_pair(f2_make(cz[rr][0], cz[rr][1]), f2_make(cz[rr][1], cz[rr][2]),
                                             f2_make(yp[0], yp[1]));
                            eacc.point2_pair(f2_make(cz[rr][2], cz[rr][3]), f2_make(cz[rr][3], right),
                                             f2_make(yp[2], yp[3]));
                        } else {
#pragma unroll
                            for (int v = 0; v < VX; ++v) eacc.point2(cz[rr][v], v == VX - 1 ? right : cz[rr][v + 1], yp[v]);
                        }
                        if (BC == ACS_BC_DIRICHLET) {
#pragma unroll
                            for (int v = 0; v < VX; ++v) {
                                const T p = cz[rr][v];
                                if (gx + v == 0) eacc.ghost_link(p);
                                if (gyr == 0) eacc.ghost_link(p);
                            }
                        }
                    }
                    continue;
                }
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    const T xm = v == 0 ? left : cz[rr][v - 1];
                    const T xp = v == VX - 1 ? right : cz[rr][v + 1];
                    xi[rr * VX + v] = predictor(cz[rr][v], nsum(ym[v], yp[v], xm, xp), c);
                }
            }
            if (MODE == kModeEnergy) {
                eacc.plane_done();
            } else {
                T out[NP];
                roots<T, SOLVE, NP>(xi, out, c);
                T* o = dst + (int64_t)gy0 * sy + gx;
#pragma unroll
                for (int rr = 0; rr < RPT; ++rr)
                    if (colok && gy0 + rr < ny) Vec<T>::put(o + rr * sy, &out[rr * VX]);
            }
            failed = __syncthreads_or(!ok);
            // block b + S reuses block b's slot, free now that every thread is past it
            if (!failed && tid == 0 && b + S < b1) {
                issue(b + S, sc);
                last_issued = b + S;
            }
            if (++sc == S) {
                sc = 0;
                pc ^= 1u;
            }
        }
    };
    // the reduction's long loop body is kept in one copy (the fix-ups test their own
    // rows), so the instruction cache holds it; the step runs a lean copy off the faces
    if ((MODE == kModeEnergy && BC != ACS_BC_DIRICHLET) || edge) run(std::true_type());
    else run(std::false_type());
    if (MODE == kModeEnergy) energy_block_write(eacc, part + (blockIdx.y * gridDim.x + blockIdx.x));
    if (failed) {
        if (tid == 0) {
            atomicExch(err, 1);
            for (int b = max(b0, last_issued - S + 1); b <= last_issued; ++b) {
                const int k = b - b0;
                mbar_wait(&full[k % S], (uint32_t)((k / S) & 1));
            }
        }
        __syncthreads();
    }
    pdl_trigger();
}

bool step2d_tma_supported(int dtype, const Geo& g) {
    const int esize = dtype == ACS_F32 ? 4 : 8;
    return g.nz == 1 && (g.nx * esize) % 16 == 0 && g.nx < (1 << 30) && g.ny < (1 << 30);
}

template <typename T, int RPT, int SS, int MODE>
static cudaError_t launch2d_variant(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int ybchunk,
                                    int* err, RedPartial* part, int* nparts, cudaStream_t st) {
    using TT = Tile3<T, RPT, SS>;
    CUtensorMap map;
    const uint64_t dims[2] = {(uint64_t)g.nx, (uint64_t)g.ny};
    const uint32_t box[2] = {(uint32_t)TT::BW, (uint32_t)TT::BH};
    if (!encode_tensor_map(&map, sizeof(T), 2, src, dims, box)) return cudaErrorNotSupported;
    const int ntx = (int)((g.nx + TT::TX - 1) / TT::TX);
    const int nyb = (int)((g.ny + TT::TY - 1) / TT::TY);
    if (ybchunk <= 0) {
        if ((int64_t)ntx * nyb <= 152 * 6) {
            // a small grid: one block per CTA, as many CTAs as there are blocks
            ybchunk = 1;
        } else {
            // about eight CTAs per SM over the launch, at least four blocks each
            const int want = 152 * 8;
            const int chunks = std::max(1, std::min(nyb / 4 > 0 ? nyb / 4 : 1, (want + ntx - 1) / ntx));
            ybchunk = (nyb + chunks - 1) / chunks;
        }
    }
    const int nchunks = (nyb + ybchunk - 1) / ybchunk;
    if (nchunks > 65535) return cudaErrorNotSupported;
    if (MODE == kModeEnergy && (int64_t)ntx * nchunks > kMaxStreamParts) return cudaErrorNotSupported;
    if (nparts) *nparts = ntx * nchunks;
    cudaError_t e = cudaSuccess;
    ACS_SOLVE_DISPATCH(c.solve, SV, {
        auto kern = bc == 0 ? k_step2d_tma<T, 0, SV, RPT, SS, MODE>
                            : (bc == 1 ? k_step2d_tma<T, 1, SV, RPT, SS, MODE> : k_step2d_tma<T, 2, SV, RPT, SS, MODE>);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TT::SMEM);
        if (e == cudaSuccess)
            e = launch_pdl(kern, dim3((unsigned)ntx, (unsigned)nchunks), dim3(32, 8), TT::SMEM, st, map, src, dst, g,
                           c, ybchunk, err, part);
    });
    return e;
}

template <typename T>
cudaError_t launch_step2d_tma(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int variant,
                              int ybchunk, int* err, cudaStream_t st) {
    cudaError_t e = cudaErrorInvalidValue;
    ACS_TILE_VARIANT_DISPATCH(variant, RPTV, SV,
                              (e = launch2d_variant<T, RPTV, SV, kModeStep>(bc, src, dst, g, c, ybchunk, err, nullptr,
                                                                          nullptr, st)));
    return e;
}

template <typename T>
cudaError_t launch_energy2d(int bc, const T* src, const Geo& g, const Coef<T>& c, int* err, RedPartial* part,
                            int* nparts, cudaStream_t st) {
    return launch2d_variant<T, 2, 6, kModeEnergy>(bc, src, nullptr, g, c, 0, err, part, nparts, st);
}
template cudaError_t launch_energy2d<float>(int, const float*, const Geo&, const Coef<float>&, int*, RedPartial*,
                                            int*, cudaStream_t);
template cudaError_t launch_energy2d<double>(int, const double*, const Geo&, const Coef<double>&, int*, RedPartial*,
                                             int*, cudaStream_t);

template cudaError_t launch_step2d_tma<float>(int, const float*, float*, const Geo&, const Coef<float>&, int, int,
                                              int*, cudaStream_t);
template cudaError_t launch_step2d_tma<double>(int, const double*, double*, const Geo&, const Coef<double>&, int,
                                               int, int*, cudaStream_t);

}  // namespace acs
