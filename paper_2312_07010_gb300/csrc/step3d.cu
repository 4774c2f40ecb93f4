// step3d.cu -- one RLB-MIE-FD step (Eq. IE-FD, Remark 1) on a 3D grid, streaming
// through z with TMA-staged xy planes.
//
// A CTA owns an xy tile of TX x TY unknowns (TX = 128 FP32 / 64 FP64, TY = 16) and a
// chunk of z.  One thread issues TMA loads of each z plane's tile plus a one-cell
// halo (the x halo widened to a 16-byte group so every box starts on a 16-byte
// boundary) into a ring of S shared-memory slots, S - 2 planes ahead of the
// compute.  Each of the 256 threads owns VX consecutive x (one 16-byte vector) in
// two rows: its z-1 and z values stay in registers, z+1 and the y neighbours come
// from shared memory, the x neighbours from its own registers and warp shuffles.
// Every unknown is read from HBM once per step and written once.
//
// Boundaries: along z the producer loads the plane the ghost rule names (wrapped for
// periodic, the edge plane itself for Neumann, an out-of-range plane -- TMA zero fill
// -- for Dirichlet).  Along x and y the zero fill gives Dirichlet; Neumann uses the
// point's own value and periodic reads the wrapped neighbour from global memory.
#include <type_traits>

#include "acs_host.h"
#include "stream_tile.cuh"
#include "tma.cuh"

namespace acs {

// A step that also reduces its input state (E_h, max-norm): both bodies in one pass.
constexpr int kModeStepEnergy = 2;

template <typename T, int BC, int SOLVE, int RPT, int SS, int MODE>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && RPT == 2) ? 3 : 2) k_step3d(const __grid_constant__ CUtensorMap tmap, const T* __restrict__ src,
                                                T* __restrict__ dst, Geo g, Coef<T> c, int ntx, int zchunk,
                                                int* err, RedPartial* part) {
    pdl_wait();  // the previous step's stores are visible from here on
    using TT = Tile3<T, RPT, SS>;
    constexpr int VX = TT::VX, TX = TT::TX, TY = TT::TY, BW = TT::BW, S = TT::S;
    constexpr int SLOT_ELEMS = TT::SLOT_STRIDE / sizeof(T);
    constexpr int NP = RPT * VX;  // points per thread per plane
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // align the ring to 128 bytes whatever the base alignment of dynamic shared memory
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(base);
    T* ring = reinterpret_cast<T*>(base + TT::BAR_BYTES);

    const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz;
    const int tile = blockIdx.x;
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
    const int z0 = blockIdx.y * zchunk;
    const int z1 = min(z0 + zchunk, nz);
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int tid = ly * 32 + lx;
    const int xl = lx * VX;
    const int gx = x0 + xl;
    const int r0 = RPT * ly;      // first tile row of this thread
    const int gy0 = y0 + r0;      // its grid row

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // plane p lives in ring slot (p - z0 + 1) % S; the z loop tracks the slot and the
    // mbarrier phase of the current plane incrementally
    auto slot_ptr = [&](int slot) { return ring + (size_t)slot * SLOT_ELEMS; };
    auto issue = [&](int p, int slot) {
        T* dstp = slot_ptr(slot);
        // self-check of the TMA preconditions: a misaligned destination or x offset is
        // recorded and the copy skipped (the consumers' bounded wait then reports it)
        if ((smem_u32(dstp) & 127u) != 0u || (((x0 - VX) * (int)sizeof(T)) & 15) != 0) {
            atomicExch(err, 2);
            return;
        }
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[slot], TT::SLOT_BYTES);
        tma_load_3d(dstp, &tmap, &full[slot], x0 - VX, y0 - 1, zsrc<BC>(p, nz));
    };
    // this thread's RPT rows x VX values of a plane
    auto read_mine = [&](const T* sl, T (&o)[RPT][VX]) {
#pragma unroll
        for (int rr = 0; rr < RPT; ++rr) Vec<T>::get(sl + (r0 + rr + 1) * BW + VX + xl, o[rr]);
    };

    int last_issued = min(z0 + S - 2, z1);
    if (tid == 0)
        for (int p = z0 - 1; p <= last_issued; ++p) issue(p, (p - z0 + 1) % S);

    T zm[RPT][VX], cz[RPT][VX];
    bool ok = mbar_wait(&full[0], 0u);
    read_mine(slot_ptr(0), zm);
    ok = mbar_wait(&full[1], 0u) && ok;
    read_mine(slot_ptr(1), cz);
    bool failed = __syncthreads_or(!ok);
    if (!failed && tid == 0 && z0 + S - 1 <= z1) issue(z0 + S - 1, 0);
    if (!failed) last_issued = min(z0 + S - 1, z1);
    int sc = 1;        // slot of the current plane
    uint32_t pc = 0u;  // its mbarrier phase parity

    const int64_t sy = g.sy, sz = g.sz;
    // Boundary handling hoisted out of the z loop: only a CTA whose tile touches an
    // x or y face (Neumann / periodic) runs the per-row fix-ups; Dirichlet needs none
    // (TMA zero fill), and z faces are handled by the producer's plane choice.  The
    // rows nx is a multiple of VX, so a thread stores its whole vector or nothing.
    const bool edge = BC != ACS_BC_DIRICHLET && (x0 == 0 || x0 + TX >= nx || y0 == 0 || y0 + TY >= ny);
    const bool xlo = gx == 0, xhi = gx + VX == nx;
    const bool colok = gx < nx;
    bool rowok[RPT];
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) rowok[rr] = colok && gy0 + rr < ny;
    T* o = dst + (int64_t)z0 * sz + (int64_t)gy0 * sy + gx;
    EnergyAcc<T> eacc;

    auto run = [&](auto edge_tag) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        // One plane: zm / cz / zp are this thread's values at z-1, z, z+1.
        auto plane = [&](int z, T (&zm)[RPT][VX], T (&cz)[RPT][VX], T (&zp)[RPT][VX]) {
            const int sn = sc + 1 == S ? 0 : sc + 1;
            const uint32_t pn = sc + 1 == S ? pc ^ 1u : pc;
            ok = mbar_wait(&full[sn], pn);
            read_mine(slot_ptr(sn), zp);
            const T* cur = slot_ptr(sc);
            T xi[NP];
            T below[VX], above[VX];  // rows r0 - 1 and r0 + RPT
            Vec<T>::get(cur + r0 * BW + VX + xl, below);
            Vec<T>::get(cur + (r0 + RPT + 1) * BW + VX + xl, above);
#pragma unroll
            for (int rr = 0; rr < RPT; ++rr) {
                const int gyr = gy0 + rr;
                T ym[VX], yp[VX];
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    ym[v] = rr == 0 ? below[v] : cz[rr - 1][v];
                    yp[v] = rr == RPT - 1 ? above[v] : cz[rr + 1][v];
                }
                // x neighbours across lanes; the tile's outer two come from the halo
                // group (every lane reads the same word: a broadcast, no branch)
                const T hl = cur[(r0 + rr + 1) * BW + VX - 1];
                const T hr = cur[(r0 + rr + 1) * BW + VX + TX];
                const T su = __shfl_up_sync(0xffffffffu, cz[rr][VX - 1], 1);
                const T sd = __shfl_down_sync(0xffffffffu, cz[rr][0], 1);
                T left = lx == 0 ? hl : su;
                T right = lx == 31 ? hr : sd;
                if (EDGE && gyr < ny) {
                    const int64_t rowoff = (int64_t)z * sz + (int64_t)gyr * sy;
                    if (gyr == 0) {
                        if (BC == ACS_BC_NEUMANN) {
#pragma unroll
                            for (int v = 0; v < VX; ++v) ym[v] = cz[rr][v];
                        } else if (gx < nx) {
                            Vec<T>::ldg(src + (int64_t)z * sz + (int64_t)(ny - 1) * sy + gx, ym);
                        }
                    }
                    if (gyr == ny - 1) {
                        if (BC == ACS_BC_NEUMANN) {
#pragma unroll
                            for (int v = 0; v < VX; ++v) yp[v] = cz[rr][v];
                        } else if (gx < nx) {
                            Vec<T>::ldg(src + (int64_t)z * sz + gx, yp);
                        }
                    }
                    if (xlo) left = BC == ACS_BC_NEUMANN ? cz[rr][0] : src[rowoff + nx - 1];
                    if (xhi) right = BC == ACS_BC_NEUMANN ? cz[rr][VX - 1] : src[rowoff];
                }
                if (MODE != kModeStep) {
                    // E_h and max-norm of this (input) state: the forward link of every
                    // unknown along x, y, z (ghost-ruled neighbours as for the step), plus
                    // the links of the first unknowns to the zero Dirichlet boundary
                    if (gyr < ny && colok) {  // rows are a multiple of VX: the whole vector
                        if constexpr (std::is_same<T, float>::value) {
                            // FP32: the four points as two packed pairs
                            eacc.point_pair(f2_make(cz[rr][0], cz[rr][1]), f2_make(cz[rr][1], cz[rr][2]),
                                            f2_make(yp[0], yp[1]), f2_make(zp[rr][0], zp[rr][1]));
                            eacc.point_pair(f2_make(cz[rr][2], cz[rr][3]), f2_make(cz[rr][3], right),
                                            f2_make(yp[2], yp[3]), f2_make(zp[rr][2], zp[rr][3]));
                        } else {
#pragma unroll
                            for (int v = 0; v < VX; ++v)
                                eacc.point(cz[rr][v], v == VX - 1 ? right : cz[rr][v + 1], yp[v], zp[rr][v]);
                        }
                        if (BC == ACS_BC_DIRICHLET) {
#pragma unroll
                            for (int v = 0; v < VX; ++v) {
                                const T p = cz[rr][v];
                                if (gx + v == 0) eacc.ghost_link(p);
                                if (gyr == 0) eacc.ghost_link(p);
                                if (z == 0) eacc.ghost_link(p);
                            }
                        }
                    }
                    if (MODE == kModeEnergy) continue;
                }
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    const T xm = v == 0 ? left : cz[rr][v - 1];
                    const T xp = v == VX - 1 ? right : cz[rr][v + 1];
                    const T s = nsum(zm[rr][v], zp[rr][v], ym[v], yp[v], xm, xp);
                    xi[rr * VX + v] = predictor(cz[rr][v], s, c);
                }
            }
            if (MODE != kModeStep) eacc.plane_done();
            if (MODE != kModeEnergy) {
                T out[NP];
                roots<T, SOLVE, NP>(xi, out, c);
#pragma unroll
                for (int rr = 0; rr < RPT; ++rr)
                    if (rowok[rr]) Vec<T>::put(o + rr * sy, &out[rr * VX]);
                o += sz;
            }
            failed = __syncthreads_or(!ok);
            // plane z + S reuses plane z's slot, free now that every thread is past it
            if (!failed && tid == 0 && z + S <= z1) issue(z + S, sc);
            if (!failed) last_issued = max(last_issued, min(z + S, z1));
            sc = sn;
            pc = pn;
        };

        // the three register sets rotate roles, so the loop is unrolled by three
        T zq[RPT][VX];
        int z = z0;
        for (; z + 3 <= z1 && !failed; z += 3) {
            plane(z, zm, cz, zq);
            if (failed) break;
            plane(z + 1, cz, zq, zm);
            if (failed) break;
            plane(z + 2, zq, zm, cz);
        }
        if (!failed && z < z1) {
            plane(z, zm, cz, zq);
            if (!failed && z + 1 < z1) plane(z + 1, cz, zq, zm);
        }
    };
    // the reduction's long loop body is kept in one copy (the fix-ups test their own
    // rows), so the instruction cache holds it; the step runs a lean copy off the faces
    if ((MODE != kModeStep && BC != ACS_BC_DIRICHLET) || edge) run(std::true_type());
    else run(std::false_type());

    if (MODE != kModeStep) energy_block_write(eacc, part + (blockIdx.y * gridDim.x + blockIdx.x));
    if (failed) {
        // record the timeout, then let the newest load of every slot land (bounded)
        // before the CTA's shared memory goes away
        if (tid == 0) {
            atomicExch(err, 1);
            for (int p = max(z0 - 1, last_issued - S + 1); p <= last_issued; ++p) {
                const int k = p - (z0 - 1);
                mbar_wait(&full[k % S], (uint32_t)((k / S) & 1));
            }
        }
        __syncthreads();
    }
    pdl_trigger();
}

bool step3d_supported(int dtype, const Geo& g) {
    const int esize = dtype == ACS_F32 ? 4 : 8;
    // TMA: row stride a multiple of 16 bytes; coordinates fit in int32
    return g.nz >= 1 && (g.nx * esize) % 16 == 0 && g.nx < (1 << 30) && g.ny < (1 << 30) && g.nz < (1 << 30);
}

// z planes per CTA: minimize (waves of resident CTAs) x (planes per CTA + pipeline
// fill), the launch's critical path; a chunk also re-reads its two halo planes.
static int choose_zchunk(int64_t tiles, int64_t nz, int resident) {
    int best = (int)nz;
    double best_cost = 1e300;
    for (int64_t zc = std::min<int64_t>(nz, 4); zc <= nz; ++zc) {
        const int64_t chunks = (nz + zc - 1) / zc;
        if (chunks > 65535) continue;
        const int64_t waves = (tiles * chunks + resident - 1) / resident;
        const double cost = (double)waves * (double)(zc + 3);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = (int)zc; }
    }
    return best;
}

template <typename T, int RPT, int SS, int MODE>
static cudaError_t launch3d_variant(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int zchunk,
                                    int* err, RedPartial* part, int* nparts, cudaStream_t st) {
    using TT = Tile3<T, RPT, SS>;
    CUtensorMap map;
    const uint64_t dims[3] = {(uint64_t)g.nx, (uint64_t)g.ny, (uint64_t)g.nz};
    const uint32_t box[3] = {(uint32_t)TT::BW, (uint32_t)TT::BH, 1u};
    if (!encode_tensor_map(&map, sizeof(T), 3, src, dims, box)) return cudaErrorNotSupported;
    const int ntx = (int)((g.nx + TT::TX - 1) / TT::TX);
    const int nty = (int)((g.ny + TT::TY - 1) / TT::TY);
    if ((int64_t)ntx * nty > 0x7fffffff) return cudaErrorNotSupported;
    cudaError_t e = cudaSuccess;
    ACS_SOLVE_DISPATCH(c.solve, SV, {
        auto kern = bc == 0 ? k_step3d<T, 0, SV, RPT, SS, MODE>
                            : (bc == 1 ? k_step3d<T, 1, SV, RPT, SS, MODE> : k_step3d<T, 2, SV, RPT, SS, MODE>);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TT::SMEM);
        if (e == cudaSuccess && zchunk <= 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, TT::SMEM);
            zchunk = choose_zchunk((int64_t)ntx * nty, g.nz, std::max(1, sms * std::max(1, per_sm)));
        }
        const int nzc = (int)((g.nz + zchunk - 1) / zchunk);
        if (e == cudaSuccess && nzc > 65535) e = cudaErrorNotSupported;
        if (e == cudaSuccess && MODE != kModeStep && (int64_t)ntx * nty * nzc > kMaxStreamParts)
            e = cudaErrorNotSupported;
        if (nparts) *nparts = ntx * nty * nzc;
        if (e == cudaSuccess)
            e = launch_pdl(kern, dim3((unsigned)(ntx * nty), (unsigned)nzc), dim3(32, 8), TT::SMEM, st, map, src, dst,
                           g, c, ntx, zchunk, err, part);
    });
    return e;
}

template <typename T>
cudaError_t launch_step3d(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int variant, int zchunk,
                          int* err, cudaStream_t st) {
    cudaError_t e = cudaErrorInvalidValue;
    ACS_TILE_VARIANT_DISPATCH(variant, RPTV, SV,
                              (e = launch3d_variant<T, RPTV, SV, kModeStep>(bc, src, dst, g, c, zchunk, err, nullptr,
                                                                          nullptr, st)));
    return e;
}

// E_h / max-norm of `src` with the streamed pipeline: per-CTA partials into `part`
// (at most kMaxStreamParts), their count in *nparts.
template <typename T>
cudaError_t launch_energy3d(int bc, const T* src, const Geo& g, const Coef<T>& c, int* err, RedPartial* part,
                            int* nparts, cudaStream_t st) {
    return launch3d_variant<T, 2, 6, kModeEnergy>(bc, src, nullptr, g, c, 0, err, part, nparts, st);
}
// One step src -> dst that also forms the E_h / max-norm partials of src (the step's
// own tiles and neighbours; the 4-slot tile shape whatever the context's variant).
template <typename T>
cudaError_t launch_step_energy3d(int bc, const T* src, T* dst, const Geo& g, const Coef<T>& c, int* err,
                                 RedPartial* part, int* nparts, cudaStream_t st) {
    return launch3d_variant<T, 2, 4, kModeStepEnergy>(bc, src, dst, g, c, 0, err, part, nparts, st);
}
template cudaError_t launch_step_energy3d<float>(int, const float*, float*, const Geo&, const Coef<float>&, int*,
                                                 RedPartial*, int*, cudaStream_t);
template cudaError_t launch_step_energy3d<double>(int, const double*, double*, const Geo&, const Coef<double>&,
                                                  int*, RedPartial*, int*, cudaStream_t);
template cudaError_t launch_energy3d<float>(int, const float*, const Geo&, const Coef<float>&, int*, RedPartial*,
                                            int*, cudaStream_t);
template cudaError_t launch_energy3d<double>(int, const double*, const Geo&, const Coef<double>&, int*, RedPartial*,
                                             int*, cudaStream_t);

template cudaError_t launch_step3d<float>(int, const float*, float*, const Geo&, const Coef<float>&, int, int, int*,
                                          cudaStream_t);
template cudaError_t launch_step3d<double>(int, const double*, double*, const Geo&, const Coef<double>&, int, int,
                                           int*, cudaStream_t);

}  // namespace acs
