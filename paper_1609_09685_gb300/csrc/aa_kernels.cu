// aa_kernels.cu -- the in-place pair of steps (gather step + local step) of the
// lattice Boltzmann permeability method (arXiv:1609.09685, Sec. 2), and the
// inlet/outlet bits the local step reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <utility>

#include "lbm_launch.h"
#include "lbm_stencil.cuh"

namespace lbmgb {

// ---------------------------------------------------------------------------
// In-place pair of steps (the "AA" access pattern of Bailey et al. 2009).
//
// Let R_i(x) be the slot the pull step reads for direction i at node x: the
// fluid source's slot (mirrored at a y/z face) or the node's own opposite slot
// (bounce-back; also the Zou-He unknowns, whose source lies outside).  Every
// slot is read by at most one (node, direction), and R_i(x) = (y, opp j)
// exactly when R_j(y) = (x, opp i) -- for streaming j = opp i, for bounce-back
// y = x and j = i, for the specular mirror y is the row image and j =
// opp(flip i).  Hence, on one buffer holding the post-collision state:
//   gather step: node x pulls f_i = g[R_i(x)] (the pull step's reads), relaxes,
//                and writes f*_opp(i) back into R_i(x);
//   local step:  node y reads its pre-collision f_j from its own slot opp(j),
//                relaxes, and writes f*_j into its own slot j.
// After the pair the buffer again holds the post-collision state in natural
// order, with the arithmetic of two pull steps.  No slot is touched by two
// threads, so both steps run in place, and the local step needs no neighbour
// index work at all.
// ---------------------------------------------------------------------------
namespace {

// Zou-He at the x faces (warp-uniform edge test), moments and BGK: the same
// operations as the pull kernel, producing the Q post-collision values.
template <class L, int EQ>
__device__ __forceinline__ void relax(float (&f)[L::Q], bool edge, bool xin, bool xout, float drho_in, float rho0,
                                      float om, float omm) {
    constexpr int Q = L::Q;
    if (edge) {
        float g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = f[i];
        zou_he<L, +1>(g, drho_in);
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = xin ? g[i] : f[i];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = f[i];
        zou_he<L, -1>(g, 0.f);
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = xout ? g[i] : f[i];
    }
    const float omc = __fsub_rn(1.0f, om);
    const bool trt = (omm != om);
    const float hw = __fmul_rn(0.5f, om), hwm = __fmul_rn(0.5f, omm);
    const float ow[3] = {__fmul_rn(om, (float)L::wd(0)), __fmul_rn(om, (float)L::wd(1)),
                         __fmul_rn(om, (float)L::wd(L::Q - 1))};
    const float ow3[3] = {__fmul_rn(3.0f, __fmul_rn(omm, (float)L::wd(0))),
                          __fmul_rn(3.0f, __fmul_rn(omm, (float)L::wd(1))),
                          __fmul_rn(3.0f, __fmul_rn(omm, (float)L::wd(L::Q - 1)))};
    float dr, jx, jy, jz, irho, a0, k45;
    moments<L>(f, dr, jx, jy, jz);
    eq_terms<L, EQ>(dr, jx, jy, jz, rho0, irho, a0, k45);
    const float f0 = f[0];
    float dsum = 0.f;  // sum over i != 0 of f_i - f*_i
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (opp<L>(i) < i) continue;
        const int o = opp<L>(i);
        const int cls = (L::c(i, 0) * L::c(i, 0) + L::c(i, 1) * L::c(i, 1) + L::c(i, 2) * L::c(i, 2));
        float sym, anti;
        pair_terms<L, EQ>(i, jx, jy, jz, a0, k45, ow[cls], ow3[cls], sym, anti);
        const float fi = f[i], fo = f[o];
        pair_relax(fi, fo, sym, anti, omc, hw, hwm, trt, f[i], f[o]);
        dsum = pair_dsum(dsum, fi, fo, f[i], f[o]);
    }
    f[0] = __fadd_rn(f0, dsum);  // mass balance: see the pull kernel
}

template <class L, int... Is>
__device__ __forceinline__ void src_elems(uint32_t (&e)[L::Q], const Win (&w)[L::NROW], uint32_t PS, uint32_t kd,
                                          bool ylo, bool yhi, bool zlo, bool zhi, std::integer_sequence<int, Is...>) {
    ((e[Is] = src_elem<L, Is>(w, PS, kd, Dir<Is, L>::cy > 0 ? ylo : yhi, Dir<Is, L>::cz > 0 ? zlo : zhi)), ...);
}

}  // namespace

// Rows batched per iteration of the direct-load gather step (the loads of all
// of them are in flight before the first is relaxed), register caps of the
// gather step, and minimum resident 256-thread blocks per SM of the local step.
#ifndef LBM_AA_ROWS_GATHER_2D
#define LBM_AA_ROWS_GATHER_2D 2
#endif
#ifndef LBM_AA_ROWS_GATHER_3D
#define LBM_AA_ROWS_GATHER_3D 1
#endif
#ifndef LBM_AA_GATHER_REGS_2D
#define LBM_AA_GATHER_REGS_2D 80
#endif
#ifndef LBM_AA_GATHER_REGS_3D
#define LBM_AA_GATHER_REGS_3D 96
#endif
#ifndef LBM_AA_MINB_LOCAL
#define LBM_AA_MINB_LOCAL 3
#endif

// Gather step of the pair: the pull step's reads, results written back to the
// slots read (direction opp(i) into R_i), in place on g.
template <class L, int EQ>
__device__ __forceinline__ void aa_gather_body(const HotArgs& A) {
    constexpr int Q = L::Q;
    constexpr int NZ = (L::NROW == 9) ? 3 : 1;
    constexpr int R = (L::Q == 9) ? LBM_AA_ROWS_GATHER_2D : LBM_AA_ROWS_GATHER_3D;
    const int lane = threadIdx.x & 31;
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= A.nitems) return;
    const uint4 it = __ldg(A.items + item);
    const uint32_t dom = it.y & 0xffffffu;
    const int nrows = (int)(it.y >> 24);
    const DomainDev D = A.dom[dom];
    if (!D.active) return;
    const int y0 = (int)(it.z & 0xffffu), z = (int)(it.z >> 16);
    const int x = (int)it.w * kSegW + lane;
    const uint32_t lmask = (1u << lane) - 1u;
    const uint32_t PS = A.pstride;
    const int ny = D.ny;
    const bool zlo = (z == 0), zhi = (z == D.nz - 1);
    const bool xin = (x == 0), xout = (x == D.nx - 1);
    const bool edge = (it.w == 0) || ((int)it.w == D.nseg - 1);
    float* const g = A.dst[0];
    const SegWindow* wcol = A.win + D.seg_base + it.w;
    const uint32_t rs = (uint32_t)D.nseg;
    uint32_t pbase[NZ];
#pragma unroll
    for (int zi = 0; zi < NZ; ++zi) {
        int zz = z + zi - (NZ == 3 ? 1 : 0);
        zz = zz < 0 ? 0 : (zz >= D.nz ? D.nz - 1 : zz);
        pbase[zi] = (uint32_t)zz * (uint32_t)ny;
    }
    auto rowc = [&](int yy) { return yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy); };
    constexpr bool kSlide = (NZ == 1);
    Win wm, wc, wp;
    if (kSlide) {
        wm = make_win(__ldg(wcol + (pbase[0] + rowc(y0 - 1)) * rs), lane, lmask);
        wc = make_win(__ldg(wcol + (pbase[0] + y0) * rs), lane, lmask);
    }
#pragma unroll 1
    for (int r0 = 0; r0 < nrows; r0 += R) {
        uint32_t e[R][Q];
        float f[R][Q];
        bool fl[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            // rows past the strip's end repeat its last row: the loads stay in
            // bounds and nothing is stored for them
            const int y = y0 + min(r0 + j, nrows - 1);
            Win w[L::NROW];
            if (kSlide) {
                wp = make_win(__ldg(wcol + (pbase[0] + rowc(y + 1)) * rs), lane, lmask);
                w[0] = wm;
                w[1] = wc;
                w[2] = wp;
                if (r0 + j + 1 < nrows) {
                    wm = wc;
                    wc = wp;
                }
            } else {
#pragma unroll
                for (int q = 0; q < L::NROW; ++q) {
                    const int zi = q / 3, dy = q % 3 - 1;
                    w[q] = make_win(__ldg(wcol + (pbase[zi] + rowc(y + dy)) * rs), lane, lmask);
                }
            }
            constexpr int C = (L::NROW == 9) ? 4 : 1;
            fl[j] = win_fluid<0>(w[C]) && (r0 + j < nrows);
            // a solid lane's kd is the next fluid slot (at most the padding
            // slot), so every read is in bounds; its values are discarded
            src_elems<L>(e[j], w, PS, win_idx<0>(w[C]), y == 0, y == ny - 1, zlo, zhi,
                         std::make_integer_sequence<int, Q>{});
#pragma unroll
            for (int i = 0; i < Q; ++i) f[j][i] = g[chk_load(e[j][i], (uint32_t)Q * PS, A.err)];
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            relax<L, EQ>(f[j], edge, xin, xout, D.drho_in, D.rho0, D.omega, D.omega_m);
            if (fl[j]) {
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (chk_store(e[j][opp<L>(i)], (uint32_t)Q * PS, A.err)) g[e[j][opp<L>(i)]] = f[j][i];
            }
        }
    }
}

// Window records staged per chunk of this many strip rows (a multiple of every
// row batch), or (0) read from global memory row by row.
#ifndef LBM_AA_WIN_STAGE
#define LBM_AA_WIN_STAGE 1
#endif
constexpr int kWinRows = 32;
// D3Q19: slide the windows down the strip as in 2D (1) or take all nine per
// row from the staged chunk (0, the default: sliding keeps six more windows
// live, spills at the register cap and measured 480 vs 429 us per launch on
// four 256x128x128 domains).
#ifndef LBM_AA_SLIDE_3D
#define LBM_AA_SLIDE_3D 0
#endif

// Gather step with the source slots parked in shared memory: a batch of RS
// rows keeps only its loaded values in registers, so more rows of loads are in
// flight per warp at the same register budget.
// Measured on GB300 (us per step, pair average; D2Q9 tau sweep / two D3Q19
// 256x128x128 domains): slots parked in shared memory 90.4 / 183.4 (the
// default for both lattices), slots kept in registers 95.3 / 207.9, and a
// cp.async row pipeline with the slots in registers 96.7 / 194.6 (removed).
#ifndef LBM_AA_GATHER_SMEM_2D
#define LBM_AA_GATHER_SMEM_2D 1
#endif
#ifndef LBM_AA_SMEM_ROWS_2D
#define LBM_AA_SMEM_ROWS_2D 4
#endif
#ifndef LBM_AA_GATHER_SMEM_3D
#define LBM_AA_GATHER_SMEM_3D 1
#endif
#ifndef LBM_AA_SMEM_ROWS_3D
#define LBM_AA_SMEM_ROWS_3D 2
#endif
template <class L>
struct GatherSmem {
    static constexpr bool on = (L::Q == 9) ? LBM_AA_GATHER_SMEM_2D : LBM_AA_GATHER_SMEM_3D;
    static constexpr int rows = (L::Q == 9) ? LBM_AA_SMEM_ROWS_2D : LBM_AA_SMEM_ROWS_3D;
};
// Population loads of the step kernels: through L1 by default; CG = true
// reads from L2 only, for a kernel whose blocks read what other blocks of the
// same launch wrote (the fused pair below).
template <bool CG>
__device__ __forceinline__ float ld_pop(const float* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}
template <bool CG, class T>
__device__ __forceinline__ T ld_pop_vec(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Population stores: plain, or (HINT) with an L2 evict-last policy so that a
// fused pair's gather results stay in L2 until its local step rewrites them.
#ifndef LBM_FUSED_L2HINT
#define LBM_FUSED_L2HINT 1
#endif
#ifndef LBM_FUSED_LOCAL_VEC
#define LBM_FUSED_LOCAL_VEC 2
#endif
template <bool HINT>
__device__ __forceinline__ void st_pop(float* p, float v) {
    if constexpr (HINT) {
        uint64_t pol;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(pol));
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;\n" ::"l"(p), "f"(v), "l"(pol) : "memory");
    } else {
        *p = v;
    }
}

// One strip work item of the gather step, by warp `wid` of the block (its
// slice of the dynamic shared memory).
template <class L, int EQ, int RS, bool CG, bool FUSED = false>
__device__ __forceinline__ void aa_gather_strip(const HotArgs& A, uint32_t item, int wid) {
    constexpr int Q = L::Q;
    constexpr int NZ = (L::NROW == 9) ? 3 : 1;
    extern __shared__ uint32_t sme[];
    const int lane = threadIdx.x & 31;
    const uint4 it = __ldg(A.items + item);
    const uint32_t dom = it.y & 0xffffffu;
    const int nrows = (int)(it.y >> 24);
    const DomainDev D = A.dom[dom];
    if (!D.active) return;
    const int y0 = (int)(it.z & 0xffffu), z = (int)(it.z >> 16);
    const int x = (int)it.w * kSegW + lane;
    const uint32_t lmask = (1u << lane) - 1u;
    const uint32_t PS = A.pstride;
    const int ny = D.ny;
    const bool zlo = (z == 0), zhi = (z == D.nz - 1);
    const bool xin = (x == 0), xout = (x == D.nx - 1);
    const bool edge = (it.w == 0) || ((int)it.w == D.nseg - 1);
    float* const g = A.dst[0];
    volatile uint32_t* const we = sme + (size_t)wid * RS * Q * 32 + lane;
    const SegWindow* wcol = A.win + D.seg_base + it.w;
    const uint32_t rs = (uint32_t)D.nseg;
    uint32_t pbase[NZ];
#pragma unroll
    for (int zi = 0; zi < NZ; ++zi) {
        int zz = z + zi - (NZ == 3 ? 1 : 0);
        zz = zz < 0 ? 0 : (zz >= D.nz ? D.nz - 1 : zz);
        pbase[zi] = (uint32_t)zz * (uint32_t)ny;
    }
    auto rowc = [&](int yy) { return yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy); };
    // Window records of a chunk of kWinRows rows (and the rows on either
    // side, in every plane the strip pulls from), staged in shared memory by
    // one load per lane, so that a batch's source loads do not wait on its
    // own window loads.  rw(zi, y) = the window of row y (clamped) in plane zi.
    constexpr int KW = kWinRows;
    const uint4* const wst = reinterpret_cast<const uint4*>(sme + (size_t)(blockDim.x >> 5) * RS * Q * 32) +
                             (size_t)wid * NZ * (KW + 2);
    auto stage = [&](int c) {  // rows y0 + c - 1 .. of the chunk starting at strip row c
        __syncwarp();
        const int nr = min(KW, nrows - c) + 2;
        uint4* const dst = const_cast<uint4*>(wst);
        for (int t = lane; t < NZ * nr; t += 32) {
            const int zi = t / nr, r = t - zi * nr;
            int zz = z + zi - (NZ == 3 ? 1 : 0);  // (not pbase[zi]: a runtime index would put it in local memory)
            zz = zz < 0 ? 0 : (zz >= D.nz ? D.nz - 1 : zz);
            dst[zi * (KW + 2) + r] = __ldg(wcol + ((uint32_t)zz * (uint32_t)ny + rowc(y0 + c - 1 + r)) * rs);
        }
        __syncwarp();
    };
    if (LBM_AA_WIN_STAGE) stage(0);
    // window of row y in plane zi; ybase = y0 + (first strip row of the staged chunk) - 1
    auto win_of = [&](int zi, int y, int ybase) {
        return LBM_AA_WIN_STAGE ? wst[zi * (KW + 2) + (y - ybase)] : __ldg(wcol + (pbase[zi] + rowc(y)) * rs);
    };
    // 2D (and 3D with LBM_AA_SLIDE_3D): windows slide down the strip, rows
    // y - 1 and y of every plane carry over and only row y + 1 is read per row
    constexpr bool kSlide = (NZ == 1) || LBM_AA_SLIDE_3D;
    Win wm[NZ], wc[NZ], wp[NZ];
    if (kSlide) {
#pragma unroll
        for (int zi = 0; zi < NZ; ++zi) {
            wm[zi] = make_win(win_of(zi, y0 - 1, y0 - 1), lane, lmask);
            wc[zi] = make_win(win_of(zi, y0, y0 - 1), lane, lmask);
        }
    }
#pragma unroll 1
    for (int r0 = 0; r0 < nrows; r0 += RS) {
        if (LBM_AA_WIN_STAGE && r0 > 0 && r0 % KW == 0) stage(r0);
        const int ybase = y0 + (r0 / KW) * KW - 1;
        float f[RS][Q];
        uint32_t flb = 0u;
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            // rows past the strip's end repeat its last row: the loads stay in
            // bounds and nothing is stored for them
            const int y = y0 + min(r0 + j, nrows - 1);
            Win w[L::NROW];
            if (kSlide) {
#pragma unroll
                for (int zi = 0; zi < NZ; ++zi) {
                    wp[zi] = make_win(win_of(zi, y + 1, ybase), lane, lmask);
                    w[3 * zi] = wm[zi];
                    w[3 * zi + 1] = wc[zi];
                    w[3 * zi + 2] = wp[zi];
                    if (r0 + j + 1 < nrows) {
                        wm[zi] = wc[zi];
                        wc[zi] = wp[zi];
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < L::NROW; ++q) {
                    const int zi = q / 3, dy = q % 3 - 1;
                    w[q] = make_win(win_of(zi, y + dy, ybase), lane, lmask);
                }
            }
            constexpr int C = (L::NROW == 9) ? 4 : 1;
            if (win_fluid<0>(w[C]) && (r0 + j < nrows)) flb |= 1u << j;
            // a solid lane's kd is the next fluid slot (at most the padding
            // slot), so every read is in bounds; its values are discarded
            uint32_t e[Q];
            src_elems<L>(e, w, PS, win_idx<0>(w[C]), y == 0, y == ny - 1, zlo, zhi,
                         std::make_integer_sequence<int, Q>{});
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[j][i] = ld_pop<CG>(g + chk_load(e[i], (uint32_t)Q * PS, A.err));
                we[(j * Q + i) * 32] = e[i];
            }
        }
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            relax<L, EQ>(f[j], edge, xin, xout, D.drho_in, D.rho0, D.omega, D.omega_m);
            if ((flb >> j) & 1u) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const uint32_t e = we[(j * Q + opp<L>(i)) * 32];
                    if (chk_store(e, (uint32_t)Q * PS, A.err)) st_pop<FUSED && LBM_FUSED_L2HINT>(g + e, f[j][i]);
                }
            }
        }
    }
}
template <class L, int EQ, int RS>
__device__ __forceinline__ void aa_gather_smem_body(const HotArgs& A) {
    const int wid = threadIdx.x >> 5;
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + wid;
    if (item >= A.nitems) return;
    aa_gather_strip<L, EQ, RS, false>(A, item, wid);
}
template <class L>
constexpr size_t gather_smem_bytes(int threads, int rs) {
    constexpr int NZ = (L::NROW == 9) ? 3 : 1;
    return GatherSmem<L>::on ? (size_t)(threads / 32) * ((size_t)rs * L::Q * 32 * sizeof(uint32_t) +
                                                         (LBM_AA_WIN_STAGE ? (size_t)NZ * (kWinRows + 2) * 16 : 0))
                             : 0;
}

// RS: rows of loads a warp keeps in flight (the "gather batch" of a launch
// configuration); 0 selects the default of the lattice.
template <class L, int EQ, int RS>
__global__ void __maxnreg__(LBM_AA_GATHER_REGS_2D) k_aa_gather2(const __grid_constant__ HotArgs A) {
    if constexpr (GatherSmem<L>::on) aa_gather_smem_body<L, EQ, RS>(A);
    else aa_gather_body<L, EQ>(A);
}
template <class L, int EQ, int RS>
__global__ void __maxnreg__(LBM_AA_GATHER_REGS_3D) k_aa_gather3(const __grid_constant__ HotArgs A) {
    if constexpr (GatherSmem<L>::on) aa_gather_smem_body<L, EQ, RS>(A);
    else aa_gather_body<L, EQ>(A);
}

// ---------------------------------------------------------------------------
// Staged gather step.  The gather step above is latency-bound: its loads
// depend on the neighbour windows, and the registers that hold loads in
// flight limit how many rows a warp can batch.  Here the loads go through the
// bulk-copy engine instead.  A block walks a list of tiles (GatherTile: up to
// TR rows x kTileSegs segment columns of one domain) with a ring of S
// shared-memory stages:
//   - one producer warp copies, for each tile, the tile record, the domain
//     record, the window records of its source rows and the compact range of
//     every source row in every plane the tile pulls from (cp.async.bulk,
//     completion counted in bytes on the stage's `full` mbarrier); it refills
//     a stage once every consumer has released it (`empty` mbarrier);
//   - kTileSegs consumer warps, one per segment column, relax the tile's nodes
//     from shared memory and write each result straight back to the global
//     slot it came from (the in-place rule of the pair), then release the
//     stage.
// A slot a tile uses is read and written only by its own node, so copying
// whole ranges is safe: slots of other tiles that come along are never used.
//
// Slot layout of a stage (2D): the row above the tile (q = 0) holds the planes
// of the c_y = +1 directions, the row below (q = nrows + 1) those of c_y = -1,
// each in slot I - Imin of its class; every tile row holds all Q planes.  A row
// above or below the domain is the specular image of the face row: its slots
// hold the face row's ranges of the y-flipped planes, so the compute needs no
// face logic to find a source, only the window of the clamped row.
// ---------------------------------------------------------------------------
namespace staged {

constexpr int TW = kTileSegs;
constexpr int RANGE = TW * 32 + 8;  // floats per (row, plane) slot
constexpr uint32_t RB = RANGE * 4;  // bytes per slot
constexpr int HDR = (int)(sizeof(DomainDev) + sizeof(GatherTile));  // domain and tile records

template <class L>
struct Cls;
template <>
struct Cls<D2Q9> {
    // directions of the row above (c_y = +1) and below (c_y = -1)
    static constexpr int up0 = find_dir<D2Q9>(0, 1, 0), up1 = find_dir<D2Q9>(1, 1, 0), up2 = find_dir<D2Q9>(-1, 1, 0);
    static constexpr int dn0 = find_dir<D2Q9>(0, -1, 0), dn1 = find_dir<D2Q9>(1, -1, 0),
                         dn2 = find_dir<D2Q9>(-1, -1, 0);
    static constexpr int up_min = 2, dn_min = 4, span = 5;
};
static_assert(Cls<D2Q9>::up0 == 2 && Cls<D2Q9>::up1 == 5 && Cls<D2Q9>::up2 == 6, "D2Q9 order");
static_assert(Cls<D2Q9>::dn0 == 4 && Cls<D2Q9>::dn1 == 8 && Cls<D2Q9>::dn2 == 7, "D2Q9 order");

template <int TR, int S>
struct Geo2 {
    static constexpr int NQ = TR + 2;
    static constexpr int SLOTS = 9 * TR + 2 * Cls<D2Q9>::span;
    static constexpr int WIN = HDR;                         // window records: NQ x TW uint4
    static constexpr int RNG = HDR + NQ * TW * 16;          // slots
    static constexpr int STAGE = RNG + SLOTS * (int)RB;     // bytes per stage
    static constexpr int BARS = S * STAGE;                  // S full, then S empty mbarriers
    static constexpr int SMEM = BARS + 16 * S;
    // first slot of source row q (slot I - Imin for the halo rows)
    __host__ __device__ static constexpr int slot0(int q, int nrows) {
        return q == 0 ? -Cls<D2Q9>::up_min
                      : (q <= nrows ? Cls<D2Q9>::span + 9 * (q - 1) : Cls<D2Q9>::span + 9 * TR - Cls<D2Q9>::dn_min);
    }
};
static_assert(HDR % 16 == 0 && Geo2<4, 2>::STAGE % 16 == 0 && RB % 16 == 0, "16-byte aligned stages and slots");

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait: false if the phase has not completed after kWaitTries polls
// (each poll may suspend the thread for a short, hardware-defined time).
constexpr int kWaitTries = 1 << 20;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int i = 0; i < kWaitTries; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}
// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of
// 16), completing `bytes` of the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// What the producer needs of a tile, loaded one tile ahead.
struct TileRegs {
    uint32_t dom, yz, shape, dims, wbase, live;
    uint32_t a0[kTileRowsMax + 2], n16[kTileRowsMax + 2];
};
__device__ __forceinline__ void load_tile(const HotArgs& A, uint32_t t, TileRegs& R) {
    const GatherTile* T = A.tiles + t;
    R.dom = __ldg(&T->dom);
    R.yz = __ldg(&T->yz);
    R.shape = __ldg(&T->shape);
    R.dims = __ldg(&T->dims);
    R.wbase = __ldg(&T->wbase);
#pragma unroll
    for (int q = 0; q < kTileRowsMax + 2; ++q) {
        R.a0[q] = __ldg(&T->a0[q]);
        R.n16[q] = __ldg(&T->n16[q]);
    }
}

// Producer: issue the copies of tile t into a stage (every lane of the
// producer warp).  Lane 0 arms the stage's mbarrier with the byte count before
// any copy is issued.  A retired domain's tile brings only the two records.
template <int TR>
__device__ __forceinline__ void issue_tile2(const HotArgs& A, uint32_t t, const TileRegs& R, unsigned char* stage,
                                            uint32_t bar) {
    using C = Cls<D2Q9>;
    constexpr int WIN = HDR;
    constexpr int RNG_ = HDR + (TR + 2) * TW * 16;
    const int lane = threadIdx.x & 31;
    const int y0 = (int)(R.yz & 0xffffu);
    const int nrows = (int)(R.shape & 0xffu), nsegs = (int)((R.shape >> 8) & 0xffu);
    const int ny = (int)(R.dims & 0xffffu), nseg = (int)(R.dims >> 16);
    const int nq = nrows + 2;
    const uint32_t PS = A.pstride;
    const uint32_t rng = saddr(stage + RNG_);
    uint32_t total = (uint32_t)HDR;
    if (R.live) {
        total += (uint32_t)(nq * nsegs * 16);
#pragma unroll
        for (int q = 0; q < kTileRowsMax + 2; ++q)
            if (q < nq) total += ((q == 0 || q == nq - 1) ? 3u : 9u) * 16u * R.n16[q];
    }
    if (lane == 0) mbar_arrive_expect(bar, total);
    __syncwarp();
    if (lane == 0) bulk_g2s(saddr(stage), A.dom + R.dom, (uint32_t)sizeof(DomainDev), bar);
    if (lane == 1) bulk_g2s(saddr(stage + sizeof(DomainDev)), A.tiles + t, (uint32_t)sizeof(GatherTile), bar);
    if (!R.live) return;
    const float* g = A.dst[0];
    const int ncopy = nq + 3 + 9 * nrows + 3;
    for (int c = lane; c < ncopy; c += 32) {
        if (c < nq) {  // window records of source row q (clamped row)
            int yc = y0 - 1 + c;
            yc = yc < 0 ? 0 : (yc >= ny ? ny - 1 : yc);
            bulk_g2s(saddr(stage + WIN + c * TW * 16), A.win + R.wbase + (uint32_t)yc * (uint32_t)nseg,
                     (uint32_t)nsegs * 16u, bar);
            continue;
        }
        const int cc = c - nq;
        int q, plane, slot;
        if (cc < 3) {  // row above: c_y = +1 planes, y-flipped when it is the image of row 0
            q = 0;
            constexpr int f0 = flip<D2Q9>(C::up0, true, false), f1 = flip<D2Q9>(C::up1, true, false),
                          f2 = flip<D2Q9>(C::up2, true, false);
            const int I = cc == 0 ? C::up0 : (cc == 1 ? C::up1 : C::up2);
            const int fI = cc == 0 ? f0 : (cc == 1 ? f1 : f2);
            slot = Geo2<TR, 1>::slot0(0, nrows) + I;
            plane = (y0 == 0) ? fI : I;
        } else if (cc < 3 + 9 * nrows) {
            q = 1 + (cc - 3) / 9;
            plane = (cc - 3) % 9;
            slot = Geo2<TR, 1>::slot0(q, nrows) + plane;
        } else {  // row below: c_y = -1 planes
            q = nrows + 1;
            constexpr int f0 = flip<D2Q9>(C::dn0, true, false), f1 = flip<D2Q9>(C::dn1, true, false),
                          f2 = flip<D2Q9>(C::dn2, true, false);
            const int j = cc - 3 - 9 * nrows;
            const int I = j == 0 ? C::dn0 : (j == 1 ? C::dn1 : C::dn2);
            const int fI = j == 0 ? f0 : (j == 1 ? f1 : f2);
            slot = Geo2<TR, 1>::slot0(q, nrows) + I;
            plane = (y0 + nrows == ny) ? fI : I;
        }
        uint32_t n = 0, a0 = 0;
#pragma unroll
        for (int k = 0; k < kTileRowsMax + 2; ++k)
            if (k == q) {
                n = R.n16[k];
                a0 = R.a0[k];
            }
        if (n == 0) continue;
        bulk_g2s(rng + (uint32_t)slot * RB, g + (size_t)plane * PS + a0, n * 16u, bar);
    }
}

__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float ldsf(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t ldsu(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(v) : "r"(a));
    return v;
}

// Source of direction I: the global element the pull step reads (and the
// gather step writes back), and the shared-memory address of its staged copy.
// rb[r]: row bases of the source rows y - 1, y, y + 1.
template <class L, int I>
__device__ __forceinline__ void src_staged(const Win (&w)[3], uint32_t PS, uint32_t kd, bool my, const uint32_t (&rb)[3],
                                           uint32_t& e, uint32_t& sa) {
    using d = Dir<I, L>;
    const Win& wn = w[d::row];
    const bool sf = win_fluid<d::cx>(wn);
    const uint32_t k = win_idx<d::cx>(wn);
    const uint32_t plane = (d::cy != 0 && my) ? (uint32_t)d::fy : (uint32_t)I;
    e = sf ? plane * PS + k : (uint32_t)d::o * PS + kd;
    sa = sf ? rb[d::row] + (uint32_t)I * RB + 4u * k : rb[1] + (uint32_t)d::o * RB + 4u * kd;
}
template <class L, int... Is>
__device__ __forceinline__ void srcs_staged(const Win (&w)[3], uint32_t PS, uint32_t kd, bool ylo, bool yhi,
                                            const uint32_t (&rb)[3], uint32_t (&e)[L::Q], uint32_t (&sa)[L::Q],
                                            std::integer_sequence<int, Is...>) {
    (src_staged<L, Is>(w, PS, kd, Dir<Is, L>::cy > 0 ? ylo : yhi, rb, e[Is], sa[Is]), ...);
}

// Consumer warp: relax the nodes of its segment column of the staged tile.
template <class L, int EQ, int TR>
__device__ __forceinline__ void compute_tile2(const HotArgs& A, const unsigned char* stage) {
    constexpr int Q = L::Q;
    constexpr int WIN = HDR;
    constexpr int RNG_ = HDR + (TR + 2) * TW * 16;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const DomainDev& D = *reinterpret_cast<const DomainDev*>(stage);
    const GatherTile& T = *reinterpret_cast<const GatherTile*>(stage + sizeof(DomainDev));
    if (!D.active) return;
    const uint32_t shape = T.shape;
    const int nsegs = (int)((shape >> 8) & 0xffu);
    if (wid >= nsegs) return;
    const int y0 = (int)(T.yz & 0xffffu);
    const int nrows = (int)(shape & 0xffu), s0 = (int)(shape >> 16);
    const int s = s0 + wid;
    const int x = s * kSegW + lane;
    const bool xin = (x == 0), xout = (x == D.nx - 1);
    const bool edge = (s == 0) || (s == D.nseg - 1);
    const int ny = D.ny;
    const float drho_in = D.drho_in, rho0 = D.rho0, om = D.omega, omm = D.omega_m;
    const uint32_t lmask = (1u << lane) - 1u;
    const uint32_t PS = A.pstride;
    float* const g = A.dst[0];
    const uint32_t wb = saddr(stage + WIN) + (uint32_t)wid * 16u;
    const uint32_t rng = saddr(stage + RNG_);
    auto rowbase = [&](int q) {
        return rng + (uint32_t)(Geo2<TR, 1>::slot0(q, nrows) * (int)RB) - 4u * T.a0[q];
    };
    // windows and row bases of the source rows y - 1, y, y + 1, slid down the column
    Win w[3];
    uint32_t rb[3];
    w[0] = make_win(lds128(wb), lane, lmask);
    w[1] = make_win(lds128(wb + TW * 16), lane, lmask);
    rb[0] = rowbase(0);
    rb[1] = rowbase(1);
#pragma unroll 1
    for (int r = 0; r < nrows; ++r) {
        const int y = y0 + r;
        w[2] = make_win(lds128(wb + (uint32_t)((r + 2) * TW * 16)), lane, lmask);
        rb[2] = rowbase(r + 2);
        const bool fl = win_fluid<0>(w[1]);
        const uint32_t kd = win_idx<0>(w[1]);
        uint32_t e[Q], sa[Q];
        srcs_staged<L>(w, PS, kd, y == 0, y == ny - 1, rb, e, sa, std::make_integer_sequence<int, Q>{});
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = ldsf(sa[i]);
        relax<L, EQ>(f, edge, xin, xout, drho_in, rho0, om, omm);
        if (fl) {
#pragma unroll
            for (int i = 0; i < Q; ++i) g[e[opp<L>(i)]] = f[i];
        }
        w[0] = w[1];
        w[1] = w[2];
        rb[0] = rb[1];
        rb[1] = rb[2];
    }
}

}  // namespace staged

// Producer warp (the last one) and kTileSegs consumer warps; see above.
template <class L, int EQ, int TR, int S>
__global__ void __launch_bounds__((kTileSegs + 1) * 32) k_aa_gather_staged(const __grid_constant__ HotArgs A) {
    using G = staged::Geo2<TR, S>;
    extern __shared__ __align__(128) unsigned char sm_stage[];
    __shared__ int failed;
    const uint32_t full0 = staged::saddr(sm_stage + G::BARS), empty0 = full0 + 8u * S;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < S; ++s) {
            staged::mbar_init(full0 + 8u * s, 1);
            staged::mbar_init(empty0 + 8u * s, kTileSegs);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    uint32_t issued = 0, consumed = 0;
    if (wid == kTileSegs) {
        // producer: one tile ahead in registers, up to S tiles ahead in shared memory
        uint32_t t = blockIdx.x;
        staged::TileRegs cur, nxt;
        if (t < A.ntiles) {
            staged::load_tile(A, t, cur);
            cur.live = __ldg(&A.dom[cur.dom].active) != 0;
        }
#pragma unroll 1
        for (uint32_t j = 0; t < A.ntiles; ++j, t += gridDim.x) {
            const uint32_t tn = t + gridDim.x;
            if (tn < A.ntiles) staged::load_tile(A, tn, nxt);
            const int s = (int)(j % S);
            if (j >= S && !staged::mbar_wait(empty0 + 8u * s, ((j / S) - 1) & 1u)) {
                if (lane == 0) atomicOr(&failed, 1);
                break;
            }
            staged::issue_tile2<TR>(A, t, cur, sm_stage + s * G::STAGE, full0 + 8u * s);
            ++issued;
            if (tn < A.ntiles) {
                nxt.live = __ldg(&A.dom[nxt.dom].active) != 0;
                cur = nxt;
            }
        }
    } else {
#pragma unroll 1
        for (uint32_t j = 0, t = blockIdx.x; t < A.ntiles; ++j, t += gridDim.x) {
            const int s = (int)(j % S);
            if (!staged::mbar_wait(full0 + 8u * s, (j / S) & 1u)) {
                if (lane == 0) atomicOr(&failed, 1);
                break;
            }
            staged::compute_tile2<L, EQ, TR>(A, sm_stage + s * G::STAGE);
            ++consumed;
            __syncwarp();
            if (lane == 0) staged::mbar_arrive(empty0 + 8u * s);
        }
    }
    __syncthreads();
    if (failed) {
        // a copy never completed: report it and give the copies the producer
        // issued one more bounded wait before the block exits
        if (threadIdx.x == 0) atomicOr(A.err, 1u);
        if (wid == kTileSegs && lane == 0)
            for (uint32_t j = 0; j < issued; ++j) staged::mbar_wait(full0 + 8u * (j % S), (j / S) & 1u);
    }
    (void)consumed;
}

// ---------------------------------------------------------------------------
// Band gather step (D2Q9).  The direct gather step waits on scattered loads;
// the staged one above moves many short ranges.  Here a block owns a band --
// up to kBandSegs consecutive segment columns (a piece of the domain's width)
// x up to kBandRowsMax rows -- and walks down its rows with a ring of NS rows
// staged in shared memory.  Two facts keep the copies few and long:
//   - in the compact (row-major) order the fluid nodes of a row piece, with
//     the node on either side, are one contiguous range of every plane;
//   - a node of row y reads plane j only in row y - c_jy (streaming) and in
//     row y itself (bounce-back, the Zou-He unknowns, the specular image), so
//     walking down, each plane needs one new row per step, and the rows just
//     above and below the band only in the three planes that stream out of
//     them.
// A staged row is therefore nine bulk copies of one range each (three for
// the two halo rows) plus the row's window records, completing on the row's
// `full` mbarrier.  Warp w relaxes segment column s0 + w of the current row
// from shared memory and writes each result straight back to the global slot
// it came from (the in-place rule of the pair; a slot is read and written
// only by its own node, so whole ranges may be copied).  After every row the
// block synchronises and warp 0 refills the slot of the row no step needs
// any more, NS - 3 rows ahead of the rows being read.
// ---------------------------------------------------------------------------
namespace band {

using staged::bulk_g2s;
using staged::lds128;
using staged::ldsf;
using staged::mbar_arrive_expect;
using staged::mbar_init;
using staged::saddr;

// Bounded wait on an mbarrier phase.  With a suspend-time hint each poll may
// keep the thread suspended until the phase completes (up to the hint), so a
// wait costs a poll or two instead of a spin.
#ifndef LBM_BAND_WAIT_HINT_NS
#define LBM_BAND_WAIT_HINT_NS 0
#endif
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
#if LBM_BAND_WAIT_HINT_NS > 0
    for (int i = 0; i < (1 << 16); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity), "n"(LBM_BAND_WAIT_HINT_NS)
            : "memory");
        if (done) return true;
    }
    return false;
#else
    return staged::mbar_wait(bar, parity);
#endif
}

template <int S, int NS>
struct Geo {
    static constexpr int RANGE = 32 * S + 8;        // floats per (row, plane): 32 S + 2 nodes, widened to 16 B
    static constexpr uint32_t RB = RANGE * 4;       // bytes per (row, plane)
    static constexpr uint32_t WINB = 16 * S;        // window records of a row
    static constexpr uint32_t SLOT = 9 * RB + WINB; // one staged row
    static constexpr uint32_t RNGT = NS * SLOT;     // range table of the band
    static constexpr uint32_t BARS = RNGT + (kBandRowsMax + 2) * 8;
    static constexpr uint32_t SMEM = BARS + 2 * NS * 8;  // full, then empty barriers
    static_assert(RB % 16 == 0 && SLOT % 16 == 0 && RNGT % 16 == 0, "16-byte aligned ring");
};

// Planes that stream out of the row above the band (c_y = +1) and out of the
// row below it (c_y = -1).
template <class L, int... Is>
__host__ __device__ constexpr uint32_t planes_cy(int cy, std::integer_sequence<int, Is...>) {
    return ((L::c(Is, 1) == cy ? (1u << Is) : 0u) | ...);
}

// Source of direction I: the global element the pull step reads (and the
// gather step writes back), and the shared-memory address of its staged
// copy.  rb[q]: shared address of row q's plane 0 minus 4 x its first staged
// compact index (q = 0, 1, 2: rows y - 1, y, y + 1, clamped onto the domain).
template <class L, int I>
__device__ __forceinline__ void src_band(const Win (&w)[3], uint32_t PS, uint32_t RB, uint32_t kd, bool my,
                                         const uint32_t (&rb)[3], uint32_t& e, uint32_t& sa) {
    using d = Dir<I, L>;
    const Win& wn = w[d::row];
    const bool sf = win_fluid<d::cx>(wn);
    const uint32_t k = win_idx<d::cx>(wn);
    const uint32_t plane = (d::cy != 0 && my) ? (uint32_t)d::fy : (uint32_t)I;
    e = sf ? plane * PS + k : (uint32_t)d::o * PS + kd;
    sa = sf ? rb[d::row] + plane * RB + 4u * k : rb[1] + (uint32_t)d::o * RB + 4u * kd;
}
template <class L, int... Is>
__device__ __forceinline__ void srcs_band(const Win (&w)[3], uint32_t PS, uint32_t RB, uint32_t kd, bool ylo,
                                          bool yhi, const uint32_t (&rb)[3], uint32_t (&e)[L::Q],
                                          uint32_t (&sa)[L::Q], std::integer_sequence<int, Is...>) {
    (src_band<L, Is>(w, PS, RB, kd, Dir<Is, L>::cy > 0 ? ylo : yhi, rb, e[Is], sa[Is]), ...);
}

}  // namespace band

template <class L, int EQ, int S, int NS>
__global__ void __launch_bounds__((S + 1) * 32, 4) k_aa_gather_band(const __grid_constant__ HotArgs A) {
    static_assert(L::Q == 9, "the band gather step is written for D2Q9");
    static_assert(NS >= 3, "a step reads three staged rows");
    using G = band::Geo<S, NS>;
    constexpr int Q = L::Q;
    constexpr uint32_t kUp = band::planes_cy<L>(1, std::make_integer_sequence<int, Q>{});
    constexpr uint32_t kDown = band::planes_cy<L>(-1, std::make_integer_sequence<int, Q>{});
    extern __shared__ __align__(128) unsigned char smb[];
    __shared__ int failed;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint4 it = __ldg(A.bands + blockIdx.x);
    const DomainDev* Dp = A.dom + it.x;
    if (!__ldg(&Dp->active)) return;
    const int ny = __ldg(&Dp->ny), nseg = __ldg(&Dp->nseg);
    const uint32_t seg_base = __ldg(&Dp->seg_base);
    const int y0 = (int)(it.y & 0xffffu), nrows = (int)(it.y >> 16);
    const int s0 = (int)(it.z & 0xffffu), nsegs = (int)(it.z >> 16);
    const int nstage = nrows + 2;
    const uint32_t ring = band::saddr(smb), full0 = ring + G::BARS, empty0 = full0 + 8u * NS;
    uint2* const rt = reinterpret_cast<uint2*>(smb + G::RNGT);
    for (int j = threadIdx.x; j < nstage; j += blockDim.x) rt[j] = __ldg(A.band_rng + it.w + j);
    if (threadIdx.x == 0) {
        failed = 0;
        for (int k = 0; k < NS; ++k) {
            band::mbar_init(full0 + 8u * k, 1);
            band::mbar_init(empty0 + 8u * k, (uint32_t)nsegs);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const uint32_t PS = A.pstride;
    float* const g = A.dst[0];
    int issued = 0;
    if (wid == S) {
        // Producer: stage row j (row y0 - 1 + j) into slot j % NS once every
        // consumer has released the row that held it.  Lane 0 arms the slot's
        // `full` barrier with the byte count first; a row outside the domain
        // arms it with none, so its phase completes at once.
#pragma unroll 1
        for (int j = 0; j < nstage; ++j) {
            const int slot = j % NS;
            if (j >= NS) {
                // release number j / NS - 1 of the slot: row j - NS
                if (!band::mbar_wait(empty0 + 8u * slot, (uint32_t)(j / NS - 1) & 1u)) {
                    if (lane == 0) atomicOr(&failed, 1);
                    break;
                }
                // the consumers' reads of the slot come before the copy engine's writes
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            }
            const int r = y0 - 1 + j;
            const bool live = r >= 0 && r < ny;
            const uint2 rr = rt[j];
            const uint32_t pm = j == 0 ? kUp : (j == nrows + 1 ? kDown : (1u << Q) - 1u);
            const uint32_t bytes = live ? (uint32_t)__popc(pm) * rr.y * 16u + (uint32_t)nsegs * 16u : 0u;
            const uint32_t bar = full0 + 8u * slot, dst = ring + (uint32_t)slot * G::SLOT;
            if (lane == 0) band::mbar_arrive_expect(bar, bytes);
            __syncwarp();
            if (live) {
                if (lane < Q) {
                    if (((pm >> lane) & 1u) && rr.y)
                        band::bulk_g2s(dst + (uint32_t)lane * G::RB, g + (size_t)lane * PS + rr.x, rr.y * 16u, bar);
                } else if (lane == Q) {
                    band::bulk_g2s(dst + (uint32_t)Q * G::RB,
                                   A.win + seg_base + (uint32_t)r * (uint32_t)nseg + (uint32_t)s0,
                                   (uint32_t)nsegs * 16u, bar);
                }
            }
            issued = j + 1;
        }
    } else if (wid < nsegs) {
        const int nx = __ldg(&Dp->nx);
        const int s = s0 + wid;
        const int x = s * kSegW + lane;
        const bool xin = (x == 0), xout = (x == nx - 1);
        const bool edge = (s == 0) || (s == nseg - 1);
        const float drho_in = __ldg(&Dp->drho_in), rho0 = __ldg(&Dp->rho0), om = __ldg(&Dp->omega),
                    omm = __ldg(&Dp->omega_m);
        const uint32_t lmask = (1u << lane) - 1u;
        const uint32_t wofs = 9u * G::RB + (uint32_t)wid * 16u;
        // slots and full-barrier parities of rows t (sm), t + 1 (sc), t + 2 (sp)
        int sm = 0, sc = 1, sp = 2;
        uint32_t pp = 0;
        bool ok = band::mbar_wait(full0, 0) && band::mbar_wait(full0 + 8u, 0) && band::mbar_wait(full0 + 16u, 0);
        Win w[3];
        uint32_t rb[3];
        if (ok) {
            // rows y0 - 1, y0, y0 + 1, clamped onto the domain (a clamped row is row y0 itself)
            const int km = y0 == 0 ? sc : sm, kp = y0 + 1 >= ny ? sc : sp;
            const int jm = y0 == 0 ? 1 : 0, jp = y0 + 1 >= ny ? 1 : 2;
            w[0] = make_win(band::lds128(ring + (uint32_t)km * G::SLOT + wofs), lane, lmask);
            w[1] = make_win(band::lds128(ring + (uint32_t)sc * G::SLOT + wofs), lane, lmask);
            w[2] = make_win(band::lds128(ring + (uint32_t)kp * G::SLOT + wofs), lane, lmask);
            rb[0] = ring + (uint32_t)km * G::SLOT - 4u * rt[jm].x;
            rb[1] = ring + (uint32_t)sc * G::SLOT - 4u * rt[1].x;
            rb[2] = ring + (uint32_t)kp * G::SLOT - 4u * rt[jp].x;
        }
#pragma unroll 1
        for (int t = 0; t < nrows && ok; ++t) {
            const int y = y0 + t;
            const bool fl = win_fluid<0>(w[1]);
            const uint32_t kd = win_idx<0>(w[1]);
            uint32_t e[Q], sa[Q];
            band::srcs_band<L>(w, PS, G::RB, kd, y == 0, y == ny - 1, rb, e, sa, std::make_integer_sequence<int, Q>{});
            float f[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = band::ldsf(sa[i]);
            relax<L, EQ>(f, edge, xin, xout, drho_in, rho0, om, omm);
            if (fl) {
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (chk_store(e[opp<L>(i)], (uint32_t)Q * PS, A.err)) g[e[opp<L>(i)]] = f[i];
            }
            // row t is read by no later step of this warp
            __syncwarp();
            if (lane == 0) staged::mbar_arrive(empty0 + 8u * sm);
            if (t + 1 == nrows) break;
            sm = sc;
            sc = sp;
            if (++sp == NS) {
                sp = 0;
                pp ^= 1u;
            }
            // next row y + 2 (row t + 3 of the band), unless y + 1 is the domain's last row
            const int jn = t + 3;
            if (!band::mbar_wait(full0 + 8u * sp, pp)) {
                ok = false;
                if (lane == 0) atomicOr(&failed, 1);
                break;
            }
            w[0] = w[1];
            w[1] = w[2];
            rb[0] = rb[1];
            rb[1] = rb[2];
            const int kn = (y + 2 >= ny) ? sc : sp;
            w[2] = make_win(band::lds128(ring + (uint32_t)kn * G::SLOT + wofs), lane, lmask);
            rb[2] = ring + (uint32_t)kn * G::SLOT - 4u * rt[(y + 2 >= ny) ? jn - 1 : jn].x;
        }
        if (!ok && lane == 0) atomicOr(&failed, 1);
    }
    __syncthreads();
    if (failed && wid == S && lane == 0) {
        // a copy or a release never completed: report it and give the staged
        // rows still in flight one more bounded wait before the block exits
        atomicOr(A.err, 1u);
        for (int j = max(0, issued - NS); j < issued; ++j) band::mbar_wait(full0 + 8u * (j % NS), (uint32_t)(j / NS) & 1u);
    }
}

// Local step of the pair: own slots only, pre-collision f_j from slot opp(j),
// post-collision f*_j to slot j.  It needs no geometry, so it runs over the
// compact index directly: each lane takes V consecutive slots as one aligned
// vector per plane (a warp moves 32 V contiguous slots per plane), and the
// face bits select the Zou-He closure for inlet and outlet nodes.  Slots
// between domains belong to no node; they hold zero, which relaxes to zero.
#ifndef LBM_LOCAL_VEC_2D
#define LBM_LOCAL_VEC_2D 4
#endif
#ifndef LBM_LOCAL_VEC_3D
#define LBM_LOCAL_VEC_3D 2
#endif
template <class L>
struct LocalVec {
    static constexpr int value = (L::Q == 9) ? LBM_LOCAL_VEC_2D : LBM_LOCAL_VEC_3D;
};
template <int V>
struct VecT;
template <>
struct VecT<1> {
    using T = float;
    __device__ static void split(const float a, float (&o)[1]) { o[0] = a; }
    __device__ static float join(const float (&o)[1]) { return o[0]; }
};
template <>
struct VecT<4> {
    using T = float4;
    __device__ static void split(const float4 a, float (&o)[4]) {
        o[0] = a.x;
        o[1] = a.y;
        o[2] = a.z;
        o[3] = a.w;
    }
    __device__ static float4 join(const float (&o)[4]) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <>
struct VecT<2> {
    using T = float2;
    __device__ static void split(const float2 a, float (&o)[2]) {
        o[0] = a.x;
        o[1] = a.y;
    }
    __device__ static float2 join(const float (&o)[2]) { return make_float2(o[0], o[1]); }
};

// One local-step work item (32 V consecutive compact slots), by one warp, in
// passes of VV slots per lane (fewer registers for VV < V).
template <class L, int EQ, bool CG, int VV = 4>
__device__ __forceinline__ void aa_local_item(const HotArgs& A, uint32_t item) {
    constexpr int Q = L::Q;
    constexpr int VI = LocalVec<L>::value;  // slots per lane of a work item
    constexpr int V = VV < VI ? VV : VI;    // slots per lane and pass (VI / V passes)
    using VT = VecT<V>;
    using T = typename VT::T;
    const int lane = threadIdx.x & 31;
    const uint2 it = __ldg(A.vitems + item);
    const DomainDev D = A.dom[it.y];
    if (!D.active) return;
    const uint32_t PS = A.pstride;
#pragma unroll 1
    for (int pass = 0; pass < VI / V; ++pass) {
    const uint32_t k = it.x + (uint32_t)(pass * 32 * V) + (uint32_t)lane * V;
    if (k >= D.fluid_end) return;
    float* const gk = A.dst[0] + k;
    float v[Q][V];
#pragma unroll
    for (int i = 0; i < Q; ++i)
        VT::split(ld_pop_vec<CG>(reinterpret_cast<const T*>(gk + (size_t)((uint32_t)opp<L>(i) * PS))), v[i]);
    const uint32_t code = (__ldg(A.face + (k >> 4)) >> ((k & 15u) * 2u)) & ((1u << (2 * V)) - 1u);
#pragma unroll
    for (int n = 0; n < V; ++n) {
        const uint32_t c = (code >> (2 * n)) & 3u;
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = v[i][n];
        relax<L, EQ>(f, c != 0u, (c & 1u) != 0u, (c & 2u) != 0u, D.drho_in, D.rho0, D.omega, D.omega_m);
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i][n] = f[i];
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) *reinterpret_cast<T*>(gk + (size_t)((uint32_t)i * PS)) = VT::join(v[i]);
    }
}

template <class L, int EQ>
__global__ void __launch_bounds__(256, LBM_AA_MINB_LOCAL) k_aa_local(const __grid_constant__ HotArgs A) {
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= A.nvitems) return;
    aa_local_item<L, EQ, false>(A, item);
}

// ---------------------------------------------------------------------------
// Fused in-place pair (L2 blocking).  The batch's strip list is cut into
// blocks of a few MB of populations (between row groups in 2D, between z
// planes in 3D).  One persistent launch runs both steps of the pair from a
// ticket queue of work units in the order
//   G(0), G(1), L(0), G(2), L(1), ..., G(K-1), L(K-2), L(K-1)
// (G(k): gather-step units of block k, L(k): local-step units of block k),
// so a block's populations, just rewritten by its gather step, are still in
// L2 when its local step reads them: the pair reads and writes DRAM about
// once instead of twice.  A local unit of block k waits until every gather
// unit of blocks k - 1, k, k + 1 is done -- the only writers of its slots --
// on counters each gather unit increments after a fence.  Every unit it waits
// for holds an earlier ticket and waits on nothing later, so the smallest
// unfinished ticket always progresses: no deadlock, whatever the number of
// resident blocks.  Blocks read populations from L2 (ld.global.cg), never
// from a possibly stale L1 line.  A wait gives up after a bounded time, sets
// bit 2 of the device error word and ends the block.
// ---------------------------------------------------------------------------
constexpr int kFusedWaitTries = 1 << 22;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <class L, int EQ, int RS>
__device__ __forceinline__ void aa_pair_fused_body(const HotArgs& A, const PairFused& F) {
    __shared__ uint32_t s_next;
    __shared__ int s_ok;
    const int wid = threadIdx.x >> 5;
    const uint32_t W = blockDim.x >> 5;
    if (threadIdx.x == 0) s_next = atomicAdd(F.ctr, 1u);
    __syncthreads();
    uint32_t u = s_next;
#pragma unroll 1
    while (u < F.nunits) {
        const uint4 U = __ldg(F.units + u);
        __syncthreads();  // every thread has read s_next
        if (threadIdx.x == 0) s_next = atomicAdd(F.ctr, 1u);  // the next ticket, fetched during this unit
        const uint32_t k = U.x >> 1;
        if ((U.x & 1u) == 0u) {
#pragma unroll 1
            for (uint32_t i = (uint32_t)wid; i < U.z; i += W) aa_gather_strip<L, EQ, RS, false, true>(A, U.y + i, wid);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(F.ctr + 2 + k, 1u);
            }
        } else {
            if (threadIdx.x == 0) {
                int ok = 1;
                for (uint32_t b = k == 0 ? 0u : k - 1u; b <= k + 1u && b < F.nblocks && ok; ++b) {
                    const uint32_t need = __ldg(F.total + b);
                    int tries = 0;
                    while (ld_acquire_u32(F.ctr + 2 + b) < need) {
                        if (++tries > kFusedWaitTries) {
                            ok = 0;
                            atomicOr(A.err, 4u);
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;
#pragma unroll 1
            for (uint32_t i = (uint32_t)wid; i < U.z; i += W) aa_local_item<L, EQ, true, LBM_FUSED_LOCAL_VEC>(A, U.y + i);
        }
        __syncthreads();  // s_next is written
        u = s_next;
    }
}
// The register caps of the gather step (the fused pair runs its code).
template <class L, int EQ, int RS>
__global__ void __maxnreg__(LBM_AA_GATHER_REGS_2D)
    k_aa_pair_fused2(const __grid_constant__ HotArgs A, const __grid_constant__ PairFused F) {
    aa_pair_fused_body<L, EQ, RS>(A, F);
}
template <class L, int EQ, int RS>
__global__ void __maxnreg__(LBM_AA_GATHER_REGS_3D)
    k_aa_pair_fused3(const __grid_constant__ HotArgs A, const __grid_constant__ PairFused F) {
    aa_pair_fused_body<L, EQ, RS>(A, F);
}

// Face bits of the compact slots: the inlet node (x = 0) is lane 0 of a row's
// first segment, the outlet node (x = N_x - 1) lane (N_x - 1) mod 32 of its
// last one.  `face` must be zeroed first.
__global__ void k_build_face(const DomainDev* __restrict__ dom, const uint32_t* __restrict__ seg_dom,
                             uint32_t nseg_total, const uint32_t* __restrict__ seg_mask,
                             const uint32_t* __restrict__ seg_off, uint32_t* __restrict__ face) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nseg_total) return;
    const DomainDev D = dom[seg_dom[g]];
    const uint32_t s = (g - D.seg_base) % (uint32_t)D.nseg;
    const uint32_t m = seg_mask[g];
    if (s == 0 && (m & 1u)) {
        const uint32_t k = seg_off[g];
        atomicOr(face + (k >> 4), 1u << ((k & 15u) * 2u));
    }
    const uint32_t last = (uint32_t)(D.nx - 1) & 31u;
    if (s == (uint32_t)D.nseg - 1 && ((m >> last) & 1u)) {
        const uint32_t k = seg_off[g] + __popc(m & ((1u << last) - 1u));
        atomicOr(face + (k >> 4), 2u << ((k & 15u) * 2u));
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
namespace {
inline unsigned aa_blocks(uint32_t nitems, int threads) {
    const uint32_t wpb = (uint32_t)threads / 32u;
    return (unsigned)((nitems + wpb - 1) / wpb);
}
}  // namespace

// Stages of the staged gather step's ring, per tile height.
#ifndef LBM_STAGED_STAGES
#define LBM_STAGED_STAGES 3
#endif
// Staged gather step: one persistent block per resident slot (occupancy x SMs,
// found once per device), each walking the tile list with stride gridDim.x.
template <class L, int EQ, int TR>
static cudaError_t staged_launch(const HotArgs& A, cudaStream_t st) {
    static_assert(L::Q == 9, "the staged gather step is written for D2Q9");
    constexpr int S = TR <= 2 ? LBM_STAGED_STAGES + 1 : LBM_STAGED_STAGES;
    using G = staged::Geo2<TR, S>;
    if (A.ntiles == 0) return cudaSuccess;
    auto kern = k_aa_gather_staged<L, EQ, TR, S>;
    static std::atomic<int> grid_of[64];  // resident blocks on device d (0 = not yet known)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    int grid = grid_of[dev].load();
    if (grid == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (kTileSegs + 1) * 32, G::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        grid = std::max(per_sm, 1) * std::max(sms, 1);
        grid_of[dev].store(grid);
    }
    const unsigned nb = (unsigned)std::min<uint32_t>(A.ntiles, (uint32_t)grid);
    kern<<<nb, (kTileSegs + 1) * 32, G::SMEM, st>>>(A);
    return cudaGetLastError();
}

template <class L, int EQ>
static cudaError_t staged_dispatch(int rows, const HotArgs& A, cudaStream_t st) {
    if constexpr (L::Q == 9) {
        switch (rows) {
            case 1: return staged_launch<L, EQ, 1>(A, st);
            case 2: return staged_launch<L, EQ, 2>(A, st);
            case 3: return staged_launch<L, EQ, 3>(A, st);
            case 4: return staged_launch<L, EQ, 4>(A, st);
        }
    }
    return cudaErrorInvalidValue;
}

// Staged rows of the band gather step's ring (3 in use, the rest in flight).
#ifndef LBM_BAND_STAGES
#define LBM_BAND_STAGES 5
#endif
// Band gather step: one block per band.
template <class L, int EQ>
static cudaError_t band_launch(const HotArgs& A, cudaStream_t st) {
    if constexpr (L::Q != 9) {
        return cudaErrorInvalidValue;
    } else {
        using G = band::Geo<kBandSegs, LBM_BAND_STAGES>;
        if (A.nbands == 0) return cudaSuccess;
        auto kern = k_aa_gather_band<L, EQ, kBandSegs, LBM_BAND_STAGES>;
        static std::atomic<uint64_t> attr_set{0};  // bit d: attribute set on device d
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        const uint64_t bit = 1ull << (dev & 63);
        if (dev >= 64 || !(attr_set.load() & bit)) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
            if (e != cudaSuccess) return e;
            if (dev < 64) attr_set.fetch_or(bit);
        }
        kern<<<A.nbands, (kBandSegs + 1) * 32, G::SMEM, st>>>(A);
        return cudaGetLastError();
    }
}

// Row batches of the direct gather step a launch configuration may choose.
template <class L>
struct GatherBatches {
    static constexpr int lo = (L::Q == 9) ? 2 : 1, hi = (L::Q == 9) ? 4 : 2;
};

template <class L, int EQ, int RS>
static cudaError_t gather_direct_launch(int threads, const HotArgs& A, cudaStream_t st) {
    const unsigned nb = aa_blocks(A.nitems, threads);
    if (nb == 0) return cudaSuccess;
    void (*kern)(HotArgs);
    if constexpr (L::Q == 9) kern = k_aa_gather2<L, EQ, RS>;
    else kern = k_aa_gather3<L, EQ, RS>;
    const size_t sm = gather_smem_bytes<L>(threads, RS);
    if (GatherSmem<L>::on) {
        // a function attribute is per device: set it once on each
        static std::atomic<uint64_t> attr_set{0};  // bit d: set on device d (per template instance)
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        const uint64_t bit = 1ull << (dev & 63);
        if (dev >= 64 || !(attr_set.load() & bit)) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gather_smem_bytes<L>(256, RS));
            if (e != cudaSuccess) return e;
            if (dev < 64) attr_set.fetch_or(bit);
        }
    }
    kern<<<nb, threads, sm, st>>>(A);
    return cudaGetLastError();
}

template <class L, int EQ>
static cudaError_t aa_half_launch(int half, const StepLaunch& cfg, const HotArgs& A, cudaStream_t st) {
    const int threads = cfg.threads > 0 ? cfg.threads : 128;
    if (half == 0 && cfg.band_rows > 0) return band_launch<L, EQ>(A, st);
    if (half == 0 && cfg.tile_rows > 0) return staged_dispatch<L, EQ>(cfg.tile_rows, A, st);
    if (half == 0) {
        const int rs = cfg.gather_batch > 0 ? cfg.gather_batch : GatherSmem<L>::rows;
        if (rs == GatherBatches<L>::lo) return gather_direct_launch<L, EQ, GatherBatches<L>::lo>(threads, A, st);
        if (rs == GatherBatches<L>::hi) return gather_direct_launch<L, EQ, GatherBatches<L>::hi>(threads, A, st);
        return cudaErrorInvalidValue;
    }
    const unsigned nv = aa_blocks(A.nvitems, threads);
    if (nv > 0) k_aa_local<L, EQ><<<nv, threads, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_aa_half(int q, int eq, int half, HotArgs A, float* g, const StepLaunch& cfg, cudaStream_t st) {
    for (int i = 0; i < 19; ++i) {
        A.dst[i] = i < q ? g + (size_t)i * A.pstride : nullptr;
        A.src[i] = A.dst[i];
    }
    if (q == 9)
        return eq == 0 ? aa_half_launch<D2Q9, 0>(half, cfg, A, st) : aa_half_launch<D2Q9, 1>(half, cfg, A, st);
    return eq == 0 ? aa_half_launch<D3Q19, 0>(half, cfg, A, st) : aa_half_launch<D3Q19, 1>(half, cfg, A, st);
}

template <class L, int EQ>
static cudaError_t fused_launch(const StepLaunch& cfg, const HotArgs& A, const PairFused& F, cudaStream_t st) {
    constexpr int RS = GatherSmem<L>::rows;  // the default row batch
    (void)cfg;
    void (*kern)(HotArgs, PairFused);
    if constexpr (L::Q == 9) kern = k_aa_pair_fused2<L, EQ, RS>;
    else kern = k_aa_pair_fused3<L, EQ, RS>;
    const size_t sm = gather_smem_bytes<L>(128, RS);
    static std::atomic<int> grid_of[64];  // resident blocks on device d (0 = not yet known)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    int grid = grid_of[dev].load();
    if (grid == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, sm);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        grid = std::max(per_sm, 1) * std::max(sms, 1);
        grid_of[dev].store(grid);
    }
    e = cudaMemsetAsync(F.ctr, 0, sizeof(uint32_t) * (2 + (size_t)F.nblocks), st);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)std::min<uint32_t>(F.nunits, (uint32_t)grid);
    if (nb == 0) return cudaSuccess;
    kern<<<nb, 128, sm, st>>>(A, F);
    return cudaGetLastError();
}

cudaError_t launch_aa_pair_fused(int q, int eq, HotArgs A, const PairFused& F, float* g, const StepLaunch& cfg,
                                 cudaStream_t st) {
    for (int i = 0; i < 19; ++i) {
        A.dst[i] = i < q ? g + (size_t)i * A.pstride : nullptr;
        A.src[i] = A.dst[i];
    }
    if (q == 9) return eq == 0 ? fused_launch<D2Q9, 0>(cfg, A, F, st) : fused_launch<D2Q9, 1>(cfg, A, F, st);
    return eq == 0 ? fused_launch<D3Q19, 0>(cfg, A, F, st) : fused_launch<D3Q19, 1>(cfg, A, F, st);
}

cudaError_t launch_aa_pair(int q, int eq, HotArgs A, float* g, const StepLaunch& cfg, cudaStream_t st) {
    cudaError_t e = launch_aa_half(q, eq, 0, A, g, cfg, st);
    if (e != cudaSuccess) return e;
    return launch_aa_half(q, eq, 1, A, g, cfg, st);
}

int staged_gather_lattice(int q) { return q == 9; }
int band_gather_lattice(int q) { return q == 9; }

void gather_batches(int q, int* lo, int* hi, int* def) {
    *lo = q == 9 ? GatherBatches<D2Q9>::lo : GatherBatches<D3Q19>::lo;
    *hi = q == 9 ? GatherBatches<D2Q9>::hi : GatherBatches<D3Q19>::hi;
    *def = q == 9 ? GatherSmem<D2Q9>::rows : GatherSmem<D3Q19>::rows;
}

int local_step_vector(int q) { return q == 9 ? LocalVec<D2Q9>::value : LocalVec<D3Q19>::value; }

cudaError_t launch_build_face(const DomainDev* dom, const uint32_t* seg_dom, uint32_t nseg_total,
                              const uint32_t* seg_mask, const uint32_t* seg_off, uint32_t* face, cudaStream_t st) {
    if (nseg_total == 0) return cudaSuccess;
    k_build_face<<<(nseg_total + 255) / 256, 256, 0, st>>>(dom, seg_dom, nseg_total, seg_mask, seg_off, face);
    return cudaGetLastError();
}

}  // namespace lbmgb
