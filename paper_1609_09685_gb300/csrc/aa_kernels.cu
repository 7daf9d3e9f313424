// aa_kernels.cu -- the in-place pair of steps (gather step + local step) of the
// lattice Boltzmann permeability method (arXiv:1609.09685, Sec. 2), and the
// inlet/outlet bits the local step reads.
#include <cuda_runtime.h>

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
    const float omc = 1.0f - om;
    const bool trt = (omm != om);
    const float hw = 0.5f * om, hwm = 0.5f * omm;
    const float ow[3] = {om * (float)L::wd(0), om * (float)L::wd(1), om * (float)L::wd(L::Q - 1)};
    const float ow3[3] = {3.0f * (omm * (float)L::wd(0)), 3.0f * (omm * (float)L::wd(1)),
                          3.0f * (omm * (float)L::wd(L::Q - 1))};
    float dr, jx, jy, jz;
    moments<L>(f, dr, jx, jy, jz);
    const float irho = __fdividef(1.0f, rho0 + dr);
    const float jj = (L::D == 3) ? jx * jx + jy * jy + jz * jz : jx * jx + jy * jy;
    const float a0 = (EQ == 0) ? fmaf(-1.5f * irho, jj, dr) : dr;
    const float k45 = 4.5f * irho;
    const float f0 = f[0];
    float dsum = 0.f;  // sum over i != 0 of f_i - f*_i
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (opp<L>(i) < i) continue;
        const int o = opp<L>(i);
        const int cls = (L::c(i, 0) * L::c(i, 0) + L::c(i, 1) * L::c(i, 1) + L::c(i, 2) * L::c(i, 2));
        const float cj = cdot<L>(i, jx, jy, jz);
        const float sym = ow[cls] * ((EQ == 0) ? fmaf(k45 * cj, cj, a0) : a0);
        const float anti = ow3[cls] * cj;
        const float fi = f[i], fo = f[o];
        pair_relax(fi, fo, sym, anti, omc, hw, hwm, trt, f[i], f[o]);
        dsum += (fi - f[i]) + (fo - f[o]);
    }
    f[0] = f0 + dsum;  // mass balance: see the pull kernel
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
            for (int i = 0; i < Q; ++i) f[j][i] = g[e[j][i]];
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            relax<L, EQ>(f[j], edge, xin, xout, D.drho_in, D.rho0, D.omega, D.omega_m);
            if (fl[j]) {
#pragma unroll
                for (int i = 0; i < Q; ++i) g[e[j][opp<L>(i)]] = f[j][i];
            }
        }
    }
}

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
template <class L, int EQ, int RS>
__device__ __forceinline__ void aa_gather_smem_body(const HotArgs& A) {
    constexpr int Q = L::Q;
    constexpr int NZ = (L::NROW == 9) ? 3 : 1;
    extern __shared__ uint32_t sme[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + wid;
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
    constexpr bool kSlide = (NZ == 1);
    Win wm, wc, wp;
    if (kSlide) {
        wm = make_win(__ldg(wcol + (pbase[0] + rowc(y0 - 1)) * rs), lane, lmask);
        wc = make_win(__ldg(wcol + (pbase[0] + y0) * rs), lane, lmask);
    }
#pragma unroll 1
    for (int r0 = 0; r0 < nrows; r0 += RS) {
        float f[RS][Q];
        uint32_t flb = 0u;
#pragma unroll
        for (int j = 0; j < RS; ++j) {
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
            if (win_fluid<0>(w[C]) && (r0 + j < nrows)) flb |= 1u << j;
            // a solid lane's kd is the next fluid slot (at most the padding
            // slot), so every read is in bounds; its values are discarded
            uint32_t e[Q];
            src_elems<L>(e, w, PS, win_idx<0>(w[C]), y == 0, y == ny - 1, zlo, zhi,
                         std::make_integer_sequence<int, Q>{});
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[j][i] = g[e[i]];
                we[(j * Q + i) * 32] = e[i];
            }
        }
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            relax<L, EQ>(f[j], edge, xin, xout, D.drho_in, D.rho0, D.omega, D.omega_m);
            if ((flb >> j) & 1u) {
#pragma unroll
                for (int i = 0; i < Q; ++i) g[we[(j * Q + opp<L>(i)) * 32]] = f[j][i];
            }
        }
    }
}
template <class L>
constexpr size_t gather_smem_bytes(int threads) {
    return GatherSmem<L>::on ? (size_t)(threads / 32) * GatherSmem<L>::rows * L::Q * 32 * sizeof(uint32_t) : 0;
}

template <class L, int EQ>
__global__ void __maxnreg__(LBM_AA_GATHER_REGS_2D) k_aa_gather2(const __grid_constant__ HotArgs A) {
    if constexpr (GatherSmem<L>::on) aa_gather_smem_body<L, EQ, GatherSmem<L>::rows>(A);
    else aa_gather_body<L, EQ>(A);
}
template <class L, int EQ>
__global__ void __maxnreg__(LBM_AA_GATHER_REGS_3D) k_aa_gather3(const __grid_constant__ HotArgs A) {
    if constexpr (GatherSmem<L>::on) aa_gather_smem_body<L, EQ, GatherSmem<L>::rows>(A);
    else aa_gather_body<L, EQ>(A);
}

// Local step of the pair: own slots only, pre-collision f_j from slot opp(j),
// post-collision f*_j to slot j.  It needs no geometry, so it runs over the
// compact index directly: each lane takes V consecutive slots as one aligned
// vector per plane (a warp moves 32 V contiguous slots per plane), and the
// face bits select the Zou-He closure for inlet and outlet nodes.  Slots
// between domains belong to no node; they hold zero, which relaxes to zero.
template <class L>
struct LocalVec {
    static constexpr int value = (L::Q == 9) ? 4 : 2;
};
template <int V>
struct VecT;
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

template <class L, int EQ>
__global__ void __launch_bounds__(256, LBM_AA_MINB_LOCAL) k_aa_local(const __grid_constant__ HotArgs A) {
    constexpr int Q = L::Q;
    constexpr int V = LocalVec<L>::value;
    using VT = VecT<V>;
    using T = typename VT::T;
    const int lane = threadIdx.x & 31;
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= A.nvitems) return;
    const uint2 it = __ldg(A.vitems + item);
    const DomainDev D = A.dom[it.y];
    if (!D.active) return;
    const uint32_t k = it.x + (uint32_t)lane * V;
    if (k >= D.fluid_end) return;
    const uint32_t PS = A.pstride;
    float* const gk = A.dst[0] + k;
    float v[Q][V];
#pragma unroll
    for (int i = 0; i < Q; ++i) VT::split(*reinterpret_cast<const T*>(gk + (size_t)((uint32_t)opp<L>(i) * PS)), v[i]);
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

template <class L, int EQ>
static cudaError_t aa_half_launch(int half, int threads, const HotArgs& A, cudaStream_t st) {
    if (half == 0) {
        const unsigned nb = aa_blocks(A.nitems, threads);
        if (nb == 0) return cudaSuccess;
        void (*kern)(HotArgs);
        if constexpr (L::Q == 9) kern = k_aa_gather2<L, EQ>;
        else kern = k_aa_gather3<L, EQ>;
        const size_t sm = gather_smem_bytes<L>(threads);
        if (GatherSmem<L>::on) {
            // a function attribute is per device: set it once on each
            static std::atomic<uint64_t> attr_set{0};  // bit d: set on device d (per template instance)
            int dev = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return e;
            const uint64_t bit = 1ull << (dev & 63);
            if (dev >= 64 || !(attr_set.load() & bit)) {
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gather_smem_bytes<L>(256));
                if (e != cudaSuccess) return e;
                if (dev < 64) attr_set.fetch_or(bit);
            }
        }
        kern<<<nb, threads, sm, st>>>(A);
        return cudaGetLastError();
    }
    const unsigned nv = aa_blocks(A.nvitems, threads);
    if (nv > 0) k_aa_local<L, EQ><<<nv, threads, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_aa_half(int q, int eq, int half, HotArgs A, float* g, int threads, cudaStream_t st) {
    if (threads <= 0) threads = 128;
    for (int i = 0; i < 19; ++i) {
        A.dst[i] = i < q ? g + (size_t)i * A.pstride : nullptr;
        A.src[i] = A.dst[i];
    }
    if (q == 9)
        return eq == 0 ? aa_half_launch<D2Q9, 0>(half, threads, A, st) : aa_half_launch<D2Q9, 1>(half, threads, A, st);
    return eq == 0 ? aa_half_launch<D3Q19, 0>(half, threads, A, st) : aa_half_launch<D3Q19, 1>(half, threads, A, st);
}

cudaError_t launch_aa_pair(int q, int eq, HotArgs A, float* g, int threads, cudaStream_t st) {
    cudaError_t e = launch_aa_half(q, eq, 0, A, g, threads, st);
    if (e != cudaSuccess) return e;
    return launch_aa_half(q, eq, 1, A, g, threads, st);
}

int local_step_vector(int q) { return q == 9 ? LocalVec<D2Q9>::value : LocalVec<D3Q19>::value; }

cudaError_t launch_build_face(const DomainDev* dom, const uint32_t* seg_dom, uint32_t nseg_total,
                              const uint32_t* seg_mask, const uint32_t* seg_off, uint32_t* face, cudaStream_t st) {
    if (nseg_total == 0) return cudaSuccess;
    k_build_face<<<(nseg_total + 255) / 256, 256, 0, st>>>(dom, seg_dom, nseg_total, seg_mask, seg_off, face);
    return cudaGetLastError();
}

}  // namespace lbmgb
