// lbm_stencil.cuh -- device helpers shared by the pull kernel (lbm_kernels.cu)
// and the in-place pair kernels (aa_kernels.cu): neighbour windows, source
// slots, Zou-He, moments, the collision of an opposite pair, cp.async.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "lbm_device.cuh"

// Checked build (-DLBM_CHECKED): every population index the step kernels take
// from the index tables (windows) is compared with the extent of the buffer it
// addresses.  An index outside is not used -- a load reads element 0 instead,
// a store is skipped -- and bit 1 of the device error word is set, which the
// next observation reports as LBM_ERR_INTERNAL.  The regular build compiles
// the checks away.
namespace lbmgb {

namespace {

__device__ __forceinline__ uint32_t chk_load(uint32_t e, uint32_t lim, uint32_t* err) {
#ifdef LBM_CHECKED
    if (e < lim) return e;
    atomicOr(err, 2u);
    return 0u;
#else
    (void)lim;
    (void)err;
    return e;
#endif
}
__device__ __forceinline__ bool chk_store(uint32_t e, uint32_t lim, uint32_t* err) {
#ifdef LBM_CHECKED
    if (e < lim) return true;
    atomicOr(err, 2u);
    return false;
#else
    (void)e;
    (void)lim;
    (void)err;
    return true;
#endif
}

constexpr unsigned kFull = 0xffffffffu;

struct SegLoc {
    int s, y, z, x;
};

__device__ __forceinline__ SegLoc locate(const DomainDev& D, uint32_t gseg, int lane) {
    const uint32_t local = gseg - D.seg_base;
    const uint32_t nseg = (uint32_t)D.nseg;
    SegLoc L;
    L.s = (int)(local % nseg);
    const uint32_t row = local / nseg;
    L.y = (int)(row % (uint32_t)D.ny);
    L.z = (int)(row / (uint32_t)D.ny);
    L.x = L.s * kSegW + lane;
    return L;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Zou-He pressure closure in shifted form for the face whose inward normal is
// `SIDE` (+1 at x = 0, -1 at x = N_x - 1), u_y = u_z = 0:
//   rho u_x = side * (drho_b - (S_0 + 2 S_in)),  S_0 = sum over c_x = 0,
//   S_in = sum over the known directions c_x = -side,
//   N_a = 1/2 sum_{c_x = 0} c_a g (transverse momentum of the c_x = 0 set),
//   g_i = g_opp(i) + side 6 w_i rho u_x - c_iy N_y - c_iz N_z  for c_ix = side.
// Written generically; in 2D it reduces to Zou & He (1997), in 3D to the
// Hecht & Harting (2010) form.  The shifted weights cancel because the c_x = 0
// weights plus twice the c_x = -side weights sum to one.
//
// Every floating-point operation of the collision helpers below is written
// out (fmaf, or the __f*_rn intrinsics, which the compiler never fuses), so
// that a node relaxed by any kernel -- pull step, gather step (direct or
// staged), local step -- gets the same bits from the same populations.
template <class L, int SIDE>
__device__ __forceinline__ void zou_he(float (&f)[L::Q], float drho_b) {
    float s0 = 0.f, sin = 0.f, ny = 0.f, nz = 0.f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        if (L::c(i, 0) == 0) {
            s0 = __fadd_rn(s0, f[i]);
            if (L::c(i, 1) > 0) ny = __fadd_rn(ny, f[i]);
            if (L::c(i, 1) < 0) ny = __fsub_rn(ny, f[i]);
            if (L::c(i, 2) > 0) nz = __fadd_rn(nz, f[i]);
            if (L::c(i, 2) < 0) nz = __fsub_rn(nz, f[i]);
        } else if (L::c(i, 0) == -SIDE) {
            sin = __fadd_rn(sin, f[i]);
        }
    }
    const float r = __fsub_rn(drho_b, __fadd_rn(s0, __fmul_rn(2.f, sin)));
    const float rux = SIDE > 0 ? r : -r;
    ny = __fmul_rn(0.5f, ny);
    nz = __fmul_rn(0.5f, nz);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        if (L::c(i, 0) == SIDE) {
            const float sw6 = (float)(SIDE * 6.0 * L::wd(i));
            float t = fmaf(sw6, rux, f[opp<L>(i)]);
            if (L::c(i, 1) > 0) t = __fsub_rn(t, ny);
            if (L::c(i, 1) < 0) t = __fadd_rn(t, ny);
            if (L::c(i, 2) > 0) t = __fsub_rn(t, nz);
            if (L::c(i, 2) < 0) t = __fadd_rn(t, nz);
            f[i] = t;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Fused stream + boundaries + BGK collide; OBS adds the per-interval FP64
// reductions (flux, residual terms, max |u|, non-finite count, mass).
//
// A warp walks one strip (consecutive rows of one segment column).  For each
// row it reads the neighbour window of every row it pulls from (the row above,
// its own, the row below; in 3D also the planes in front and behind).  Lane l
// shifts the 34-bit window by l: bits 0, 1, 2 are the fluid flags of the
// sources at x - 1, x, x + 1, i.e. for c_x = +1, 0, -1, and the compact index
// of the c_x = +1 source is the window base plus a popcount below lane l.
// ---------------------------------------------------------------------------
namespace {

struct Win {
    uint32_t tri;  // fluid flags of nodes x - 1, x, x + 1 in the window's row
    uint32_t i0;   // compact index of node x - 1 (valid when that node is fluid)
};

__device__ __forceinline__ Win make_win(const uint4 r, int lane, uint32_t lmask) {
    const uint64_t W = ((uint64_t)r.y << 32) | r.x;
    Win w;
    w.tri = (uint32_t)(W >> lane) & 7u;
    w.i0 = r.z + __popc(r.x & lmask);
    return w;
}
template <int CX>
__device__ __forceinline__ uint32_t win_idx(const Win& w) {
    return CX == 1 ? w.i0 : (CX == 0 ? w.i0 + (w.tri & 1u) : w.i0 + (w.tri & 1u) + ((w.tri >> 1) & 1u));
}
template <int CX>
__device__ __forceinline__ bool win_fluid(const Win& w) {
    return (w.tri >> (1 - CX)) & 1u;
}
// c_i . v using only the non-zero components of c_i (without fast-math the
// compiler must keep 0 * v, which is not 0 for a non-finite v).
template <class L>
__device__ __forceinline__ float cdot(int i, float vx, float vy, float vz) {
    float r = 0.f;
    if (L::c(i, 0) > 0) r = __fadd_rn(r, vx);
    if (L::c(i, 0) < 0) r = __fsub_rn(r, vx);
    if (L::c(i, 1) > 0) r = __fadd_rn(r, vy);
    if (L::c(i, 1) < 0) r = __fsub_rn(r, vy);
    if (L::c(i, 2) > 0) r = __fadd_rn(r, vz);
    if (L::c(i, 2) < 0) r = __fsub_rn(r, vz);
    return r;
}
// first moments: density deviation and the momentum components, from the
// non-zero velocity components only
template <class L>
__device__ __forceinline__ void moments(const float (&f)[L::Q], float& dr, float& jx, float& jy, float& jz) {
    dr = 0.f;
    jx = 0.f;
    jy = 0.f;
    jz = 0.f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        dr = __fadd_rn(dr, f[i]);
        if (L::c(i, 0) > 0) jx = __fadd_rn(jx, f[i]);
        if (L::c(i, 0) < 0) jx = __fsub_rn(jx, f[i]);
        if (L::c(i, 1) > 0) jy = __fadd_rn(jy, f[i]);
        if (L::c(i, 1) < 0) jy = __fsub_rn(jy, f[i]);
        if (L::c(i, 2) > 0) jz = __fadd_rn(jz, f[i]);
        if (L::c(i, 2) < 0) jz = __fsub_rn(jz, f[i]);
    }
}

// Node terms of the (shifted) equilibrium: 1/rho, a0 = drho - 1.5 |j|^2 / rho
// (quadratic) or drho (linear), and 4.5/rho.
template <class L, int EQ>
__device__ __forceinline__ void eq_terms(float dr, float jx, float jy, float jz, float rho0, float& irho, float& a0,
                                         float& k45) {
    irho = __fdividef(1.0f, __fadd_rn(rho0, dr));
    const float jj =
        (L::D == 3) ? fmaf(jx, jx, fmaf(jy, jy, __fmul_rn(jz, jz))) : fmaf(jx, jx, __fmul_rn(jy, jy));
    a0 = (EQ == 0) ? fmaf(__fmul_rn(-1.5f, irho), jj, dr) : dr;
    k45 = __fmul_rn(4.5f, irho);
}

// Even and odd equilibrium terms of the opposite pair (i, opp i):
// sym = omega w (a0 + 4.5 (c_i . j)^2 / rho), anti = omega_m 3 w (c_i . j);
// ow, ow3 are omega w and 3 omega_m w of the pair's weight class.
template <class L, int EQ>
__device__ __forceinline__ void pair_terms(int i, float jx, float jy, float jz, float a0, float k45, float ow,
                                           float ow3, float& sym, float& anti) {
    const float cj = cdot<L>(i, jx, jy, jz);
    sym = __fmul_rn(ow, (EQ == 0) ? fmaf(__fmul_rn(k45, cj), cj, a0) : a0);
    anti = __fmul_rn(ow3, cj);
}

// Post-collision values of the opposite pair (i, opp i) from the pair's even
// and odd equilibrium terms sym = omega w (even part of f_eq - w rho_0) and
// anti = omega_m 3 w (c_i . j).  BGK (omega_m == omega, warp-uniform per
// domain): f* = (1 - omega) f + sym +- anti.  TRT (Ginzburg 2005): the even
// part (f_i + f_o)/2 relaxes with omega, the odd part (f_i - f_o)/2 with
// omega_m; hw = omega/2, hwm = omega_m/2.
__device__ __forceinline__ void pair_relax(float fi, float fo, float sym, float anti, float omc, float hw,
                                           float hwm, bool trt, float& oi, float& oo) {
    if (!trt) {
        oi = fmaf(omc, fi, __fadd_rn(sym, anti));
        oo = fmaf(omc, fo, __fsub_rn(sym, anti));
    } else {
        const float hp = __fmul_rn(hw, __fadd_rn(fi, fo)), hm = __fmul_rn(hwm, __fsub_rn(fi, fo));
        oi = __fadd_rn(__fsub_rn(__fsub_rn(fi, hp), hm), __fadd_rn(sym, anti));
        oo = __fadd_rn(__fadd_rn(__fsub_rn(fo, hp), hm), __fsub_rn(sym, anti));
    }
}
// Running sum of f_i - f*_i over the pairs, for the mass-balanced rest
// population f*_0 = f_0 + sum_{i != 0} (f_i - f*_i).
__device__ __forceinline__ float pair_dsum(float dsum, float fi, float fo, float oi, float oo) {
    return __fadd_rn(dsum, __fadd_rn(__fsub_rn(fi, oi), __fsub_rn(fo, oo)));
}

template <int I, class L>
struct Dir {
    static constexpr int cx = L::c(I, 0), cy = L::c(I, 1), cz = L::c(I, 2);
    static constexpr int o = opp<L>(I);
    static constexpr int fy = flip<L>(I, true, false), fz = flip<L>(I, false, true),
                         fyz = flip<L>(I, true, true);
    static constexpr int row = (1 - cy) + (L::NROW == 9 ? 3 * (1 - cz) : 0);
};

// Source element of direction I for the node of window set w (pull
// streaming): the fluid source's compact slot in the (possibly mirrored)
// direction plane, or the node's own opposite slot when the source is solid
// (bounce-back).  Plane offsets are compile-time multiples of the uniform
// plane stride, so they stay in uniform registers.
template <class L, int I>
__device__ __forceinline__ uint32_t src_elem(const Win (&w)[L::NROW], uint32_t PS, uint32_t kd, bool my, bool mz) {
    using d = Dir<I, L>;
    const Win& wn = w[d::row];
    const bool sf = win_fluid<d::cx>(wn);
    uint32_t plane = (uint32_t)I * PS;
    if (d::cy != 0 && d::cz != 0)
        plane = my ? (mz ? (uint32_t)d::fyz * PS : (uint32_t)d::fy * PS) : (mz ? (uint32_t)d::fz * PS : plane);
    else if (d::cy != 0) plane = my ? (uint32_t)d::fy * PS : plane;
    else if (d::cz != 0) plane = mz ? (uint32_t)d::fz * PS : plane;
    return sf ? plane + win_idx<d::cx>(wn) : (uint32_t)d::o * PS + kd;
}

// Bit i set when the pull source of direction i is fluid.  The destination of
// direction i is the source of opp(i), so bit opp(i) tells whether a
// post-collision population in direction i reaches a fluid node.
template <class L, int... Is>
__device__ __forceinline__ uint32_t src_fluid_mask(const Win (&w)[L::NROW], std::integer_sequence<int, Is...>) {
    return ((win_fluid<Dir<Is, L>::cx>(w[Dir<Is, L>::row]) ? (1u << Is) : 0u) | ...);
}

__device__ __forceinline__ void cp_async4(uint32_t saddr, const float* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Issue the Q source loads of one row into shared-memory stage `sbase`
// (slot (i, lane) at sbase + 4 (32 i + lane)).  For a solid lane kd is the
// slot of the next fluid node (at most the padding slot nfluid < pstride), so
// every address is in bounds; the value is discarded.
template <class L, int... Is>
__device__ __forceinline__ void issue_row(const float* __restrict__ src, uint32_t PS, const Win (&w)[L::NROW],
                                          uint32_t kd, bool ylo, bool yhi, bool zlo, bool zhi, uint32_t sbase,
                                          uint32_t* err, std::integer_sequence<int, Is...>) {
    // a direction with c_y = +1 pulls from row y - 1, mirrored when y = 0, etc.
    (void)err;
    (cp_async4(sbase + 4u * (32u * Is),
               src + chk_load(src_elem<L, Is>(w, PS, kd, Dir<Is, L>::cy > 0 ? ylo : yhi,
                                                  Dir<Is, L>::cz > 0 ? zlo : zhi),
                                  (uint32_t)L::Q * PS, err)),
     ...);
}

}  // namespace

}  // namespace lbmgb
