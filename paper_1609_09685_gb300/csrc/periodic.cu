// periodic.cu -- force-driven flow with every face periodic: the 3D experiment
// of arXiv:1609.09685, Sec. 2 (permeability from Eq. 2, k = nu <u> / g).
//
// One pull step per launch over the strip work items of the pressure-driven
// kernels (same compact storage, same neighbour windows).  Differences:
//   - rows and planes wrap (no specular mirror), and the lanes at x = 0 and
//     x = N_x - 1 take their x neighbour from the other end of the source row,
//     whose fluid flag and compact slot come from that row's end segment;
//   - no Zou-He faces;
//   - BGK with the forcing of Guo, Zheng & Shi (2002): force density
//     F = rho_0 g e_x, equilibrium momentum j' = j + F/2, source
//     S_i = w_i [3 (c_i - u') . F + 9 (c_i . u')(c_i . F)] (quadratic) or
//     3 w_i c_i . F (linear), f* = f - omega (f - f_eq(j')) + (1 - omega/2) S_i;
//     the rest population from the mass balance, as in the pressure-driven
//     kernels (the forcing adds no mass);
//   - TRT (omega_m != omega): the even and odd parts of f - f_eq and of the
//     source relax with omega and omega_m (factors 1 - omega/2, 1 - omega_m/2);
//   - the observing variant sums the fluid momentum of Guo's scheme, the
//     pre-collision j_x plus F/2, into slot 0: the Eq. 2 flux.
#include <cuda_runtime.h>

#include <utility>

#include "lbm_device.cuh"
#include "lbm_launch.h"
#include "lbm_stencil.cuh"

namespace lbmgb {

namespace {

constexpr unsigned kAll = 0xffffffffu;

struct PWin {
    uint32_t tri;  // fluid flags of x - 1, x, x + 1
    uint32_t i0;   // compact slot of x - 1 (when fluid)
};

__device__ __forceinline__ PWin pwin(const uint4 r, int lane, uint32_t lmask) {
    const uint64_t W = ((uint64_t)r.y << 32) | r.x;
    PWin w;
    w.tri = (uint32_t)(W >> lane) & 7u;
    w.i0 = r.z + __popc(r.x & lmask);
    return w;
}

// Forced BGK / TRT collision of one node (Guo forcing, see above), every
// floating-point operation written out (fmaf or the __f*_rn intrinsics, never
// fused by the compiler), so that the pull step, the gather step and the
// local step relax a node to the same bits.  f: pre-collision on entry,
// post-collision on return; dr, jx, jy, jz: the node's density deviation and
// pre-collision momentum, irho = 1 / rho (for the observables).
template <class L, int EQ>
__device__ __forceinline__ void forced_relax(float (&f)[L::Q], float rho0, float F, float om, float omm, float& dr,
                                             float& jx, float& jy, float& jz, float& irho) {
    constexpr int Q = L::Q;
    moments<L>(f, dr, jx, jy, jz);
    irho = __fdividef(1.0f, __fadd_rn(rho0, dr));
    const float jsx = fmaf(0.5f, F, jx);  // equilibrium momentum j' = j + F/2
    const float ux = __fmul_rn(jsx, irho), uy = __fmul_rn(jy, irho), uz = __fmul_rn(jz, irho);
    const float jj = (L::D == 3) ? fmaf(jsx, jsx, fmaf(jy, jy, __fmul_rn(jz, jz))) : fmaf(jsx, jsx, __fmul_rn(jy, jy));
    const float omc = __fsub_rn(1.0f, om), hf = __fsub_rn(1.0f, __fmul_rn(0.5f, om));
    const float hfm = __fsub_rn(1.0f, __fmul_rn(0.5f, omm));
    const bool trt = (omm != om);
    const float uF = __fmul_rn(ux, F);
    auto eqs = [&](int i, float& eqi, float& Si) {
        const float wi = (float)L::wd(i);
        const float cj = cdot<L>(i, jsx, jy, jz);
        const float cF = L::c(i, 0) > 0 ? F : (L::c(i, 0) < 0 ? -F : 0.f);
        if (EQ == 0) {
            const float quad = fmaf(4.5f, __fmul_rn(cj, cj), __fmul_rn(-1.5f, jj));
            eqi = __fmul_rn(wi, fmaf(irho, quad, fmaf(3.0f, cj, dr)));
            const float cu = cdot<L>(i, ux, uy, uz);
            Si = __fmul_rn(wi, fmaf(9.0f, __fmul_rn(cu, cF), __fmul_rn(3.0f, __fsub_rn(cF, uF))));
        } else {
            eqi = __fmul_rn(wi, fmaf(3.0f, cj, dr));
            Si = __fmul_rn(3.0f, __fmul_rn(wi, cF));
        }
    };
    float dsum = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (opp<L>(i) < i) continue;
        const int o = opp<L>(i);
        float ei, si, eo, so;
        eqs(i, ei, si);
        eqs(o, eo, so);
        const float fi = f[i], fo = f[o];
        float oi, oo;
        if (!trt) {
            oi = fmaf(omc, fi, fmaf(om, ei, __fmul_rn(hf, si)));
            oo = fmaf(omc, fo, fmaf(om, eo, __fmul_rn(hf, so)));
        } else {
            const float fp = __fmul_rn(0.5f, __fadd_rn(fi, fo)), fm = __fmul_rn(0.5f, __fsub_rn(fi, fo));
            const float ep = __fmul_rn(0.5f, __fadd_rn(ei, eo)), em = __fmul_rn(0.5f, __fsub_rn(ei, eo));
            const float sp = __fmul_rn(0.5f, __fadd_rn(si, so)), sm = __fmul_rn(0.5f, __fsub_rn(si, so));
            const float even = fmaf(hf, sp, __fmul_rn(-om, __fsub_rn(fp, ep)));
            const float odd = fmaf(hfm, sm, __fmul_rn(-omm, __fsub_rn(fm, em)));
            oi = __fadd_rn(fi, __fadd_rn(even, odd));
            oo = __fadd_rn(fo, __fsub_rn(even, odd));
        }
        dsum = pair_dsum(dsum, fi, fo, oi, oo);
        f[i] = oi;
        f[o] = oo;
    }
    f[0] = __fadd_rn(f[0], dsum);  // mass balance
}

// Source of direction i for the lane's node (periodic pull streaming): the
// global element of the fluid source, or of the node's own opposite slot
// (bounce-back from a solid source; a solid lane's kd is the next fluid slot,
// at most the padding slot).
template <class L, int I>
__device__ __forceinline__ uint32_t psrc(const PWin (&w)[L::NROW], const uint32_t (&fl_l)[L::NROW],
                                         const uint32_t (&ix_l)[L::NROW], const uint32_t (&fl_r)[L::NROW],
                                         const uint32_t (&ix_r)[L::NROW], bool wrapl, bool wrapr, uint32_t kd,
                                         uint32_t PS) {
    constexpr int cx = L::c(I, 0);
    constexpr int q = (1 - L::c(I, 1)) + (L::NROW == 9 ? 3 * (1 - L::c(I, 2)) : 0);  // source row
    bool sf;
    uint32_t idx;
    if (cx == 0) {
        sf = (w[q].tri >> 1) & 1u;
        idx = w[q].i0 + (w[q].tri & 1u);
    } else if (cx > 0) {  // source x - 1
        sf = wrapl ? (fl_l[q] != 0u) : ((w[q].tri & 1u) != 0u);
        idx = wrapl ? ix_l[q] : w[q].i0;
    } else {  // source x + 1
        sf = wrapr ? (fl_r[q] != 0u) : (((w[q].tri >> 2) & 1u) != 0u);
        idx = wrapr ? ix_r[q] : w[q].i0 + (w[q].tri & 1u) + ((w[q].tri >> 1) & 1u);
    }
    return sf ? (uint32_t)I * PS + idx : (uint32_t)opp<L>(I) * PS + kd;
}
// The lanes at x = 0 (wrapl) and x = N_x - 1 (wrapr) take the x neighbour of
// their c_x = +1 (resp. -1) directions from the other end of each source row:
// that row's end segment gives its fluid flag and compact slot.  Applied
// after the interior rule for the two lanes only.
template <class L, int I>
__device__ __forceinline__ void pwrap(uint32_t& e, const SegWindow* wdom, int y, int z, int ny, int nz, int nseg,
                                      int lastl, bool wrapl, bool wrapr, uint32_t kd, uint32_t PS) {
    constexpr int cx = L::c(I, 0);
    if constexpr (cx != 0) {
        if ((cx > 0 && wrapl) || (cx < 0 && wrapr)) {
            const int yy = (y - L::c(I, 1) + ny) % ny, zz = (z - L::c(I, 2) + nz) % nz;
            const uint4 r = __ldg(wdom + ((uint32_t)zz * ny + (uint32_t)yy) * nseg + (cx > 0 ? nseg - 1 : 0));
            uint32_t fl, ix;
            if (cx > 0) {  // node N_x - 1 of the source row: lane lastl of its last segment
                fl = (r.w >> lastl) & 1u;
                ix = r.z + (r.x & 1u) + __popc(r.w & ((1u << lastl) - 1u));
            } else {  // node 0 of the source row: lane 0 of its first segment
                fl = r.w & 1u;
                ix = r.z + (r.x & 1u);
            }
            e = fl ? (uint32_t)I * PS + ix : (uint32_t)opp<L>(I) * PS + kd;
        }
    }
}
template <class L, int... Is>
__device__ __forceinline__ void pwraps(uint32_t (&e)[L::Q], const SegWindow* wdom, int y, int z, int ny, int nz,
                                       int nseg, int lastl, bool wrapl, bool wrapr, uint32_t kd, uint32_t PS,
                                       std::integer_sequence<int, Is...>) {
    (pwrap<L, Is>(e[Is], wdom, y, z, ny, nz, nseg, lastl, wrapl, wrapr, kd, PS), ...);
}
template <class L, int... Is>
__device__ __forceinline__ void psrcs(uint32_t (&e)[L::Q], const PWin (&w)[L::NROW], const uint32_t (&fl_l)[L::NROW],
                                      const uint32_t (&ix_l)[L::NROW], const uint32_t (&fl_r)[L::NROW],
                                      const uint32_t (&ix_r)[L::NROW], bool wrapl, bool wrapr, uint32_t kd,
                                      uint32_t PS, std::integer_sequence<int, Is...>) {
    ((e[Is] = psrc<L, Is>(w, fl_l, ix_l, fl_r, ix_r, wrapl, wrapr, kd, PS)), ...);
}

__device__ __forceinline__ float pwarp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
    return v;
}
__device__ __forceinline__ float pwarp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kAll, v, o));
    return v;
}

}  // namespace

// Pull step (OBS: the observing variant) and the gather step of an in-place
// pair (GATHER: each result written back to the slot it was read from, the
// rule of the pressure-driven pair; periodic streaming and bounce-back keep
// the pairing exact).
template <class L, int EQ, bool OBS, bool GATHER>
__device__ __forceinline__ void periodic_strip(const HotArgs& A, const float* __restrict__ gforce,
                                               float* __restrict__ uprev, double* __restrict__ partials) {
    constexpr int Q = L::Q;
    const int lane = threadIdx.x & 31;
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= A.nitems) return;
    const uint4 it = __ldg(A.items + item);
    const uint32_t dom = it.y & 0xffffffu;
    const int nrows = (int)(it.y >> 24);
    const DomainDev D = A.dom[dom];
    if (!D.active) {
        if (OBS && lane < kNumObs) partials[(size_t)item * kNumObs + lane] = 0.0;
        return;
    }
    const int y0 = (int)(it.z & 0xffffu), z = (int)(it.z >> 16);
    const int s = (int)it.w;
    const uint32_t lmask = (1u << lane) - 1u;
    const uint32_t PS = A.pstride;
    const int ny = D.ny, nz = D.nz, nseg = D.nseg;
    const int lastl = (D.nx - 1) & 31;
    const bool wrapl = (s == 0 && lane == 0);             // x = 0: its x - 1 is N_x - 1
    const bool wrapr = (s == nseg - 1 && lane == lastl);  // x = N_x - 1: its x + 1 is 0
    const float om = D.omega, omm = D.omega_m;
    const float F = __fmul_rn(gforce[dom], D.rho0);
    const float* src = A.src[0];
    float* const dst0 = A.dst[0];
    const SegWindow* wdom = A.win + D.seg_base;
    float a0s = 0.f, a1s = 0.f, a2s = 0.f, a5s = 0.f, a6s = 0.f, umax2 = 0.f;
    int nbad = 0;
#pragma unroll 1
    for (int r = 0; r < nrows; ++r) {
        const int y = y0 + r;
        PWin w[L::NROW];
#pragma unroll
        for (int q = 0; q < L::NROW; ++q) {
            const int dy = q % 3 - 1, dz = (L::NROW == 9) ? q / 3 - 1 : 0;
            const int yy = (y + dy + ny) % ny, zz = (z + dz + nz) % nz;
            w[q] = pwin(__ldg(wdom + ((uint32_t)zz * ny + (uint32_t)yy) * nseg + s), lane, lmask);
        }
        constexpr int C = (L::NROW == 9) ? 4 : 1;
        const bool fl = (w[C].tri >> 1) & 1u;
        const uint32_t kd = w[C].i0 + (w[C].tri & 1u);
        uint32_t e[Q];
        {
            const uint32_t zero[L::NROW] = {};
            psrcs<L>(e, w, zero, zero, zero, zero, false, false, kd, PS, std::make_integer_sequence<int, Q>{});
        }
        if (wrapl || wrapr)
            pwraps<L>(e, wdom, y, z, ny, nz, nseg, lastl, wrapl, wrapr, kd, PS, std::make_integer_sequence<int, Q>{});
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = src[e[i]];
        if (!fl) continue;
        float dr, jx, jy, jz, irho;
        forced_relax<L, EQ>(f, D.rho0, F, om, omm, dr, jx, jy, jz, irho);
        if (GATHER) {
#pragma unroll
            for (int i = 0; i < Q; ++i) dst0[e[opp<L>(i)]] = f[i];
            continue;
        }
        float* const dk = dst0 + kd;
#pragma unroll
        for (int i = 0; i < Q; ++i) dk[(uint32_t)i * PS] = f[i];
        if (OBS) {
            // stored post-collision momentum: j + F
            const float pux = __fmul_rn(__fadd_rn(jx, F), irho), puy = __fmul_rn(jy, irho),
                        puz = (L::D == 3) ? __fmul_rn(jz, irho) : 0.f;
            const float px = uprev[kd], py = uprev[PS + kd];
            const float pz = (L::D == 3) ? uprev[2u * PS + kd] : 0.f;
            const float ex = pux - px, ey = puy - py, ez = puz - pz;
            const float uu = pux * pux + puy * puy + puz * puz;
            a0s += fmaf(0.5f, F, jx);
            a1s += ex * ex + ey * ey + ez * ez;
            a2s += uu;
            umax2 = fmaxf(umax2, uu);
            nbad += (isfinite(pux) && isfinite(puy) && isfinite(puz)) ? 0 : 1;
            a5s += dr;
            a6s += jx;
            uprev[kd] = pux;
            uprev[PS + kd] = puy;
            if (L::D == 3) uprev[2u * PS + kd] = puz;
        }
    }
    if (OBS) {
        a0s = pwarp_sum(a0s);
        a1s = pwarp_sum(a1s);
        a2s = pwarp_sum(a2s);
        a5s = pwarp_sum(a5s);
        a6s = pwarp_sum(a6s);
        umax2 = pwarp_max(umax2);
        nbad = __reduce_add_sync(kAll, nbad);
        if (lane == 0) {
            double* p = partials + (size_t)item * kNumObs;
            p[0] = a0s;
            p[1] = a1s;
            p[2] = a2s;
            p[3] = sqrt((double)umax2);
            p[4] = (double)nbad;
            p[5] = a5s;
            p[6] = a6s;
            p[7] = 0.0;
        }
    }
}

// Minimum resident 128-thread blocks per SM of the forced pair kernels, which
// caps their registers: gather / local step in 2D (no spills at 6) and 3D
// (the gather step fits 5 without spilling; the local step stays uncapped,
// at 4, where it does not spill).
template <class L, int HALF>
struct PeriodicMinB {
    static constexpr int value = L::Q == 9 ? 6 : (HALF == 0 ? 5 : 1);
};
template <class L, int EQ, bool OBS>
__global__ void __launch_bounds__(128) k_periodic_step(const __grid_constant__ HotArgs A, const float* __restrict__ gforce,
                                                      float* __restrict__ uprev, double* __restrict__ partials) {
    periodic_strip<L, EQ, OBS, false>(A, gforce, uprev, partials);
}
template <class L, int EQ>
__global__ void __launch_bounds__(128, (PeriodicMinB<L, 0>::value)) k_periodic_gather(const __grid_constant__ HotArgs A,
                                                        const float* __restrict__ gforce) {
    periodic_strip<L, EQ, false, true>(A, gforce, nullptr, nullptr);
}

// Local step of the forced pair: each node's pre-collision f_j from its own
// slot opp(j), post-collision f*_j to slot j; one lane per compact slot over
// the local-step work items (slots between domains hold zero and stay zero:
// no force acts there, they are never read as fluid).
template <class L, int EQ>
__global__ void __launch_bounds__(128, (PeriodicMinB<L, 1>::value)) k_periodic_local(const __grid_constant__ HotArgs A,
                                                       const float* __restrict__ gforce, uint32_t span) {
    constexpr int Q = L::Q;
    const int lane = threadIdx.x & 31;
    const uint32_t witem = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (witem >= A.nvitems) return;
    const uint2 it = __ldg(A.vitems + witem);
    const DomainDev D = A.dom[it.y];
    if (!D.active) return;
    const uint32_t PS = A.pstride;
    const float F = __fmul_rn(gforce[it.y], D.rho0);
    float* const g = A.dst[0];  // a work item covers `span` slots, one per lane and pass
#pragma unroll 1
    for (uint32_t k = it.x + (uint32_t)lane; k < it.x + span; k += 32u) {
        if (k >= D.fluid_end) return;
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = g[(uint32_t)opp<L>(i) * PS + k];
        float dr, jx, jy, jz, irho;
        forced_relax<L, EQ>(f, D.rho0, F, D.omega, D.omega_m, dr, jx, jy, jz, irho);
#pragma unroll
        for (int i = 0; i < Q; ++i) g[(uint32_t)i * PS + k] = f[i];
    }
}

namespace {
template <class L, int EQ>
cudaError_t periodic_dispatch(bool obs, unsigned nb, int threads, const HotArgs& A, const float* gforce,
                              float* uprev, double* partials, cudaStream_t st) {
    if (obs) k_periodic_step<L, EQ, true><<<nb, threads, 0, st>>>(A, gforce, uprev, partials);
    else k_periodic_step<L, EQ, false><<<nb, threads, 0, st>>>(A, gforce, uprev, partials);
    return cudaGetLastError();
}
template <class L, int EQ>
cudaError_t periodic_pair_dispatch(int half, const HotArgs& A, const float* gforce, cudaStream_t st) {
    constexpr int threads = 128;
    if (half == 0) {
        const unsigned nb = (A.nitems + (threads / 32) - 1) / (threads / 32);
        if (nb) k_periodic_gather<L, EQ><<<nb, threads, 0, st>>>(A, gforce);
    } else {
        const unsigned nb = (A.nvitems + (threads / 32) - 1) / (threads / 32);
        if (nb) k_periodic_local<L, EQ><<<nb, threads, 0, st>>>(A, gforce, 32u * (uint32_t)local_step_vector(L::Q));
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_periodic_step(int q, int eq, bool obs, HotArgs A, const float* gforce, const float* src,
                                 float* dst, float* uprev, double* partials, cudaStream_t st) {
    const int threads = 128;
    for (int i = 0; i < 19; ++i) {
        A.src[i] = i < q ? src + (size_t)i * A.pstride : nullptr;
        A.dst[i] = i < q ? dst + (size_t)i * A.pstride : nullptr;
    }
    const unsigned nb = (A.nitems + (threads / 32) - 1) / (threads / 32);
    if (nb == 0) return cudaSuccess;
    if (q == 9)
        return eq == 0 ? periodic_dispatch<D2Q9, 0>(obs, nb, threads, A, gforce, uprev, partials, st)
                       : periodic_dispatch<D2Q9, 1>(obs, nb, threads, A, gforce, uprev, partials, st);
    return eq == 0 ? periodic_dispatch<D3Q19, 0>(obs, nb, threads, A, gforce, uprev, partials, st)
                   : periodic_dispatch<D3Q19, 1>(obs, nb, threads, A, gforce, uprev, partials, st);
}

cudaError_t launch_periodic_half(int q, int eq, int half, HotArgs A, const float* gforce, float* g, cudaStream_t st) {
    for (int i = 0; i < 19; ++i) {
        A.src[i] = i < q ? g + (size_t)i * A.pstride : nullptr;
        A.dst[i] = A.src[i] ? g + (size_t)i * A.pstride : nullptr;
    }
    if (q == 9)
        return eq == 0 ? periodic_pair_dispatch<D2Q9, 0>(half, A, gforce, st)
                       : periodic_pair_dispatch<D2Q9, 1>(half, A, gforce, st);
    return eq == 0 ? periodic_pair_dispatch<D3Q19, 0>(half, A, gforce, st)
                   : periodic_pair_dispatch<D3Q19, 1>(half, A, gforce, st);
}

}  // namespace lbmgb
