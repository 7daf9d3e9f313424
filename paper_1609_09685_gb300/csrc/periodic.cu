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

template <class L>
__device__ __forceinline__ void pmoments(const float (&f)[L::Q], float& dr, float& jx, float& jy, float& jz) {
    dr = jx = jy = jz = 0.f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        dr += f[i];
        if (L::c(i, 0) > 0) jx += f[i];
        if (L::c(i, 0) < 0) jx -= f[i];
        if (L::c(i, 1) > 0) jy += f[i];
        if (L::c(i, 1) < 0) jy -= f[i];
        if (L::c(i, 2) > 0) jz += f[i];
        if (L::c(i, 2) < 0) jz -= f[i];
    }
}

template <class L>
__device__ __forceinline__ float pdot(int i, float vx, float vy, float vz) {
    float r = 0.f;
    if (L::c(i, 0) > 0) r += vx;
    if (L::c(i, 0) < 0) r -= vx;
    if (L::c(i, 1) > 0) r += vy;
    if (L::c(i, 1) < 0) r -= vy;
    if (L::c(i, 2) > 0) r += vz;
    if (L::c(i, 2) < 0) r -= vz;
    return r;
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

template <class L, int EQ, bool OBS>
__global__ void __launch_bounds__(128) k_periodic_step(const __grid_constant__ HotArgs A, const float* __restrict__ gforce,
                                                      float* __restrict__ uprev, double* __restrict__ partials) {
    constexpr int Q = L::Q;
    constexpr int NZ = (L::NROW == 9) ? 3 : 1;
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
    const int x = s * kSegW + lane;
    const uint32_t lmask = (1u << lane) - 1u;
    const uint32_t PS = A.pstride;
    const int ny = D.ny, nz = D.nz, nseg = D.nseg;
    const int lastl = (D.nx - 1) & 31;
    const bool wrapl = (s == 0 && lane == 0);                     // x = 0: its x - 1 is N_x - 1
    const bool wrapr = (s == nseg - 1 && lane == lastl);          // x = N_x - 1: its x + 1 is 0
    const float om = D.omega, omc = 1.0f - om, hf = 1.0f - 0.5f * om;
    const float omm = D.omega_m, hfm = 1.0f - 0.5f * omm;
    const bool trt = (omm != om);
    const float F = gforce[dom] * D.rho0;
    const float* src = A.src[0];
    float* const dst0 = A.dst[0];
    const SegWindow* wdom = A.win + D.seg_base;
    auto rec = [&](int zz, int yy, int ss) { return __ldg(wdom + ((uint32_t)zz * ny + (uint32_t)yy) * nseg + ss); };
    float a0s = 0.f, a1s = 0.f, a2s = 0.f, a5s = 0.f, a6s = 0.f, umax2 = 0.f;
    int nbad = 0;
#pragma unroll 1
    for (int r = 0; r < nrows; ++r) {
        const int y = y0 + r;
        PWin w[L::NROW];
        uint32_t fl_l[L::NROW], ix_l[L::NROW], fl_r[L::NROW], ix_r[L::NROW];
#pragma unroll
        for (int q = 0; q < L::NROW; ++q) {
            const int dy = q % 3 - 1, dz = (NZ == 3) ? q / 3 - 1 : 0;
            const int yy = (y + dy + ny) % ny, zz = (z + dz + nz) % nz;
            w[q] = pwin(rec(zz, yy, s), lane, lmask);
            fl_l[q] = ix_l[q] = fl_r[q] = ix_r[q] = 0u;
            if (wrapl) {  // node N_x - 1 of the source row: lane lastl of its last segment
                const uint4 e = rec(zz, yy, nseg - 1);
                fl_l[q] = (e.w >> lastl) & 1u;
                ix_l[q] = e.z + (e.x & 1u) + __popc(e.w & ((1u << lastl) - 1u));
            }
            if (wrapr) {  // node 0 of the source row: lane 0 of its first segment
                const uint4 e = rec(zz, yy, 0);
                fl_r[q] = e.w & 1u;
                ix_r[q] = e.z + (e.x & 1u);
            }
        }
        constexpr int C = (L::NROW == 9) ? 4 : 1;
        const bool fl = (w[C].tri >> 1) & 1u;
        const uint32_t kd = w[C].i0 + (w[C].tri & 1u);
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0);
            const int q = (1 - L::c(i, 1)) + (L::NROW == 9 ? 3 * (1 - L::c(i, 2)) : 0);  // source row
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
            // solid source: halfway bounce-back from the node's own opposite slot;
            // a solid lane's kd is the next fluid slot (at most the padding slot)
            f[i] = sf ? src[(uint32_t)i * PS + idx] : src[(uint32_t)opp<L>(i) * PS + kd];
        }
        if (!fl) continue;
        float dr, jx, jy, jz;
        pmoments<L>(f, dr, jx, jy, jz);
        const float rho = D.rho0 + dr;
        const float irho = __fdividef(1.0f, rho);
        const float jsx = jx + 0.5f * F;  // equilibrium momentum j' = j + F/2
        const float ux = jsx * irho, uy = jy * irho, uz = jz * irho;
        const float jj = jsx * jsx + jy * jy + jz * jz;
        float dsum = 0.f;
        float* const dk = dst0 + kd;
        auto eqs = [&](int i, float& eqi, float& Si) {
            const float wi = (float)L::wd(i);
            const float cj = pdot<L>(i, jsx, jy, jz);
            const float cF = (float)L::c(i, 0) * F;
            if (EQ == 0) {
                eqi = wi * (dr + 3.0f * cj + irho * (4.5f * cj * cj - 1.5f * jj));
                const float cu = pdot<L>(i, ux, uy, uz);
                Si = wi * (3.0f * (cF - ux * F) + 9.0f * cu * cF);
            } else {
                eqi = wi * (dr + 3.0f * cj);
                Si = 3.0f * wi * cF;
            }
        };
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (opp<L>(i) < i) continue;
            const int o = opp<L>(i);
            float ei, si, eo, so;
            eqs(i, ei, si);
            eqs(o, eo, so);
            float oi, oo;
            if (!trt) {
                oi = fmaf(omc, f[i], fmaf(om, ei, hf * si));
                oo = fmaf(omc, f[o], fmaf(om, eo, hf * so));
            } else {
                const float fp = 0.5f * (f[i] + f[o]), fm = 0.5f * (f[i] - f[o]);
                const float ep = 0.5f * (ei + eo), em = 0.5f * (ei - eo);
                const float sp = 0.5f * (si + so), sm = 0.5f * (si - so);
                const float even = hf * sp - om * (fp - ep), odd = hfm * sm - omm * (fm - em);
                oi = f[i] + even + odd;
                oo = f[o] + even - odd;
            }
            dsum += (f[i] - oi) + (f[o] - oo);
            dk[(uint32_t)i * PS] = oi;
            dk[(uint32_t)o * PS] = oo;
        }
        dk[0] = f[0] + dsum;  // mass balance
        if (OBS) {
            // stored post-collision momentum: j + F
            const float pux = (jx + F) * irho, puy = jy * irho, puz = (L::D == 3) ? jz * irho : 0.f;
            const float px = uprev[kd], py = uprev[PS + kd];
            const float pz = (L::D == 3) ? uprev[2u * PS + kd] : 0.f;
            const float ex = pux - px, ey = puy - py, ez = puz - pz;
            const float uu = pux * pux + puy * puy + puz * puz;
            a0s += jx + 0.5f * F;
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

namespace {
template <class L, int EQ>
cudaError_t periodic_dispatch(bool obs, unsigned nb, int threads, const HotArgs& A, const float* gforce,
                              float* uprev, double* partials, cudaStream_t st) {
    if (obs) k_periodic_step<L, EQ, true><<<nb, threads, 0, st>>>(A, gforce, uprev, partials);
    else k_periodic_step<L, EQ, false><<<nb, threads, 0, st>>>(A, gforce, uprev, partials);
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

}  // namespace lbmgb
