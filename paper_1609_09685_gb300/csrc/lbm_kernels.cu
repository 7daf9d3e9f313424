// lbm_kernels.cu -- CUDA kernels (sm_103a) of the lattice Boltzmann permeability
// method of Li, Ho, Wu & Zhang (arXiv:1609.09685, Sec. 2).
//
// Storage.  Each x-row of a domain is cut into 32-node segments.  A segment
// carries a 32-bit fluid mask and the compact index of its first fluid node;
// populations live only at fluid nodes, as FP32 structure-of-arrays planes
// g[i][k] (k = compact fluid index, plane stride `pstride`), shifted by the
// outlet density: g_i = f_i - w_i rho_0.  Solid nodes therefore cost no
// population bandwidth.  One warp owns one segment: lane l is node x = 32 s + l.
// The compact index of any neighbour is the neighbour segment's offset plus a
// popcount of its mask below the neighbour's lane, so pull streaming needs no
// per-node index table.
//
// One time step (pull form, the method of Sec. 2 with the boundary readings
// Zou-He pressure at x = 0 / N_x - 1, specular symmetry on the y (z) faces,
// halfway bounce-back at solids):
//   f_i(d) = f*_i(d - c_i)            source fluid
//          = f*_opp(i)(d)             source solid          (bounce-back)
//          = f*_flip(i)(d - c_i|row d)  source row outside    (specular mirror)
//   unknown at the x faces -> Zou-He; then BGK toward the (shifted)
//   equilibrium with relaxation 1/tau.
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include <utility>

#include "lbm_device.cuh"
#include "lbm_launch.h"
#include "lbm_stencil.cuh"

namespace lbmgb {
// Minimum resident 256-thread blocks per SM for the stream-collide kernel
// (caps registers per thread: 65536 / (256 * MINB)).
#ifndef LBM_SC_MINB_2D
#define LBM_SC_MINB_2D 4
#endif
#ifndef LBM_SC_MINB_3D
#define LBM_SC_MINB_3D 2
#endif
template <class L>
struct MinBlocks {
    static constexpr int value = (L::Q == 9) ? LBM_SC_MINB_2D : LBM_SC_MINB_3D;
};

// Rows in flight per warp in the cp.async pipeline (D2Q9 / D3Q19).
#ifndef LBM_SC_STAGES_2D
#define LBM_SC_STAGES_2D 3
#endif
#ifndef LBM_SC_STAGES_3D
#define LBM_SC_STAGES_3D 3
#endif
template <class L>
__host__ __device__ constexpr int stages() {
    return L::Q == 9 ? LBM_SC_STAGES_2D : LBM_SC_STAGES_3D;
}

// Shared-memory slots per stage: the Q source populations, plus the D
// components of u_prev when the step also observes.
template <class L, bool OBS>
__host__ __device__ constexpr int stage_slots() {
    return L::Q + (OBS ? L::D : 0);
}
template <class L, bool OBS>
constexpr size_t sc_smem_bytes(int threads) {
    return (size_t)(threads / 32) * stages<L>() * stage_slots<L, OBS>() * 32 * sizeof(float);
}

// A warp walks its strip row by row.  Rows k+1 .. k+S-1 are already in
// flight as cp.async copies into the warp's shared-memory stages while row k
// is relaxed and stored, so loads overlap compute without holding registers.
template <class L, int EQ, bool OBS>
__global__ void __launch_bounds__(256, MinBlocks<L>::value)
    k_stream_collide(const __grid_constant__ HotArgs A, float* __restrict__ uprev, double* __restrict__ partials) {
    constexpr int Q = L::Q;
    constexpr int NZ = (L::NROW == 9) ? 3 : 1;
    constexpr int S = stages<L>();
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + wid;
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
    const int x = (int)it.w * kSegW + lane;
    const uint32_t lmask = (1u << lane) - 1u;
    const uint32_t PS = A.pstride;
    const int ny = D.ny;
    const bool zlo = (z == 0), zhi = (z == D.nz - 1);
    const bool xin = (x == 0), xout = (x == D.nx - 1);
    // a slab's ghost columns are pulled from, never written or observed
    const bool ghost = ((D.ghost & 1u) && xin) || ((D.ghost & 2u) && xout);
    const bool edge = (it.w == 0) || ((int)it.w == D.nseg - 1);
    // omega-scaled weights by |c|^2 class (0 rest, 1 axis, 2 diagonal), and 3x
    // the omega_m-scaled ones (the odd part's rate; omega_m = omega for BGK)
    const float om = D.omega, omc = __fsub_rn(1.0f, D.omega), omm = D.omega_m;
    const bool trt = (omm != om);
    const float hw = __fmul_rn(0.5f, om), hwm = __fmul_rn(0.5f, omm);
    const float ow[3] = {__fmul_rn(om, (float)L::wd(0)), __fmul_rn(om, (float)L::wd(1)),
                         __fmul_rn(om, (float)L::wd(L::Q - 1))};
    const float ow3[3] = {__fmul_rn(3.0f, __fmul_rn(omm, (float)L::wd(0))),
                          __fmul_rn(3.0f, __fmul_rn(omm, (float)L::wd(1))),
                          __fmul_rn(3.0f, __fmul_rn(omm, (float)L::wd(L::Q - 1)))};
    float* const dst0 = A.dst[0];  // plane i starts at dst0 + i * PS
    constexpr int SL = stage_slots<L, OBS>();
    float* wbuf = smem + (size_t)wid * S * SL * 32;
    const uint32_t sb0 = (uint32_t)__cvta_generic_to_shared(wbuf) + 4u * lane;
    // Window records of planes z-1, z, z+1 and rows clamped onto the domain
    // (the clamped row or plane is the mirror image at a specular face).
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
    // D2Q9 slides the windows of rows r-1, r, r+1 down the strip (one new
    // record per row, prefetched one issue ahead); D3Q19 would need 9 sliding
    // windows, so it reloads its 9 records per row from L1 instead.
    constexpr bool kSlide = (NZ == 1);
    constexpr int NW = kSlide ? NZ : 1;
    Win wm[NW], wc[NW], wp[NW];
    uint4 rn[NW];
    if (kSlide) {
#pragma unroll
        for (int zi = 0; zi < NW; ++zi) {
            wm[zi] = make_win(__ldg(wcol + (pbase[zi] + rowc(y0 - 1)) * rs), lane, lmask);
            wc[zi] = make_win(__ldg(wcol + (pbase[zi] + y0) * rs), lane, lmask);
            wp[zi] = make_win(__ldg(wcol + (pbase[zi] + rowc(y0 + 1)) * rs), lane, lmask);
            rn[zi] = __ldg(wcol + (pbase[zi] + rowc(y0 + 2)) * rs);
        }
    }
    int next = 0;  // next row (relative to y0) to issue
    bool flq[S];
    uint32_t kdq[S];
    uint32_t sfq[S];  // source-fluid masks (observing step only)
    // issue row `next` into stage st, then slide the windows one row down
    auto issue = [&](int st) {
        if (next < nrows) {
            const int y = y0 + next;
            Win w[L::NROW];
            if (kSlide) {
#pragma unroll
                for (int r = 0; r < L::NROW; ++r) {
                    const int dy = r % 3;
                    w[r] = dy == 0 ? wm[0] : (dy == 1 ? wc[0] : wp[0]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < L::NROW; ++r) {
                    const int zi = r / 3, dy = r % 3 - 1;
                    w[r] = make_win(__ldg(wcol + (pbase[zi] + rowc(y + dy)) * rs), lane, lmask);
                }
            }
            constexpr int C = (L::NROW == 9) ? 4 : 1;
            flq[st] = win_fluid<0>(w[C]);
            kdq[st] = win_idx<0>(w[C]);
            sfq[st] = OBS ? src_fluid_mask<L>(w, std::make_integer_sequence<int, Q>{}) : 0u;
            const uint32_t sbase = sb0 + 4u * (uint32_t)(st * SL * 32);
            issue_row<L>(A.src[0], PS, w, kdq[st], y == 0, y == ny - 1, zlo, zhi, sbase, A.err,
                         std::make_integer_sequence<int, Q>{});
            if (OBS) {
#pragma unroll
                for (int a = 0; a < L::D; ++a)
                    cp_async4(sbase + 4u * (32u * (Q + a)), uprev + (size_t)a * PS + chk_load(kdq[st], PS, A.err));
            }
            if (kSlide && next + 1 < nrows) {
#pragma unroll
                for (int zi = 0; zi < NW; ++zi) {
                    wm[zi] = wc[zi];
                    wc[zi] = wp[zi];
                    wp[zi] = make_win(rn[zi], lane, lmask);
                    rn[zi] = __ldg(wcol + (pbase[zi] + rowc(y + 3)) * rs);
                }
            }
        } else {
            flq[st] = false;
            kdq[st] = 0u;
            sfq[st] = 0u;
        }
        ++next;
        cp_async_commit();
    };
#pragma unroll
    for (int st = 0; st < S - 1; ++st) issue(st);

    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0, v5 = 0.0;
    float a0s = 0.f, a1s = 0.f, a2s = 0.f, a5s = 0.f, a6s = 0.f, umax2 = 0.f;
    int nbad = 0;
    for (int k = 0; k < nrows; k += S) {
#pragma unroll
        for (int st = 0; st < S; ++st) {
            if (k + st >= nrows) break;
            issue((st + S - 1) % S);
            cp_async_wait<S - 1>();
            const float* sf = wbuf + st * SL * 32 + lane;
            float f[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = sf[i * 32];
            const bool fl = flq[st] && !ghost && chk_store(kdq[st], PS, A.err);
            const uint32_t kk = kdq[st];
            if (edge) {  // warp-uniform: only the first and last segment columns hold x faces
                float g[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = f[i];
                zou_he<L, +1>(g, D.drho_in);
#pragma unroll
                for (int i = 0; i < Q; ++i) f[i] = xin ? g[i] : f[i];
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = f[i];
                zou_he<L, -1>(g, 0.f);
#pragma unroll
                for (int i = 0; i < Q; ++i) f[i] = xout ? g[i] : f[i];
            }
            float dr, jx, jy, jz, irho, a0, k45;
            moments<L>(f, dr, jx, jy, jz);
            eq_terms<L, EQ>(dr, jx, jy, jz, D.rho0, irho, a0, k45);
            if (fl) {
                // BGK (or TRT) by opposite pairs: f* = (1 - omega) f + omega w (a0 + 4.5 (c.j)^2/rho +- 3 c.j),
                // a0 = drho - 1.5 |j|^2 / rho (quadratic) or drho (linear).
                float* const dk = dst0 + kk;
                float dsum = 0.f;  // sum over i != 0 of f_i - f*_i
                float link = 0.f;  // post-collision populations that cross an interior x plane
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    if (opp<L>(i) < i) continue;
                    const int o = opp<L>(i);
                    const int cls = (L::c(i, 0) * L::c(i, 0) + L::c(i, 1) * L::c(i, 1) + L::c(i, 2) * L::c(i, 2));
                    float sym, anti;
                    pair_terms<L, EQ>(i, jx, jy, jz, a0, k45, ow[cls], ow3[cls], sym, anti);
                    float out_i, out_o;
                    pair_relax(f[i], f[o], sym, anti, omc, hw, hwm, trt, out_i, out_o);
                    dk[(uint32_t)i * PS] = out_i;
                    dk[(uint32_t)o * PS] = out_o;
                    dsum = pair_dsum(dsum, f[i], f[o], out_i, out_o);
                    if (OBS && L::c(i, 0) != 0) {
                        // direction i reaches fluid iff the source of o is fluid, and vice versa
                        if ((sfq[st] >> o) & 1u) link += (float)L::c(i, 0) * out_i;
                        if ((sfq[st] >> i) & 1u) link += (float)L::c(o, 0) * out_o;
                    }
                }
                // Mass balance.  BGK conserves mass, so f*_0 = f_0 + sum over
                // i != 0 of (f_i - f*_i); taking the rest population this way
                // instead of from its own formula leaves one rounding of the
                // node's mass per step instead of one per population.  Each
                // difference is exact in FP32 whenever f_i and f*_i lie within a
                // factor 2 (Sterbenz), which holds near steady state.  At a
                // steady state the rounding repeats every step and acts as a
                // fixed mass source; the slow pressure modes of a porous domain
                // amplify it (a 512 x 256 domain's k drifted 4e-4 from the FP64
                // value with the rest population from its own formula, 3e-6
                // with this balance).
                dk[0] = __fadd_rn(f[0], dsum);
                if (OBS) {
                    // Within one strip (at most 8 rows x 32 lanes) the sums are
                    // FP32 -- the FP64 rate of this part is low -- and each
                    // strip hands one FP64 partial to the cross-strip FP64 pass.
                    const float ux = jx * irho, uy = jy * irho, uz = (L::D == 3) ? jz * irho : 0.f;
                    const float px = sf[Q * 32], py = sf[(Q + 1) * 32];
                    const float pz = (L::D == 3) ? sf[(Q + 2) * 32] : 0.f;
                    const float ex = ux - px, ey = uy - py, ez = uz - pz;
                    const float uu = (L::D == 3) ? ux * ux + uy * uy + uz * uz : ux * ux + uy * uy;
                    a0s += link;
                    a6s += jx;
                    a1s += (L::D == 3) ? ex * ex + ey * ey + ez * ez : ex * ex + ey * ey;
                    a2s += uu;
                    umax2 = fmaxf(umax2, uu);
                    nbad += (isfinite(ux) && isfinite(uy) && isfinite(uz)) ? 0 : 1;  // uz = 0 in 2D
                    a5s += dr;
                    uprev[kk] = ux;
                    uprev[PS + kk] = uy;
                    if (L::D == 3) uprev[2u * PS + kk] = uz;
                }
            }
        }
    }
    cp_async_wait<0>();
    if (OBS) {
        a0s = warp_sumf(a0s);
        a1s = warp_sumf(a1s);
        a2s = warp_sumf(a2s);
        a5s = warp_sumf(a5s);
        a6s = warp_sumf(a6s);
        umax2 = warp_maxf(umax2);
        nbad = __reduce_add_sync(kFull, nbad);
        v0 = a0s;
        v1 = a1s;
        v2 = a2s;
        v3 = sqrt((double)umax2);
        v4 = (double)nbad;
        v5 = a5s;
        if (lane == 0) {
            double* p = partials + (size_t)item * kNumObs;
            p[0] = v0;
            p[1] = v1;
            p[2] = v2;
            p[3] = v3;
            p[4] = v4;
            p[5] = v5;
            p[6] = a6s;
            p[7] = 0.0;
        }
    }
}

// Neighbour windows of every segment (see SegWindow).
__global__ void k_build_windows(const DomainDev* __restrict__ dom, const uint32_t* __restrict__ seg_dom,
                                uint32_t nseg_total, const uint32_t* __restrict__ seg_mask,
                                const uint32_t* __restrict__ seg_off, uint4* __restrict__ win) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nseg_total) return;
    const DomainDev D = dom[seg_dom[g]];
    const uint32_t s = (g - D.seg_base) % (uint32_t)D.nseg;
    const uint32_t own = seg_mask[g];
    const uint32_t left = s > 0 ? seg_mask[g - 1] >> 31 : 0u;
    const uint32_t right = (s + 1 < (uint32_t)D.nseg) ? seg_mask[g + 1] & 1u : 0u;
    uint4 r;
    r.x = left | (own << 1);
    r.y = (own >> 31) | (right << 1);
    r.z = seg_off[g] - left;
    r.w = own;
    win[g] = r;
}

// Observation of the current state without stepping: the same reductions as
// the OBS step, from the stored post-collision populations (whose moments equal
// the pre-collision ones, BGK conserving rho and j).
template <class L>
__global__ void __launch_bounds__(256)
    k_observe(Geometry G, const float* __restrict__ g, float* __restrict__ uprev,
              double* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const uint32_t gseg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gseg >= G.nseg_total) return;
    const DomainDev D = G.dom[__ldg(G.seg_dom + gseg)];
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    const SegLoc P = locate(D, gseg, lane);
    const bool ghost = ((D.ghost & 1u) && P.x == 0) || ((D.ghost & 2u) && P.x == D.nx - 1);
    const bool fluid = ((mc >> lane) & 1u) && !ghost;
    const size_t PS = G.pstride;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0, v5 = 0.0, v6 = 0.0;
    if (fluid) {
        const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
        float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, link = 0.f;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const float v = g[(size_t)i * PS + kd];
            dr += v;
            jx += (float)L::c(i, 0) * v;
            jy += (float)L::c(i, 1) * v;
            jz += (float)L::c(i, 2) * v;
            if (L::c(i, 0) != 0) {
                // does the population reach a fluid node across the x plane?
                const int tx = P.x + L::c(i, 0);
                int ty = P.y + L::c(i, 1), tz = P.z + L::c(i, 2);
                if (ty < 0 || ty >= D.ny) ty = P.y;
                if (tz < 0 || tz >= D.nz) tz = P.z;
                if (tx >= 0 && tx < D.nx) {
                    const uint32_t ts = D.seg_base + ((uint32_t)tz * D.ny + ty) * D.nseg + (tx >> 5);
                    if ((__ldg(G.seg_mask + ts) >> (tx & 31)) & 1u) link += (float)L::c(i, 0) * v;
                }
            }
        }
        const float irho = 1.0f / (D.rho0 + dr);
        const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
        const float px = uprev[kd], py = uprev[PS + kd];
        const float pz = (L::D == 3) ? uprev[2 * PS + kd] : 0.f;
        const float ex = ux - px, ey = uy - py, ez = uz - pz;
        v0 = (double)link;
        v1 = (double)ex * ex + (double)ey * ey + (double)ez * ez;
        v2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
        v3 = sqrt(v2);
        v4 = isfinite(ux) && isfinite(uy) && isfinite(uz) ? 0.0 : 1.0;
        v5 = (double)dr;
        v6 = (double)jx;
        uprev[kd] = ux;
        uprev[PS + kd] = uy;
        if (L::D == 3) uprev[2 * PS + kd] = uz;
    }
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    v3 = warp_max(v3);
    v4 = warp_sum(v4);
    v5 = warp_sum(v5);
    v6 = warp_sum(v6);
    if (lane == 0) {
        double* p = partials + (size_t)gseg * kNumObs;
        p[0] = v0;
        p[1] = v1;
        p[2] = v2;
        p[3] = v3;
        p[4] = v4;
        p[5] = v5;
        p[6] = v6;
        p[7] = 0.0;
    }
}

// Per-domain second pass over the warp partials in a fixed order (deterministic).
__global__ void __launch_bounds__(256)
    k_reduce_obs(const DomainDev* __restrict__ dom, const double* __restrict__ partials,
                 double* __restrict__ obs, int item_mode) {
    constexpr int K = 7;  // slots 0..6; slot 3 is a maximum, the others sums
    __shared__ double sh[K][256];
    const int d = blockIdx.x;
    const uint32_t base = item_mode ? dom[d].item_base : dom[d].seg_base;
    const uint32_t n = item_mode ? dom[d].nitems : dom[d].nseg_dom;
    double a[K] = {0, 0, 0, 0, 0, 0, 0};
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double* p = partials + (size_t)(base + i) * kNumObs;
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] = (k == 3) ? fmax(a[k], p[k]) : a[k] + p[k];
    }
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            for (int k = 0; k < K; ++k) {
                const double o = sh[k][threadIdx.x + w];
                sh[k][threadIdx.x] = (k == 3) ? fmax(sh[k][threadIdx.x], o) : sh[k][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < kNumObs) obs[(size_t)d * kNumObs + threadIdx.x] = threadIdx.x < K ? sh[threadIdx.x][0] : 0.0;
}

// Rest equilibrium with a linear density ramp: drho(x) = drho_in (N_x-1-x)/(N_x-1)
// (global x and N_x for a slab).
template <class L>
__global__ void __launch_bounds__(256) k_init(Geometry G, float* __restrict__ g, float* __restrict__ uprev) {
    const int lane = threadIdx.x & 31;
    const uint32_t gseg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gseg >= G.nseg_total) return;
    const DomainDev D = G.dom[__ldg(G.seg_dom + gseg)];
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    if (!((mc >> lane) & 1u)) return;
    const SegLoc P = locate(D, gseg, lane);
    const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
    const float dr = D.drho_in * (float)(D.nx_glob - 1 - D.x0 - P.x) / (float)(D.nx_glob - 1);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) g[(size_t)i * G.pstride + kd] = (float)L::wd(i) * dr;
    for (int a = 0; a < L::D; ++a) uprev[(size_t)a * G.pstride + kd] = 0.f;
}

// Dense unshifted populations of one domain: out[n*Q + i] = g + w rho_0 (0 on solids).
template <class L>
__global__ void __launch_bounds__(256)
    k_export_pops(Geometry G, uint32_t base, uint32_t nseg, double rho0, const float* __restrict__ g,
                  double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nseg) return;
    const uint32_t gseg = base + w;
    const DomainDev D = G.dom[__ldg(G.seg_dom + gseg)];
    const SegLoc P = locate(D, gseg, lane);
    if (P.x >= D.nx) return;
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    const size_t n = ((size_t)P.z * D.ny + P.y) * D.nx + P.x;
    const bool fluid = (mc >> lane) & 1u;
    const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        out[n * L::Q + i] = fluid ? (double)g[(size_t)i * G.pstride + kd] + L::wd(i) * rho0 : 0.0;
}

// Inverse of k_export_pops: g = (float)(f - w rho_0) at fluid nodes.
template <class L>
__global__ void __launch_bounds__(256)
    k_import_pops(Geometry G, uint32_t base, uint32_t nseg, double rho0, const double* __restrict__ in,
                  float* __restrict__ g) {
    const int lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nseg) return;
    const uint32_t gseg = base + w;
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    if (!((mc >> lane) & 1u)) return;
    const DomainDev D = G.dom[__ldg(G.seg_dom + gseg)];
    const SegLoc P = locate(D, gseg, lane);
    const size_t n = ((size_t)P.z * D.ny + P.y) * D.nx + P.x;
    const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
#pragma unroll
    for (int i = 0; i < L::Q; ++i) g[(size_t)i * G.pstride + kd] = (float)(in[n * L::Q + i] - L::wd(i) * rho0);
}

// Dense FP64 fields of one domain from the populations (zero on solids).
template <class L>
__global__ void __launch_bounds__(256)
    k_export_fields(Geometry G, uint32_t base, uint32_t nseg, double rho0, const float* __restrict__ g,
                    double* __restrict__ rho, double* __restrict__ ux, double* __restrict__ uy,
                    double* __restrict__ uz) {
    const int lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nseg) return;
    const uint32_t gseg = base + w;
    const DomainDev D = G.dom[__ldg(G.seg_dom + gseg)];
    const SegLoc P = locate(D, gseg, lane);
    if (P.x >= D.nx) return;
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    const size_t n = ((size_t)P.z * D.ny + P.y) * D.nx + P.x;
    double r = 0.0, a = 0.0, b = 0.0, c = 0.0;
    if ((mc >> lane) & 1u) {
        const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
        double dr = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double v = (double)g[(size_t)i * G.pstride + kd];
            dr += v;
            jx += L::c(i, 0) * v;
            jy += L::c(i, 1) * v;
            jz += L::c(i, 2) * v;
        }
        r = rho0 + dr;
        a = jx / r;
        b = jy / r;
        c = jz / r;
    }
    rho[n] = r;
    ux[n] = a;
    uy[n] = b;
    if (uz) uz[n] = c;
}

// Warm start: g = g_eq(drho, rho u) from dense float fields; u_prev = u.
template <class L, int EQ>
__global__ void __launch_bounds__(256)
    k_set_fields(Geometry G, uint32_t base, uint32_t nseg, const float* __restrict__ drho,
                 const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
                 float* __restrict__ g, float* __restrict__ uprev) {
    const int lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nseg) return;
    const uint32_t gseg = base + w;
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    if (!((mc >> lane) & 1u)) return;
    const DomainDev D = G.dom[__ldg(G.seg_dom + gseg)];
    const SegLoc P = locate(D, gseg, lane);
    const size_t n = ((size_t)P.z * D.ny + P.y) * D.nx + P.x;
    const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
    const float dr = drho[n];
    const float u[3] = {ux[n], uy[n], (L::D == 3 && uz) ? uz[n] : 0.f};
    const float rho = D.rho0 + dr;
    const float j[3] = {rho * u[0], rho * u[1], rho * u[2]};
    const float jj = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const float cj = (float)L::c(i, 0) * j[0] + (float)L::c(i, 1) * j[1] + (float)L::c(i, 2) * j[2];
        float geq = dr + 3.0f * cj;
        if (EQ == 0) geq += (4.5f * cj * cj - 1.5f * jj) / rho;
        g[(size_t)i * G.pstride + kd] = (float)L::wd(i) * geq;
    }
    for (int a = 0; a < L::D; ++a) uprev[(size_t)a * G.pstride + kd] = u[a];
}

// Normalised steady fields of one 2D domain, the training targets of the
// warm-start network: out[n*3 + 0] = (rho - rho_0)/drho - (1 - x/(N_x - 1)),
// the density's deviation from the linear inlet-to-outlet ramp; out[n*3 + 1..2]
// = u * scale_u with scale_u = nu (N_x - 1)/(c_s^2 drho); zero on solids.  In
// the Stokes regime these depend on the geometry (and weakly on tau) only.
template <class L>
__global__ void __launch_bounds__(256)
    k_export_targets(Geometry G, uint32_t base, uint32_t nseg, double rho0, double inv_drho, double scale_u,
                     const float* __restrict__ g, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nseg) return;
    const uint32_t gseg = base + w;
    const DomainDev D = G.dom[__ldg(G.seg_dom + gseg)];
    const SegLoc P = locate(D, gseg, lane);
    if (P.x >= D.nx) return;
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    const size_t n = ((size_t)P.z * D.ny + P.y) * D.nx + P.x;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
    if ((mc >> lane) & 1u) {
        const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
        double dr = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double v = (double)g[(size_t)i * G.pstride + kd];
            dr += v;
            jx += L::c(i, 0) * v;
            jy += L::c(i, 1) * v;
        }
        const double r = rho0 + dr;
        t0 = (float)(dr * inv_drho - (1.0 - (double)P.x / (double)(D.nx - 1)));
        t1 = (float)(jx / r * scale_u);
        t2 = (float)(jy / r * scale_u);
    }
    out[n * 3 + 0] = t0;
    out[n * 3 + 1] = t1;
    out[n * 3 + 2] = t2;
}

// Warm start from a normalised prediction (bf16, channel stride ld): drho =
// drho_scale (p0 + 1 - x/(N_x - 1)), u = (p1, p2) / scale_u clipped to
// |u| <= umax; populations = g_eq(drho, u), u_prev = u.  Solid nodes are
// untouched (they hold nothing).
template <class L, int EQ>
__global__ void __launch_bounds__(256)
    k_warm_start(Geometry G, uint32_t base, uint32_t nseg, const __nv_bfloat16* __restrict__ pred, int ld,
                 float drho_scale, float inv_scale_u, float umax, float* __restrict__ g, float* __restrict__ uprev) {
    const int lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nseg) return;
    const uint32_t gseg = base + w;
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    if (!((mc >> lane) & 1u)) return;
    const DomainDev D = G.dom[__ldg(G.seg_dom + gseg)];
    const SegLoc P = locate(D, gseg, lane);
    const size_t n = ((size_t)P.z * D.ny + P.y) * D.nx + P.x;
    const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
    const float ramp = 1.0f - (float)P.x / (float)(D.nx - 1);
    const float dr = (__bfloat162float(pred[n * ld]) + ramp) * drho_scale;
    float ux = __bfloat162float(pred[n * ld + 1]) * inv_scale_u;
    float uy = __bfloat162float(pred[n * ld + 2]) * inv_scale_u;
    const float um = sqrtf(ux * ux + uy * uy);
    if (um > umax) {
        ux *= umax / um;
        uy *= umax / um;
    }
    const float rho = D.rho0 + dr;
    const float jx = rho * ux, jy = rho * uy, jj = jx * jx + jy * jy;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const float cj = (float)L::c(i, 0) * jx + (float)L::c(i, 1) * jy;
        float geq = dr + 3.0f * cj;
        if (EQ == 0) geq += (4.5f * cj * cj - 1.5f * jj) / rho;
        g[(size_t)i * G.pstride + kd] = (float)L::wd(i) * geq;
    }
    uprev[kd] = ux;
    uprev[G.pstride + kd] = uy;
}

cudaError_t launch_export_targets(const Geometry& G, uint32_t base, uint32_t nseg, double rho0, double inv_drho,
                                  double scale_u, const float* g, float* out, cudaStream_t st) {
    const unsigned nb = (nseg + 7) / 8;
    if (nb == 0) return cudaSuccess;
    k_export_targets<D2Q9><<<nb, 256, 0, st>>>(G, base, nseg, rho0, inv_drho, scale_u, g, out);
    return cudaGetLastError();
}

cudaError_t launch_warm_start(int eq, const Geometry& G, uint32_t base, uint32_t nseg, const void* pred, int ld,
                              float drho_scale, float inv_scale_u, float umax, float* g, float* uprev,
                              cudaStream_t st) {
    const unsigned nb = (nseg + 7) / 8;
    if (nb == 0) return cudaSuccess;
    const __nv_bfloat16* p = (const __nv_bfloat16*)pred;
    if (eq == 0) k_warm_start<D2Q9, 0><<<nb, 256, 0, st>>>(G, base, nseg, p, ld, drho_scale, inv_scale_u, umax, g, uprev);
    else k_warm_start<D2Q9, 1><<<nb, 256, 0, st>>>(G, base, nseg, p, ld, drho_scale, inv_scale_u, umax, g, uprev);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Segment tables: domain of each segment, fluid bits, fluid counts, offsets.
// ---------------------------------------------------------------------------
__global__ void k_seg_locate(const uint32_t* __restrict__ dom_begin, int ndom, uint32_t nseg_total,
                             uint32_t* __restrict__ seg_dom) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nseg_total) return;
    int lo = 0, hi = ndom - 1;  // largest d with dom_begin[d] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (dom_begin[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    seg_dom[g] = (uint32_t)lo;
}

__global__ void __launch_bounds__(256)
    k_seg_build(const DomainDev* __restrict__ dom, const uint32_t* __restrict__ seg_dom,
                uint32_t nseg_total, const uint8_t* __restrict__ mask, uint32_t* __restrict__ seg_mask,
                uint32_t* __restrict__ seg_cnt) {
    const int lane = threadIdx.x & 31;
    const uint32_t gseg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gseg >= nseg_total) return;
    const DomainDev D = dom[seg_dom[gseg]];
    const SegLoc P = locate(D, gseg, lane);
    bool fl = false;
    if (P.x < D.nx) fl = mask[D.mask_base + ((size_t)P.z * D.ny + P.y) * D.nx + P.x] == 0;
    const uint32_t b = __ballot_sync(kFull, fl);
    if (lane == 0) {
        seg_mask[gseg] = b;
        seg_cnt[gseg] = __popc(b);
    }
}

// Exclusive scan of n uint32 values: block scans, a scan of block totals, add.
__global__ void __launch_bounds__(1024)
    k_scan_blocks(const uint32_t* __restrict__ in, uint32_t n, uint32_t* __restrict__ out,
                  uint32_t* __restrict__ totals) {
    __shared__ uint32_t wsum[32];
    const uint32_t i = blockIdx.x * 1024u + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t v = i < n ? in[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += t;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    const uint32_t incl = x + (wid > 0 ? wsum[wid - 1] : 0u);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == 1023) totals[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(1024) k_scan_totals(uint32_t* __restrict__ totals, uint32_t nb,
                                                       uint32_t* __restrict__ grand) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += 1024u) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? totals[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            uint32_t s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += t;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const uint32_t incl = x + (wid > 0 ? wsum[wid - 1] : 0u);
        if (i < nb) totals[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, uint32_t n, const uint32_t* __restrict__ totals) {
    const uint32_t i = blockIdx.x * 1024u + threadIdx.x;
    if (i < n) out[i] += totals[blockIdx.x];
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
namespace {
inline unsigned seg_blocks(uint32_t nseg, int threads) {
    const uint32_t wpb = (uint32_t)threads / 32u;
    return (unsigned)((nseg + wpb - 1) / wpb);
}
}  // namespace

template <class L, int EQ, bool OBS>
static cudaError_t sc_launch(unsigned nb, int threads, const HotArgs& A, float* uprev, double* partials,
                             cudaStream_t st) {
    const size_t sm = sc_smem_bytes<L, OBS>(threads);
    static bool attr_set = false;  // per template instance; the attribute is per device function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_stream_collide<L, EQ, OBS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sc_smem_bytes<L, OBS>(256));
        if (e != cudaSuccess) return e;
        // (no carveout preference: the default keeps a large L1, which the
        // cp.async loads need for the sectors neighbouring segments share)
        attr_set = true;
    }
    k_stream_collide<L, EQ, OBS><<<nb, threads, sm, st>>>(A, uprev, partials);
    return cudaGetLastError();
}

template <class L>
static cudaError_t sc_dispatch(int eq, bool obs, const HotArgs& A, float* uprev, double* partials, int threads,
                               cudaStream_t st) {
    const unsigned nb = seg_blocks(A.nitems, threads);
    if (nb == 0) return cudaSuccess;
    if (eq == 0) {
        if (obs) return sc_launch<L, 0, true>(nb, threads, A, uprev, partials, st);
        return sc_launch<L, 0, false>(nb, threads, A, uprev, partials, st);
    }
    if (obs) return sc_launch<L, 1, true>(nb, threads, A, uprev, partials, st);
    return sc_launch<L, 1, false>(nb, threads, A, uprev, partials, st);
}

cudaError_t launch_stream_collide(int q, int eq, bool obs, HotArgs A, const float* src, float* dst,
                                  float* uprev, double* partials, int threads, cudaStream_t st) {
    if (threads <= 0) threads = 128;  // measured best on GB300 for both lattices
    for (int i = 0; i < 19; ++i) {
        A.src[i] = i < q ? src + (size_t)i * A.pstride : nullptr;
        A.dst[i] = i < q ? dst + (size_t)i * A.pstride : nullptr;
    }
    if (q == 9) return sc_dispatch<D2Q9>(eq, obs, A, uprev, partials, threads, st);
    return sc_dispatch<D3Q19>(eq, obs, A, uprev, partials, threads, st);
}

cudaError_t launch_build_windows(const DomainDev* dom, const uint32_t* seg_dom, uint32_t nseg_total,
                                 const uint32_t* seg_mask, const uint32_t* seg_off, uint4* win,
                                 cudaStream_t st) {
    if (nseg_total == 0) return cudaSuccess;
    k_build_windows<<<(nseg_total + 255) / 256, 256, 0, st>>>(dom, seg_dom, nseg_total, seg_mask, seg_off, win);
    return cudaGetLastError();
}

cudaError_t launch_observe(int q, const Geometry& G, const float* g, float* uprev, double* partials,
                           cudaStream_t st) {
    const unsigned nb = seg_blocks(G.nseg_total, 256);
    if (nb == 0) return cudaSuccess;
    if (q == 9) k_observe<D2Q9><<<nb, 256, 0, st>>>(G, g, uprev, partials);
    else k_observe<D3Q19><<<nb, 256, 0, st>>>(G, g, uprev, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce_obs(const DomainDev* dom, int ndom, const double* partials, double* obs,
                              bool item_mode, cudaStream_t st) {
    if (ndom <= 0) return cudaSuccess;
    k_reduce_obs<<<ndom, 256, 0, st>>>(dom, partials, obs, item_mode ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_init(int q, const Geometry& G, float* g, float* uprev, cudaStream_t st) {
    const unsigned nb = seg_blocks(G.nseg_total, 256);
    if (nb == 0) return cudaSuccess;
    if (q == 9) k_init<D2Q9><<<nb, 256, 0, st>>>(G, g, uprev);
    else k_init<D3Q19><<<nb, 256, 0, st>>>(G, g, uprev);
    return cudaGetLastError();
}

cudaError_t launch_export_pops(int q, const Geometry& G, uint32_t base, uint32_t nseg, double rho0,
                               const float* g, double* out, cudaStream_t st) {
    const unsigned nb = seg_blocks(nseg, 256);
    if (nb == 0) return cudaSuccess;
    if (q == 9) k_export_pops<D2Q9><<<nb, 256, 0, st>>>(G, base, nseg, rho0, g, out);
    else k_export_pops<D3Q19><<<nb, 256, 0, st>>>(G, base, nseg, rho0, g, out);
    return cudaGetLastError();
}

cudaError_t launch_import_pops(int q, const Geometry& G, uint32_t base, uint32_t nseg, double rho0,
                               const double* in, float* g, cudaStream_t st) {
    const unsigned nb = seg_blocks(nseg, 256);
    if (nb == 0) return cudaSuccess;
    if (q == 9) k_import_pops<D2Q9><<<nb, 256, 0, st>>>(G, base, nseg, rho0, in, g);
    else k_import_pops<D3Q19><<<nb, 256, 0, st>>>(G, base, nseg, rho0, in, g);
    return cudaGetLastError();
}

cudaError_t launch_export_fields(int q, const Geometry& G, uint32_t base, uint32_t nseg, double rho0,
                                 const float* g, double* rho, double* ux, double* uy, double* uz,
                                 cudaStream_t st) {
    const unsigned nb = seg_blocks(nseg, 256);
    if (nb == 0) return cudaSuccess;
    if (q == 9) k_export_fields<D2Q9><<<nb, 256, 0, st>>>(G, base, nseg, rho0, g, rho, ux, uy, uz);
    else k_export_fields<D3Q19><<<nb, 256, 0, st>>>(G, base, nseg, rho0, g, rho, ux, uy, uz);
    return cudaGetLastError();
}

cudaError_t launch_set_fields(int q, int eq, const Geometry& G, uint32_t base, uint32_t nseg,
                              const float* drho, const float* ux, const float* uy, const float* uz,
                              float* g, float* uprev, cudaStream_t st) {
    const unsigned nb = seg_blocks(nseg, 256);
    if (nb == 0) return cudaSuccess;
    if (q == 9) {
        if (eq == 0) k_set_fields<D2Q9, 0><<<nb, 256, 0, st>>>(G, base, nseg, drho, ux, uy, uz, g, uprev);
        else k_set_fields<D2Q9, 1><<<nb, 256, 0, st>>>(G, base, nseg, drho, ux, uy, uz, g, uprev);
    } else {
        if (eq == 0) k_set_fields<D3Q19, 0><<<nb, 256, 0, st>>>(G, base, nseg, drho, ux, uy, uz, g, uprev);
        else k_set_fields<D3Q19, 1><<<nb, 256, 0, st>>>(G, base, nseg, drho, ux, uy, uz, g, uprev);
    }
    return cudaGetLastError();
}

cudaError_t launch_seg_setup(const DomainDev* dom, const uint32_t* dom_begin, int ndom,
                             uint32_t nseg_total, const uint8_t* mask, uint32_t* seg_dom,
                             uint32_t* seg_mask, uint32_t* seg_cnt, uint32_t* seg_off,
                             uint32_t* scan_totals, uint32_t* grand_total, cudaStream_t st) {
    if (nseg_total == 0) return cudaSuccess;
    k_seg_locate<<<(nseg_total + 255) / 256, 256, 0, st>>>(dom_begin, ndom, nseg_total, seg_dom);
    k_seg_build<<<seg_blocks(nseg_total, 256), 256, 0, st>>>(dom, seg_dom, nseg_total, mask, seg_mask,
                                                             seg_cnt);
    const uint32_t nb = (nseg_total + 1023u) / 1024u;
    k_scan_blocks<<<nb, 1024, 0, st>>>(seg_cnt, nseg_total, seg_off, scan_totals);
    k_scan_totals<<<1, 1024, 0, st>>>(scan_totals, nb, grand_total);
    k_scan_add<<<nb, 1024, 0, st>>>(seg_off, nseg_total, scan_totals);
    return cudaGetLastError();
}

}  // namespace lbmgb
