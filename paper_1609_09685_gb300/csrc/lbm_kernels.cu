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

#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbmgb {

namespace {

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

// Zou-He pressure closure in shifted form for the face whose inward normal is
// `SIDE` (+1 at x = 0, -1 at x = N_x - 1), u_y = u_z = 0:
//   rho u_x = side * (drho_b - (S_0 + 2 S_in)),  S_0 = sum over c_x = 0,
//   S_in = sum over the known directions c_x = -side,
//   N_a = 1/2 sum_{c_x = 0} c_a g (transverse momentum of the c_x = 0 set),
//   g_i = g_opp(i) + side 6 w_i rho u_x - c_iy N_y - c_iz N_z  for c_ix = side.
// Written generically; in 2D it reduces to Zou & He (1997), in 3D to the
// Hecht & Harting (2010) form.  The shifted weights cancel because the c_x = 0
// weights plus twice the c_x = -side weights sum to one.
template <class L, int SIDE>
__device__ __forceinline__ void zou_he(float (&f)[L::Q], float drho_b) {
    float s0 = 0.f, sin = 0.f, ny = 0.f, nz = 0.f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        if (L::c(i, 0) == 0) {
            s0 += f[i];
            ny += (float)L::c(i, 1) * f[i];
            nz += (float)L::c(i, 2) * f[i];
        } else if (L::c(i, 0) == -SIDE) {
            sin += f[i];
        }
    }
    const float rux = (float)SIDE * (drho_b - (s0 + 2.f * sin));
    ny *= 0.5f;
    nz *= 0.5f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        if (L::c(i, 0) == SIDE) {
            const float w6 = (float)(6.0 * L::wd(i));
            f[i] = f[opp<L>(i)] + (float)SIDE * w6 * rux - (float)L::c(i, 1) * ny -
                   (float)L::c(i, 2) * nz;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Fused stream + boundaries + BGK collide; OBS adds the per-interval FP64
// reductions (flux, residual terms, max |u|, non-finite count, mass).
// ---------------------------------------------------------------------------
template <class L, int EQ, bool OBS>
__global__ void __launch_bounds__(256)
    k_stream_collide(Geometry G, const float* __restrict__ src, float* __restrict__ dst,
                     float* __restrict__ uprev, double* __restrict__ partials) {
    constexpr int Q = L::Q;
    const int lane = threadIdx.x & 31;
    const uint32_t gseg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gseg >= G.nseg_total) return;
    const uint32_t d = __ldg(G.seg_dom + gseg);
    const DomainDev D = G.dom[d];
    const uint32_t mc = __ldg(G.seg_mask + gseg);
    if (!D.active || mc == 0u) {
        if (OBS && lane < kNumObs) partials[(size_t)gseg * kNumObs + lane] = 0.0;
        return;
    }
    const SegLoc P = locate(D, gseg, lane);

    // Neighbourhood metadata: lane e < 3 NROW holds segment s + (e % 3) - 1 of
    // row (y + dy, z + dz) with e / 3 = (dy + 1) + 3 (dz + 1); a row outside the
    // domain is replaced by the node's own row (the mirror image).
    uint32_t nbm = 0u, nbo = 0u;
    if (lane < 3 * L::NROW) {
        const int r = lane / 3, cs = lane - 3 * r;
        int yy = P.y + (r % 3) - 1;
        int zz = P.z + (L::NROW == 9 ? r / 3 - 1 : 0);
        if (yy < 0 || yy >= D.ny) yy = P.y;
        if (zz < 0 || zz >= D.nz) zz = P.z;
        const int ss = P.s + cs - 1;
        if (ss >= 0 && ss < D.nseg) {
            const uint32_t g2 = D.seg_base + ((uint32_t)zz * D.ny + yy) * D.nseg + ss;
            nbm = __ldg(G.seg_mask + g2);
            nbo = __ldg(G.seg_off + g2);
        }
    }
    const bool fluid = (mc >> lane) & 1u;
    const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
    const size_t PS = G.pstride;

    float f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        const int sx = P.x - cx;
        const bool fy = (cy != 0) && (P.y - cy < 0 || P.y - cy >= D.ny);
        const bool fz = (cz != 0) && (P.z - cz < 0 || P.z - cz >= D.nz);
        const int r = (1 - cy) + (L::NROW == 9 ? 3 * (1 - cz) : 0);
        const int e = 3 * r + ((sx >> 5) - P.s + 1);
        const uint32_t m = __shfl_sync(kFull, nbm, e);
        const uint32_t o = __shfl_sync(kFull, nbo, e);
        const int j = fy ? (fz ? flip<L>(i, true, true) : flip<L>(i, true, false))
                         : (fz ? flip<L>(i, false, true) : i);
        const uint32_t bit = (uint32_t)sx & 31u;
        const bool sf = (m >> bit) & 1u;
        const size_t a = sf ? (size_t)j * PS + o + __popc(m & ((1u << bit) - 1u))
                            : (size_t)opp<L>(i) * PS + kd;
        f[i] = fluid ? __ldg(src + a) : 0.f;
    }
    if (P.x == 0) zou_he<L, +1>(f, D.drho_in);
    if (P.x == D.nx - 1) zou_he<L, -1>(f, 0.f);

    float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        dr += f[i];
        jx += (float)L::c(i, 0) * f[i];
        jy += (float)L::c(i, 1) * f[i];
        jz += (float)L::c(i, 2) * f[i];
    }
    const float rho = D.rho0 + dr;
    const float irho = 1.0f / rho;
    const float jj = jx * jx + jy * jy + jz * jz;
    if (fluid) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float cj = (float)L::c(i, 0) * jx + (float)L::c(i, 1) * jy + (float)L::c(i, 2) * jz;
            const float w = (float)L::wd(i);
            float geq = dr + 3.0f * cj;
            if (EQ == 0) geq += (4.5f * cj * cj - 1.5f * jj) * irho;
            geq *= w;
            dst[(size_t)i * PS + kd] = f[i] + D.omega * (geq - f[i]);
        }
    }
    if (OBS) {
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0, v5 = 0.0;
        if (fluid) {
            const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
            const float px = uprev[kd], py = uprev[PS + kd];
            const float pz = (L::D == 3) ? uprev[2 * PS + kd] : 0.f;
            const float ex = ux - px, ey = uy - py, ez = uz - pz;
            v0 = (double)jx;
            v1 = (double)ex * ex + (double)ey * ey + (double)ez * ez;
            v2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
            v3 = sqrt(v2);
            v4 = isfinite(ux) && isfinite(uy) && isfinite(uz) ? 0.0 : 1.0;
            v5 = (double)dr;
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
        if (lane == 0) {
            double* p = partials + (size_t)gseg * kNumObs;
            p[0] = v0;
            p[1] = v1;
            p[2] = v2;
            p[3] = v3;
            p[4] = v4;
            p[5] = v5;
            p[6] = 0.0;
            p[7] = 0.0;
        }
    }
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
    const bool fluid = (mc >> lane) & 1u;
    const size_t PS = G.pstride;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0, v5 = 0.0;
    if (fluid) {
        const uint32_t kd = __ldg(G.seg_off + gseg) + __popc(mc & ((1u << lane) - 1u));
        float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const float v = g[(size_t)i * PS + kd];
            dr += v;
            jx += (float)L::c(i, 0) * v;
            jy += (float)L::c(i, 1) * v;
            jz += (float)L::c(i, 2) * v;
        }
        const float irho = 1.0f / (D.rho0 + dr);
        const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
        const float px = uprev[kd], py = uprev[PS + kd];
        const float pz = (L::D == 3) ? uprev[2 * PS + kd] : 0.f;
        const float ex = ux - px, ey = uy - py, ez = uz - pz;
        v0 = (double)jx;
        v1 = (double)ex * ex + (double)ey * ey + (double)ez * ez;
        v2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
        v3 = sqrt(v2);
        v4 = isfinite(ux) && isfinite(uy) && isfinite(uz) ? 0.0 : 1.0;
        v5 = (double)dr;
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
    if (lane == 0) {
        double* p = partials + (size_t)gseg * kNumObs;
        p[0] = v0;
        p[1] = v1;
        p[2] = v2;
        p[3] = v3;
        p[4] = v4;
        p[5] = v5;
        p[6] = 0.0;
        p[7] = 0.0;
    }
}

// Per-domain second pass over the warp partials in a fixed order (deterministic).
__global__ void __launch_bounds__(256)
    k_reduce_obs(const DomainDev* __restrict__ dom, const double* __restrict__ partials,
                 double* __restrict__ obs) {
    __shared__ double sh[kNumObs][256];
    const int d = blockIdx.x;
    const uint32_t base = dom[d].seg_base, n = dom[d].nseg_dom;
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double* p = partials + (size_t)(base + i) * kNumObs;
        a[0] += p[0];
        a[1] += p[1];
        a[2] += p[2];
        a[3] = fmax(a[3], p[3]);
        a[4] += p[4];
        a[5] += p[5];
    }
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            for (int k = 0; k < 6; ++k) {
                const double o = sh[k][threadIdx.x + w];
                sh[k][threadIdx.x] = (k == 3) ? fmax(sh[k][threadIdx.x], o) : sh[k][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < kNumObs) obs[(size_t)d * kNumObs + threadIdx.x] = threadIdx.x < 6 ? sh[threadIdx.x][0] : 0.0;
}

// Rest equilibrium with a linear density ramp: drho(x) = drho_in (N_x-1-x)/(N_x-1).
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
    const float dr = D.drho_in * (float)(D.nx - 1 - P.x) / (float)(D.nx - 1);
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

template <class L>
static cudaError_t sc_dispatch(int eq, bool obs, const Geometry& G, const float* src, float* dst,
                               float* uprev, double* partials, int threads, cudaStream_t st) {
    const unsigned nb = seg_blocks(G.nseg_total, threads);
    if (nb == 0) return cudaSuccess;
    if (eq == 0) {
        if (obs) k_stream_collide<L, 0, true><<<nb, threads, 0, st>>>(G, src, dst, uprev, partials);
        else k_stream_collide<L, 0, false><<<nb, threads, 0, st>>>(G, src, dst, uprev, partials);
    } else {
        if (obs) k_stream_collide<L, 1, true><<<nb, threads, 0, st>>>(G, src, dst, uprev, partials);
        else k_stream_collide<L, 1, false><<<nb, threads, 0, st>>>(G, src, dst, uprev, partials);
    }
    return cudaGetLastError();
}

cudaError_t launch_stream_collide(int q, int eq, bool obs, const Geometry& G, const float* src,
                                  float* dst, float* uprev, double* partials, int threads,
                                  cudaStream_t st) {
    if (threads <= 0) threads = 256;
    if (q == 9) return sc_dispatch<D2Q9>(eq, obs, G, src, dst, uprev, partials, threads, st);
    return sc_dispatch<D3Q19>(eq, obs, G, src, dst, uprev, partials, threads, st);
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
                              cudaStream_t st) {
    if (ndom <= 0) return cudaSuccess;
    k_reduce_obs<<<ndom, 256, 0, st>>>(dom, partials, obs);
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
