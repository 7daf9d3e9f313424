// pore.cu -- local pore size and local Knudsen number (arXiv:1609.09685, Sec. 2:
// the local Kn of narrow pores can be much larger than the domain's).
//
// Pore size of a fluid node: h = 2 D - 1, D the Euclidean distance in nodes to
// the nearest solid node of the domain (the centre node of a channel of h fluid
// rows gets h).  D^2 is computed exactly in integers by the separable
// transform: D^2(x, y, z) = min over j of [ min over i of (G_x(i, j, z) + (y - j)^2) ... ],
// one 1D pass per axis, G starting as 0 on solids and "infinite" on fluid.  In
// each pass a thread scans outward from its node along the axis and stops once
// the squared offset reaches its best candidate, so a pass costs about D per
// node; a line without any finite value costs its length.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "lbm_launch.h"

namespace lbmgb {

namespace {

constexpr uint32_t kInf = 0xffffffffu;

// One 1D pass along `axis` (0 = x, 1 = y, 2 = z) of a dense nz x ny x nx grid.
// in == nullptr: the first pass, taking G from the mask.
__global__ void k_edt_pass(const uint8_t* __restrict__ mask, const uint32_t* __restrict__ in,
                           uint32_t* __restrict__ out, int nx, int ny, int nz, int axis) {
    const uint64_t n = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t total = (uint64_t)nx * ny * nz;
    if (n >= total) return;
    const int x = (int)(n % (uint64_t)nx);
    const int y = (int)((n / (uint64_t)nx) % (uint64_t)ny);
    const int z = (int)(n / ((uint64_t)nx * ny));
    const int len = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int pos = axis == 0 ? x : (axis == 1 ? y : z);
    const int64_t stride = axis == 0 ? 1 : (axis == 1 ? (int64_t)nx : (int64_t)nx * ny);
    auto g = [&](int64_t idx) -> uint32_t {
        if (in == nullptr) return mask[idx] ? 0u : kInf;
        return in[idx];
    };
    uint64_t best = g((int64_t)n);
    for (int k = 1;; ++k) {
        const uint64_t k2 = (uint64_t)k * (uint64_t)k;
        if (k2 >= best) break;
        const bool lo = pos - k >= 0, hi = pos + k < len;
        if (!lo && !hi) break;
        if (lo) {
            const uint32_t v = g((int64_t)n - k * stride);
            if (v != kInf && (uint64_t)v + k2 < best) best = (uint64_t)v + k2;
        }
        if (hi) {
            const uint32_t v = g((int64_t)n + k * stride);
            if (v != kInf && (uint64_t)v + k2 < best) best = (uint64_t)v + k2;
        }
    }
    out[n] = best >= (uint64_t)kInf ? kInf : (uint32_t)best;
}

__global__ void k_local_kn(const uint8_t* __restrict__ mask, const uint32_t* __restrict__ d2, uint64_t total,
                           double kn_num, double* __restrict__ h_out, double* __restrict__ kn_out) {
    const uint64_t n = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= total) return;
    double h = 0.0, kn = 0.0;
    if (!mask[n]) {
        if (d2[n] == kInf) {
            h = INFINITY;
        } else {
            h = 2.0 * sqrt((double)d2[n]) - 1.0;
            kn = kn_num / h;
        }
    }
    if (h_out) h_out[n] = h;
    if (kn_out) kn_out[n] = kn;
}

}  // namespace

cudaError_t launch_pore_d2(const uint8_t* mask, int nx, int ny, int nz, uint32_t* d2, uint32_t* tmp,
                           cudaStream_t st) {
    const uint64_t total = (uint64_t)nx * ny * nz;
    if (total == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((total + 255) / 256);
    // x pass into d2, y pass into tmp, z pass (3D) back into d2
    k_edt_pass<<<nb, 256, 0, st>>>(mask, nullptr, d2, nx, ny, nz, 0);
    k_edt_pass<<<nb, 256, 0, st>>>(mask, d2, tmp, nx, ny, nz, 1);
    if (nz > 1) {
        k_edt_pass<<<nb, 256, 0, st>>>(mask, tmp, d2, nx, ny, nz, 2);
    } else {
        cudaError_t e = cudaMemcpyAsync(d2, tmp, sizeof(uint32_t) * total, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_local_kn(const uint8_t* mask, const uint32_t* d2, uint64_t total, double tau, double* h_out,
                            double* kn_out, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    const double num = std::sqrt(M_PI / 6.0) * (tau - 0.5);
    k_local_kn<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(mask, d2, total, num, h_out, kn_out);
    return cudaGetLastError();
}

}  // namespace lbmgb
