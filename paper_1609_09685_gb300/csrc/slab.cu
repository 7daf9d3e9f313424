// slab.cu -- halo transfer of an x-slab of a larger domain (the domain
// decomposition of one lattice Boltzmann domain over several solvers, each a
// slab of columns with a ghost column at each cut; the method of Sec. 2 is
// unchanged).
//
// One pull step of a slab's first real column reads, from the ghost column to
// its left, only the directions with c_x = +1 (its Q = 9 lattice: 3 of them;
// D3Q19: 5); the last real column reads the c_x = -1 directions from the
// ghost to its right.  So a cut exchanges those planes of one column per step:
// the sending slab packs the column's fluid nodes (in the order of the
// column's compact index list) into a dense buffer, the receiving slab
// unpacks it into its ghost column, whose fluid nodes come in the same order
// (both columns have the same mask).
#include <cuda_runtime.h>

#include "lbm_launch.h"

namespace lbmgb {

namespace {

__global__ void k_halo_pack(const float* __restrict__ g, uint32_t PS, const uint32_t* __restrict__ idx, uint32_t n,
                            HaloPlanes P, float* __restrict__ out) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (m >= n || j >= P.n) return;
    out[(size_t)j * n + m] = g[(size_t)P.plane[j] * PS + idx[m]];
}

__global__ void k_halo_unpack(float* __restrict__ g, uint32_t PS, const uint32_t* __restrict__ idx, uint32_t n,
                              HaloPlanes P, const float* __restrict__ in) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (m >= n || j >= P.n) return;
    g[(size_t)P.plane[j] * PS + idx[m]] = in[(size_t)j * n + m];
}

}  // namespace

cudaError_t launch_halo(bool pack, float* g, uint32_t PS, const uint32_t* idx, uint32_t n, const HaloPlanes& P,
                        float* buf, cudaStream_t st) {
    if (n == 0 || P.n == 0) return cudaSuccess;
    const dim3 grid((n + 127) / 128, (unsigned)P.n);
    if (pack) k_halo_pack<<<grid, 128, 0, st>>>(g, PS, idx, n, P, buf);
    else k_halo_unpack<<<grid, 128, 0, st>>>(g, PS, idx, n, P, buf);
    return cudaGetLastError();
}

}  // namespace lbmgb
