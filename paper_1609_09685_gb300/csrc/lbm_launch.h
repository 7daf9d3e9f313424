// lbm_launch.h -- host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "lbm_device.cuh"

namespace lbmgb {

cudaError_t launch_stream_collide(int q, int eq, bool obs, HotArgs A, const float* src, float* dst,
                                  float* uprev, double* partials, int threads, cudaStream_t st);
// Launch configuration of the plain steps (chosen per solver; every choice
// gives bit-identical results).
struct StepLaunch {
    int threads;       // block size of the direct gather, local and pull steps (0 = 128)
    int tile_rows;     // > 0: staged gather step over A.tiles (built with that many rows per tile)
    int gather_batch;  // rows of loads in flight per warp of the direct gather step (0 = default)
    int band_rows;     // > 0: band gather step over A.bands (built with up to that many rows per band)
};
// Two steps in place on g (gather step, then local step); see k_aa_gather.
cudaError_t launch_aa_pair(int q, int eq, HotArgs A, float* g, const StepLaunch& cfg, cudaStream_t st);
// Both steps of the pair in one persistent launch over the work queue F
// (L2-blocked; see k_aa_pair_fused); zeroes F.ctr first.
cudaError_t launch_aa_pair_fused(int q, int eq, HotArgs A, const PairFused& F, float* g, const StepLaunch& cfg,
                                 cudaStream_t st);
// One half of the pair: half 0 = gather step, 1 = local step.
cudaError_t launch_aa_half(int q, int eq, int half, HotArgs A, float* g, const StepLaunch& cfg, cudaStream_t st);
// Nonzero when the lattice with q directions has a staged gather step.
int staged_gather_lattice(int q);
// Nonzero when the lattice with q directions has a band gather step.
int band_gather_lattice(int q);
// Row batches of the direct gather step: the two compiled ones and the default.
void gather_batches(int q, int* lo, int* hi, int* def);
// Slots per lane of the local step (its work items cover 32 x this many slots).
int local_step_vector(int q);
// Inlet/outlet bits of the compact slots (face zeroed beforehand).
cudaError_t launch_build_face(const DomainDev* dom, const uint32_t* seg_dom, uint32_t nseg_total,
                              const uint32_t* seg_mask, const uint32_t* seg_off, uint32_t* face, cudaStream_t st);
cudaError_t launch_build_windows(const DomainDev* dom, const uint32_t* seg_dom, uint32_t nseg_total,
                                 const uint32_t* seg_mask, const uint32_t* seg_off, uint4* win,
                                 cudaStream_t st);
cudaError_t launch_observe(int q, const Geometry& G, const float* g, float* uprev, double* partials,
                           cudaStream_t st);
// item_mode: partials are per strip item (stream-collide) rather than per
// segment (observe-only kernel).
cudaError_t launch_reduce_obs(const DomainDev* dom, int ndom, const double* partials, double* obs,
                              bool item_mode, cudaStream_t st);
cudaError_t launch_init(int q, const Geometry& G, float* g, float* uprev, cudaStream_t st);
cudaError_t launch_export_pops(int q, const Geometry& G, uint32_t base, uint32_t nseg, double rho0,
                               const float* g, double* out, cudaStream_t st);
cudaError_t launch_import_pops(int q, const Geometry& G, uint32_t base, uint32_t nseg, double rho0,
                               const double* in, float* g, cudaStream_t st);
cudaError_t launch_export_fields(int q, const Geometry& G, uint32_t base, uint32_t nseg, double rho0,
                                 const float* g, double* rho, double* ux, double* uy, double* uz,
                                 cudaStream_t st);
cudaError_t launch_set_fields(int q, int eq, const Geometry& G, uint32_t base, uint32_t nseg,
                              const float* drho, const float* ux, const float* uy, const float* uz,
                              float* g, float* uprev, cudaStream_t st);
cudaError_t launch_seg_setup(const DomainDev* dom, const uint32_t* dom_begin, int ndom,
                             uint32_t nseg_total, const uint8_t* mask, uint32_t* seg_dom,
                             uint32_t* seg_mask, uint32_t* seg_cnt, uint32_t* seg_off,
                             uint32_t* scan_totals, uint32_t* grand_total, cudaStream_t st);

cudaError_t launch_export_targets(const Geometry& G, uint32_t base, uint32_t nseg, double rho0, double inv_drho,
                                  double scale_u, const float* g, float* out, cudaStream_t st);
cudaError_t launch_warm_start(int eq, const Geometry& G, uint32_t base, uint32_t nseg, const void* pred, int ld,
                              float drho_scale, float inv_scale_u, float umax, float* g, float* uprev,
                              cudaStream_t st);

// QSGS (qsgs.cu).  keys: N uint64 scratch; counter: one uint64 scratch.
struct QsgsScratch {
    uint64_t* keys;
    uint8_t* start;
    unsigned long long* counter;
    unsigned long long* host_counter;  // pinned
};
// Growth iterations after which qsgs_generate gives up (the solid count has
// stopped growing, e.g. every remaining fluid cell is out of reach).
constexpr int kMaxGrowthIterations = 1000000;
// Returns 0 on success, -1 argument error, -2 CUDA error (cuda_err set),
// -3 no solid core to grow from, -4 kMaxGrowthIterations reached.
int qsgs_generate(uint64_t seed, int nx, int ny, int nz, double core_p, double porosity,
                  double d_face, uint8_t* d_mask, const QsgsScratch& sc, cudaStream_t st,
                  int* iterations, cudaError_t* cuda_err);

// Force-driven flow with every face periodic (periodic.cu): one pull step,
// observing when obs; gforce = body acceleration per domain (device).
cudaError_t launch_periodic_step(int q, int eq, bool obs, HotArgs A, const float* gforce, const float* src,
                                 float* dst, float* uprev, double* partials, cudaStream_t st);
// One half of a force-driven in-place pair on g: half 0 = gather step (pull
// reads, results written back to the slots read), 1 = local step.
cudaError_t launch_periodic_half(int q, int eq, int half, HotArgs A, const float* gforce, float* g, cudaStream_t st);

// Local pore size (pore.cu): exact squared distance to the nearest solid node of
// a dense mask (d2, tmp: nx*ny*nz uint32 each), then h = 2 D - 1 and the local Kn.
cudaError_t launch_pore_d2(const uint8_t* mask, int nx, int ny, int nz, uint32_t* d2, uint32_t* tmp,
                           cudaStream_t st);
cudaError_t launch_local_kn(const uint8_t* mask, const uint32_t* d2, uint64_t total, double tau, double* h_out,
                            double* kn_out, cudaStream_t st);

// Halo transfer of a slab (slab.cu): the planes a cut exchanges, packed from
// (pack) or unpacked into (!pack) the column whose fluid nodes' compact
// indices are idx[0..n), buf dense [P.n][n].
struct HaloPlanes {
    int n;
    int plane[5];
};
cudaError_t launch_halo(bool pack, float* g, uint32_t PS, const uint32_t* idx, uint32_t n, const HaloPlanes& P,
                        float* buf, cudaStream_t st);

// Warm-start network convolution on the tcgen05 tensor cores (unet_tc.cu), and
// the device flag its bounded waits set (taken and cleared by tc_error_take).
namespace nn {
cudaError_t launch_conv_fwd_tc(const void* in, int N, int H, int W, int Cin, const void* w, const float* bias,
                               int taps, int Cout, int relu, void* out, float* out_f32, cudaStream_t st);
cudaError_t tc_error_take(unsigned int* word, cudaStream_t st);
}  // namespace nn

// Record the detail string lbm_last_error(NULL) returns on this thread (capi.cu).
void set_thread_error(const std::string& msg);

}  // namespace lbmgb
