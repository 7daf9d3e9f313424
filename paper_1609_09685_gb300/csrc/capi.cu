// capi.cu -- C ABI and host runtime of the GB300 LBM permeability library.
//
// The runtime owns device memory, builds the segment tables, enqueues the
// kernels of lbm_kernels.cu / qsgs.cu on the solver's stream, captures each
// convergence-check interval as a CUDA graph, and takes the scalar decisions
// of the steady-state control (Sec. 2: "iterated to steady state") on the host
// from the FP64 observables the kernels reduce.  Permeability and Kn follow
// Sec. 2 (Darcy's law with the mass flow rate; Kn = sqrt(pi/6)(tau-1/2)/N_x)
// with nu = (tau - 1/2)/3 from Eq. (1).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_launch.h"

using namespace lbmgb;

namespace {
// NVTX range for the lifetime of a scope (named ranges in Nsight timelines;
// header-only, no cost without a tool attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};
}  // namespace

namespace {

thread_local std::string t_err;

struct DomainHost {
    int32_t nx = 0, ny = 0, nz = 1;
    double tau = 1.0, drho = 0.0;
    double g = 0.0;           // body acceleration along +x (force-driven solvers)
    uint32_t seg_begin = 0, nseg = 0;
    uint32_t fluid_begin = 0, fluid_count = 0;
    uint64_t mask_base = 0;
    int32_t active = 1;
    lbm_status status = LBM_NOT_CONVERGED;
    int64_t steps = 0;
    double residual = INFINITY;
    std::vector<double> rhist;
    std::vector<double> kq;   // recent k values for the k-based stop
    int32_t k_ok = 0;         // consecutive checks meeting the k-based stop
    int32_t k_dead = 0;       // consecutive checks with |k| below 0.1 k_tol of its peak
    double k_peak = 0.0;      // largest |k| seen in this run
    bool has_obs = false;
    bool forced_state = false;  // populations are the post-collision state of a forced step
    double obs[kNumObs] = {0};
    // per check interval of the last lbm_run_to_steady: step, k, residual,
    // host seconds since the call began
    std::vector<int64_t> h_step;
    std::vector<double> h_k, h_r, h_t;
};

struct GraphKey {
    int64_t n;
    int obs;
    int parity;
    bool operator<(const GraphKey& o) const {
        if (n != o.n) return n < o.n;
        if (obs != o.obs) return obs < o.obs;
        return parity < o.parity;
    }
};

const char* kVersion = "0.1.0";

}  // namespace

struct lbm_solver {
    int q = 9, eq = 0;
    lbm_options opt{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<DomainHost> dom;
    uint64_t mask_bytes = 0;     // bytes of d_mask (all domains' dense masks)
    std::vector<DomainDev> hdom;
    DomainDev* d_dom = nullptr;
    uint32_t* d_dom_begin = nullptr;
    uint32_t* d_seg_dom = nullptr;
    uint32_t* d_seg_mask = nullptr;
    uint32_t* d_seg_off = nullptr;
    uint32_t* d_seg_cnt = nullptr;
    uint32_t* d_scan = nullptr;
    uint4* d_win = nullptr;
    uint4* d_items = nullptr;
    uint2* d_vitems = nullptr;  // local-step work items
    uint32_t nvitems = 0;
    uint32_t* d_face = nullptr;  // inlet/outlet bits per compact slot
    GatherTile* d_tiles = nullptr;  // staged gather step: tile list
    uint32_t ntiles = 0;
    int tile_rows = 0;              // rows per tile of the staged gather step (0: direct gather step)
    BandItem* d_bands = nullptr;    // band gather step: band list and range records
    uint2* d_band_rng = nullptr;
    uint32_t nbands = 0;
    int band_rows = 0;              // rows per band of the band gather step (0: not used)
    // L2-blocked pairs: the plain steps of a pair run block by block -- gather
    // step of block k + 1, then local step of block k -- so that each block's
    // populations are still in L2 when its local step reads them.  blk_item[k]
    // / blk_vitem[k]: first strip / local-step item of block k (K + 1 entries;
    // empty: one block, the plain pair).
    int pair_block_mb = 0;
    std::vector<uint32_t> blk_item, blk_vitem;
    std::vector<uint4> h_items;     // host copy of the strip work list
    // work queue of the fused pair kernel over those blocks
    uint4* d_units = nullptr;
    uint32_t* d_utotal = nullptr;   // gather units per block
    uint32_t* d_uctr = nullptr;     // ticket and per-block counters
    uint32_t nunits = 0;
    int gather_batch = 0;           // rows in flight per warp of the direct gather step (0: default)
    int strip_rows = 8;             // rows per strip work item
    std::vector<uint32_t> h_off, h_smask;  // segment offsets and fluid masks (host copies)
    // x-slab solvers (lbm_slab_create): compact indices of the exchanged
    // columns: [0] first real column, [1] last real column (packed), [2] left
    // ghost, [3] right ghost (unpacked)
    bool slab = false;
    uint32_t* d_col[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t ncol[4] = {0, 0, 0, 0};
    bool forced = false;         // force-driven, every face periodic (lbm_batch_create_forced)
    bool obs_only = false;       // the last observation was taken without stepping
    float* d_gforce = nullptr;   // body acceleration per domain (force-driven solvers)
    uint32_t nitems = 0;
    uint8_t* d_mask = nullptr;
    uint32_t nseg_total = 0;
    uint64_t nfluid = 0, pstride = 0;
    float* d_g[2] = {nullptr, nullptr};
    int cur = 0;
    float* d_uprev = nullptr;
    double* d_partials = nullptr;
    double* d_obs = nullptr;
    double* h_obs = nullptr;  // pinned
    int64_t step = 0;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::string err;

    Geometry geom() const {
        Geometry G;
        G.dom = d_dom;
        G.seg_dom = d_seg_dom;
        G.seg_mask = d_seg_mask;
        G.seg_off = d_seg_off;
        G.nseg_total = nseg_total;
        G.pstride = pstride;
        return G;
    }
    StepLaunch launch_cfg() const { return StepLaunch{opt.block_threads, tile_rows, gather_batch, band_rows}; }
    HotArgs hot() const {
        HotArgs A;
        A.dom = d_dom;
        A.win = d_win;
        A.items = d_items;
        A.nitems = nitems;
        A.pstride = (uint32_t)pstride;
        A.vitems = d_vitems;
        A.nvitems = nvitems;
        A.face = d_face;
        A.tiles = d_tiles;
        A.ntiles = ntiles;
        A.err = err_word();
        A.bands = d_bands;
        A.nbands = nbands;
        A.band_rng = d_band_rng;
        return A;
    }
    // device error word, kept right after the observables so that every
    // observation brings it back to the host
    uint32_t* err_word() const {
        return d_obs ? reinterpret_cast<uint32_t*>(d_obs + (size_t)kNumObs * dom.size()) : nullptr;
    }
};

namespace {

lbm_status fail(lbm_handle h, lbm_status s, const std::string& msg) {
    if (h) h->err = msg;
    t_err = msg;
    return s;
}

lbm_status cuda_fail(lbm_handle h, cudaError_t e, const char* what) {
    const lbm_status s = (e == cudaErrorMemoryAllocation) ? LBM_ERR_OOM : LBM_ERR_CUDA;
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();  // clear a sticky launch error where possible
    return fail(h, s, m);
}

#define CK(h, call)                                      \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

// Device memory of solvers comes from one stream-ordered pool per device.  The
// pool keeps up to kPoolKeep bytes of freed blocks, so creating and destroying
// solvers in a loop reuses memory instead of returning it to the CUDA driver each
// time; larger frees go back to the CUDA driver at the next synchronisation.
constexpr uint64_t kPoolKeep = 8ull << 30;

cudaError_t solver_pool(cudaMemPool_t* pool) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) {
        *pool = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = kPoolKeep;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(p);
        return e;
    }
    pools[dev] = p;
    *pool = p;
    return cudaSuccess;
}

template <class T>
cudaError_t dmalloc(lbm_handle h, T** ptr, size_t bytes) {
    if (h->opt.alloc_fn) {  // the caller's allocator
        void* p = h->opt.alloc_fn(h->opt.alloc_ctx, bytes, h->st);
        if (!p) return cudaErrorMemoryAllocation;
        *ptr = static_cast<T*>(p);
        return cudaSuccess;
    }
    cudaMemPool_t pool = nullptr;
    cudaError_t e = solver_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(reinterpret_cast<void**>(ptr), bytes, pool, h->st);
}

template <class T>
void dfree(lbm_handle h, T*& p) {
    if (p) {
        if (h->opt.free_fn) h->opt.free_fn(h->opt.alloc_ctx, (void*)p, h->st);
        else cudaFreeAsync(p, h->st);
    }
    p = nullptr;
}

void free_solver(lbm_handle h) {
    if (!h) return;
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    if (h->st) {
        dfree(h, h->d_dom);
        dfree(h, h->d_dom_begin);
        dfree(h, h->d_seg_dom);
        dfree(h, h->d_seg_mask);
        dfree(h, h->d_seg_off);
        dfree(h, h->d_seg_cnt);
        dfree(h, h->d_scan);
        dfree(h, h->d_win);
        dfree(h, h->d_items);
        dfree(h, h->d_vitems);
        dfree(h, h->d_face);
        dfree(h, h->d_tiles);
        dfree(h, h->d_bands);
        dfree(h, h->d_band_rng);
        dfree(h, h->d_units);
        dfree(h, h->d_utotal);
        dfree(h, h->d_uctr);
        for (auto& p : h->d_col) dfree(h, p);
        dfree(h, h->d_mask);
        dfree(h, h->d_g[0]);
        dfree(h, h->d_g[1]);
        dfree(h, h->d_uprev);
        dfree(h, h->d_partials);
        dfree(h, h->d_obs);
        dfree(h, h->d_gforce);
    }
    if (h->h_obs) cudaFreeHost(h->h_obs);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    delete h;
}

double knudsen(double tau, int nx) { return std::sqrt(M_PI / 6.0) * (tau - 0.5) / (double)nx; }

// Darcy's law with the simulated mass flow rate (Sec. 2).  sum_link is the
// mass crossing the N_x - 1 interior x planes in one step, summed over the
// planes; its plane average <J> = sum_link / (N_x - 1) is the mass flow rate,
// U = <J> / (rho A) with A = N_y N_z, mu = rho nu, nu = (tau - 1/2)/3 (Eq. 1),
// dP = c_s^2 drho over L = N_x - 1:  k = nu <J> (N_x - 1) / (A c_s^2 drho).
// Force-driven solvers (Eq. 2): k = nu <u> / g, <u> the sum over fluid nodes of
// rho u_x (observable 0) over rho_0 N_grid.
double darcy_k(const DomainHost& D, double sum_link, bool forced, double rho0) {
    const double nu = (D.tau - 0.5) / 3.0;
    if (forced) return nu * sum_link / (rho0 * (double)D.nx * D.ny * D.nz) / D.g;
    const double jmean = sum_link / (double)(D.nx - 1);
    return nu * jmean * (double)(D.nx - 1) / ((double)D.ny * D.nz * (1.0 / 3.0) * D.drho);
}

lbm_status upload_dom(lbm_handle h) {
    for (size_t d = 0; d < h->dom.size(); ++d) h->hdom[d].active = h->dom[d].active;
    CK(h, cudaMemcpyAsync(h->d_dom, h->hdom.data(), sizeof(DomainDev) * h->hdom.size(),
                          cudaMemcpyHostToDevice, h->st));
    return LBM_OK;
}

// Pull steps (buffer swaps) among n steps: the observing step, and with
// in-place pairs only an odd plain step left over.
int64_t pull_steps(lbm_handle h, int64_t n, bool obs) {
    const int64_t o = (obs && n > 0) ? 1 : 0;
    const int64_t plain = n - o;
    return o + (h->opt.in_place_pairs ? (plain & 1) : plain);
}

// Per-kernel timing for lbm_profile_steps: an event pair around every launch.
struct KernelProf {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    cudaError_t mark(cudaStream_t st) {
        cudaEvent_t e = nullptr;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev.push_back(e);
        return cudaEventRecord(e, st);
    }
    ~KernelProf() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// Enqueue n steps (the last one observing when obs) plus the reduction and the
// copy of the observables to pinned host memory.  Plain steps run as in-place
// pairs on the current buffer (when enabled); the remaining steps pull from
// the current buffer into the other one.  Advances h->cur.  With prof, every
// kernel is bracketed by events (kinds: 0 gather, 1 local, 2 pull, 3 observing
// pull).
lbm_status enqueue_steps(lbm_handle h, int64_t n, bool obs, KernelProf* prof = nullptr) {
    const Geometry G = h->geom();
    const HotArgs A = h->hot();
    const int64_t o = (obs && n > 0) ? 1 : 0;
    int64_t plain = n - o;
    if (h->forced) {
        // plain steps two at a time in place (forced gather step + local
        // step), the rest as pull steps
        int64_t k0 = 0;
        if (h->opt.in_place_pairs) {
            for (; plain >= 2; plain -= 2, k0 += 2)
                for (int half = 0; half < 2; ++half) {
                    if (prof) CK(h, prof->mark(h->st));
                    CK(h, launch_periodic_half(h->q, h->eq, half, A, h->d_gforce, h->d_g[h->cur], h->st));
                    if (prof) {
                        CK(h, prof->mark(h->st));
                        prof->kind.push_back(half);
                    }
                }
        }
        for (int64_t k = k0; k < n; ++k) {
            const bool ob = (o == 1) && (k == n - 1);
            if (prof) CK(h, prof->mark(h->st));
            CK(h, launch_periodic_step(h->q, h->eq, ob, A, h->d_gforce, h->d_g[h->cur], h->d_g[h->cur ^ 1],
                                       h->d_uprev, h->d_partials, h->st));
            if (prof) {
                CK(h, prof->mark(h->st));
                prof->kind.push_back(ob ? 3 : 2);
            }
            h->cur ^= 1;
        }
        plain = 0;
    } else if (h->opt.in_place_pairs) {
        const StepLaunch cfg = h->launch_cfg();
        const size_t K = h->blk_item.empty() ? 0 : h->blk_item.size() - 1;
        const bool blocked = K >= 2 && h->nunits > 0 && cfg.tile_rows <= 0 && cfg.band_rows <= 0;
        PairFused F{};
        F.units = h->d_units;
        F.nunits = h->nunits;
        F.nblocks = (uint32_t)K;
        F.total = h->d_utotal;
        F.ctr = h->d_uctr;
        for (; plain >= 2; plain -= 2) {
            if (blocked) {
                // both steps in one persistent launch, block by block through L2
                if (prof) CK(h, prof->mark(h->st));
                CK(h, launch_aa_pair_fused(h->q, h->eq, A, F, h->d_g[h->cur], cfg, h->st));
                if (prof) {
                    CK(h, prof->mark(h->st));
                    prof->kind.push_back(4);
                }
                continue;
            }
            if (!prof) {
                CK(h, launch_aa_pair(h->q, h->eq, A, h->d_g[h->cur], cfg, h->st));
                continue;
            }
            for (int half = 0; half < 2; ++half) {
                CK(h, prof->mark(h->st));
                CK(h, launch_aa_half(h->q, h->eq, half, A, h->d_g[h->cur], h->launch_cfg(), h->st));
                CK(h, prof->mark(h->st));
                prof->kind.push_back(half);
            }
        }
    }
    for (int64_t k = 0; k < (h->forced ? 0 : plain + o); ++k) {
        const bool ob = (o == 1) && (k == plain);
        if (prof) CK(h, prof->mark(h->st));
        CK(h, launch_stream_collide(h->q, h->eq, ob, A, h->d_g[h->cur], h->d_g[h->cur ^ 1], h->d_uprev,
                                    h->d_partials, h->opt.block_threads, h->st));
        if (prof) {
            CK(h, prof->mark(h->st));
            prof->kind.push_back(ob ? 3 : 2);
        }
        h->cur ^= 1;
    }
    if (obs) {
        h->obs_only = (n == 0);
        if (n == 0) CK(h, launch_observe(h->q, G, h->d_g[h->cur], h->d_uprev, h->d_partials, h->st));
        CK(h, launch_reduce_obs(h->d_dom, (int)h->dom.size(), h->d_partials, h->d_obs, n > 0, h->st));
        CK(h, cudaMemcpyAsync(h->h_obs, h->d_obs, sizeof(double) * (kNumObs * h->dom.size() + 1),
                              cudaMemcpyDeviceToHost, h->st));
    }
    return LBM_OK;
}

// After n > 0 steps of a force-driven solver, the active domains hold the
// post-collision state of a forced step.
void mark_forced_state(lbm_handle h, int64_t n) {
    if (!h->forced || n <= 0) return;
    for (auto& D : h->dom)
        if (D.active) D.forced_state = true;
}

// Same work through a cached CUDA graph (one per step count, observe flag and
// starting buffer parity).
lbm_status run_steps(lbm_handle h, int64_t n, bool obs) {
    mark_forced_state(h, n);
    if (!h->opt.use_graphs || n <= 1 || h->st == nullptr) return enqueue_steps(h, n, obs);
    GraphKey key{n, obs ? 1 : 0, h->cur};
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        const int cur0 = h->cur;
        CK(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
        lbm_status s = enqueue_steps(h, n, obs);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->st, &g);
        h->cur = cur0;
        if (s != LBM_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
        it = h->graphs.emplace(key, ex).first;
    }
    CK(h, cudaGraphLaunch(it->second, h->st));
    if (pull_steps(h, n, obs) & 1) h->cur ^= 1;
    return LBM_OK;
}

lbm_status device_error(lbm_handle h, uint32_t word) {
    if (word == 0) return LBM_OK;
    std::string m = "device error word " + std::to_string(word) + ":";
    if (word & 1u) m += " a staged gather copy did not complete within its wait limit;";
    if (word & 2u) m += " a population index from the index tables was out of range (access skipped);";
    return fail(h, LBM_ERR_INTERNAL, m);
}

lbm_status store_obs(lbm_handle h) {
    uint32_t word = 0;
    std::memcpy(&word, h->h_obs + (size_t)kNumObs * h->dom.size(), sizeof(word));
    if (word) return device_error(h, word);
    for (size_t d = 0; d < h->dom.size(); ++d) {
        if (!h->dom[d].active) continue;
        std::memcpy(h->dom[d].obs, h->h_obs + d * kNumObs, sizeof(double) * kNumObs);
        // An observation without a step comes from the pressure-driven observe
        // kernel (slot 0 = link flux).  For force-driven solvers slot 0 must be
        // the Eq. 2 flux: when the populations come from a forced step, the
        // fluid momentum of Guo's scheme is the stored post-collision momentum
        // (slot 6) minus F/2 per fluid node; a state that no forced step has
        // produced yet (fresh, or set by the caller) holds its fluid momentum
        // as it is.
        if (h->forced && h->obs_only)
            h->dom[d].obs[0] = h->dom[d].obs[6] - (h->dom[d].forced_state ? 0.5 * h->dom[d].g * h->opt.rho_out *
                                                                         h->dom[d].fluid_count
                                                                   : 0.0);
        h->dom[d].has_obs = true;
    }
    return LBM_OK;
}

// Copy a retired domain's populations into the other buffer so both hold its
// final state (no kernel writes a retired domain).
// Permeability-based stop.  The domain-summed FP64 mass flow rate averages out
// most of the FP32 rounding that makes the per-node residual jitter, so k(t)
// converges smoothly until a small jitter floor.  Over windows of W = 10
// checks, the changes D1 = k_i - k_(i-W) and D0 = k_(i-W) - k_(i-2W) of a
// geometric approach shrink by q = |D1 / D0| per window and the remaining error
// is at most |D1| q / (1 - q).  The domain stops once that bound is below
// k_tol |k| at 10 consecutive checks while the velocity residual r is below
// 10 k_tol (early on, a fast mode can set q and hide a slow one; the residual
// still sees the slow mode), or once k has stayed within 0.05 k_tol |k| over
// the last 40 checks (the jitter floor, where the ratio carries no
// information).  The scale of the tolerance is |k|, but at least 1e-3 of the
// largest |k| of the run, so that a domain whose flow dies out also stops.
bool k_converged(DomainHost& D, double k, double r, double k_tol) {
    constexpr size_t W = 10, KEEP = 41;
    D.kq.push_back(k);
    if (D.kq.size() > KEEP) D.kq.erase(D.kq.begin());
    const size_t n = D.kq.size();
    D.k_peak = std::max(D.k_peak, std::fabs(k));
    const double tolk = k_tol * std::max(std::fabs(k), 1e-3 * D.k_peak);
    bool ok = false;
    // a flow that dies out (no connected fluid path) keeps a relative residual
    // of order one while it decays, so the residual gate does not apply there
    const bool vanishing = std::fabs(k) < 1e-3 * D.k_peak;
    if (n >= 2 * W + 1 && (r < 10.0 * k_tol || vanishing)) {
        const double d1 = D.kq[n - 1] - D.kq[n - 1 - W], d0 = D.kq[n - 1 - W] - D.kq[n - 1 - 2 * W];
        if (d0 != 0.0) {
            const double q = std::fabs(d1 / d0);
            if (q < 1.0) ok = std::fabs(d1) * q / (1.0 - q) < tolk;
        } else {
            ok = (d1 == 0.0);
        }
    }
    D.k_ok = ok ? D.k_ok + 1 : 0;
    if (D.k_ok >= 10) return true;
    // vanishing flow: |k| below 0.1 k_tol of its peak for 10 checks in a row
    D.k_dead = (std::fabs(k) < 0.1 * k_tol * D.k_peak) ? D.k_dead + 1 : 0;
    if (D.k_dead >= 10) return true;
    if (n == KEEP) {
        double lo = D.kq[0], hi = D.kq[0];
        for (double v : D.kq) {
            lo = std::min(lo, v);
            hi = std::max(hi, v);
        }
        if (hi - lo < 0.05 * tolk) return true;
    }
    return false;
}

lbm_status mirror_domain(lbm_handle h, size_t d) {
    const DomainHost& D = h->dom[d];
    if (D.fluid_count == 0) return LBM_OK;
    for (int i = 0; i < h->q; ++i) {
        const size_t off = (size_t)i * h->pstride + D.fluid_begin;
        CK(h, cudaMemcpyAsync(h->d_g[h->cur ^ 1] + off, h->d_g[h->cur] + off, sizeof(float) * D.fluid_count,
                              cudaMemcpyDeviceToDevice, h->st));
    }
    return LBM_OK;
}

lbm_status check_domain(lbm_handle h, int32_t d) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (d < 0 || d >= (int32_t)h->dom.size()) return fail(h, LBM_ERR_ARG, "domain index out of range");
    return LBM_OK;
}

}  // namespace

void lbmgb::set_thread_error(const std::string& msg) { t_err = msg; }

// ---------------------------------------------------------------------------
extern "C" {

const char* lbm_version(void) { return kVersion; }

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_NOT_CONVERGED: return "not converged (max_steps reached)";
        case LBM_STALLED: return "stalled at the FP32 residual floor";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_OOM: return "out of device memory";
        case LBM_DIVERGED: return "diverged (non-finite velocity)";
        case LBM_TIMEOUT: return "timeout";
        case LBM_ERR_IO: return "I/O error";
        case LBM_ERR_INTERNAL: return "internal error";
        case LBM_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

const char* lbm_last_error(lbm_handle h) { return h ? h->err.c_str() : t_err.c_str(); }

}  // extern "C"

namespace {
template <class L>
void lattice_tables(int32_t* c, double* w, int32_t* o, int32_t* fy, int32_t* fz) {
    for (int i = 0; i < L::Q; ++i) {
        if (c)
            for (int a = 0; a < 3; ++a) c[3 * i + a] = L::c(i, a);
        if (w) w[i] = L::wd(i);
        if (o) o[i] = opp<L>(i);
        if (fy) fy[i] = flip<L>(i, true, false);
        if (fz) fz[i] = flip<L>(i, false, true);
    }
}
}  // namespace

extern "C" {

lbm_status lbm_lattice(int32_t q, int32_t* c, double* w, int32_t* opp_out, int32_t* flip_y, int32_t* flip_z) {
    if (q == 9) lattice_tables<D2Q9>(c, w, opp_out, flip_y, flip_z);
    else if (q == 19) lattice_tables<D3Q19>(c, w, opp_out, flip_y, flip_z);
    else return fail(nullptr, LBM_ERR_ARG, "q must be 9 (D2Q9) or 19 (D3Q19)");
    return LBM_OK;
}

void lbm_options_default(lbm_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->struct_size = (int32_t)sizeof(lbm_options);
    o->equilibrium = LBM_EQ_QUADRATIC;
    o->check_interval = 100;
    o->stall_checks = 200;
    o->stall_floor = 1e-5;
    o->rho_out = 1.0;
    o->stream = nullptr;
    o->block_threads = 0;
    o->use_graphs = 1;
    o->cancel_flag = nullptr;
    o->strip_rows = 0;
    o->k_tol = 1e-5;
    o->in_place_pairs = 1;
    o->collision = LBM_COLL_BGK;
    o->trt_lambda = 3.0 / 16.0;
    o->band_rows = 0;
    o->pair_block_mb = 0;
}

lbm_status lbm_qsgs(uint64_t seed, int32_t nx, int32_t ny, int32_t nz, double core_p, double porosity,
                    double d_face, void* stream, uint8_t* mask_out, int32_t* iterations) {
    Range r("lbm_qsgs");
    if (!mask_out) return fail(nullptr, LBM_ERR_ARG, "mask_out is null");
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_ERR_ARG, "sizes must be >= 1");
    const uint64_t N = (uint64_t)nx * ny * nz;
    if (N > (1ull << 31)) return fail(nullptr, LBM_ERR_ARG, "more than 2^31 cells");
    if (!(porosity >= 0.0 && porosity <= 1.0)) return fail(nullptr, LBM_ERR_ARG, "porosity outside [0,1]");
    if (!(core_p >= 0.0 && core_p <= 1.0) || !(d_face >= 0.0 && d_face <= 1.0))
        return fail(nullptr, LBM_ERR_ARG, "probabilities outside [0,1]");
    cudaStream_t st = (cudaStream_t)stream;
    QsgsScratch sc{};
    uint8_t* d_mask = nullptr;
    lbm_status rs = LBM_OK;
    // scratch from the solvers' stream-ordered pool, on the caller's stream
    cudaMemPool_t pool = nullptr;
    cudaError_t e = solver_pool(&pool);
    auto palloc = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes, pool, st);
    };
    palloc(&sc.keys, sizeof(uint64_t) * N);
    palloc(&sc.start, N);
    palloc(&sc.counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&sc.host_counter, sizeof(unsigned long long));
    palloc(&d_mask, N);
    if (e != cudaSuccess) {
        rs = cuda_fail(nullptr, e, "qsgs allocation");
    } else {
        int it = 0;
        cudaError_t ce = cudaSuccess;
        const int r = qsgs_generate(seed, nx, ny, nz, core_p, porosity, d_face, d_mask, sc, st, &it, &ce);
        if (r == -2) rs = cuda_fail(nullptr, ce, "qsgs kernels");
        else if (r == -1) rs = fail(nullptr, LBM_ERR_ARG, "bad qsgs arguments");
        else if (r == -3) rs = fail(nullptr, LBM_ERR_INTERNAL, "no solid core to grow from");
        else if (r == -4) rs = fail(nullptr, LBM_ERR_INTERNAL, "growth iteration cap reached before the target porosity");
        else {
            e = cudaMemcpyAsync(mask_out, d_mask, N, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rs = cuda_fail(nullptr, e, "qsgs copy-out");
            if (iterations) *iterations = it;
        }
    }
    for (void* p : {(void*)sc.keys, (void*)sc.start, (void*)sc.counter, (void*)d_mask})
        if (p) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);  // the pinned counter may be read by work still queued on an error path
    if (sc.host_counter) cudaFreeHost(sc.host_counter);
    return rs;
}

namespace {

// Strip work list of the pull and direct gather steps: per domain and z
// plane, runs of up to R rows at each segment column, with the column
// innermost so that warps of one block (and neighbouring blocks) sweep
// adjacent segments of the same rows -- contiguous compact ranges in every
// population plane.  Strips whose segments are all solid are left out.  Sets
// each domain's item range and uploads the list and the domain records.
lbm_status build_items(lbm_handle h, int R) {
    const int n = (int)h->dom.size();
    const std::vector<uint32_t>& smask = h->h_smask;
    std::vector<uint4> items;
    for (int d = 0; d < n; ++d) {
        DomainDev& G = h->hdom[d];
        G.item_base = (uint32_t)items.size();
        for (int z = 0; z < G.nz; ++z)
            for (int y0 = 0; y0 < G.ny; y0 += R)
                for (int sidx = 0; sidx < G.nseg; ++sidx) {
                    const int nr = std::min(R, G.ny - y0);
                    const uint32_t g0 = G.seg_base + ((uint32_t)z * G.ny + y0) * G.nseg + sidx;
                    bool any = false;
                    for (int k = 0; k < nr && !any; ++k) any = smask[g0 + (uint32_t)k * G.nseg] != 0u;
                    if (!any) continue;
                    items.push_back(make_uint4(g0, (uint32_t)d | ((uint32_t)nr << 24),
                                               (uint32_t)y0 | ((uint32_t)z << 16), (uint32_t)sidx));
                }
        G.nitems = (uint32_t)items.size() - G.item_base;
    }
    dfree(h, h->d_items);
    h->h_items = items;
    h->nitems = (uint32_t)items.size();
    CK(h, dmalloc(h, &h->d_items, sizeof(uint4) * std::max<size_t>(items.size(), 1)));
    CK(h, cudaMemcpyAsync(h->d_items, items.data(), sizeof(uint4) * items.size(), cudaMemcpyHostToDevice, h->st));
    for (int d = 0; d < n; ++d) h->hdom[d].active = h->dom[d].active;
    CK(h, cudaMemcpyAsync(h->d_dom, h->hdom.data(), sizeof(DomainDev) * n, cudaMemcpyHostToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    h->strip_rows = R;
    return LBM_OK;
}

// Tiles of the staged gather step (D2Q9 in-place pairs): per domain and z
// plane, tr rows x kTileSegs segment columns, column groups innermost;
// all-solid tiles are left out.  For each source row (the rows above and
// below included, clamped onto the domain) the 16-byte aligned compact range
// that covers nodes 32 s0 - 1 .. 32 (s0 + nsegs).  tr = 0 drops the list
// (direct gather step).
lbm_status build_tiles(lbm_handle h, int tr) {
    const int n = (int)h->dom.size();
    if (tr && (h->q != 9 || !h->opt.in_place_pairs || h->forced)) tr = 0;
    for (int d = 0; d < n && tr; ++d)
        if (h->hdom[d].nseg > 65535) tr = 0;  // s0 is packed in 16 bits
    const std::vector<uint32_t>& smask = h->h_smask;
    const std::vector<uint32_t>& off = h->h_off;
    std::vector<GatherTile> tiles;
    for (int d = 0; d < n && tr; ++d) {
        const DomainDev& G = h->hdom[d];
        for (int z = 0; z < G.nz; ++z)
            for (int y0 = 0; y0 < G.ny; y0 += tr)
                for (int s0 = 0; s0 < G.nseg; s0 += kTileSegs) {
                    const int nr = std::min(tr, G.ny - y0), ns = std::min(kTileSegs, G.nseg - s0);
                    auto seg = [&](int y, int sx) {
                        return G.seg_base + ((uint32_t)z * G.ny + (uint32_t)y) * (uint32_t)G.nseg + (uint32_t)sx;
                    };
                    bool any = false;
                    for (int r = 0; r < nr && !any; ++r)
                        for (int k = 0; k < ns && !any; ++k) any = smask[seg(y0 + r, s0 + k)] != 0u;
                    if (!any) continue;
                    GatherTile T{};
                    T.dom = (uint32_t)d;
                    T.yz = (uint32_t)y0 | ((uint32_t)z << 16);
                    T.shape = (uint32_t)nr | ((uint32_t)ns << 8) | ((uint32_t)s0 << 16);
                    T.dims = (uint32_t)G.ny | ((uint32_t)G.nseg << 16);
                    T.wbase = seg(0, s0);
                    for (int qq = 0; qq < nr + 2; ++qq) {
                        const int yc = std::min(std::max(y0 - 1 + qq, 0), G.ny - 1);
                        const uint32_t g0 = seg(yc, s0), g1 = seg(yc, s0 + ns - 1);
                        const uint32_t left = s0 > 0 ? (smask[g0 - 1] >> 31) & 1u : 0u;
                        const uint32_t right = s0 + ns < G.nseg ? smask[g1 + 1] & 1u : 0u;
                        const uint32_t lo = off[g0] - left;
                        const uint32_t hi = off[g1] + (uint32_t)__builtin_popcount(smask[g1]) + right;
                        const uint32_t a0 = lo & ~3u, a1 = (hi + 3u) & ~3u;
                        T.a0[qq] = a0;
                        T.n16[qq] = (uint16_t)(hi > lo ? (a1 - a0) / 4u : 0u);
                    }
                    tiles.push_back(T);
                }
    }
    dfree(h, h->d_tiles);
    h->tile_rows = tr;
    h->ntiles = (uint32_t)tiles.size();
    if (tr) {
        CK(h, dmalloc(h, &h->d_tiles, sizeof(GatherTile) * std::max<size_t>(tiles.size(), 1)));
        CK(h, cudaMemcpyAsync(h->d_tiles, tiles.data(), sizeof(GatherTile) * tiles.size(), cudaMemcpyHostToDevice,
                              h->st));
        CK(h, cudaStreamSynchronize(h->st));
    }
    return LBM_OK;
}

// Bands of the band gather step (D2Q9 in-place pairs): per domain, runs of up
// to br rows at each piece of the width -- the domain's segment columns split
// into ceil(nseg / kBandSegs) pieces as even as possible -- pieces innermost;
// all-solid bands are left out.  Range records for the rows y0 - 1 ..
// y0 + nrows of each band: the 16-byte aligned compact range covering nodes
// 32 s0 - 1 .. 32 (s0 + nsegs) (length 0 for a row outside the domain or
// without fluid there).  br = 0 drops the list.
lbm_status build_bands(lbm_handle h, int br) {
    const int n = (int)h->dom.size();
    if (br && (!band_gather_lattice(h->q) || !h->opt.in_place_pairs || h->forced || h->slab)) br = 0;
    for (int d = 0; d < n && br; ++d)
        if (h->hdom[d].nseg > 65535 || h->hdom[d].ny > 65535 || h->hdom[d].nz != 1) br = 0;
    const std::vector<uint32_t>& smask = h->h_smask;
    const std::vector<uint32_t>& off = h->h_off;
    std::vector<uint4> bands;
    std::vector<uint2> rng;
    for (int d = 0; d < n && br; ++d) {
        const DomainDev& G = h->hdom[d];
        const int pieces = (G.nseg + kBandSegs - 1) / kBandSegs;
        auto seg = [&](int y, int sx) { return G.seg_base + (uint32_t)y * (uint32_t)G.nseg + (uint32_t)sx; };
        for (int y0 = 0; y0 < G.ny; y0 += br)
            for (int p = 0, s0 = 0; p < pieces; ++p) {
                const int ns = G.nseg / pieces + (p < G.nseg % pieces ? 1 : 0);
                const int nr = std::min(br, G.ny - y0);
                bool any = false;
                for (int r = 0; r < nr && !any; ++r)
                    for (int k = 0; k < ns && !any; ++k) any = smask[seg(y0 + r, s0 + k)] != 0u;
                if (any) {
                    bands.push_back(make_uint4((uint32_t)d, (uint32_t)y0 | ((uint32_t)nr << 16),
                                               (uint32_t)s0 | ((uint32_t)ns << 16), (uint32_t)rng.size()));
                    for (int r = y0 - 1; r <= y0 + nr; ++r) {
                        if (r < 0 || r >= G.ny) {
                            rng.push_back(make_uint2(0u, 0u));
                            continue;
                        }
                        const uint32_t g0 = seg(r, s0), g1 = seg(r, s0 + ns - 1);
                        const uint32_t left = s0 > 0 ? (smask[g0 - 1] >> 31) & 1u : 0u;
                        const uint32_t right = s0 + ns < G.nseg ? smask[g1 + 1] & 1u : 0u;
                        const uint32_t lo = off[g0] - left;
                        const uint32_t hi = off[g1] + (uint32_t)__builtin_popcount(smask[g1]) + right;
                        const uint32_t a0 = lo & ~3u, a1 = (hi + 3u) & ~3u;
                        rng.push_back(make_uint2(a0, hi > lo ? (a1 - a0) / 4u : 0u));
                    }
                }
                s0 += ns;
            }
    }
    dfree(h, h->d_bands);
    dfree(h, h->d_band_rng);
    h->band_rows = br;
    h->nbands = (uint32_t)bands.size();
    if (br) {
        CK(h, dmalloc(h, &h->d_bands, sizeof(uint4) * std::max<size_t>(bands.size(), 1)));
        CK(h, dmalloc(h, &h->d_band_rng, sizeof(uint2) * std::max<size_t>(rng.size(), 1)));
        CK(h, cudaMemcpyAsync(h->d_bands, bands.data(), sizeof(uint4) * bands.size(), cudaMemcpyHostToDevice, h->st));
        CK(h, cudaMemcpyAsync(h->d_band_rng, rng.data(), sizeof(uint2) * rng.size(), cudaMemcpyHostToDevice, h->st));
        CK(h, cudaStreamSynchronize(h->st));
    }
    return LBM_OK;
}

// Blocks of the L2-blocked pairs: consecutive runs of the strip list holding
// about mb MB of populations each, cut only where the local step of one block
// can follow the gather step of the next -- between row groups of a 2D domain,
// between z planes of a 3D one, or between domains.  Local-step items go to
// the block holding their last slot: a slot's writers in the gather step are
// its own row and the neighbouring rows (planes in 3D), so every writer of a
// block-k item lies in blocks <= k + 1.  mb = 0 drops the blocks.
lbm_status build_pair_blocks(lbm_handle h, int mb) {
    h->blk_item.clear();
    h->blk_vitem.clear();
    h->pair_block_mb = 0;
    h->nunits = 0;
    if (mb <= 0 || !h->opt.in_place_pairs || h->forced || h->slab) return LBM_OK;
    const uint64_t target = std::max<uint64_t>((uint64_t)mb << 20, 1) / (4ull * (uint64_t)h->q);
    std::vector<uint32_t> cstart;  // compact index where each block begins
    uint32_t prev_d = ~0u, prev_z = ~0u, prev_y = ~0u;
    uint64_t block_c0 = 0;
    for (uint32_t i = 0; i < (uint32_t)h->h_items.size(); ++i) {
        const uint4 it = h->h_items[i];
        const uint32_t d = it.y & 0xffffffu, y0 = it.z & 0xffffu, z = it.z >> 16;
        if (d == prev_d && z == prev_z && y0 == prev_y) continue;
        const DomainDev& G = h->hdom[d];
        const bool cut_ok = d != prev_d || (G.nz == 1 ? y0 != prev_y : z != prev_z);
        const uint32_t c = h->h_off[G.seg_base + ((uint32_t)z * (uint32_t)G.ny + y0) * (uint32_t)G.nseg];
        if (h->blk_item.empty() || (cut_ok && (uint64_t)c - block_c0 >= target)) {
            h->blk_item.push_back(i);
            cstart.push_back(h->blk_item.size() == 1 ? 0u : c);
            block_c0 = c;
        }
        prev_d = d;
        prev_z = z;
        prev_y = y0;
    }
    h->pair_block_mb = mb;
    if (h->blk_item.size() < 2) {  // one block: whole-batch pairs
        h->blk_item.clear();
        return LBM_OK;
    }
    h->blk_item.push_back((uint32_t)h->h_items.size());
    // local-step items, in the order the create call made them
    const uint32_t span = 32u * (uint32_t)local_step_vector(h->q);
    const size_t K = cstart.size();
    h->blk_vitem.assign(K + 1, 0u);
    uint32_t j = 0;
    size_t k = 0;
    for (size_t d = 0; d < h->hdom.size(); ++d)
        for (uint32_t c = h->hdom[d].fluid_begin; c < h->hdom[d].fluid_end; c += span, ++j) {
            const uint32_t last = std::min(c + span, h->hdom[d].fluid_end) - 1u;
            while (k + 1 < K && cstart[k + 1] <= last) h->blk_vitem[++k] = j;
        }
    while (k + 1 <= K) h->blk_vitem[++k] = j;
    // work queue: G(k) = the gather units of block k (kFusedGather strips
    // each), L(k) = its local units (kFusedLocal items each), L(k) after
    // G(k + lag); lag = about kFusedLagMb of blocks ahead
    const uint32_t lag = (uint32_t)std::max(1, (kFusedLagMb + mb / 2) / mb);
    std::vector<uint4> units;
    std::vector<uint32_t> total(K, 0u);
    for (size_t b = 0; b < K + lag; ++b) {
        if (b < K)
            for (uint32_t i = h->blk_item[b]; i < h->blk_item[b + 1]; i += kFusedGather, ++total[b])
                units.push_back(make_uint4((uint32_t)b << 1, i, std::min(kFusedGather, h->blk_item[b + 1] - i), 0u));
        if (b >= lag) {
            const size_t c = b - lag;
            for (uint32_t i = h->blk_vitem[c]; i < h->blk_vitem[c + 1]; i += kFusedLocal)
                units.push_back(make_uint4(((uint32_t)c << 1) | 1u, i, std::min(kFusedLocal, h->blk_vitem[c + 1] - i), 0u));
        }
    }
    dfree(h, h->d_units);
    dfree(h, h->d_utotal);
    dfree(h, h->d_uctr);
    h->nunits = (uint32_t)units.size();
    CK(h, dmalloc(h, &h->d_units, sizeof(uint4) * std::max<size_t>(units.size(), 1)));
    CK(h, dmalloc(h, &h->d_utotal, sizeof(uint32_t) * K));
    CK(h, dmalloc(h, &h->d_uctr, sizeof(uint32_t) * (K + 2)));
    CK(h, cudaMemcpyAsync(h->d_units, units.data(), sizeof(uint4) * units.size(), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->d_utotal, total.data(), sizeof(uint32_t) * K, cudaMemcpyHostToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return LBM_OK;
}

// Compact indices of a slab's exchanged columns, fluid nodes in (z, y) order.
lbm_status build_slab_columns(lbm_handle h) {
    const DomainDev& G = h->hdom[0];
    const int first = (G.ghost & 1u) ? 1 : 0, last = G.nx - 1 - ((G.ghost & 2u) ? 1 : 0);
    const int cols[4] = {first, last, 0, G.nx - 1};
    const bool used[4] = {(G.ghost & 1u) != 0, (G.ghost & 2u) != 0, (G.ghost & 1u) != 0, (G.ghost & 2u) != 0};
    for (int c = 0; c < 4; ++c) {
        if (!used[c]) continue;
        std::vector<uint32_t> idx;
        const int xc = cols[c];
        for (int z = 0; z < G.nz; ++z)
            for (int y = 0; y < G.ny; ++y) {
                const uint32_t g = G.seg_base + ((uint32_t)z * G.ny + (uint32_t)y) * (uint32_t)G.nseg + (uint32_t)(xc >> 5);
                const uint32_t m = h->h_smask[g], bit = (uint32_t)(xc & 31);
                if ((m >> bit) & 1u) idx.push_back(h->h_off[g] + (uint32_t)__builtin_popcount(m & ((1u << bit) - 1u)));
            }
        h->ncol[c] = (uint32_t)idx.size();
        CK(h, dmalloc(h, &h->d_col[c], sizeof(uint32_t) * std::max<size_t>(idx.size(), 1)));
        CK(h, cudaMemcpyAsync(h->d_col[c], idx.data(), sizeof(uint32_t) * idx.size(), cudaMemcpyHostToDevice, h->st));
    }
    CK(h, cudaStreamSynchronize(h->st));
    return LBM_OK;
}

}  // namespace

struct SlabInfo {
    int32_t x0, nx_glob;
    uint32_t ghost;
};

static lbm_status create_impl(int32_t n, const lbm_domain_desc* descs, const lbm_options* opt, int force_q,
                              lbm_handle* out, const double* gforce = nullptr, const SlabInfo* slab = nullptr) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is null");
    *out = nullptr;
    if (n < 1 || !descs) return fail(nullptr, LBM_ERR_ARG, "need at least one domain");
    lbm_options o;
    lbm_options_default(&o);
    if (opt) {
        if (opt->struct_size != (int32_t)sizeof(lbm_options))
            return fail(nullptr, LBM_ERR_ARG, "lbm_options.struct_size mismatch");
        o = *opt;
    }
    if (o.check_interval < 1 || o.stall_checks < 1 || !(o.rho_out > 0.0) || !(o.k_tol >= 0.0) ||
        (o.equilibrium != LBM_EQ_QUADRATIC && o.equilibrium != LBM_EQ_LINEAR) || o.block_threads < 0 ||
        o.block_threads > 256 || (o.block_threads % 32) != 0 || o.strip_rows < 0 || o.strip_rows > 255 ||
        (o.in_place_pairs != 0 && o.in_place_pairs != 1) ||
        (o.collision != LBM_COLL_BGK && o.collision != LBM_COLL_TRT) ||
        !(o.trt_lambda > 0.0 && std::isfinite(o.trt_lambda)) || o.tile_rows < -1 || o.tile_rows > kTileRowsMax ||
        o.band_rows < -1 || o.band_rows > kBandRowsMax || (o.tile_rows > 0 && o.band_rows > 0) ||
        o.pair_block_mb < -1 || o.pair_block_mb > kPairBlockMbMax ||
        (o.autotune != 0 && o.autotune != 1) || o.gather_batch < 0 || (!o.alloc_fn != !o.free_fn))
        return fail(nullptr, LBM_ERR_ARG, "invalid options");
    if (slab) o.in_place_pairs = 0;  // a slab's ghost columns are refreshed between single pull steps
    if (gforce) {
        for (int d = 0; d < n; ++d)
            if (!std::isfinite(gforce[d])) return fail(nullptr, LBM_ERR_ARG, "g must be finite");
    }
    int q = force_q;
    if (!q) {
        q = 9;
        for (int d = 0; d < n; ++d)
            if (descs[d].nz > 1) q = 19;
    }
    uint64_t segs = 0, cells = 0;
    for (int d = 0; d < n; ++d) {
        const lbm_domain_desc& D = descs[d];
        if (!D.mask) return fail(nullptr, LBM_ERR_ARG, "domain mask is null");
        if (D.nx < 3 || D.ny < 1 || D.nz < 1) return fail(nullptr, LBM_ERR_ARG, "need nx >= 3, ny >= 1, nz >= 1");
        if (D.ny > 65535 || D.nz > 65535) return fail(nullptr, LBM_ERR_ARG, "ny and nz must be <= 65535");
        if (q == 9 && D.nz != 1) return fail(nullptr, LBM_ERR_ARG, "D2Q9 domains need nz = 1");
        if (!(D.tau > 0.5) || !std::isfinite(D.tau)) return fail(nullptr, LBM_ERR_ARG, "tau must be > 0.5");
        if (!gforce && (!std::isfinite(D.drho) || std::fabs(D.drho) >= o.rho_out))
            return fail(nullptr, LBM_ERR_ARG, "drho must be finite and |drho| < rho_out");
        const uint64_t N = (uint64_t)D.nx * D.ny * D.nz;
        uint8_t bad = 0;  // OR of the bits above bit 0 (a branch-free loop the compiler vectorises)
        for (uint64_t k = 0; k < N; ++k) bad |= (uint8_t)(D.mask[k] & 0xFEu);
        if (bad) return fail(nullptr, LBM_ERR_ARG, "mask bytes must be 0 (fluid) or 1 (solid)");
        segs += (uint64_t)((D.nx + kSegW - 1) / kSegW) * D.ny * D.nz;
        cells += N;
    }
    if (segs >= (1ull << 32) || (cells + 32ull * (n + 2)) * q >= (1ull << 32) || n >= (1 << 24))
        return fail(nullptr, LBM_ERR_ARG, "batch too large (Q x nodes must stay below 2^32)");

    lbm_handle h = new lbm_solver();
    h->q = q;
    h->eq = o.equilibrium;
    h->forced = gforce != nullptr;
    h->slab = slab != nullptr;
    h->opt = o;
    if (o.stream) {
        h->st = (cudaStream_t)o.stream;
    } else {
        cudaError_t e = cudaStreamCreate(&h->st);
        if (e != cudaSuccess) {
            lbm_status s = cuda_fail(nullptr, e, "cudaStreamCreate");
            free_solver(h);
            return s;
        }
        h->own_stream = true;
    }
    h->dom.resize(n);
    h->hdom.resize(n);
    std::vector<uint32_t> begin(n + 1);
    uint64_t mb = 0;
    uint32_t sb = 0;
    for (int d = 0; d < n; ++d) {
        const lbm_domain_desc& S = descs[d];
        DomainHost& D = h->dom[d];
        D.nx = S.nx;
        D.ny = S.ny;
        D.nz = S.nz;
        D.tau = S.tau;
        D.drho = gforce ? 0.0 : S.drho;
        D.g = gforce ? gforce[d] : 0.0;
        D.seg_begin = sb;
        D.nseg = (uint32_t)((S.nx + kSegW - 1) / kSegW) * S.ny * S.nz;
        D.mask_base = mb;
        begin[d] = sb;
        DomainDev& G = h->hdom[d];
        G.nx = S.nx;
        G.ny = S.ny;
        G.nz = S.nz;
        G.nseg = (S.nx + kSegW - 1) / kSegW;
        G.seg_base = sb;
        G.nseg_dom = D.nseg;
        G.omega = (float)(1.0 / S.tau);
        G.omega_m = o.collision == LBM_COLL_TRT ? (float)(1.0 / (0.5 + o.trt_lambda / (S.tau - 0.5))) : G.omega;
        G.drho_in = gforce ? 0.0f : (float)S.drho;
        G.rho0 = (float)o.rho_out;
        G.active = 1;
        G.mask_base = mb;
        G.x0 = slab ? slab->x0 : 0;
        G.nx_glob = slab ? slab->nx_glob : S.nx;
        G.ghost = slab ? slab->ghost : 0u;
        mb += (uint64_t)S.nx * S.ny * S.nz;
        sb += D.nseg;
    }
    begin[n] = sb;
    h->nseg_total = sb;
    *out = h;

#define CKC(call)                                  \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            lbm_status s_ = cuda_fail(nullptr, e_, #call); \
            free_solver(h);                        \
            *out = nullptr;                        \
            return s_;                             \
        }                                          \
    } while (0)

    CKC(dmalloc(h, &h->d_dom, sizeof(DomainDev) * n));
    CKC(dmalloc(h, &h->d_dom_begin, sizeof(uint32_t) * (n + 1)));
    CKC(dmalloc(h, &h->d_seg_dom, sizeof(uint32_t) * std::max<uint32_t>(sb, 1)));
    CKC(dmalloc(h, &h->d_seg_mask, sizeof(uint32_t) * std::max<uint32_t>(sb, 1)));
    CKC(dmalloc(h, &h->d_seg_off, sizeof(uint32_t) * std::max<uint32_t>(sb, 1)));
    CKC(dmalloc(h, &h->d_seg_cnt, sizeof(uint32_t) * std::max<uint32_t>(sb, 1)));
    CKC(dmalloc(h, &h->d_scan, sizeof(uint32_t) * ((sb + 1023) / 1024 + 2)));
    CKC(dmalloc(h, &h->d_mask, std::max<uint64_t>(mb, 1)));
    CKC(cudaMemcpyAsync(h->d_dom, h->hdom.data(), sizeof(DomainDev) * n, cudaMemcpyHostToDevice, h->st));
    CKC(cudaMemcpyAsync(h->d_dom_begin, begin.data(), sizeof(uint32_t) * (n + 1), cudaMemcpyHostToDevice, h->st));
    h->mask_bytes = mb;
    for (int d = 0; d < n; ++d)  // straight from the caller's buffers (DMA when they are pinned)
        CKC(cudaMemcpyAsync(h->d_mask + h->hdom[d].mask_base, descs[d].mask,
                            (size_t)descs[d].nx * descs[d].ny * descs[d].nz, cudaMemcpyHostToDevice, h->st));
    const uint32_t nscan = (sb + 1023) / 1024;
    CKC(launch_seg_setup(h->d_dom, h->d_dom_begin, n, sb, h->d_mask, h->d_seg_dom, h->d_seg_mask, h->d_seg_cnt,
                         h->d_seg_off, h->d_scan, h->d_scan + nscan + 1, h->st));
    std::vector<uint32_t> off(sb + 1), smask(std::max<uint32_t>(sb, 1));
    uint32_t total = 0;
    CKC(cudaMemcpyAsync(off.data(), h->d_seg_off, sizeof(uint32_t) * sb, cudaMemcpyDeviceToHost, h->st));
    CKC(cudaMemcpyAsync(smask.data(), h->d_seg_mask, sizeof(uint32_t) * sb, cudaMemcpyDeviceToHost, h->st));
    CKC(cudaMemcpyAsync(&total, h->d_scan + nscan + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->st));
    CKC(cudaStreamSynchronize(h->st));
    off[sb] = total;
    h->nfluid = total;
    // Each domain's compact range starts on a 32-slot boundary, so that the
    // local step of the in-place pair moves whole aligned vectors; the slots
    // in between belong to no node and stay zero.
    {
        uint32_t pos = 0;
        for (int d = 0; d < n; ++d) {
            const uint32_t b0 = off[begin[d]], cnt = off[begin[d + 1]] - b0;
            const uint32_t nb = (pos + 31u) / 32u * 32u;
            for (uint32_t g = begin[d]; g < begin[d + 1]; ++g) off[g] = off[g] - b0 + nb;
            h->dom[d].fluid_begin = nb;
            h->dom[d].fluid_count = cnt;
            h->hdom[d].fluid_begin = nb;
            h->hdom[d].fluid_end = nb + cnt;
            pos = nb + cnt;
        }
        total = (pos + 31u) / 32u * 32u;
        off[sb] = total;
        CKC(cudaMemcpyAsync(h->d_seg_off, off.data(), sizeof(uint32_t) * sb, cudaMemcpyHostToDevice, h->st));
    }
    // local-step work items: 32 lanes x V slots of one domain each
    {
        const uint32_t span = 32u * (uint32_t)local_step_vector(q);
        std::vector<uint2> vit;
        for (int d = 0; d < n; ++d)
            for (uint32_t k = h->hdom[d].fluid_begin; k < h->hdom[d].fluid_end; k += span)
                vit.push_back(make_uint2(k, (uint32_t)d));
        h->nvitems = (uint32_t)vit.size();
        CKC(dmalloc(h, &h->d_vitems, sizeof(uint2) * std::max<size_t>(vit.size(), 1)));
        CKC(cudaMemcpyAsync(h->d_vitems, vit.data(), sizeof(uint2) * vit.size(), cudaMemcpyHostToDevice, h->st));
        CKC(cudaStreamSynchronize(h->st));
    }
    {
        int lo, hi, def;
        gather_batches(q, &lo, &hi, &def);
        if (o.gather_batch != 0 && o.gather_batch != lo && o.gather_batch != hi) {
            free_solver(h);
            *out = nullptr;
            return fail(nullptr, LBM_ERR_ARG, "gather_batch must be 0 or one of the lattice's compiled batches");
        }
        h->gather_batch = o.gather_batch;
    }
    h->h_off.assign(off.begin(), off.end() - 1);
    h->h_smask.assign(smask.begin(), smask.begin() + sb);
    {
        lbm_status bs = build_items(h, o.strip_rows > 0 ? o.strip_rows : 8);
        if (bs == LBM_OK) bs = build_tiles(h, o.tile_rows > 0 ? o.tile_rows : 0);
        if (bs == LBM_OK) bs = build_bands(h, o.band_rows > 0 ? o.band_rows : (o.band_rows == 0 && o.tile_rows <= 0 ? kBandRowsDefault : 0));
        if (bs == LBM_OK)
            bs = build_pair_blocks(h, o.pair_block_mb > 0 ? o.pair_block_mb
                                                          : (o.pair_block_mb == 0 ? kPairBlockMbDefault : 0));
        if (bs == LBM_OK && slab) bs = build_slab_columns(h);
        if (bs != LBM_OK) {
            free_solver(h);
            *out = nullptr;
            return bs;
        }
    }
    CKC(dmalloc(h, &h->d_win, sizeof(uint4) * std::max<uint32_t>(sb, 1)));
    CKC(launch_build_windows(h->d_dom, h->d_seg_dom, sb, h->d_seg_mask, h->d_seg_off, h->d_win, h->st));
    CKC(cudaStreamSynchronize(h->st));
    // one padding slot past the last fluid node: the stream-collide kernel
    // loads unconditionally and a solid lane may address slot nfluid
    h->pstride = ((uint64_t)total + 1 + 31) / 32 * 32;
    CKC(dmalloc(h, &h->d_face, sizeof(uint32_t) * (h->pstride / 16)));
    CKC(cudaMemsetAsync(h->d_face, 0, sizeof(uint32_t) * (h->pstride / 16), h->st));
    CKC(launch_build_face(h->d_dom, h->d_seg_dom, sb, h->d_seg_mask, h->d_seg_off, h->d_face, h->st));
    const int D = (q == 9) ? 2 : 3;
    CKC(dmalloc(h, &h->d_g[0], sizeof(float) * q * h->pstride));
    CKC(dmalloc(h, &h->d_g[1], sizeof(float) * q * h->pstride));
    CKC(dmalloc(h, &h->d_uprev, sizeof(float) * D * h->pstride));
    // partials: one per strip item (at most one per segment, whatever the strip
    // rows) or one per segment (observation without a step)
    CKC(dmalloc(h, &h->d_partials, sizeof(double) * kNumObs * std::max<uint32_t>(sb, 1)));
    CKC(dmalloc(h, &h->d_obs, sizeof(double) * (kNumObs * n + 1)));
    CKC(cudaMemsetAsync(h->d_obs, 0, sizeof(double) * (kNumObs * n + 1), h->st));
    if (gforce) {
        std::vector<float> gf(n);
        for (int d = 0; d < n; ++d) gf[d] = (float)gforce[d];
        CKC(dmalloc(h, &h->d_gforce, sizeof(float) * n));
        CKC(cudaMemcpyAsync(h->d_gforce, gf.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->st));
        CKC(cudaStreamSynchronize(h->st));
    }
    CKC(cudaMallocHost(&h->h_obs, sizeof(double) * (kNumObs * n + 1)));
    CKC(cudaMemsetAsync(h->d_g[0], 0, sizeof(float) * q * h->pstride, h->st));
    CKC(cudaMemsetAsync(h->d_g[1], 0, sizeof(float) * q * h->pstride, h->st));
    CKC(launch_init(q, h->geom(), h->d_g[0], h->d_uprev, h->st));
    CKC(cudaStreamSynchronize(h->st));
#undef CKC
    if (o.autotune) {
        lbm_status ts = lbm_autotune(h, o.tune_cache, 0, nullptr);
        if (ts != LBM_OK) {
            std::string msg = std::string("autotune at creation: ") + h->err;
            free_solver(h);
            *out = nullptr;
            return fail(nullptr, ts, msg);
        }
    }
    return LBM_OK;
}

lbm_status lbm_slab_create(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz, double tau, double drho,
                           int32_t x_offset, int32_t nx_global, int32_t ghosts, const lbm_options* opt,
                           lbm_handle* out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is null");
    *out = nullptr;
    if (ghosts < 0 || ghosts > 3) return fail(nullptr, LBM_ERR_ARG, "ghosts must be 0..3");
    if (x_offset < 0 || nx < 3 || nx_global < 3 || (int64_t)x_offset + nx > nx_global)
        return fail(nullptr, LBM_ERR_ARG, "need 0 <= x_offset, x_offset + nx <= nx_global, nx >= 3");
    // a column 0 past the global inlet is the left neighbour's column, and a
    // last column short of the global outlet the right neighbour's
    if (((ghosts & 1) != 0) != (x_offset > 0) || ((ghosts & 2) != 0) != ((int64_t)x_offset + nx < nx_global))
        return fail(nullptr, LBM_ERR_ARG, "ghost columns must be exactly the cuts to neighbouring slabs");
    const SlabInfo info{x_offset, nx_global, (uint32_t)ghosts};
    lbm_domain_desc d{mask, nx, ny, nz, tau, drho};
    return create_impl(1, &d, opt, nz > 1 ? 19 : 9, out, nullptr, &info);
}

static HaloPlanes halo_planes(int q, int cx) {
    HaloPlanes P{};
    for (int i = 0; i < q; ++i) {
        const int c = q == 9 ? D2Q9::c(i, 0) : D3Q19::c(i, 0);
        if (c == cx) P.plane[P.n++] = i;
    }
    return P;
}

lbm_status lbm_slab_halo_floats(lbm_handle h, int32_t side, int32_t incoming, int64_t* n) {
    if (!h || !n) return fail(h, LBM_ERR_ARG, "null argument");
    if (!h->slab) return fail(h, LBM_ERR_ARG, "not a slab solver");
    if (side != 0 && side != 1) return fail(h, LBM_ERR_ARG, "side must be 0 (left cut) or 1 (right cut)");
    if (!(h->hdom[0].ghost & (1u << side))) return fail(h, LBM_ERR_ARG, "no neighbouring slab on that side");
    const int cx = incoming ? (side == 0 ? 1 : -1) : (side == 0 ? -1 : 1);
    *n = (int64_t)halo_planes(h->q, cx).n * h->ncol[incoming ? 2 + side : side];
    return LBM_OK;
}

static lbm_status slab_halo(lbm_handle h, int32_t side, bool pack, float* buf) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (!h->slab) return fail(h, LBM_ERR_ARG, "not a slab solver");
    if (side != 0 && side != 1) return fail(h, LBM_ERR_ARG, "side must be 0 (left cut) or 1 (right cut)");
    if (!(h->hdom[0].ghost & (1u << side))) return fail(h, LBM_ERR_ARG, "no neighbouring slab on that side");
    if (!buf) return fail(h, LBM_ERR_ARG, "null buffer");
    // the left cut carries the c_x = -1 planes leftwards and the c_x = +1 planes rightwards
    const int cx = pack ? (side == 0 ? -1 : 1) : (side == 0 ? 1 : -1);
    const int c = pack ? side : 2 + side;
    CK(h, launch_halo(pack, h->d_g[h->cur], (uint32_t)h->pstride, h->d_col[c], h->ncol[c], halo_planes(h->q, cx), buf,
                      h->st));
    if (!pack) h->dom[0].has_obs = false;
    return LBM_OK;
}

lbm_status lbm_slab_export(lbm_handle h, int32_t side, float* buf) { return slab_halo(h, side, true, buf); }

lbm_status lbm_slab_import(lbm_handle h, int32_t side, const float* buf) {
    return slab_halo(h, side, false, const_cast<float*>(buf));
}

lbm_status lbm_slab_observables(lbm_handle h, const double* obs_sum, double* k, double* kn, double* residual) {
    if (!h || !obs_sum) return fail(h, LBM_ERR_ARG, "null argument");
    if (!h->slab) return fail(h, LBM_ERR_ARG, "not a slab solver");
    const DomainHost& D = h->dom[0];
    const DomainDev& G = h->hdom[0];
    if (k) {
        if (D.drho == 0.0) return fail(h, LBM_ERR_ARG, "drho = 0: permeability undefined");
        DomainHost whole = D;  // Darcy's law over the whole domain: only N_y N_z and drho enter
        whole.nx = G.nx_glob;
        *k = darcy_k(whole, obs_sum[0], false, h->opt.rho_out);
    }
    if (kn) *kn = knudsen(D.tau, G.nx_glob);
    if (residual) *residual = obs_sum[2] > 0.0 ? std::sqrt(obs_sum[1] / obs_sum[2]) : (obs_sum[1] == 0.0 ? 0.0 : INFINITY);
    return LBM_OK;
}

lbm_status lbm_batch_create(int32_t n, const lbm_domain_desc* descs, const lbm_options* opt, lbm_handle* out) {
    Range r("lbm_batch_create");
    return create_impl(n, descs, opt, 0, out);
}

lbm_status lbm_batch_create_forced(int32_t n, const lbm_domain_desc* descs, const double* g, const lbm_options* opt,
                                   lbm_handle* out) {
    if (!g) return fail(nullptr, LBM_ERR_ARG, "g is null");
    return create_impl(n, descs, opt, 0, out, g);
}

lbm_status lbm_create_domain(const uint8_t* mask, int32_t nx, int32_t ny, double tau, double drho,
                             const lbm_options* opt, lbm_handle* out) {
    lbm_domain_desc d{mask, nx, ny, 1, tau, drho};
    return create_impl(1, &d, opt, 9, out);
}

lbm_status lbm_create_domain_3d(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz, double tau, double drho,
                                const lbm_options* opt, lbm_handle* out) {
    lbm_domain_desc d{mask, nx, ny, nz, tau, drho};
    return create_impl(1, &d, opt, 19, out);
}

void lbm_destroy(lbm_handle h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    free_solver(h);
}

lbm_status lbm_info(lbm_handle h, int32_t* n_domains, int32_t* q, int64_t* fluid_nodes_total) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (n_domains) *n_domains = (int32_t)h->dom.size();
    if (q) *q = h->q;
    if (fluid_nodes_total) *fluid_nodes_total = (int64_t)h->nfluid;
    return LBM_OK;
}

lbm_status lbm_domain_fluid_nodes(lbm_handle h, int32_t d, int64_t* fluid_nodes) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    if (fluid_nodes) *fluid_nodes = h->dom[d].fluid_count;
    return LBM_OK;
}

lbm_status lbm_step(lbm_handle h, int64_t nsteps) {
    Range r("lbm_step");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    lbm_status s = run_steps(h, nsteps, false);
    if (s == LBM_OK) {
        h->step += nsteps;
        for (auto& D : h->dom)
            if (D.active) D.has_obs = false;
    }
    return s;
}

lbm_status lbm_local_knudsen(lbm_handle h, int32_t d, uint32_t* d2_out, double* h_out, double* kn_out) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    if (!d2_out && !h_out && !kn_out) return fail(h, LBM_ERR_ARG, "no output requested");
    const DomainHost& D = h->dom[d];
    const uint64_t total = (uint64_t)D.nx * D.ny * D.nz;
    const uint8_t* mask = h->d_mask + D.mask_base;
    uint32_t *d2 = nullptr, *tmp = nullptr;
    double* dev = nullptr;  // h then kn, total doubles each
    auto release = [&]() {
        dfree(h, d2);
        dfree(h, tmp);
        dfree(h, dev);
    };
    cudaError_t e = dmalloc(h, &d2, sizeof(uint32_t) * total);
    if (e == cudaSuccess) e = dmalloc(h, &tmp, sizeof(uint32_t) * total);
    if (e == cudaSuccess) e = dmalloc(h, &dev, sizeof(double) * 2 * total);
    if (e == cudaSuccess) e = launch_pore_d2(mask, D.nx, D.ny, D.nz, d2, tmp, h->st);
    if (e == cudaSuccess) e = launch_local_kn(mask, d2, total, D.tau, dev, dev + total, h->st);
    if (e == cudaSuccess && d2_out)
        e = cudaMemcpyAsync(d2_out, d2, sizeof(uint32_t) * total, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && h_out)
        e = cudaMemcpyAsync(h_out, dev, sizeof(double) * total, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && kn_out)
        e = cudaMemcpyAsync(kn_out, dev + total, sizeof(double) * total, cudaMemcpyDeviceToHost, h->st);
    release();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_local_knudsen");
    return LBM_OK;
}

lbm_status lbm_profile_steps(lbm_handle h, int64_t nsteps, double* times_us, int64_t* counts) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (nsteps < 0 || nsteps > 100000) return fail(h, LBM_ERR_ARG, "nsteps must be in [0, 100000]");
    if (!times_us || !counts) return fail(h, LBM_ERR_ARG, "times_us and counts are required");
    for (int k = 0; k < LBM_NUM_KERNEL_KINDS; ++k) {
        times_us[k] = 0.0;
        counts[k] = 0;
    }
    if (nsteps == 0) return LBM_OK;
    KernelProf prof;
    mark_forced_state(h, nsteps);
    lbm_status s = enqueue_steps(h, nsteps, false, &prof);
    if (s != LBM_OK) return s;
    CK(h, cudaStreamSynchronize(h->st));
    {
        uint32_t word = 0;
        CK(h, cudaMemcpy(&word, h->err_word(), sizeof(word), cudaMemcpyDeviceToHost));
        s = device_error(h, word);
        if (s != LBM_OK) return s;
    }
    for (size_t i = 0; i < prof.kind.size(); ++i) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, prof.ev[2 * i], prof.ev[2 * i + 1]));
        times_us[prof.kind[i]] += 1e3 * (double)ms;
        counts[prof.kind[i]] += 1;
    }
    h->step += nsteps;
    for (auto& D : h->dom)
        if (D.active) D.has_obs = false;
    return LBM_OK;
}

lbm_status lbm_step_observe(lbm_handle h, int64_t nsteps, double* obs) {
    Range r("lbm_step_observe");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps < 0");
    lbm_status s = run_steps(h, nsteps, true);
    if (s != LBM_OK) return s;
    CK(h, cudaStreamSynchronize(h->st));
    h->step += nsteps;
    s = store_obs(h);
    if (s != LBM_OK) return s;
    if (obs) std::memcpy(obs, h->h_obs, sizeof(double) * kNumObs * h->dom.size());
    return LBM_OK;
}

lbm_status lbm_run_to_steady(lbm_handle h, double tol, int64_t max_steps, lbm_status* status, int64_t* steps,
                             double* residual) {
    Range rr("lbm_run_to_steady");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (h->slab) return fail(h, LBM_ERR_ARG, "a slab is stepped by a driver that exchanges its halos");
    if (!(tol > 0.0) || max_steps < 0) return fail(h, LBM_ERR_ARG, "need tol > 0 and max_steps >= 0");
    const size_t n = h->dom.size();
    for (auto& D : h->dom) {
        D.active = 1;
        D.status = LBM_NOT_CONVERGED;
        D.steps = 0;
        D.residual = INFINITY;
        D.rhist.clear();
        D.kq.clear();
        D.k_ok = 0;
        D.k_dead = 0;
        D.k_peak = 0.0;
        D.h_step.clear();
        D.h_k.clear();
        D.h_r.clear();
        D.h_t.clear();
    }
    lbm_status s = upload_dom(h);
    if (s != LBM_OK) return s;
    const auto t_start = std::chrono::steady_clock::now();
    const int64_t N = h->opt.check_interval;
    int64_t taken = 0;
    size_t nactive = n;
    bool cancelled = false;
    while (nactive > 0 && taken < max_steps) {
        if (h->opt.cancel_flag && *h->opt.cancel_flag) {
            cancelled = true;
            break;
        }
        const int64_t k = std::min<int64_t>(N, max_steps - taken);
        Range ri("check interval");
        s = run_steps(h, k, true);
        if (s != LBM_OK) return s;
        CK(h, cudaStreamSynchronize(h->st));
        taken += k;
        h->step += k;
        s = store_obs(h);
        if (s != LBM_OK) return s;
        bool retired = false;
        for (size_t d = 0; d < n; ++d) {
            DomainHost& D = h->dom[d];
            if (!D.active) continue;
            const double* o = D.obs;
            D.steps = taken;
            double r;
            if (o[2] > 0.0) r = std::sqrt(o[1] / o[2]);
            else r = (o[1] == 0.0) ? 0.0 : INFINITY;
            D.residual = r;
            D.h_step.push_back(h->step);
            D.h_k.push_back((h->forced ? D.g != 0.0 : D.drho != 0.0) ? darcy_k(D, o[0], h->forced, h->opt.rho_out)
                                                                     : NAN);
            D.h_r.push_back(r);
            D.h_t.push_back(std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
            lbm_status ds = LBM_NOT_CONVERGED;
            const double kt = D.h_k.back();
            if (o[4] > 0.0 || !std::isfinite(o[0])) ds = LBM_DIVERGED;
            else if (r < tol) ds = LBM_OK;
            else if (h->opt.k_tol > 0.0 && std::isfinite(kt) && k_converged(D, kt, r, h->opt.k_tol)) ds = LBM_OK;
            else {
                // FP32 floor: below stall_floor the residual jitters instead of
                // decaying, so it stops setting new minima; a slow but genuine
                // decay sets one at every check.  A residual far above the
                // best so far is a transient (e.g. after a warm start, whose
                // first interval barely moves u) and restarts the count.
                if (D.rhist.empty() || r < D.rhist[0] || r > 30.0 * D.rhist[0]) {
                    D.rhist.assign(1, r);  // rhist[0] = best residual since the last restart
                } else {
                    D.rhist.push_back(r);  // checks since the best
                }
                if (r < h->opt.stall_floor && (int64_t)D.rhist.size() > (int64_t)h->opt.stall_checks)
                    ds = LBM_STALLED;
            }
            if (ds != LBM_NOT_CONVERGED) {
                D.status = ds;
                D.active = 0;
                --nactive;
                retired = true;
                s = mirror_domain(h, d);
                if (s != LBM_OK) return s;
            }
        }
        if (retired) {
            s = upload_dom(h);
            if (s != LBM_OK) return s;
        }
    }
    CK(h, cudaStreamSynchronize(h->st));
    // leave every domain active for later lbm_step calls
    bool any_div = false, any_stall = false, any_open = false;
    for (size_t d = 0; d < n; ++d) {
        DomainHost& D = h->dom[d];
        if (D.active) {
            D.status = cancelled ? LBM_CANCELLED : LBM_NOT_CONVERGED;
            any_open = true;
        }
        any_div |= D.status == LBM_DIVERGED;
        any_stall |= D.status == LBM_STALLED;
        if (status) status[d] = D.status;
        if (steps) steps[d] = D.steps;
        if (residual) residual[d] = D.residual;
        D.active = 1;
    }
    s = upload_dom(h);
    if (s != LBM_OK) return s;
    CK(h, cudaStreamSynchronize(h->st));
    if (cancelled) return fail(h, LBM_CANCELLED, "cancelled by cancel_flag");
    if (any_div) return fail(h, LBM_DIVERGED, "non-finite velocity in at least one domain");
    if (any_open) return LBM_NOT_CONVERGED;
    if (any_stall) return LBM_STALLED;
    return LBM_OK;
}

lbm_status lbm_batch_run_to_steady(lbm_batch b, double tol, int64_t max_steps, lbm_status* per_domain) {
    return lbm_run_to_steady(b, tol, max_steps, per_domain, nullptr, nullptr);
}

lbm_status lbm_batch_permeability(lbm_batch b, double* k) { return lbm_permeability(b, k, nullptr); }

void lbm_batch_destroy(lbm_batch b) { lbm_destroy(b); }

lbm_status lbm_permeability(lbm_handle h, double* k, double* kn) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (h->slab) return fail(h, LBM_ERR_ARG, "a slab's permeability needs the observables of every slab "
                                             "(lbm_slab_observables)");
    if (!k) return fail(h, LBM_ERR_ARG, "k is null");
    bool need = false;
    for (auto& D : h->dom) need |= !D.has_obs;
    if (need) {
        // observe the current state (this also refreshes u_prev)
        lbm_status s = enqueue_steps(h, 0, true);
        if (s != LBM_OK) return s;
        CK(h, cudaStreamSynchronize(h->st));
        s = store_obs(h);
        if (s != LBM_OK) return s;
    }
    lbm_status rs = LBM_OK;
    for (size_t d = 0; d < h->dom.size(); ++d) {
        const DomainHost& D = h->dom[d];
        if (h->forced ? D.g == 0.0 : D.drho == 0.0) {
            k[d] = NAN;
            rs = fail(h, LBM_ERR_ARG, h->forced ? "g = 0: permeability undefined" : "drho = 0: permeability undefined");
        } else {
            k[d] = darcy_k(D, D.obs[0], h->forced, h->opt.rho_out);
        }
        if (kn) kn[d] = knudsen(D.tau, D.nx);
    }
    return rs;
}

lbm_status lbm_get_fields(lbm_handle h, int32_t d, double* rho, double* ux, double* uy, double* uz) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    if (!rho || !ux || !uy || (h->q == 19 && !uz)) return fail(h, LBM_ERR_ARG, "null output");
    const DomainHost& D = h->dom[d];
    const size_t N = (size_t)D.nx * D.ny * D.nz;
    double* buf = nullptr;
    CK(h, dmalloc(h, &buf, sizeof(double) * N * 4));
    const cudaError_t e1 = launch_export_fields(h->q, h->geom(), D.seg_begin, D.nseg, h->opt.rho_out,
                                                h->d_g[h->cur], buf, buf + N, buf + 2 * N,
                                                h->q == 19 ? buf + 3 * N : nullptr, h->st);
    cudaError_t e = e1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(rho, buf, sizeof(double) * N, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ux, buf + N, sizeof(double) * N, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(uy, buf + 2 * N, sizeof(double) * N, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && h->q == 19)
        e = cudaMemcpyAsync(uz, buf + 3 * N, sizeof(double) * N, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    dfree(h, buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_get_fields");
    if (h->q == 9 && uz) std::memset(uz, 0, sizeof(double) * N);
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_handle h, int32_t d, double* f) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    if (!f) return fail(h, LBM_ERR_ARG, "null output");
    const DomainHost& D = h->dom[d];
    const size_t M = (size_t)D.nx * D.ny * D.nz * h->q;
    double* buf = nullptr;
    CK(h, dmalloc(h, &buf, sizeof(double) * M));
    cudaError_t e = launch_export_pops(h->q, h->geom(), D.seg_begin, D.nseg, h->opt.rho_out, h->d_g[h->cur],
                                       buf, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, buf, sizeof(double) * M, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    dfree(h, buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_get_populations");
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_handle h, int32_t d, const double* f) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    if (!f) return fail(h, LBM_ERR_ARG, "null input");
    const DomainHost& D = h->dom[d];
    const size_t M = (size_t)D.nx * D.ny * D.nz * h->q;
    double* buf = nullptr;
    CK(h, dmalloc(h, &buf, sizeof(double) * M));
    cudaError_t e = cudaMemcpyAsync(buf, f, sizeof(double) * M, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess)
        e = launch_import_pops(h->q, h->geom(), D.seg_begin, D.nseg, h->opt.rho_out, buf, h->d_g[h->cur], h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    dfree(h, buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_set_populations");
    h->dom[d].has_obs = false;
    h->dom[d].forced_state = false;
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_handle h, int32_t d, const float* drho, const float* ux, const float* uy,
                          const float* uz, int32_t on_device) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    if (!drho || !ux || !uy || (h->q == 19 && !uz)) return fail(h, LBM_ERR_ARG, "null input");
    const DomainHost& D = h->dom[d];
    const size_t N = (size_t)D.nx * D.ny * D.nz;
    float* buf = nullptr;
    const float *a = drho, *b = ux, *c = uy, *z = (h->q == 19) ? uz : nullptr;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        CK(h, dmalloc(h, &buf, sizeof(float) * N * 4));
        e = cudaMemcpyAsync(buf, drho, sizeof(float) * N, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(buf + N, ux, sizeof(float) * N, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(buf + 2 * N, uy, sizeof(float) * N, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess && z)
            e = cudaMemcpyAsync(buf + 3 * N, uz, sizeof(float) * N, cudaMemcpyHostToDevice, h->st);
        a = buf;
        b = buf + N;
        c = buf + 2 * N;
        z = z ? buf + 3 * N : nullptr;
    }
    if (e == cudaSuccess)
        e = launch_set_fields(h->q, h->eq, h->geom(), D.seg_begin, D.nseg, a, b, c, z, h->d_g[h->cur],
                              h->d_uprev, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    dfree(h, buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_set_fields");
    h->dom[d].has_obs = false;
    h->dom[d].forced_state = false;
    return LBM_OK;
}

lbm_status lbm_get_history(lbm_handle h, int32_t d, int64_t* steps, double* k, double* residual, double* seconds,
                           int32_t capacity, int32_t* count) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    const DomainHost& D = h->dom[d];
    const int32_t n = (int32_t)D.h_k.size();
    if (count) *count = n;
    const int32_t m = std::min(n, std::max(capacity, 0));
    for (int32_t i = 0; i < m; ++i) {
        if (steps) steps[i] = D.h_step[i];
        if (k) k[i] = D.h_k[i];
        if (residual) residual[i] = D.h_r[i];
        if (seconds) seconds[i] = D.h_t[i];
    }
    return LBM_OK;
}

// nu (N_x - 1) / (c_s^2 drho): the velocity scale of the warm-start targets.
static double target_u_scale(const DomainHost& D) { return (D.tau - 0.5) / 3.0 * (double)(D.nx - 1) / (D.drho / 3.0); }

lbm_status lbm_nn_targets(lbm_handle h, int32_t d, float* out_dev) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    if (!out_dev) return fail(h, LBM_ERR_ARG, "null output");
    if (h->forced || h->slab) return fail(h, LBM_ERR_ARG, "targets are defined for whole pressure-driven domains");
    if (h->q != 9) return fail(h, LBM_ERR_ARG, "warm-start targets are defined for 2D (D2Q9) domains");
    const DomainHost& D = h->dom[d];
    if (D.drho == 0.0) return fail(h, LBM_ERR_ARG, "drho = 0: targets undefined");
    CK(h, launch_export_targets(h->geom(), D.seg_begin, D.nseg, h->opt.rho_out, 1.0 / D.drho, target_u_scale(D),
                                h->d_g[h->cur], out_dev, h->st));
    return LBM_OK;
}

lbm_status lbm_warm_start(lbm_handle h, int32_t d, const void* pred_dev, int32_t ld) {
    lbm_status s = check_domain(h, d);
    if (s != LBM_OK) return s;
    if (!pred_dev || ld < 3) return fail(h, LBM_ERR_ARG, "need a prediction with at least 3 channels");
    if (h->forced || h->slab)
        return fail(h, LBM_ERR_ARG, "the warm start is defined for whole pressure-driven domains");
    if (h->q != 9) return fail(h, LBM_ERR_ARG, "the warm start is defined for 2D (D2Q9) domains");
    DomainHost& D = h->dom[d];
    if (D.drho == 0.0) return fail(h, LBM_ERR_ARG, "drho = 0: nothing to predict");
    const double umax = 0.1 / std::sqrt(3.0);  // |u| <= 0.1 c_s
    CK(h, launch_warm_start(h->eq, h->geom(), D.seg_begin, D.nseg, pred_dev, ld, (float)D.drho,
                            (float)(1.0 / target_u_scale(D)), (float)umax, h->d_g[h->cur], h->d_uprev, h->st));
    D.has_obs = false;
    return LBM_OK;
}

lbm_status lbm_get_step(lbm_handle h, int64_t* step) {
    if (!h || !step) return fail(h, LBM_ERR_ARG, "null argument");
    *step = h->step;
    return LBM_OK;
}

// Checkpoint layout: magic, version, header ints, per-domain records, masks,
// then per domain its compact populations (Q planes) and u_prev (D planes).
static const char kMagic[8] = {'L', 'B', 'M', 'G', 'B', '3', '0', '0'};

lbm_status lbm_save(lbm_handle h, const char* path) {
    if (!h || !path) return fail(h, LBM_ERR_ARG, "null argument");
    if (h->forced || h->slab) return fail(h, LBM_ERR_ARG, "checkpoints hold whole pressure-driven domains only");
    CK(h, cudaStreamSynchronize(h->st));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(h, LBM_ERR_IO, std::string("cannot open ") + path);
    const int D = (h->q == 9) ? 2 : 3;
    bool ok = true;
    auto W = [&](const void* p, size_t sz) { ok = ok && std::fwrite(p, 1, sz, fp) == sz; };
    const int32_t hdr[4] = {1, h->q, h->eq, (int32_t)h->dom.size()};
    W(kMagic, 8);
    W(hdr, sizeof(hdr));
    W(&h->step, sizeof(h->step));
    W(&h->opt.rho_out, sizeof(double));
    for (const DomainHost& d : h->dom) {
        const int32_t dims[3] = {d.nx, d.ny, d.nz};
        W(dims, sizeof(dims));
        W(&d.tau, sizeof(double));
        W(&d.drho, sizeof(double));
        const int32_t st = (int32_t)d.status;
        W(&st, sizeof(st));
        W(&d.steps, sizeof(d.steps));
        W(&d.residual, sizeof(double));
        const int32_t ho = d.has_obs ? 1 : 0;
        W(&ho, sizeof(ho));
        W(d.obs, sizeof(d.obs));
    }
    {
        std::vector<uint8_t> masks(h->mask_bytes);
        CK(h, cudaMemcpy(masks.data(), h->d_mask, h->mask_bytes, cudaMemcpyDeviceToHost));
        W(masks.data(), masks.size());
    }
    std::vector<float> tmp;
    for (const DomainHost& d : h->dom) {
        tmp.resize((size_t)d.fluid_count);
        for (int i = 0; i < h->q + D && ok; ++i) {
            const float* src = (i < h->q) ? h->d_g[h->cur] + (size_t)i * h->pstride
                                          : h->d_uprev + (size_t)(i - h->q) * h->pstride;
            if (d.fluid_count) {
                cudaError_t e = cudaMemcpy(tmp.data(), src + d.fluid_begin, sizeof(float) * d.fluid_count,
                                           cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) {
                    std::fclose(fp);
                    return cuda_fail(h, e, "lbm_save copy");
                }
            }
            W(tmp.data(), sizeof(float) * tmp.size());
        }
    }
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(h, LBM_ERR_IO, "write failed");
    return LBM_OK;
}

lbm_status lbm_load(const char* path, const lbm_options* opt, lbm_handle* out) {
    if (!path || !out) return fail(nullptr, LBM_ERR_ARG, "null argument");
    *out = nullptr;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(nullptr, LBM_ERR_IO, std::string("cannot open ") + path);
    bool ok = true;
    auto R = [&](void* p, size_t sz) { ok = ok && std::fread(p, 1, sz, fp) == sz; };
    char magic[8];
    int32_t hdr[4];
    int64_t step = 0;
    double rho_out = 1.0;
    R(magic, 8);
    R(hdr, sizeof(hdr));
    R(&step, sizeof(step));
    R(&rho_out, sizeof(double));
    if (!ok || std::memcmp(magic, kMagic, 8) != 0 || hdr[0] != 1 || (hdr[1] != 9 && hdr[1] != 19) || hdr[3] < 1 ||
        hdr[3] > (1 << 24)) {
        std::fclose(fp);
        return fail(nullptr, LBM_ERR_IO, "not a checkpoint of this library version");
    }
    const int n = hdr[3];
    struct Rec {
        int32_t dims[3];
        double tau, drho;
        int32_t st;
        int64_t steps;
        double residual;
        int32_t has_obs;
        double obs[kNumObs];
    };
    std::vector<Rec> recs(n);
    uint64_t cells = 0;
    for (int d = 0; d < n && ok; ++d) {
        Rec& r = recs[d];
        R(r.dims, sizeof(r.dims));
        R(&r.tau, sizeof(double));
        R(&r.drho, sizeof(double));
        R(&r.st, sizeof(int32_t));
        R(&r.steps, sizeof(int64_t));
        R(&r.residual, sizeof(double));
        R(&r.has_obs, sizeof(int32_t));
        R(r.obs, sizeof(r.obs));
        if (r.dims[0] < 3 || r.dims[1] < 1 || r.dims[2] < 1 || r.dims[0] > (1 << 20) || r.dims[1] > (1 << 20) ||
            r.dims[2] > (1 << 20))
            ok = false;
        else
            cells += (uint64_t)r.dims[0] * r.dims[1] * r.dims[2];
    }
    if (!ok || cells >= (1ull << 32)) {
        std::fclose(fp);
        return fail(nullptr, LBM_ERR_IO, "truncated or corrupt checkpoint header");
    }
    std::vector<uint8_t> masks(cells);
    R(masks.data(), cells);
    if (!ok) {
        std::fclose(fp);
        return fail(nullptr, LBM_ERR_IO, "truncated checkpoint (masks)");
    }
    lbm_options o;
    lbm_options_default(&o);
    if (opt) o = *opt;
    o.equilibrium = hdr[2];
    o.rho_out = rho_out;
    std::vector<lbm_domain_desc> descs(n);
    uint64_t mb = 0;
    for (int d = 0; d < n; ++d) {
        descs[d] = lbm_domain_desc{masks.data() + mb, recs[d].dims[0], recs[d].dims[1], recs[d].dims[2],
                                   recs[d].tau, recs[d].drho};
        mb += (uint64_t)recs[d].dims[0] * recs[d].dims[1] * recs[d].dims[2];
    }
    lbm_handle h = nullptr;
    lbm_status s = create_impl(n, descs.data(), &o, hdr[1], &h);
    if (s != LBM_OK) {
        std::fclose(fp);
        return s;
    }
    const int D = (h->q == 9) ? 2 : 3;
    std::vector<float> tmp;
    for (int d = 0; d < n && ok; ++d) {
        DomainHost& dh = h->dom[d];
        tmp.resize((size_t)dh.fluid_count);
        for (int i = 0; i < h->q + D && ok; ++i) {
            R(tmp.data(), sizeof(float) * tmp.size());
            if (!ok) break;
            float* dst = (i < h->q) ? h->d_g[0] + (size_t)i * h->pstride : h->d_uprev + (size_t)(i - h->q) * h->pstride;
            if (dh.fluid_count) {
                cudaError_t e = cudaMemcpy(dst + dh.fluid_begin, tmp.data(), sizeof(float) * dh.fluid_count,
                                           cudaMemcpyHostToDevice);
                if (e != cudaSuccess) {
                    std::fclose(fp);
                    lbm_status cs = cuda_fail(nullptr, e, "lbm_load copy");
                    free_solver(h);
                    return cs;
                }
            }
        }
        dh.status = (lbm_status)recs[d].st;
        dh.steps = recs[d].steps;
        dh.residual = recs[d].residual;
        dh.has_obs = recs[d].has_obs != 0;
        std::memcpy(dh.obs, recs[d].obs, sizeof(dh.obs));
    }
    std::fclose(fp);
    if (!ok) {
        free_solver(h);
        return fail(nullptr, LBM_ERR_IO, "truncated checkpoint (populations)");
    }
    h->cur = 0;
    h->step = step;
    *out = h;
    return LBM_OK;
}


// ---------------------------------------------------------------------------
// Launch configuration and autotuner
// ---------------------------------------------------------------------------
#ifndef LBM_KERNEL_HASH
#define LBM_KERNEL_HASH "unversioned"
#endif

}  // extern "C"

namespace {

lbm_launch current_launch(lbm_handle h) {
    int lo, hi, def;
    gather_batches(h->q, &lo, &hi, &def);
    lbm_launch c;
    c.block_threads = h->opt.block_threads > 0 ? h->opt.block_threads : 128;
    c.strip_rows = h->strip_rows;
    c.gather_batch = h->gather_batch > 0 ? h->gather_batch : def;
    c.tile_rows = h->tile_rows;
    c.band_rows = h->band_rows;
    c.pair_block_mb = h->pair_block_mb;
    return c;
}

bool launch_valid(lbm_handle h, const lbm_launch& c) {
    int lo, hi, def;
    gather_batches(h->q, &lo, &hi, &def);
    return c.block_threads >= 32 && c.block_threads <= 256 && c.block_threads % 32 == 0 && c.strip_rows >= 1 &&
           c.strip_rows <= 255 && (c.gather_batch == lo || c.gather_batch == hi) && c.tile_rows >= 0 &&
           c.tile_rows <= kTileRowsMax && (c.tile_rows == 0 || staged_gather_lattice(h->q)) && c.band_rows >= 0 &&
           c.band_rows <= kBandRowsMax && (c.band_rows == 0 || band_gather_lattice(h->q)) &&
           !(c.tile_rows > 0 && c.band_rows > 0) && c.pair_block_mb >= 0 && c.pair_block_mb <= kPairBlockMbMax;
}

lbm_status apply_launch(lbm_handle h, const lbm_launch& c) {
    if (!launch_valid(h, c)) return fail(h, LBM_ERR_ARG, "launch configuration outside the allowed ranges");
    const lbm_launch cur = current_launch(h);
    lbm_status s = LBM_OK;
    if (c.strip_rows != cur.strip_rows) s = build_items(h, c.strip_rows);
    if (s == LBM_OK && c.tile_rows != cur.tile_rows) s = build_tiles(h, c.tile_rows);
    if (s == LBM_OK && c.band_rows != cur.band_rows) s = build_bands(h, c.band_rows);
    if (s == LBM_OK && (c.pair_block_mb != cur.pair_block_mb || c.strip_rows != cur.strip_rows))
        s = build_pair_blocks(h, c.pair_block_mb);
    if (s != LBM_OK) return s;
    h->opt.block_threads = c.block_threads;
    h->gather_batch = c.gather_batch;
    // cached graphs hold the old launches
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    return LBM_OK;
}

std::string key_part(const char* s) {
    std::string r;
    for (const char* p = s; *p; ++p) r += (*p == ' ' || *p == '"' || *p == '\\' || *p == '|') ? '_' : *p;
    return r;
}

lbm_status write_key(const std::string& k, char* key, size_t cap) {
    if (!key || cap < k.size() + 1) return fail(nullptr, LBM_ERR_ARG, "key buffer too small");
    std::memcpy(key, k.c_str(), k.size() + 1);
    return LBM_OK;
}

std::string make_key(const char* device, int q, int64_t fluid, int eq, int coll) {
    int b = 0;
    while ((int64_t(1) << (b + 1)) <= fluid && b < 62) ++b;
    return key_part(device) + "|q" + std::to_string(q) + "|n2^" + std::to_string(b) + "|eq" + std::to_string(eq) +
           "|coll" + std::to_string(coll) + "|" + LBM_KERNEL_HASH;
}

// The cache file holds one member per line:  "KEY": {"block_threads": B, ...},
struct CacheEntry {
    lbm_launch c;
    double us;
};
std::map<std::string, CacheEntry> read_cache(const char* path) {
    std::map<std::string, CacheEntry> m;
    FILE* fp = path ? std::fopen(path, "r") : nullptr;
    if (!fp) return m;
    char line[1024];
    while (std::fgets(line, sizeof(line), fp)) {
        const char* a = std::strchr(line, '"');
        if (!a) continue;
        const char* b = std::strchr(a + 1, '"');
        if (!b) continue;
        const std::string key(a + 1, b);
        CacheEntry e{};
        auto field = [&](const char* name, double* v) {
            const char* f = std::strstr(b, name);
            if (!f) return false;
            f = std::strchr(f + std::strlen(name), ':');
            return f && std::sscanf(f + 1, "%lf", v) == 1;
        };
        double bt, sr, gb, tr, us, br = 0.0, pb = 0.0;
        if (field("\"block_threads\"", &bt) && field("\"strip_rows\"", &sr) && field("\"gather_batch\"", &gb) &&
            field("\"tile_rows\"", &tr) && field("\"us_per_step\"", &us)) {
            field("\"band_rows\"", &br);  // absent in entries written before band gather steps existed
            field("\"pair_block_mb\"", &pb);
            e.c.block_threads = (int32_t)bt;
            e.c.strip_rows = (int32_t)sr;
            e.c.gather_batch = (int32_t)gb;
            e.c.tile_rows = (int32_t)tr;
            e.c.band_rows = (int32_t)br;
            e.c.pair_block_mb = (int32_t)pb;
            e.us = us;
            m[key] = e;
        }
    }
    std::fclose(fp);
    return m;
}
bool write_cache(const char* path, const std::map<std::string, CacheEntry>& m) {
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)std::chrono::steady_clock::now()
                                                                            .time_since_epoch()
                                                                            .count() % 1000000007);
    FILE* fp = std::fopen(tmp.c_str(), "w");
    if (!fp) return false;
    bool ok = std::fprintf(fp, "{\n") > 0;
    size_t i = 0;
    for (const auto& kv : m) {
        const CacheEntry& e = kv.second;
        ok = ok && std::fprintf(fp,
                                "\"%s\": {\"block_threads\": %d, \"strip_rows\": %d, \"gather_batch\": %d, "
                                "\"tile_rows\": %d, \"band_rows\": %d, \"pair_block_mb\": %d, \"us_per_step\": %.3f}%s\n",
                                kv.first.c_str(), e.c.block_threads, e.c.strip_rows, e.c.gather_batch, e.c.tile_rows,
                                e.c.band_rows, e.c.pair_block_mb, e.us, ++i < m.size() ? "," : "") > 0;
    }
    ok = ok && std::fprintf(fp, "}\n") > 0;
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

lbm_status lbm_get_launch(lbm_handle h, lbm_launch* cfg) {
    if (!h || !cfg) return fail(h, LBM_ERR_ARG, "null argument");
    *cfg = current_launch(h);
    return LBM_OK;
}

lbm_status lbm_set_launch(lbm_handle h, const lbm_launch* cfg) {
    if (!h || !cfg) return fail(h, LBM_ERR_ARG, "null argument");
    return apply_launch(h, *cfg);
}

lbm_status lbm_time_steps(lbm_handle h, int32_t nsteps, double* us_per_step) {
    if (!h || !us_per_step) return fail(h, LBM_ERR_ARG, "null argument");
    if (nsteps < 2 || nsteps > 10000 || (nsteps & 1)) return fail(h, LBM_ERR_ARG, "nsteps must be even, 2..10000");
    const size_t bytes = sizeof(float) * (size_t)h->q * h->pstride;
    float* save = nullptr;
    CK(h, dmalloc(h, &save, bytes));
    const int cur0 = h->cur;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemcpyAsync(save, h->d_g[cur0], bytes, cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    lbm_status s = LBM_OK;
    if (e == cudaSuccess) s = enqueue_steps(h, 2, false);
    if (e == cudaSuccess && s == LBM_OK) e = cudaEventRecord(e0, h->st);
    if (e == cudaSuccess && s == LBM_OK) s = enqueue_steps(h, nsteps, false);
    if (e == cudaSuccess && s == LBM_OK) e = cudaEventRecord(e1, h->st);
    if (e == cudaSuccess && s == LBM_OK) e = cudaStreamSynchronize(h->st);
    float ms = 0.f;
    if (e == cudaSuccess && s == LBM_OK) e = cudaEventElapsedTime(&ms, e0, e1);
    // restore the state (an even number of steps leaves the current buffer in place)
    h->cur = cur0;
    cudaError_t e2 = cudaMemcpyAsync(h->d_g[cur0], save, bytes, cudaMemcpyDeviceToDevice, h->st);
    dfree(h, save);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(h->st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s != LBM_OK) return s;
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_time_steps");
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "lbm_time_steps restore");
    uint32_t word = 0;
    CK(h, cudaMemcpy(&word, h->err_word(), sizeof(word), cudaMemcpyDeviceToHost));
    s = device_error(h, word);
    if (s != LBM_OK) return s;
    *us_per_step = 1e3 * (double)ms / nsteps;
    return LBM_OK;
}

lbm_status lbm_tune_key_for(const char* device_name, int32_t q, int64_t fluid_nodes, int32_t eq, int32_t collision,
                            char* key, size_t cap) {
    if (!device_name) return fail(nullptr, LBM_ERR_ARG, "null device name");
    return write_key(make_key(device_name, q, fluid_nodes, eq, collision), key, cap);
}

lbm_status lbm_tune_key(lbm_handle h, char* key, size_t cap) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    int dev = 0;
    cudaDeviceProp prop{};
    CK(h, cudaGetDevice(&dev));
    CK(h, cudaGetDeviceProperties(&prop, dev));
    return write_key(make_key(prop.name, h->q, (int64_t)h->nfluid, h->eq, h->opt.collision), key, cap);
}

lbm_status lbm_tune_cache_get(const char* path, const char* key, lbm_launch* cfg, double* us_per_step,
                              int32_t* found) {
    if (!path || !key || !found) return fail(nullptr, LBM_ERR_ARG, "null argument");
    const auto m = read_cache(path);
    const auto it = m.find(key);
    *found = it != m.end();
    if (*found) {
        if (cfg) *cfg = it->second.c;
        if (us_per_step) *us_per_step = it->second.us;
    }
    return LBM_OK;
}

lbm_status lbm_tune_cache_put(const char* path, const char* key, const lbm_launch* cfg, double us_per_step) {
    if (!path || !key || !cfg) return fail(nullptr, LBM_ERR_ARG, "null argument");
    if (std::strchr(key, '"') || std::strchr(key, '\n')) return fail(nullptr, LBM_ERR_ARG, "key holds a quote or newline");
    auto m = read_cache(path);
    m[key] = CacheEntry{*cfg, us_per_step};
    if (!write_cache(path, m)) return fail(nullptr, LBM_ERR_IO, std::string("cannot write ") + path);
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_handle h, const char* cache_path, int32_t nsteps, lbm_tune_result* out) {
    Range rg("lbm_autotune");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
    if (nsteps < 0 || nsteps > 10000) return fail(h, LBM_ERR_ARG, "nsteps must be in [0, 10000]");
    const int steps = nsteps == 0 ? 20 : (nsteps + 1) / 2 * 2;
    int lo, hi, def;
    gather_batches(h->q, &lo, &hi, &def);
    lbm_tune_result r{};
    const bool bands_apply = band_gather_lattice(h->q) && h->opt.in_place_pairs && !h->forced && !h->slab;
    const bool blocks_apply = h->opt.in_place_pairs && !h->forced && !h->slab;
    r.defaults = lbm_launch{128, 8, def, 0, bands_apply ? kBandRowsDefault : 0,
                            blocks_apply ? kPairBlockMbDefault : 0};
    r.chosen = current_launch(h);
    if (h->forced) {  // pull steps of the periodic kernel only: nothing to choose
        if (out) *out = r;
        return LBM_OK;
    }
    char key[512];
    lbm_status s = lbm_tune_key(h, key, sizeof(key));
    if (s != LBM_OK) return s;
    if (cache_path) {
        const auto m = read_cache(cache_path);
        const auto it = m.find(key);
        if (it != m.end() && launch_valid(h, it->second.c)) {
            s = apply_launch(h, it->second.c);
            if (s != LBM_OK) return s;
            r.chosen = it->second.c;
            r.us_per_step = it->second.us;
            r.from_cache = 1;
            if (out) *out = r;
            return LBM_OK;
        }
    }
    std::vector<lbm_launch> cands{r.defaults};
    for (int bt : {64, 128, 256})
        for (int sr : {4, 8, 16})
            for (int gb : {lo, hi}) {
                const lbm_launch c{bt, sr, gb, 0, 0};
                if (std::memcmp(&c, &r.defaults, sizeof(c)) != 0) cands.push_back(c);
            }
    if (staged_gather_lattice(h->q) && h->opt.in_place_pairs && !h->slab)
        for (int tr : {2, 3}) cands.push_back(lbm_launch{128, 8, def, tr, 0});
    if (bands_apply)
        for (int br : {16, 32, 64}) {
            const lbm_launch c{128, 8, def, 0, br};
            if (std::memcmp(&c, &r.defaults, sizeof(c)) != 0) cands.push_back(c);
        }
    double best = INFINITY;
    lbm_launch best_c = r.defaults;
    for (size_t i = 0; i < cands.size(); ++i) {
        s = apply_launch(h, cands[i]);
        if (s != LBM_OK) return s;
        double t = 0.0;
        s = lbm_time_steps(h, steps, &t);
        if (s != LBM_OK) return s;
        if (i == 0) r.us_per_step_default = t;
        if (t < best) {
            best = t;
            best_c = cands[i];
        }
    }
    s = apply_launch(h, best_c);
    if (s != LBM_OK) return s;
    r.chosen = best_c;
    r.us_per_step = best;
    r.candidates = (int32_t)cands.size();
    if (cache_path) {
        s = lbm_tune_cache_put(cache_path, key, &best_c, best);
        if (s != LBM_OK) return fail(h, s, lbm_last_error(nullptr));
    }
    if (out) *out = r;
    return LBM_OK;
}


lbm_status lbm_debug_corrupt_window(lbm_handle h, uint32_t seg, uint32_t value) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "null handle");
#ifdef LBM_CHECKED
    if (seg >= h->nseg_total) return fail(h, LBM_ERR_ARG, "segment out of range");
    CK(h, cudaStreamSynchronize(h->st));
    CK(h, cudaMemcpy(reinterpret_cast<uint32_t*>(h->d_win + seg) + 2, &value, sizeof(value), cudaMemcpyHostToDevice));
    return LBM_OK;
#else
    (void)seg;
    (void)value;
    return fail(h, LBM_ERR_ARG, "only a checked build (LBM_CHECKED) accepts a corrupted index table");
#endif
}

lbm_status lbm_build_checked(int32_t* checked) {
    if (!checked) return fail(nullptr, LBM_ERR_ARG, "null argument");
#ifdef LBM_CHECKED
    *checked = 1;
#else
    *checked = 0;
#endif
    return LBM_OK;
}

}  // extern "C"
