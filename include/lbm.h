/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann permeability library.
 *
 * The library computes the intrinsic permeability of a porous solid mask the
 * way Li, Ho, Wu & Zhang ("Lattice Boltzmann modelling of intrinsic
 * permeability", arXiv:1609.09685) do in Sec. 2: a BGK lattice Boltzmann run of
 * pressure-driven flow along x (D2Q9 in 2D, D3Q19 in 3D), iterated to steady
 * state, with the permeability taken from the simulated mass flow rate by
 * Darcy's law and reported against Kn = sqrt(pi/6) (tau - 1/2) / N_x.  It also
 * runs the paper's force-driven periodic 3D setup (Eq. 2), a TRT collision and
 * local pore-size / local-Kn diagnostics.
 *
 * Every lattice update, reduction, mask-generation and field conversion step
 * runs in the library's own CUDA kernels (sm_103a).  Host code only validates
 * arguments, moves buffers and takes scalar decisions between kernel launches.
 *
 * Conventions (all entry points):
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3, nu = (tau - 1/2)/3 (Eq. 1).
 *   - Masks are host arrays of uint8, x fastest: index (z*ny + y)*nx + x,
 *     1 = solid, 0 = fluid.  Any other byte value is rejected (LBM_ERR_ARG).
 *     Masks are copied; the caller keeps ownership.
 *   - Output arrays are caller-allocated host arrays unless stated otherwise.
 *   - Direction order, D2Q9: 0 (0,0); 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1);
 *     5 (1,1); 6 (-1,1); 7 (-1,-1); 8 (1,-1).
 *     D3Q19: 0 rest; 1 (1,0,0); 2 (-1,0,0); 3 (0,1,0); 4 (0,-1,0); 5 (0,0,1);
 *     6 (0,0,-1); 7 (1,1,0); 8 (-1,-1,0); 9 (1,-1,0); 10 (-1,1,0); 11 (1,0,1);
 *     12 (-1,0,-1); 13 (1,0,-1); 14 (-1,0,1); 15 (0,1,1); 16 (0,-1,-1);
 *     17 (0,1,-1); 18 (0,-1,1).
 *   - Device state is FP32 "shifted" populations g_i = f_i - w_i rho_0 with
 *     rho_0 = rho_out, so Stokes-regime density differences are not lost to
 *     round-off; flux, residual and permeability arithmetic is FP64.
 *   - Nothing aborts, prints or exits.  Every failure is an lbm_status with a
 *     detail string from lbm_last_error().  A handle is not thread-safe.
 *   - Work is enqueued on lbm_options.stream (NULL = legacy default stream);
 *     calls that return host data synchronise that stream.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_NOT_CONVERGED = 1, /* max_steps reached before tol */
    LBM_STALLED = 2,       /* FP32 residual floor reached (see lbm_run_to_steady) */
    LBM_ERR_ARG = -1,
    LBM_ERR_CUDA = -2,
    LBM_ERR_OOM = -3,
    LBM_DIVERGED = -4, /* a non-finite velocity appeared */
    LBM_TIMEOUT = -5,
    LBM_ERR_IO = -6,
    LBM_ERR_INTERNAL = -7, /* a kernel's bounded wait gave up (a staged or band gather step's copy, a fused
                              pair's wait on its neighbouring blocks), or a checked build met an out-of-range
                              index; reported at the next observation from the device error word */
    LBM_CANCELLED = -8
} lbm_status;

enum { LBM_EQ_QUADRATIC = 0, LBM_EQ_LINEAR = 1 };

/*
 * Collision.  BGK is the paper's single-relaxation model (Sec. 2, Eq. 1).  TRT
 * (Ginzburg 2005) follows the paper's pointer to multi-relaxation models for a
 * wall location that does not move with the viscosity: the parts of f - f_eq
 * even and odd under i -> opp(i) relax with 1/tau (viscosity, as in BGK) and
 * 1/tau_minus, tau_minus = 1/2 + Lambda/(tau - 1/2).  Steady states then
 * depend on tau only through the viscosity; with Lambda = 3/16 a straight
 * bounce-back wall sits exactly half way between nodes.
 */
enum { LBM_COLL_BGK = 0, LBM_COLL_TRT = 1 };

/* Solver options.  Fill with lbm_options_default() and override fields. */
typedef struct lbm_options {
    int32_t struct_size;     /* sizeof(lbm_options) */
    int32_t equilibrium;     /* LBM_EQ_QUADRATIC (default) or LBM_EQ_LINEAR (Stokes, Sec. 2's 3D case) */
    int32_t check_interval;  /* steps between convergence checks N (default 100, >= 1) */
    int32_t stall_checks;    /* checks without a new minimum residual before LBM_STALLED (default 200) */
    double stall_floor;      /* stall rule applies only while r < stall_floor (default 1e-5) */
    double rho_out;          /* outlet density rho_0 (default 1.0) */
    void* stream;            /* cudaStream_t; NULL = legacy default stream */
    int32_t block_threads;   /* block size of the step kernels, a multiple of 32 up to 256; 0 = 128 */
    int32_t use_graphs;      /* capture each check interval as a CUDA graph (default 1) */
    volatile const int32_t* cancel_flag; /* host flag polled between intervals; nonzero cancels */
    int32_t strip_rows;      /* rows per work item of the pull and gather steps (0 = default 8, max 255) */
    double k_tol;            /* permeability-based stop (see lbm_run_to_steady); 0 disables (default 1e-5) */
    int32_t in_place_pairs;  /* 1 (default): advance plain steps two at a time in place (a gather step that
                                writes each result back to the slot it read, then a step on each node's own
                                slots); same arithmetic as two pull steps.  0: one pull step at a time. */
    int32_t collision;       /* LBM_COLL_BGK (default) or LBM_COLL_TRT */
    double trt_lambda;       /* TRT: Lambda = (tau - 1/2)(tau_minus - 1/2), > 0 (default 3/16) */
    int32_t tile_rows;       /* gather step of the in-place pair (D2Q9): 1..4 = staged through shared memory in
                                tiles of this many rows x 128 nodes (bulk copies by a producer warp, consumed by
                                four compute warps); 0 or -1 = direct loads per strip (the default, faster on
                                GB300; D3Q19 always direct).  Every choice gives bit-identical results. */
    int32_t gather_batch;    /* rows of loads in flight per warp of the direct gather step: 2 or 4 (D2Q9), 1 or 2
                                (D3Q19); 0 = default (4 / 2).  Bit-identical results either way. */
    int32_t autotune;        /* 1: run lbm_autotune at creation (with tune_cache); 0 (default): keep the launch
                                configuration given by the fields above, i.e. force the defaults */
    const char* tune_cache;  /* JSON cache file of lbm_autotune (NULL: none); read and updated */
    /* Device memory of the solver's buffers: NULL, NULL (default) = the library's stream-ordered pool;
       otherwise every buffer comes from alloc_fn(alloc_ctx, bytes, stream) -- NULL return = out of memory,
       the call then fails with LBM_ERR_OOM after returning what it had -- and goes back through
       free_fn(alloc_ctx, ptr, stream).  Both or neither.  (How a framework such as PyTorch lends its
       caching allocator to the solver.) */
    void* (*alloc_fn)(void* ctx, size_t bytes, void* stream);
    void (*free_fn)(void* ctx, void* ptr, void* stream);
    void* alloc_ctx;
    int32_t band_rows;       /* gather step of the in-place pair (D2Q9): 1..64 = band gather step -- a block walks
                                down up to this many rows of a piece of up to 256 nodes (8 segments) of the
                                width, staging each row's compact range of every plane in a shared-memory ring
                                by bulk copies (one copy per plane and row) -- ; -1 = not used; 0 = the
                                library's default (not used: the direct gather step measured faster).  Both
                                band_rows and tile_rows > 0 is an error; ignored for D3Q19 and for force-driven
                                or slab solvers.  Bit-identical results either way. */
    int32_t pair_block_mb;   /* L2-blocked pairs (1..4096): both steps of an in-place pair in one persistent
                                launch over blocks of about this many MB of populations -- the gather step runs
                                about 32 MB of blocks ahead of the local step, which then reads each block
                                while it is still in L2 -- instead of two whole-batch launches; -1 = whole-batch
                                pairs; 0 = the library's default (whole-batch pairs, measured faster).  Used with
                                the direct gather step only.  Bit-identical results either way. */
} lbm_options;

/* One domain of a batch. */
typedef struct lbm_domain_desc {
    const uint8_t* mask; /* host, nx*ny*nz bytes */
    int32_t nx, ny, nz;  /* nz = 1 for D2Q9; all domains of a batch share the lattice */
    double tau;          /* relaxation time, > 0.5 */
    double drho;         /* rho_in - rho_out (pressure difference / c_s^2) */
} lbm_domain_desc;

typedef struct lbm_solver* lbm_handle;

/* Library version string ("major.minor.patch"). */
const char* lbm_version(void);
/* Static description of a status code. */
const char* lbm_status_string(lbm_status s);
/* Detail of the last failure on h, or of the last failure of a call without a
 * handle on this thread when h is NULL.  Valid until the next call. */
const char* lbm_last_error(lbm_handle h);
/* Defaults described in lbm_options. */
void lbm_options_default(lbm_options* opt);
/*
 * The lattice tables the kernels use (Qian, d'Humieres & Lallemand 1992; the
 * direction order above): for q = 9 (D2Q9) or 19 (D3Q19), c[3 q] the
 * velocities (x, y, z per direction), w[q] the weights, opp[q] the reversed
 * direction, flip_y[q] / flip_z[q] the direction with its y / z component
 * reversed (the specular reflection at the symmetry planes, Sec. 2 Fig. 1).
 * Host arrays, each nullable.  Host only; no device is touched.
 * LBM_ERR_ARG for any other q.
 */
lbm_status lbm_lattice(int32_t q, int32_t* c, double* w, int32_t* opp, int32_t* flip_y, int32_t* flip_z);

/*
 * QSGS porous mask (Sec. 2, "randomly generated quartet structure"; QSGS
 * after Wang et al. 2007) on the GPU.  Grows the solid phase from cores
 * (probability core_p) with growth probability d_face to the 4 (2D) / 6 (3D)
 * axis neighbours, d_face/2 to 3D edge neighbours and d_face/4 to 2D diagonal
 * or 3D corner neighbours, in synchronous iterations driven by a counter-based
 * splitmix64 hash of (seed, iteration, cell, neighbour slot), until exactly
 * S = round((1 - porosity) nx ny nz) cells are solid (ties in the last
 * iteration broken by ascending (draw, cell index)).  nz = 1 gives a 2D mask.
 * mask_out: host, nx*ny*nz bytes.  iterations (nullable): growth iterations.
 * Errors: LBM_ERR_ARG for bad sizes / porosity outside [0,1] / more than 2^31
 * cells; LBM_ERR_INTERNAL if no solid core appears while S > 0, or if 10^6
 * growth iterations pass before S cells are solid (each with its own detail
 * string).
 */
lbm_status lbm_qsgs(uint64_t seed, int32_t nx, int32_t ny, int32_t nz, double core_p,
                    double porosity, double d_face, void* stream, uint8_t* mask_out,
                    int32_t* iterations);

/*
 * Allocation-free variant of lbm_qsgs, for callers that cannot allocate GPU
 * memory while they run (for example a host whose device memory is owned by
 * its own pool allocator, or code under a policy that forbids cudaMalloc and
 * cudaFree after set-up).  The paper has no counterpart to this entry point:
 * it only changes where the scratch lives.  It produces the same mask as
 * lbm_qsgs, written to mask_dev_out, a caller-owned DEVICE buffer of
 * nx*ny*nz bytes on the current device, enqueued on `stream` (NULL = legacy
 * default stream); the call returns after the mask is complete.
 *   - Scratch is a file-scope device array inside the library, sized for at
 *     most 1,048,576 cells (about 9 MB, held on every GPU that loads the
 *     library until the process exits).  Larger grids return LBM_ERR_ARG.
 *   - Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 *   - The first call on a device looks up the scratch array's device address
 *     (once per device, with that device current); make that first call before
 *     any stream capture.
 *   - Every call, the first and the later ones, synchronises `stream` and reads
 *     a candidate counter back to the host between its kernel launches.
 *   - All calls share the scratch array and it keeps the last call's contents
 *     (every value a call reads is written by that call first).  Calls that
 *     overlap on the GPU -- from several host threads or several streams --
 *     race on it: serialise them.
 * Errors are reported like lbm_qsgs's, with detail from lbm_last_error(NULL).
 */
lbm_status lbm_qsgs_noalloc(uint64_t seed, int32_t nx, int32_t ny, int32_t nz, double core_p,
                            double porosity, double d_face, void* stream, uint8_t* mask_dev_out,
                            int32_t* iterations);

/*
 * Create a solver for a batch of n independent domains (Sec. 2's sweeps of
 * tau x resolution x geometry), all D2Q9 (every nz = 1) or all D3Q19 (every
 * nz > 1, or lattice forced by lbm_create_domain_3d).  Per domain: pressure
 * rho_out + drho at the fluid nodes of x = 0 and rho_out at x = nx - 1
 * (Zou-He), specular symmetry planes on the y (and z) faces, halfway
 * bounce-back at solids, and the initial state of rest equilibrium with rho
 * falling linearly from inlet to outlet.  Requires nx >= 3, ny >= 1, nz >= 1,
 * tau > 0.5.  opt may be NULL.  On success *out owns all device memory.
 */
lbm_status lbm_batch_create(int32_t n, const lbm_domain_desc* descs, const lbm_options* opt,
                            lbm_handle* out);

/*
 * Force-driven flow with every face periodic: the paper's 3D experiment
 * (Sec. 2, Eq. 2).  n domains as in lbm_batch_create (descs[d].drho is
 * ignored), each driven by a body acceleration g[d] along +x (host array of n
 * doubles) instead of the pressure boundaries.  Solids bounce back half way;
 * the forcing is Guo, Zheng & Shi (2002) with force density F = rho_out g;
 * lbm_permeability then returns Eq. 2's k = nu <u>/g, <u> the sum over fluid
 * nodes of rho u_x over rho_out N_grid, with rho u the fluid momentum of Guo's
 * scheme (the pre-collision momentum plus F/2, i.e. the stored post-collision
 * momentum minus F/2).  BGK or TRT (opt->collision).  Plain steps run as
 * in-place pairs of kernels of their own (a forced gather step that writes
 * each result back to the slot it read, then a forced step on each node's own
 * slots) when opt->in_place_pairs is 1 (the default), else as pull steps; the
 * two give bit-identical populations.
 * lbm_save, lbm_nn_targets and lbm_warm_start return LBM_ERR_ARG on such a
 * solver.
 */
lbm_status lbm_batch_create_forced(int32_t n, const lbm_domain_desc* descs, const double* g,
                                   const lbm_options* opt, lbm_handle* out);
/* Single 2D (D2Q9) domain: a batch of one. */
lbm_status lbm_create_domain(const uint8_t* mask, int32_t nx, int32_t ny, double tau,
                             double drho, const lbm_options* opt, lbm_handle* out);
/* Single 3D (D3Q19) domain: a batch of one. */
lbm_status lbm_create_domain_3d(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz,
                                double tau, double drho, const lbm_options* opt,
                                lbm_handle* out);
/*
 * Batch names of the three calls that act on a whole batch.  Every solver is a
 * batch (a single domain is a batch of one), so lbm_batch is the same handle
 * and these are the batch forms of the calls below:
 *   lbm_batch_run_to_steady: lbm_run_to_steady (Sec. 2, "iterated to steady
 *     state") with only the per-domain statuses (host array of n, nullable);
 *   lbm_batch_permeability: lbm_permeability (Sec. 2, Darcy's law with the
 *     simulated mass flow rate; nu from Eq. 1) without the Kn output;
 *   lbm_batch_destroy: lbm_destroy.
 * Statuses and errors are those of the calls they stand for.
 */
typedef lbm_handle lbm_batch;
lbm_status lbm_batch_run_to_steady(lbm_batch b, double tol, int64_t max_steps, lbm_status* per_domain);
lbm_status lbm_batch_permeability(lbm_batch b, double* k);
void lbm_batch_destroy(lbm_batch b);

/*
 * x-slab of a larger domain: one domain of N_x columns cut into slabs of
 * consecutive columns, each run by its own solver (on its own GPU or process),
 * so that a domain larger than one GPU runs as several; the method (Sec. 2) is
 * unchanged.  mask: the slab's columns x_offset .. x_offset + nx - 1 of the
 * whole domain's mask (host, nx*ny*nz, x fastest), including one ghost column
 * at each cut: bit 0 of `ghosts` says column 0 is a copy of the left
 * neighbour's last real column, bit 1 that column nx - 1 is a copy of the right
 * neighbour's first; a ghost is required exactly at every cut (x_offset > 0,
 * x_offset + nx < nx_global).  drho is the whole domain's; the inlet (Zou-He,
 * rho_out + drho) acts only on the slab holding x = 0, the outlet only on the
 * slab holding x = nx_global - 1, and the initial density ramp runs over the
 * whole domain.  A slab advances by pull steps (opt.in_place_pairs is
 * ignored); its ghost columns are pulled from but never written, and no
 * observable counts them.  After every step each cut is exchanged:
 *   lbm_slab_export(h, side, buf): pack the real column next to the cut
 *     (side 0: first real column, 1: last real column) -- the planes whose
 *     direction crosses the cut towards the neighbour (c_x = -1 leftwards,
 *     +1 rightwards; 3 of 9 in D2Q9, 5 of 19 in D3Q19), dense [planes][fluid
 *     nodes of the column in (z, y) order] -- into buf;
 *   lbm_slab_import(h, side, buf): unpack the neighbour's buffer into the
 *     ghost column on that side;
 * buf is a DEVICE buffer of lbm_slab_halo_floats(h, side, incoming) floats
 * (incoming = 0: what export packs, 1: what import unpacks; a receiver's
 * incoming count equals its neighbour's outgoing one), owned by the caller;
 * both calls are enqueued on the solver's stream (order them against the
 * neighbour's stream, or share one).  lbm_slab_observables turns observables summed
 * over all slabs (lbm_step_observe's 8 slots, slot 3 as a maximum) into the
 * whole domain's permeability (Darcy's law with the mass flow rate, Sec. 2;
 * nu from Eq. 1), Kn = sqrt(pi/6)(tau - 1/2)/nx_global and residual
 * r = sqrt(sum |du|^2 / sum |u|^2); each null output is skipped.
 * lbm_run_to_steady, lbm_permeability and lbm_save return LBM_ERR_ARG on a slab
 * (its driver exchanges the halos and sums the observables).  Errors:
 * LBM_ERR_ARG for inconsistent geometry or a side without a neighbour.
 */
lbm_status lbm_slab_create(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz, double tau, double drho,
                           int32_t x_offset, int32_t nx_global, int32_t ghosts, const lbm_options* opt,
                           lbm_handle* out);
lbm_status lbm_slab_halo_floats(lbm_handle h, int32_t side, int32_t incoming, int64_t* n);
lbm_status lbm_slab_export(lbm_handle h, int32_t side, float* buf);
lbm_status lbm_slab_import(lbm_handle h, int32_t side, const float* buf);
lbm_status lbm_slab_observables(lbm_handle h, const double* obs_sum, double* k, double* kn, double* residual);

/* Synchronises the solver's stream and frees its resources.  Device memory of
 * solvers comes from one stream-ordered pool per device; up to 8 GB of freed
 * blocks stay cached there for the next solver, the rest returns to the
 * CUDA driver at the next synchronisation. */
void lbm_destroy(lbm_handle h);

/*
 * Launch configuration of the plain steps, and the runtime autotuner.  The
 * paper has no counterpart: these choose how the step of Sec. 2 is mapped onto
 * the GPU, never what it computes -- every configuration gives bit-identical
 * populations.
 *   block_threads  block size of the gather, local and pull steps (32..256, a
 *                  multiple of 32)
 *   strip_rows     rows per work item of the pull and direct gather steps (1..255)
 *   gather_batch   rows of loads a warp of the direct gather step keeps in
 *                  flight: 2 or 4 (D2Q9), 1 or 2 (D3Q19)
 *   tile_rows      0: direct gather step; 1..4: staged gather step (D2Q9)
 *   band_rows      0: not used; 1..64: band gather step with up to this many
 *                  rows per band (D2Q9; not together with tile_rows)
 *   pair_block_mb  0: whole-batch pairs; 1..4096: L2-blocked pairs with blocks
 *                  of about this many MB (with the direct gather step)
 * lbm_get_launch reports the solver's configuration; lbm_set_launch changes
 * it (LBM_ERR_ARG for a value outside the ranges above).
 */
typedef struct lbm_launch {
    int32_t block_threads, strip_rows, gather_batch, tile_rows, band_rows, pair_block_mb;
} lbm_launch;
lbm_status lbm_get_launch(lbm_handle h, lbm_launch* cfg);
lbm_status lbm_set_launch(lbm_handle h, const lbm_launch* cfg);
/* Device time per plain step: nsteps (even, 2..10000) plain steps of every
 * active domain, launched one by one on the solver's stream, timed with CUDA
 * events after two warm-up steps.  The populations are saved before and
 * restored after, and the step counter does not move.  Synchronises. */
lbm_status lbm_time_steps(lbm_handle h, int32_t nsteps, double* us_per_step);

/*
 * Autotuner.  Times each candidate configuration with lbm_time_steps (nsteps
 * per candidate, 0 = 20) and keeps the fastest; the candidates are block size
 * {64, 128, 256} x strip rows {4, 8, 16} x gather batch (both compiled ones),
 * plus, for D2Q9, the staged gather step with 2 and 3 tile rows and the band
 * gather step with 16, 32 and 64 band rows.  With
 * cache_path (nullable), the choice is looked up first under the key of
 * lbm_tune_key and stored after a search.  Force-driven solvers have nothing
 * to tune (their steps run kernels of their own in one fixed configuration):
 * the call only reports their configuration.  out (nullable) receives the chosen and the
 * default configuration with their times per plain step, the number of
 * configurations timed (0 when the cache answered) and whether it did.
 */
typedef struct lbm_tune_result {
    lbm_launch chosen;
    double us_per_step;
    lbm_launch defaults;
    double us_per_step_default;
    int32_t candidates;
    int32_t from_cache;
} lbm_tune_result;
lbm_status lbm_autotune(lbm_handle h, const char* cache_path, int32_t nsteps, lbm_tune_result* out);
/* Cache key of a solver: "<device>|q<Q>|n2^<b>|eq<e>|coll<c>|<kernel hash>",
 * b = floor(log2(fluid nodes)), spaces of the device name replaced by '_',
 * the kernel hash that of the library's CUDA sources.  lbm_tune_key_for
 * builds the same key from its parts (host only).  LBM_ERR_ARG if cap is too
 * small. */
lbm_status lbm_tune_key(lbm_handle h, char* key, size_t cap);
lbm_status lbm_tune_key_for(const char* device_name, int32_t q, int64_t fluid_nodes, int32_t eq,
                            int32_t collision, char* key, size_t cap);
/* The cache file: a JSON object with one member per key, each an object with
 * the four lbm_launch fields and "us_per_step".  lbm_tune_cache_get sets
 * *found to 1 and fills cfg / us_per_step (nullable) when key is present
 * (a missing or unreadable file counts as empty); lbm_tune_cache_put adds or
 * replaces key and rewrites the file (LBM_ERR_IO if it cannot).  Host only. */
lbm_status lbm_tune_cache_get(const char* path, const char* key, lbm_launch* cfg, double* us_per_step,
                              int32_t* found);
lbm_status lbm_tune_cache_put(const char* path, const char* key, const lbm_launch* cfg, double us_per_step);

/*
 * Checked build (compiled with -DLBM_CHECKED; the paper has no counterpart:
 * a failure-detection aid).  Its pull and direct gather steps compare every
 * population index they take from the neighbour-window table with the
 * buffer's extent; an index outside is not used and sets a device error bit
 * that the next observation (lbm_step_observe, lbm_run_to_steady,
 * lbm_permeability, lbm_profile_steps) returns as LBM_ERR_INTERNAL, so a
 * corrupted table never turns into a bad memory access.
 * lbm_build_checked: *checked = 1 in such a build, else 0.
 * lbm_debug_corrupt_window: overwrite the compact base index of segment seg's
 * window record with value (synchronises the solver's stream) -- a fault
 * injection for testing the checks; LBM_ERR_ARG in a regular build.
 */
lbm_status lbm_build_checked(int32_t* checked);
lbm_status lbm_debug_corrupt_window(lbm_handle h, uint32_t seg, uint32_t value);

/* Number of domains, lattice size Q, and fluid node count of domain d. */
lbm_status lbm_info(lbm_handle h, int32_t* n_domains, int32_t* q, int64_t* fluid_nodes_total);
lbm_status lbm_domain_fluid_nodes(lbm_handle h, int32_t d, int64_t* fluid_nodes);

/* Enqueue nsteps fused stream + boundary + collide steps on every active
 * domain.  Does not synchronise. */
lbm_status lbm_step(lbm_handle h, int64_t nsteps);

/*
 * Local pore size and local Knudsen number of domain d (Sec. 2 notes that the
 * local Kn in narrow pores can be much larger than Kn = sqrt(pi/6)(tau-1/2)/N_x).
 * The paper defines no pore size; here a fluid node's pore size is
 * h = 2 D - 1, D the Euclidean distance in nodes to the nearest solid node of
 * the domain (exact, integer D^2), so that the centre node of a channel of h
 * fluid rows gets h; the local Kn is sqrt(pi/6)(tau - 1/2)/h.  The faces are
 * not walls: a node that sees no solid node has D^2 = UINT32_MAX, h = +inf and
 * Kn = 0.  Outputs are host arrays in the mask's dense layout (nz*ny*nx, x
 * fastest), each nullable (at least one given): d2_out the squared distance
 * (0 on solids), h_out the pore size and kn_out the local Kn (both 0 on
 * solids).  Device scratch of 16 bytes per node comes from the solver's memory
 * pool for the duration of the call; the call synchronises.
 */
lbm_status lbm_local_knudsen(lbm_handle h, int32_t d, uint32_t* d2_out, double* h_out, double* kn_out);

/*
 * Measurement: advance nsteps plain steps exactly as lbm_step does (same
 * kernels, same pairing), but launch every kernel on its own with a CUDA event
 * recorded before and after it on the solver's stream, instead of through the
 * cached graph.  On return (the call synchronises) times_us[k] holds the summed
 * device time in microseconds and counts[k] the launches of each kernel kind
 * k: LBM_KERNEL_GATHER (the gather step of an in-place pair),
 * LBM_KERNEL_LOCAL (its local step), LBM_KERNEL_PULL (a pull step),
 * LBM_KERNEL_PULL_OBSERVE (unused here: always 0), LBM_KERNEL_PAIR_FUSED
 * (both steps of an L2-blocked pair in one launch, lbm_options.pair_block_mb).
 * Both arrays are host memory of LBM_NUM_KERNEL_KINDS entries; nsteps is at
 * most 100000.
 * No counterpart in the paper (a timing aid for the kernels of Sec. 2's step).
 */
enum { LBM_KERNEL_GATHER = 0, LBM_KERNEL_LOCAL = 1, LBM_KERNEL_PULL = 2, LBM_KERNEL_PULL_OBSERVE = 3,
       LBM_KERNEL_PAIR_FUSED = 4, LBM_NUM_KERNEL_KINDS = 5 };
lbm_status lbm_profile_steps(lbm_handle h, int64_t nsteps, double* times_us, int64_t* counts);

/*
 * Enqueue nsteps steps of which the last also reduces, per domain, in FP64:
 *   obs[d*8 + 0] = sum over the N_x - 1 interior planes x + 1/2 of the mass
 *                  crossing each plane in the next streaming (the link flux
 *                  of the post-collision populations); /(N_x - 1) = mass flow rate
 *   obs[d*8 + 1] = sum |u - u_prev|^2   (u_prev = u at the previous observation)
 *   obs[d*8 + 2] = sum |u|^2
 *   obs[d*8 + 3] = max |u|
 *   obs[d*8 + 4] = count of nodes with a non-finite velocity
 *   obs[d*8 + 5] = sum of (rho - rho_0)
 *   obs[d*8 + 6] = sum of j_x over fluid nodes (node momentum, a diagnostic)
 *   obs[d*8 + 7] = 0 (reserved)
 * and stores u as the new u_prev.  nsteps = 0 observes the current state
 * without stepping.  obs: host, 8*n doubles; the call synchronises.
 */
lbm_status lbm_step_observe(lbm_handle h, int64_t nsteps, double* obs);

/*
 * Iterate every domain to steady state (the paper's "iterated to steady
 * state").  Every check_interval steps the residual
 *   r = sqrt( sum |u^t - u^{t-N}|^2 / sum |u^t|^2 )
 * is formed per domain; a domain with r < tol is converged and retired from
 * further stepping.  A domain is also converged (LBM_OK) when its permeability
 * k(t), from the FP64 mass flow rate of each check, has settled: over windows
 * of 10 checks, with D1 and D0 the last two changes of k and q = |D1/D0|, the
 * remaining error of a geometric approach is at most |D1| q/(1 - q); the
 * domain stops once that bound is below opt.k_tol |k| at 10 consecutive checks
 * with r < 10 opt.k_tol (or with |k| below 1e-3 of its largest value in the
 * run: a flow that dies out keeps r of order one), once k has stayed within
 * 0.05 opt.k_tol |k| over 40 checks, or once |k| has stayed below
 * 0.1 opt.k_tol times its largest value for 10 checks (no connected fluid
 * path: k -> 0) (|k| is taken
 * as at least 1e-3 of its largest value in the run, so that a domain whose
 * flow dies out, having no through-path, stops too).  This is the
 * stop that matters in FP32: in the Stokes regime the per-node residual
 * reaches its rounding floor long before the mass flow rate does.  Because the state is FP32, r eventually stops decaying
 * and jitters at a rounding floor: a domain whose r is below stall_floor and
 * has not set a new minimum for stall_checks consecutive checks is retired as
 * LBM_STALLED (a residual more than 30x above the minimum so far counts as a
 * transient and restarts the count).  Returns LBM_OK when every domain converged,
 * LBM_STALLED when all finished and some stalled, LBM_NOT_CONVERGED when
 * max_steps was reached first, LBM_DIVERGED on a non-finite velocity,
 * LBM_CANCELLED if opt.cancel_flag was raised.  Per-domain arrays (each
 * nullable, n entries): status, steps taken, last residual.
 */
lbm_status lbm_run_to_steady(lbm_handle h, double tol, int64_t max_steps,
                             lbm_status* status, int64_t* steps, double* residual);

/*
 * Darcy permeability of each domain from its last observed mass flow rate
 * (Sec. 2, "Darcy law with simulated mass flow rate"):
 *   k = nu <J> (nx - 1) / (ny nz c_s^2 drho),  nu = (tau - 1/2)/3 (Eq. 1),
 *   <J> = the mass crossing an interior x plane per step, averaged over the
 *   nx - 1 planes (obs slot 0 / (nx - 1)).  Fluid off the through-paths (closed
 *   pockets, boundary nodes boxed in by solid) carries no such flux.
 * and Kn = sqrt(pi/6) (tau - 1/2) / nx (Sec. 2).  If no observation exists yet
 * the current state is observed first.  k, kn: host arrays of n (kn nullable).
 */
lbm_status lbm_permeability(lbm_handle h, double* k, double* kn);

/* Dense fields of domain d (host, nx*ny*nz each, zero on solids), from the
 * current populations in FP64: rho = rho_0 + sum g, u = sum c g / rho. */
lbm_status lbm_get_fields(lbm_handle h, int32_t d, double* rho, double* ux, double* uy,
                          double* uz /* nullable in 2D */);
/* Dense unshifted populations of domain d: host double [nz][ny][nx][Q],
 * f = g + w rho_0 on fluid nodes, 0 on solids. */
lbm_status lbm_get_populations(lbm_handle h, int32_t d, double* f);
/* Overwrite domain d's populations from the same dense layout (host double). */
lbm_status lbm_set_populations(lbm_handle h, int32_t d, const double* f);
/*
 * Warm start: set domain d's populations to the equilibrium of given fields,
 * g_i = g_eq_i(rho - rho_0, u).  drho, ux, uy, uz: dense float arrays of
 * nx*ny*nz (uz ignored in 2D, may be NULL); device pointers when on_device is
 * nonzero (read on the solver's stream), else host.  Resets u_prev to u.
 */
lbm_status lbm_set_fields(lbm_handle h, int32_t d, const float* drho, const float* ux,
                          const float* uy, const float* uz, int32_t on_device);

/* Per-check-interval record of domain d from the last lbm_run_to_steady:
 * global step counter, permeability k(t) from that interval's flux (as
 * lbm_permeability), residual r, and host seconds since the call began.  Up to
 * `capacity` entries are written to each non-null array; *count receives the
 * number recorded.  Used to measure time-to-permeability a posteriori. */
lbm_status lbm_get_history(lbm_handle h, int32_t d, int64_t* steps, double* k, double* residual,
                           double* seconds, int32_t capacity, int32_t* count);

/* Steps taken since creation (the batch's global step counter). */
lbm_status lbm_get_step(lbm_handle h, int64_t* step);

/* Checkpoint: masks, parameters, populations, u_prev, step counter and
 * per-domain run state; lbm_load restores a solver that continues bit for bit. */
lbm_status lbm_save(lbm_handle h, const char* path);
lbm_status lbm_load(const char* path, const lbm_options* opt, lbm_handle* out);

/* ------------------------------------------------------------------------ */
/* Learned warm start (U-Net).                                               */
/* ------------------------------------------------------------------------ */
/*
 * The network maps a 2D mask, x / (nx - 1) and (tau - 1/2) to the normalised
 * steady fields: the density's deviation from the linear inlet-to-outlet ramp,
 * (rho - rho_out)/drho - (1 - x/(nx - 1)), and u nu (nx - 1)/(c_s^2 drho).  In the
 * Stokes regime of Sec. 2 these depend on the geometry (and weakly on tau)
 * only.  Its prediction only initialises the populations; the lattice
 * Boltzmann iteration (Sec. 2) then converges from there, so the network
 * changes how fast the steady state is reached, not what it is.  The paper has
 * no learned component; this is the acceleration layer built on it.
 *
 * Tensor conventions: NHWC, H = ny rows, W = nx columns.  Activations and
 * gradients are bf16 with channel counts that are multiples of 16.  Weights
 * are bf16 [taps][cout][cin] (taps = 9 for 3x3 with zero padding, 1 for 1x1),
 * with an FP32 master copy for the optimiser; biases are FP32.  All pointers
 * are DEVICE pointers, 16-byte aligned, owned by the caller.  Work is enqueued
 * on `stream` (NULL = legacy default stream) and nothing is synchronised.
 * Shapes are validated before any launch (LBM_ERR_ARG); launch failures
 * return LBM_ERR_CUDA.  Details come from lbm_last_error(NULL).
 */

/* Tensor-core path of the convolutions (process-wide; all give the same
 * result up to FP32 summation order):
 *   LBM_NN_CONV_MMA_SYNC  warp-level mma.sync m16n8k16, operands in registers;
 *   LBM_NN_CONV_TCGEN05   5th-generation tcgen05.mma issued by one thread per
 *                         block, operands in shared memory, the FP32
 *                         accumulator in tensor memory;
 *   LBM_NN_CONV_AUTO      (default) tcgen05 for layers with cin >= 32,
 *                         cout >= 64 and images of w >= 64 and h w >= 2048
 *                         (where it measured faster on GB300), else mma.sync.
 * lbm_nn_sync_status synchronises `stream` and returns LBM_ERR_INTERNAL if a
 * tcgen05 convolution gave up one of its bounded waits since the last call
 * (its output is then incomplete); it clears that record. */
enum { LBM_NN_CONV_MMA_SYNC = 0, LBM_NN_CONV_TCGEN05 = 1, LBM_NN_CONV_AUTO = 2 };
lbm_status lbm_nn_set_conv_impl(int32_t impl);
int32_t lbm_nn_get_conv_impl(void);
lbm_status lbm_nn_sync_status(void* stream);

/* out = act(b + sum_{tap, ci} in[p + off_tap, ci] w[tap][co][ci]), act = ReLU if
 * relu != 0.  BF16 tensor-core implicit GEMM (the path lbm_nn_set_conv_impl
 * selects), FP32 accumulation.  bias and out_f32 (an FP32 copy of out) may be
 * NULL. */
lbm_status lbm_nn_conv_fwd(const void* in, int32_t n, int32_t h, int32_t w, int32_t cin, const void* wts,
                           const float* bias, int32_t taps, int32_t cout, int32_t relu, void* out,
                           float* out_f32, void* stream);
/* gin = adjoint of the convolution applied to gout (no activation).
 * wflip_scratch: taps*cin*cout bf16. */
lbm_status lbm_nn_conv_bwd_data(const void* gout, int32_t n, int32_t h, int32_t w, int32_t cout,
                                const void* wts, int32_t taps, int32_t cin, void* wflip_scratch,
                                void* gin, void* stream);
/* dw[tap][co][ci] (+)= sum_p gout[p, co] in[p + off_tap, ci], db[co] (+)= sum_p gout[p, co]
 * (FP32; accumulate != 0 adds to dw/db).  scratch: FP32 partial sums; at least
 * taps*cout*cin + cout floats, more allows more parallel blocks.  db may be NULL. */
lbm_status lbm_nn_conv_bwd_weight(const void* in, const void* gout, int32_t n, int32_t h, int32_t w,
                                  int32_t cin, int32_t cout, int32_t taps, float* dw, float* db,
                                  int32_t accumulate, float* scratch, size_t scratch_floats, void* stream);
/* gx = gy where y > 0, else 0 (gradient through a ReLU with output y). */
lbm_status lbm_nn_relu_bwd(const void* y, const void* gy, void* gx, size_t count, void* stream);
/* 2x2 average pooling of an h x w input (h, w even) and its adjoint. */
lbm_status lbm_nn_pool2_fwd(const void* in, int32_t n, int32_t h, int32_t w, int32_t c, void* out, void* stream);
lbm_status lbm_nn_pool2_bwd(const void* gout, int32_t n, int32_t h, int32_t w, int32_t c, void* gin,
                            void* stream);
/* Nearest-neighbour 2x upsampling of an h x w input and its adjoint. */
lbm_status lbm_nn_up2_fwd(const void* in, int32_t n, int32_t h, int32_t w, int32_t c, void* out, void* stream);
lbm_status lbm_nn_up2_bwd(const void* gout, int32_t n, int32_t h, int32_t w, int32_t c, void* gin, void* stream);
/* dst[p, dc0 + c] = src[p, sc0 + c] for c < nc over npix pixels (channel
 * concatenation and its adjoint); sld/dld are the channel strides. */
lbm_status lbm_nn_copy_channels(const void* src, int32_t sld, int32_t sc0, void* dst, int32_t dld, int32_t dc0,
                                int32_t nc, size_t npix, void* stream);
/* Masked, channel-weighted mean squared error over fluid pixels (solid[p] ==
 * 0) and the first nout <= 8 channels: *loss (device) = inv_count sum w_c d^2
 * and grad = 2 w_c d inv_count (bf16, stride ld; zero on solids and padding
 * channels; grad may be NULL).  target: FP32 [npix][nout].  weights: HOST
 * array of nout floats (NULL = all 1).  scratch256: 256 floats. */
lbm_status lbm_nn_mse(const void* pred, int32_t ld, const float* target, const uint8_t* solid, size_t npix,
                      int32_t nout, const float* weights, float inv_count, void* grad, float* scratch256,
                      float* loss, void* stream);
/* AdamW step (bias-corrected, decoupled weight decay) on FP32 parameters;
 * refreshes the bf16 copy p_bf16 when non-NULL.  step >= 1. */
lbm_status lbm_nn_adamw(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                        float eps, float wd, int32_t step, void* p_bf16, void* stream);
/* out = a + b elementwise (bf16; used to merge gradients of a tensor read twice). */
lbm_status lbm_nn_add(const void* a, const void* b, void* out, size_t n, void* stream);
/* b = bf16(a) elementwise. */
lbm_status lbm_nn_f32_to_bf16(const float* a, void* b, size_t n, void* stream);
/* Network input of one h x w sample: channel 0 = solid flag, 1 = x / (w - 1),
 * 2 = tau_feat, 3..15 = 0 (bf16, 16 channels). */
lbm_status lbm_nn_make_input(const uint8_t* solid, int32_t h, int32_t w, float tau_feat, void* out, void* stream);
/* Training targets from 2D domain d's current populations (on the solver's
 * stream): out_dev FP32 [ny*nx][3] = ((rho - rho_out)/drho - (1 - x/(nx-1)),
 * u_x s, u_y s) with s = nu (nx - 1)/(c_s^2 drho); zero on solids. */
lbm_status lbm_nn_targets(lbm_handle h, int32_t d, float* out_dev);
/* Warm start of 2D domain d from a normalised prediction pred_dev (bf16
 * [ny*nx][ld], channels 0..2 as in lbm_nn_targets): populations = g_eq of
 * rho = rho_out + drho (p0 + 1 - x/(nx-1)) and u = (p1, p2)/s, |u| clipped to
 * 0.1 c_s. */
lbm_status lbm_warm_start(lbm_handle h, int32_t d, const void* pred_dev, int32_t ld);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
