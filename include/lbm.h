/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann permeability library.
 *
 * The library computes the intrinsic permeability of a porous solid mask the
 * way Li, Ho, Wu & Zhang ("Lattice Boltzmann modelling of intrinsic
 * permeability", arXiv:1609.09685) do in Sec. 2: a BGK lattice Boltzmann run of
 * pressure-driven flow along x (D2Q9 in 2D, D3Q19 in 3D), iterated to steady
 * state, with the permeability taken from the simulated mass flow rate by
 * Darcy's law and reported against Kn = sqrt(pi/6) (tau - 1/2) / N_x.
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
    LBM_ERR_INTERNAL = -7,
    LBM_CANCELLED = -8
} lbm_status;

enum { LBM_EQ_QUADRATIC = 0, LBM_EQ_LINEAR = 1 };

/* Solver options.  Fill with lbm_options_default() and override fields. */
typedef struct lbm_options {
    int32_t struct_size;     /* sizeof(lbm_options) */
    int32_t equilibrium;     /* LBM_EQ_QUADRATIC (default) or LBM_EQ_LINEAR (Stokes, Sec. 2's 3D case) */
    int32_t check_interval;  /* steps between convergence checks N (default 100, >= 1) */
    int32_t stall_checks;    /* checks without a new minimum residual before LBM_STALLED (default 50) */
    double stall_floor;      /* stall rule applies only while r < stall_floor (default 1e-5) */
    double rho_out;          /* outlet density rho_0 (default 1.0) */
    void* stream;            /* cudaStream_t; NULL = legacy default stream */
    int32_t block_threads;   /* stream-collide block size, a multiple of 32 up to 256; 0 = 256 */
    int32_t use_graphs;      /* capture each check interval as a CUDA graph (default 1) */
    volatile const int32_t* cancel_flag; /* host flag polled between intervals; nonzero cancels */
    int32_t strip_rows;      /* rows per stream-collide work item (0 = default 8, max 255) */
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
 * cells; LBM_ERR_INTERNAL if no solid core appears while S > 0.
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
/* Single 2D (D2Q9) domain: a batch of one. */
lbm_status lbm_create_domain(const uint8_t* mask, int32_t nx, int32_t ny, double tau,
                             double drho, const lbm_options* opt, lbm_handle* out);
/* Single 3D (D3Q19) domain: a batch of one. */
lbm_status lbm_create_domain_3d(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz,
                                double tau, double drho, const lbm_options* opt,
                                lbm_handle* out);
void lbm_destroy(lbm_handle h);

/* Number of domains, lattice size Q, and fluid node count of domain d. */
lbm_status lbm_info(lbm_handle h, int32_t* n_domains, int32_t* q, int64_t* fluid_nodes_total);
lbm_status lbm_domain_fluid_nodes(lbm_handle h, int32_t d, int64_t* fluid_nodes);

/* Enqueue nsteps fused stream + boundary + collide steps on every active
 * domain.  Does not synchronise. */
lbm_status lbm_step(lbm_handle h, int64_t nsteps);

/*
 * Enqueue nsteps steps of which the last also reduces, per domain, in FP64:
 *   obs[d*8 + 0] = sum of j_x over fluid nodes (mass flux, Eq. 2's sum)
 *   obs[d*8 + 1] = sum |u - u_prev|^2   (u_prev = u at the previous observation)
 *   obs[d*8 + 2] = sum |u|^2
 *   obs[d*8 + 3] = max |u|
 *   obs[d*8 + 4] = count of nodes with a non-finite velocity
 *   obs[d*8 + 5] = sum of (rho - rho_0)
 *   obs[d*8 + 6..7] = 0 (reserved)
 * and stores u as the new u_prev.  nsteps = 0 observes the current state
 * without stepping.  obs: host, 8*n doubles; the call synchronises.
 */
lbm_status lbm_step_observe(lbm_handle h, int64_t nsteps, double* obs);

/*
 * Iterate every domain to steady state (the paper's "iterated to steady
 * state").  Every check_interval steps the residual
 *   r = sqrt( sum |u^t - u^{t-N}|^2 / sum |u^t|^2 )
 * is formed per domain; a domain with r < tol is converged and retired from
 * further stepping.  Because the state is FP32, r eventually stops decaying
 * and jitters at a rounding floor: a domain whose r is below stall_floor and
 * has not set a new minimum for stall_checks consecutive checks is retired as
 * LBM_STALLED.  Returns LBM_OK when every domain converged,
 * LBM_STALLED when all finished and some stalled, LBM_NOT_CONVERGED when
 * max_steps was reached first, LBM_DIVERGED on a non-finite velocity,
 * LBM_CANCELLED if opt.cancel_flag was raised.  Per-domain arrays (each
 * nullable, n entries): status, steps taken, last residual.
 */
lbm_status lbm_run_to_steady(lbm_handle h, double tol, int64_t max_steps,
                             lbm_status* status, int64_t* steps, double* residual);

/*
 * Darcy permeability of each domain from its last observed mass flux (Sec. 2):
 *   k = nu <j_x> (nx - 1) / (c_s^2 drho),  nu = (tau - 1/2)/3 (Eq. 1),
 *   <j_x> = sum of j_x over fluid nodes / (nx ny nz)   (superficial, as Eq. 2)
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
 * number recorded.  Used to judge time-to-permeability a posteriori. */
lbm_status lbm_get_history(lbm_handle h, int32_t d, int64_t* steps, double* k, double* residual,
                           double* seconds, int32_t capacity, int32_t* count);

/* Steps taken since creation (the batch's global step counter). */
lbm_status lbm_get_step(lbm_handle h, int64_t* step);

/* Checkpoint: masks, parameters, populations, u_prev, step counter and
 * per-domain run state; lbm_load restores a solver that continues bit for bit. */
lbm_status lbm_save(lbm_handle h, const char* path);
lbm_status lbm_load(const char* path, const lbm_options* opt, lbm_handle* out);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
