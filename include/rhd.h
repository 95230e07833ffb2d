/*
 * rhd.h -- C ABI of librhd.so: the subcycled gray M1 radiation update under the reduced speed of
 * light approximation (RSLA) of Skinner & Ostriker (2013), "A two-moment radiation hydrodynamics
 * module in Athena using a time-explicit Godunov method", run on one NVIDIA GB300 (sm_103a).
 *
 * What one subcycle computes (Section 3.1, algorithm step 4; Sections 3.3 and 3.4):
 *   the radiation subsystem  d_t U + div F(U) = S  for U = (E, F/c) (Eq. algorithm:compactform,
 *   radiation rows of Eq. algorithm:variables, with chat in the time derivatives) is advanced by
 *   dt = dt_rad with the van Leer predictor/corrector integrator: first-order HLL fluxes
 *   (Eq. hyperbolic:hllflux2) and a half step, then piecewise-linear reconstruction of the half-step
 *   state, the M1 closure (Eqs. m1:m1tns, m1:chi), the wave speeds lambda_1,3 (Eq.
 *   hyperbolic:evals13), HLL fluxes and the full step; the non-stiff O(beta tau) sources
 *   (Eq. algorithm:source:explicit:rad with Eq. m1:simplifiedsource) are added in both stages, the
 *   absorption of F by the theta scheme of Eq. (source:stiff:radmomentum:soln), and the gas-radiation
 *   energy exchange by the quartic theta scheme of Eqs. (source:energyupdate)-(source:polynomial)
 *   (or its absorption-only, frozen-temperature or radiative-equilibrium variants) against the
 *   frozen gas state.  The flux-limiting condition |F| <= cE (Eq. m1:fluxlimit) is re-imposed after
 *   each stage.
 *
 * Around the subcycles (Section 3.1 steps 1-3 and 6): the time steps (rhd_max_signal_speed,
 * rhd_max_optical_depth, rhd_suggest_chat, rhd_time_steps), the gas step (rhd_gas_step: the Euler
 * equations with the explicit gas sources, one van Leer step with HLLC fluxes) and its second-order
 * source correction after the subcycles (rhd_gas_correct).
 *
 * Conventions
 *   - Every array is dense FP64 over the interior cells only, x fastest: idx = i + nx*(j + ny*k).
 *     A direction with n = 1 is inactive (1D: ny = nz = 1; 2D: nz = 1).  Active directions need
 *     n >= 3.
 *   - Pointers are borrowed, never kept: host arrays are copied during the call; device arrays
 *     (on_device = 1, e.g. torch CUDA tensors) are read or written on the context's stream during
 *     the call.  The library owns its own device buffers, which hold E and G = F/c.
 *   - Every function returns an rhd_status and never aborts, throws or exits.  Arguments are checked
 *     before any launch.  On failure rhd_last_error() describes the problem; the context stays
 *     usable unless the status is RHD_ERR_CUDA from a sticky device error.
 *   - A context is bound to one CUDA stream and is not thread-safe; separate contexts are
 *     independent.  A non-default stream given in the descriptor is used directly; with NULL (the
 *     legacy default stream) the library runs on a stream of its own, ordered after the caller's
 *     legacy stream on entry and before it on return.
 */
#ifndef RHD_H
#define RHD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RHD_ABI_VERSION 2  /* 2: rhd_stats gained the gas-step counters; the gas-step entry points */

typedef struct rhd_ctx rhd_ctx; /* opaque, library-owned */

typedef enum {
    RHD_OK = 0,
    RHD_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, out-of-range parameter) */
    RHD_ERR_STATE = 2,      /* call not valid in the current state (e.g. state not set yet) */
    RHD_ERR_CUDA = 3,       /* a CUDA runtime call failed; see rhd_last_error */
    RHD_ERR_OOM = 4,        /* device or pinned-host allocation failed */
    RHD_ERR_CFL = 5,        /* dt > cfl * min(dx) / chat, or chat > c (Eqs. algorithm:radtimestep) */
    RHD_ERR_NONFINITE = 6,  /* non-finite values were produced (reported by rhd_get_stats) */
    RHD_ERR_TIMEOUT = 7,    /* a bounded wait gave up */
    RHD_ERR_UNSUPPORTED = 8, /* the operation is not part of this library */
    RHD_ERR_BOUNDS = 9       /* debug build only: kernels met out-of-range array indices (rhd_get_stats) */
} rhd_status;

/* Environment (read by the library, none required):
 *   RHD_LOG=1                   print every error status and its message to stderr; 2: also the launch
 *                               configurations the autotuner chooses
 *   RHD_DEVICE_MEMORY_LIMIT=B   cap (bytes) on the cumulative device allocations of each context created
 *                               afterwards; allocations beyond it return RHD_ERR_OOM (a test hook for the
 *                               out-of-memory paths)
 * Every API call is also marked as an NVTX range of the same name for Nsight tools. */
typedef enum { RHD_BC_PERIODIC = 0, RHD_BC_OUTFLOW = 1, RHD_BC_REFLECT = 2, RHD_BC_DIRICHLET = 3 } rhd_bc;

/* Energy-exchange treatment (Section 3.4):
 *   FULL        implicit quartic theta scheme for e and E (Eqs. source:energyupdate - source:eradupdate),
 *               once per subcycle after the corrector; updates T
 *   ABSORB      absorption only, E <- E [1-(1-theta)x]/[1+theta x], x = chat kP dt (Eq.
 *               source:stiff:radenergy:soln), in both stages
 *   EQUILIBRIUM radiative equilibrium: no exchange term
 *   FROZEN_T    absorption and emission against the fixed gas temperature,
 *               E <- [E(1-(1-theta)x) + x a_R T^4]/[1+theta x], in both stages
 *   LINEAR      the Pomraning material of the Marshak wave (Section 4.1.4, c_v = alpha T^3): v = a_R T^4
 *               and E relax by Eqs. marshak:update (linear_eps = 4 a_R / alpha), once per subcycle after
 *               the corrector; updates T.  Runs in the fused kernels (split grids and ensembles with it
 *               use them) */
typedef enum { RHD_EX_FULL = 0, RHD_EX_ABSORB = 1, RHD_EX_EQUILIBRIUM = 2, RHD_EX_FROZEN_T = 3, RHD_EX_LINEAR = 4 } rhd_exchange;
typedef enum { RHD_LIM_MINMOD = 0, RHD_LIM_MC = 1, RHD_LIM_NONE = 2 } rhd_limiter;
typedef enum { RHD_CLOSURE_M1 = 0, RHD_CLOSURE_P1 = 1 } rhd_closure;     /* P1: T = I/3 (Section 2.3) */
typedef enum { RHD_SPEEDS_M1 = 0, RHD_SPEEDS_FIXED = 1 } rhd_speeds;     /* FIXED: -+chat/sqrt(3) */
/* FP64: every step in FP64.
 * SPLIT: reconstruction, closure, wave speeds, HLL fluxes, the flux divergence and the explicit O(beta
 * tau) and emissivity sources in FP32, giving an FP32 increment of each cell's state; the predictor's
 * half-step state U^{m+1/2} is FP32.  The state (E, G and T) is FP64 and accumulates that increment in
 * FP64.  The corrector's stiff sources (the theta updates of F and E and the FULL energy exchange) act
 * on the FP64 state at FP64 accuracy: double-float arithmetic (about 48 bits) seeded by an FP32 Newton
 * iteration, their results added to the FP64 state in FP64; their error is a few 2^-48 of the state
 * and does not grow with the ratio of gas to radiation energy.  The gas inputs enter as FP32 copies
 * (rho, v, kP, kF, j; the opacity law is evaluated at the FP32 density).  E_floor must be at least the
 * smallest normal FP32 number (1.2e-38) on SPLIT grids. */
typedef enum { RHD_FP64 = 0, RHD_SPLIT = 1 } rhd_precision;
/* RHD_FLAG_NO_GRAPH: issue the n_sub launches one by one instead of replaying a captured CUDA graph. */
#define RHD_FLAG_NO_GRAPH 1
/* RHD_FLAG_SPLIT_FUSED: for RHD_SPLIT grids (and ensembles) with three active directions, run each
 * subcycle as one fused kernel (predictor recomputed on the tile halo) instead of the default
 * predictor + corrector pair, which keeps U^{m+1/2} in an extra FP32 buffer of 16 bytes per cell of the
 * grid with two ghost layers in each direction that is not periodic on both faces.  Ignored
 * elsewhere. */
#define RHD_FLAG_SPLIT_FUSED 2
/* RHD_FLAG_AUTOTUNE: the first rhd_radiation_subcycle / rhd_ensemble_subcycle call runs the
 * autotuner (rhd_autotune / rhd_ensemble_autotune, 3 timed subcycles per candidate) on the state
 * then loaded, unless a context of the same shape and mode was tuned before in this process, whose
 * choice is reused. */
#define RHD_FLAG_AUTOTUNE 4
/* RHD_FLAG_EXCHANGE_ON_GAS_STEP: the paper's placement of the stiff energy exchange (Section 3.1 step 2,
 * Section 3.4: S_i integrated once per gas step): with exchange = RHD_EX_FULL the subcycles carry no
 * exchange term and rhd_gas_exchange integrates it over Delta t_gas before the gas step.  Single grids
 * only; requires RHD_EX_FULL. */
#define RHD_FLAG_EXCHANGE_ON_GAS_STEP 8

typedef struct {
    int n[3];                   /* nx, ny, nz */
    double dx[3];               /* uniform spacing per direction (ignored when inactive) */
    int bc_lo[3], bc_hi[3];     /* rhd_bc per face */
    double c;                   /* true speed of light: source terms and f = |F|/(cE) */
    double a_rad;               /* radiation constant a_R */
    double gamma;               /* adiabatic index, e = P/(gamma-1) */
    double mu_over_kB;          /* mean particle mass over k_B: P = rho T / mu_over_kB */
    double theta_F, theta_E;    /* theta of the F absorption and of the E exchange, in (0, 1] */
    double E_floor;             /* E is kept >= E_floor; a normal number: >= DBL_MIN, and >= FLT_MIN on SPLIT grids
                                   (RHD_ERR_ARG otherwise) */
    double cfl;                 /* Courant number K0 of Eq. (algorithm:radtimestep), (0, 1] */
    int exchange;               /* rhd_exchange */
    int beta_tau;               /* 1: include the O(beta tau) source terms (Section 3.4 code switch) */
    int limiter;                /* rhd_limiter */
    int closure;                /* rhd_closure */
    int speeds;                 /* rhd_speeds */
    int precision;              /* rhd_precision */
    int flags;                  /* RHD_FLAG_* bits */
    int z_chunk;                /* z planes per CTA of the fused kernel; 0 chooses automatically */
    double kappa_P, kappa_F;    /* opacity law used where kP / kF arrays are not given: */
    int kappa_rho_pow;          /*   k = kappa * rho^p, p in {0, 1, 2} (absorption coefficients) */
    void* cuda_stream;          /* cudaStream_t to run on (NULL: legacy default stream, see above) */
    double linear_eps;          /* RHD_EX_LINEAR only: retardation eps = 4 a_R / alpha (> 0) of the Pomraning
                                   material c_v = alpha T^3 (Section 4.1.4); v = a_R T^4 and E relax by
                                   Eqs. marshak:update, with chat in the radiation rows (T is updated) */
} rhd_grid_desc;

typedef struct {
    int64_t n_subcycles;         /* subcycles run since the last reset */
    int64_t n_realizability_fix; /* cells rescaled onto |F| = cE (both stages, interior cells) */
    int64_t n_face_fallback;     /* (cell, direction) pairs whose limited slope was zeroed */
    int64_t n_theta_fallback;    /* energy-exchange solves redone with theta = 1 (no feasible root) */
    int64_t n_newton_fallback;   /* energy-exchange solves finished by bisection (FP64 path) or by FP64
                                    Newton steps (split path) */
    int64_t n_nonfinite;         /* interior cells that produced a non-finite value (split grids: also a
                                    state beyond the FP32 range of their transport) */
    int32_t newton_iter_max;     /* largest Newton iteration count of one solve (split path: the FP32
                                    iterations plus the double-float step) */
    int32_t wait_timeouts;       /* bounded device-side waits that ran out; nonzero makes rhd_get_stats
                                    return RHD_ERR_TIMEOUT (the affected tiles were not updated) */
    double sum_E;                /* sum of E over the interior (current state), FP64, fixed order */
    double sum_F[3];             /* sums of Fx, Fy, Fz */
    double max_f;                /* max |F|/(cE) */
    int64_t bounds_violations;   /* debug build (librhd_debug.so, rhd_bounds_checked() = 1): array indices
                                    found out of range by the kernels' checks since the last reset (each
                                    access was redirected to element 0); nonzero makes rhd_get_stats
                                    return RHD_ERR_BOUNDS.  The counter is per process (shared by all
                                    contexts; rhd_reset_stats of any context clears it).  Always 0 in
                                    the release build. */
    int64_t gas_energy_floors;   /* gas step: cells whose internal energy went negative and was set to 0 */
    int64_t gas_nonfinite;       /* gas step: interior cells with a non-finite result (nonzero makes
                                    rhd_get_stats return RHD_ERR_NONFINITE) */
} rhd_stats;

/* Create a context for one grid (Section 3.1).  Validates d, allocates the device state and makes
 * the stream current.  *out is set only on success.  Errors: RHD_ERR_ARG, RHD_ERR_OOM, RHD_ERR_CUDA. */
rhd_status rhd_init_grid(rhd_ctx** out, const rhd_grid_desc* d);

/* Set the frozen gas state of the subcycles (Section 3.4: rho, T and v are held fixed; T changes only
 * through the FULL exchange).  rho and T are required; vx, vy, vz NULL mean 0; kP, kF NULL mean the
 * opacity law of the descriptor; j (emissivity, energy per volume per time, entering as chat j / c in
 * the E row, cf. Eq. radshell:sourceprofile) NULL means 0.  Errors: RHD_ERR_ARG, RHD_ERR_CUDA. */
rhd_status rhd_set_gas_state(rhd_ctx* ctx, const double* rho, const double* T, const double* vx,
                             const double* vy, const double* vz, const double* kP, const double* kF,
                             const double* j, int on_device);

/* Set the radiation moments E, Fx, Fy, Fz (Eq. mixedframe:radmoments).  Errors: RHD_ERR_ARG, RHD_ERR_CUDA. */
rhd_status rhd_set_moments(rhd_ctx* ctx, const double* E, const double* Fx, const double* Fy,
                           const double* Fz, int on_device);

/* Fixed radiation state (E, Fx, Fy, Fz) seen through a Dirichlet face; face = 2*dir + (0 low, 1 high). */
rhd_status rhd_set_dirichlet(rhd_ctx* ctx, int face, const double state[4]);

/* Run n_sub >= 0 radiation subcycles of length dt with reduced speed of light chat (Section 3.1 steps
 * 4-5).  Requires chat <= c and dt <= cfl * min(dx) / chat (RHD_ERR_CFL otherwise).  The loop is
 * replayed from a cached CUDA graph of n_sub kernel launches on the context stream; the call returns
 * without synchronising.  Errors: RHD_ERR_ARG, RHD_ERR_STATE (moments or gas not set), RHD_ERR_CFL,
 * RHD_ERR_CUDA. */
rhd_status rhd_radiation_subcycle(rhd_ctx* ctx, int n_sub, double chat, double dt);

/* Gas step of Section 3.1 step 3 (Section 3.4): advance (rho, rho v, E_gas) of the Euler equations over
 * dt_gas >= 0 with the explicit gas sources S_e,gas of Eq. (algorithm:source:explicit:gas) without gravity,
 *     rho v:  k_F (G - (4/3) (v/c) E),   E_gas:  -k_F v . G        (G = F/c, k_F = rho kappa_0;
 * the terms with v are the O(beta tau) terms, included when beta_tau = 1), by one van Leer predictor /
 * corrector step: a first-order half step whose sources use the gas and the radiation at t^n, then a
 * second-order full step (piecewise-linear primitives with the grid's limiter, HLLC fluxes) whose
 * sources use the gas at t^{n+1/2} and the radiation still at t^n.  k_F is the kF array if one was
 * given, else kappa_F rho^kappa_rho_pow.  P = rho T / mu_over_kB, E_gas = P/(gamma-1) + rho v^2/2; the
 * gas state (rho, v, T) is updated in place on the device and velocity components never given become
 * arrays (starting at zero).  Ghost cells follow the grid's boundary conditions (a Dirichlet face
 * takes the nearest cell for the gas).  A negative internal energy is set to zero (counted in
 * rhd_stats.gas_energy_floors).  The step leaves a source correction pending: run the radiation
 * subcycles that span dt_gas, then rhd_gas_correct.  The energy exchange stays in the subcycles unless
 * the grid has RHD_FLAG_EXCHANGE_ON_GAS_STEP (then rhd_gas_exchange runs it once, before this step).
 * RHD_SPLIT grids compute the face fluxes (reconstruction, wave speeds, HLLC), their differences, the
 * sources, the half step and the increments of (rho, v, T) in FP32 and add the increments to the FP64
 * state in FP64 (rhd_gas_correct likewise).  Does not synchronise.  Scratch, allocated by the first
 * call, for n cells and m = (n0+4)(n1+4)(n2+4) (2D / 1D: no padding in inactive directions): 8 n
 * doubles; 5 m doubles and 15 m face doubles (FP64 grids) or 5 m floats and 15 m face floats
 * (RHD_SPLIT grids).  Single grids only.  Errors: RHD_ERR_ARG (dt_gas), RHD_ERR_STATE
 * (ensemble, gas or moments not set), RHD_ERR_OOM, RHD_ERR_CUDA. */
rhd_status rhd_gas_step(rhd_ctx* ctx, double dt_gas);

/* Section 3.1 step 6: correct the gas sources of the pending gas step to second order with the current
 * radiation state U_rad^{n+1}: rho v and E_gas change by
 *     dt_gas/2 [S_e,gas(U_gas^{n+1/2}, U_rad^{n+1}) - S_e,gas(U_gas^{n+1/2}, U_rad^n)]
 * (Section 3.4), where U_gas^{n+1/2} and U_rad^n are those the step used.  Does not synchronise.
 * Errors: RHD_ERR_STATE (no pending step, ensemble), RHD_ERR_CUDA. */
rhd_status rhd_gas_correct(rhd_ctx* ctx);

/* Section 3.1 step 2 with the paper's placement of the stiff exchange S_i (Eq. algorithm:source:implicit):
 * integrate the gas-radiation energy exchange once over dt_gas, before the gas step, in every cell: E
 * floored at E_floor, then the FULL quartic theta scheme of the subcycles (Eqs. source:energyupdate -
 * source:polynomial, updating E and T, with the grid's theta_E, a_rad, gamma, mu_over_kB and kP) over
 * dt_gas with this chat, then |F| <= c E by rescaling F.  FP64 on every grid (it runs once per gas step).
 * The grid must have exchange = RHD_EX_FULL and RHD_FLAG_EXCHANGE_ON_GAS_STEP, whose subcycles then
 * carry no exchange term.  Counts theta fallbacks, Newton fallbacks, flux rescalings and non-finite
 * cells in rhd_stats.  Does not synchronise.  Errors: RHD_ERR_ARG (dt_gas < 0 or not finite, chat not in
 * (0, c]), RHD_ERR_STATE (the flag is not set, ensemble, gas or moments not set), RHD_ERR_CUDA. */
rhd_status rhd_gas_exchange(rhd_ctx* ctx, double dt_gas, double chat);

/* Copy the gas state out: rho, vx, vy, vz, T (any may be NULL to skip it; an absent velocity component
 * reads as zero).  Layout as rhd_set_gas_state.  Synchronises the stream.  Errors: RHD_ERR_ARG,
 * RHD_ERR_STATE (gas not set, ensemble), RHD_ERR_CUDA. */
rhd_status rhd_get_gas(rhd_ctx* ctx, double* rho, double* vx, double* vy, double* vz, double* T, int on_device);

/* Copy the current moments out (synchronises the stream).  Errors: RHD_ERR_ARG, RHD_ERR_STATE, RHD_ERR_CUDA. */
rhd_status rhd_get_moments(rhd_ctx* ctx, double* E, double* Fx, double* Fy, double* Fz, int on_device);

/* The radiation state in the variables the solver advances, E and G = F / c (the radiation rows of
 * Eq. algorithm:variables with the momentum rows divided by c), copied without arithmetic: a state
 * saved with rhd_get_conserved and given back with rhd_set_conserved continues bit for bit (the
 * F = c G conversion of rhd_get/set_moments rounds).  Same layout, ownership and synchronisation as
 * rhd_set_moments / rhd_get_moments.  Errors: RHD_ERR_ARG, RHD_ERR_STATE (get before any set, or an
 * ensemble context), RHD_ERR_CUDA. */
rhd_status rhd_set_conserved(rhd_ctx* ctx, const double* E, const double* Gx, const double* Gy,
                             const double* Gz, int on_device);
rhd_status rhd_get_conserved(rhd_ctx* ctx, double* E, double* Gx, double* Gy, double* Gz, int on_device);

/* Copy the current gas temperature out (changes only in FULL mode).  Synchronises the stream. */
rhd_status rhd_get_gas_state(rhd_ctx* ctx, double* T, int on_device);

/* Counters accumulated since the last reset plus sums over the current state (synchronises). */
rhd_status rhd_get_stats(rhd_ctx* ctx, rhd_stats* out);
rhd_status rhd_reset_stats(rhd_ctx* ctx);

/* Block until the context stream is idle, or give up after timeout_ms (RHD_ERR_TIMEOUT; the work keeps
 * running and the context stays usable).  timeout_ms < 0 waits without limit. */
rhd_status rhd_synchronize(rhd_ctx* ctx, int timeout_ms);

/* Message of the last failure of this context (or of rhd_init_grid when ctx is NULL); never NULL. */
const char* rhd_last_error(const rhd_ctx* ctx);

/* Release the context and its device buffers.  NULL is accepted. */
rhd_status rhd_destroy(rhd_ctx* ctx);

/* ---------------------------------------------------------------------------------------------
 * Batched ensemble: many independent grids of uneven sizes advanced together.  Each subcycle is one
 * persistent launch whose CTAs pull (grid, tile) work items from a global counter; n_sub launches are
 * replayed from one CUDA graph.  Grids never exchange data.  All grids share precision, exchange mode,
 * limiter, closure and speeds (taken from descs[0]); sizes, spacing, boundaries, physics constants
 * and opacity laws are per grid.
 * ------------------------------------------------------------------------------------------- */
rhd_status rhd_ensemble_create(rhd_ctx** out, int n_grids, const rhd_grid_desc* descs);
/* Per-grid state setters/getters of an ensemble context (grid in [0, n_grids)). */
rhd_status rhd_ensemble_set_gas_state(rhd_ctx* ctx, int grid, const double* rho, const double* T,
                                      const double* vx, const double* vy, const double* vz,
                                      const double* kP, const double* kF, const double* j, int on_device);
rhd_status rhd_ensemble_set_moments(rhd_ctx* ctx, int grid, const double* E, const double* Fx,
                                    const double* Fy, const double* Fz, int on_device);
rhd_status rhd_ensemble_get_moments(rhd_ctx* ctx, int grid, double* E, double* Fx, double* Fy,
                                    double* Fz, int on_device);
rhd_status rhd_ensemble_get_gas_state(rhd_ctx* ctx, int grid, double* T, int on_device);
/* n_sub subcycles of every grid, grid g with its own dt_per_grid[g] (host array), common chat. */
rhd_status rhd_ensemble_subcycle(rhd_ctx* ctx, int n_sub, double chat, const double* dt_per_grid);

/* ---------------------------------------------------------------------------------------------
 * Launch configuration and autotuner.  The paper has no counterpart (its code runs on CPUs); these
 * pick how the subcycle kernels are laid out on the GPU, never what they compute: every candidate
 * gives results within the error bound of its precision.
 *   variant   RHD_VARIANT_FUSED: one kernel per subcycle; the predictor (U^{m+1/2}) is recomputed
 *             on the 2-cell halo of each x-y tile.  RHD_VARIANT_TWOPASS (RHD_SPLIT, 3D grids only):
 *             a predictor kernel writes U^{m+1/2} (FP32) for the grid plus 2 ghost layers per face
 *             in each direction that is not periodic on both faces, then a corrector kernel reads
 *             it back; extra device memory (n0+p0)(n1+p1)(n2+p2) x 16 bytes, p = 0 for a direction
 *             periodic on both faces, else 4.
 *   tile_x, tile_y   cells per CTA tile in x and y (the supported shapes are those the tuner lists)
 *   z_chunk   planes per CTA along z (each CTA marches its tile through a chunk of planes)
 *   staging   RHD_STAGING_CPASYNC: the tile and its halo are staged into shared memory with per-
 *             thread asynchronous copies.  RHD_STAGING_TMA (two-pass corrector): the tile + 2-cell
 *             halo of U^{m+1/2} is fetched with one tensor-memory-accelerator copy per plane.
 * ------------------------------------------------------------------------------------------- */
#define RHD_VARIANT_FUSED 0
#define RHD_VARIANT_TWOPASS 1
#define RHD_STAGING_CPASYNC 0
#define RHD_STAGING_TMA 1
typedef struct {
    int variant, tile_x, tile_y, z_chunk, staging;
    double ms_per_subcycle;     /* rhd_autotune: measured mean time per subcycle; < 0: candidate failed */
} rhd_launch_config;

/* Time every candidate configuration of a single-grid context on its current state (moments and
 * gas must be set; chat and dt as for rhd_radiation_subcycle) with reps >= 1 timed subcycles each
 * (plain launches, after one warm-up), then keep the fastest.  The grid's state (E, F, T) and the
 * statistics are left exactly as they were; captured graphs are dropped.  table (may be NULL)
 * receives up to capacity entries, *n_entries (may be NULL) the number of candidates, *chosen (may
 * be NULL) the configuration kept.  Synchronises the context's stream.  Errors: RHD_ERR_ARG,
 * RHD_ERR_STATE (state not set, or an ensemble context), RHD_ERR_OOM / RHD_ERR_CUDA. */
rhd_status rhd_autotune(rhd_ctx* ctx, double chat, double dt, int reps, rhd_launch_config* table, int capacity,
                        int* n_entries, rhd_launch_config* chosen);
/* The same for an ensemble context: candidates are the z_chunk values shared by all grids. */
rhd_status rhd_ensemble_autotune(rhd_ctx* ctx, double chat, const double* dt_per_grid, int reps,
                                 rhd_launch_config* table, int capacity, int* n_entries,
                                 rhd_launch_config* chosen);
/* Read the configuration in use (ms_per_subcycle is that of the last tuning, or -1). */
rhd_status rhd_get_launch_config(rhd_ctx* ctx, rhd_launch_config* out);
/* Select a configuration explicitly (single-grid contexts); RHD_ERR_ARG if it is not supported for
 * this grid's precision and dimension.  Drops captured graphs. */
rhd_status rhd_set_launch_config(rhd_ctx* ctx, const rhd_launch_config* cfg);

/* Poll limit of the waits on the TMA staging of the two-pass corrector (each plane's tensor copy is
 * awaited on an mbarrier by at most `polls` try-wait polls): polls < 0 restores the default (2^22 polls,
 * far beyond a copy's time), 0 makes every such wait give up at once.  For tests of the timeout path
 * (failure detection without a GPU fault): a tile whose wait gives up abandons its work (its cells keep
 * no new values), its one copy in flight is still awaited with the default bound before the block exits,
 * and rhd_get_stats reports RHD_ERR_TIMEOUT with rhd_stats.wait_timeouts.  Applies to later calls (the
 * context's captured graphs are dropped).  No paper counterpart.  Errors: RHD_ERR_ARG. */
rhd_status rhd_set_wait_limit(rhd_ctx* ctx, long long polls);

/* ---------------------------------------------------------------------------------------------
 * Kernel timer.  While enabled, subcycles are issued as plain launches (no graph) with a CUDA event
 * recorded on the context's stream before and after every kernel.  rhd_get_kernel_times
 * synchronises the stream and returns, per kernel, the launches and their summed event-measured
 * duration since the timer was enabled or last read (then starts a new interval), and the
 * algorithmic bytes of one launch: every input array read once and every output written once
 * (U^m and U^{m+1} 32 B/cell in FP64, U^{m+1/2} 16 B/cell in FP32, gas arrays 4 B (split) or 8 B
 * (FP64) each, T 8 B read and / or written as the exchange mode needs).
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    char name[48];              /* e.g. "twopass_corrector_split" */
    int64_t launches;
    double total_ms;
    double alg_bytes_per_launch;
} rhd_kernel_time;
rhd_status rhd_set_kernel_timing(rhd_ctx* ctx, int enable);
rhd_status rhd_get_kernel_times(rhd_ctx* ctx, rhd_kernel_time* out, int capacity, int* n_entries);

/* ---------------------------------------------------------------------------------------------
 * Subcycles without device allocation.  The paper has no counterpart: this is an interface for
 * callers that cannot call cudaMalloc, for example code running while another component owns the
 * device memory through its own pool allocator, or an application that must keep the device
 * footprint fixed once the library is loaded.  It runs n_sub FP64 subcycles exactly as
 * rhd_radiation_subcycle does, reading and writing only the caller's DEVICE arrays (interior cells,
 * x fastest) plus one static scratch array that librhd.so reserves on every GPU that loads it, held
 * until the process exits: 32 MiB for the working state, so grids of at most RHD_NOALLOC_MAX_CELLS
 * cells (larger grids return RHD_ERR_ARG).  It calls no cudaMalloc, cudaFree or allocating routine.
 *   d         grid descriptor; precision must be RHD_FP64; d->cuda_stream is the stream used (NULL:
 *             legacy default stream); the call synchronises that stream before it returns (it reads
 *             the call's event counters back, so that non-finite results are always reported)
 *   dirichlet 6 x 4 values (E, Fx, Fy, Fz) for faces 2*dir + side, or NULL (zeros)
 *   E..Fz     input moments; rho, T required; vx, vy, vz, kP, kF, j may be NULL (as in
 *             rhd_set_gas_state)
 *   *_out     output moments and gas temperature (may equal the inputs: the inputs are read first)
 *   stats     NULL, or counters of this call (sums are not computed)
 * The first call on a device looks up the scratch address on that device (make it before any stream
 * capture).  The scratch is shared by all calls and keeps the last call's contents; each call resets
 * what must start at zero.  Calls whose work overlaps on the GPU (other streams or threads) race on
 * the scratch and must be serialised by the caller.  Errors: RHD_ERR_ARG, RHD_ERR_CFL, RHD_ERR_CUDA,
 * RHD_ERR_NONFINITE (non-finite results, with or without stats); the message is in
 * rhd_last_error(NULL). */
#define RHD_NOALLOC_MAX_CELLS 1048576
rhd_status rhd_subcycle_noalloc(const rhd_grid_desc* d, const double dirichlet[24], int n_sub, double chat,
                                double dt, const double* E, const double* Fx, const double* Fy, const double* Fz,
                                const double* rho, const double* T, const double* vx, const double* vy,
                                const double* vz, const double* kP, const double* kF, const double* j,
                                double* E_out, double* Fx_out, double* Fy_out, double* Fz_out, double* T_out,
                                rhd_stats* stats);

/* ---------------------------------------------------------------------------------------------
 * Reduced-speed-of-light helpers (Sections 3.1 and 3.2): the signal speeds and time steps around the
 * subcycle loop.  The two grid maxima run as reductions on the context's stream and synchronise it;
 * single-grid contexts only (RHD_ERR_STATE on an ensemble).
 * --------------------------------------------------------------------------------------------- */

/* v_max = max over cells of |v| + c_eff, with the effective sound speed of Eq. algorithm:ceff
 * c_eff = sqrt((gamma P + (4/9) E (1 - exp(-k_F dx))) / rho), P = rho T / mu_over_kB, from the frozen
 * gas state (current T) and the current E; k_F is the per-cell flux-mean absorption coefficient (the
 * kF array, else the opacity law) and dx the smallest active spacing.  Errors: RHD_ERR_ARG,
 * RHD_ERR_STATE (gas or moments not set), RHD_ERR_NONFINITE (*v_max is then NaN or inf), RHD_ERR_OOM,
 * RHD_ERR_CUDA. */
rhd_status rhd_max_signal_speed(rhd_ctx* ctx, double* v_max);

/* tau_max = the largest optical depth sum(k_F dx_d) along any grid line parallel to an active axis:
 * the domain's optical depth along the axes, the tau_max of Eq. rsla:diffcrit measured on the grid.
 * Errors as rhd_max_signal_speed (only the gas state is required). */
rhd_status rhd_max_optical_depth(rhd_ctx* ctx, double* tau_max);

/* chat from the RSLA static-diffusion criterion (Eq. rsla:staticdiffreq), "much greater than" taken
 * as the factor ratio (the paper uses R ~ 10 to 100): chat = min(c, ratio v_max max(1, tau_max)), i.e.
 * chat = c where c is not far above the gas speeds (Section 3.1).  Pure host arithmetic.  Errors:
 * RHD_ERR_ARG (c, v_max, ratio not positive and finite, tau_max negative or not finite, NULL chat). */
rhd_status rhd_suggest_chat(double c, double v_max, double tau_max, double ratio, double* chat);

/* Time steps of one gas cycle: dt_gas = cfl dx_min / v_max (Eq. algorithm:gastimestep) and the
 * radiation subcycles that span it (Eq. algorithm:radtimestep, "about R" of them, Section 3.1 step 5):
 * n_sub = the smallest n with dt_gas / n <= cfl dx_min / chat, dt_rad = dt_gas / n_sub, so that
 * n_sub subcycles end exactly at t + dt_gas and dt_rad passes rhd_radiation_subcycle's CFL check.  Pure
 * host arithmetic.  Errors: RHD_ERR_ARG (non-positive or non-finite input, NULL output, more than
 * 2^31 - 1 subcycles). */
rhd_status rhd_time_steps(double cfl, double dx_min, double v_max, double chat, double* dt_gas, double* dt_rad,
                          int* n_sub);

/* The radiation subcycles that span a given gas step dt_gas (Eq. algorithm:radtimestep, as in
 * rhd_time_steps but with dt_gas chosen by the caller): n_sub = the smallest n with
 * dt_gas / n <= cfl dx_min / chat, dt_rad = dt_gas / n_sub.  Pure host arithmetic.  Errors: RHD_ERR_ARG
 * (non-positive or non-finite input, NULL output, more than 2^31 - 1 subcycles). */
rhd_status rhd_subcycle_steps(double cfl, double dx_min, double chat, double dt_gas, double* dt_rad, int* n_sub);

/* 1 for the debug library librhd_debug.so, whose kernels check every global-memory index and the
 * shared-memory indices of the two-pass kernels against their arrays' extents (a substitute for a
 * memory checker: an out-of-range index is counted and redirected to element 0, no trap), else 0. */
int rhd_bounds_checked(void);

/* Left-boundary state of the non-equilibrium Marshak wave (Section 4.1.4): E(0, t) from the Su & Olson
 * surface value u(0, tau) of Eq. marshak:suolson at chi = 0 (integrals by the midpoint rule with n_quad
 * points, as in the paper), F(0, t) from c E + 2 F = 4 F_inc (Eq. marshak:bc_ix1); tau = eps c rho kappa_0 t.
 * state = (E, F, 0, 0), the Dirichlet state of the low x face (rhd_set_dirichlet face 0) for the
 * subcycles starting at t.  Pure host arithmetic.  Errors: RHD_ERR_ARG (tau < 0, eps <= 0, F_inc < 0,
 * c <= 0, n_quad < 1, non-finite input, NULL state). */
rhd_status rhd_marshak_boundary(double tau, double eps, double F_inc, double c, int n_quad, double state[4]);

/* n_sub subcycles of the Marshak wave from time t0, the low x face's Dirichlet state of subcycle m
 * computed on the device by the same quadrature as rhd_marshak_boundary at tau = tau_rate (t0 + (m + 1/2) dt)
 * (the subcycle's midpoint; tau_rate = eps c rho kappa_0): one launch computes all n_sub states (one block
 * each, kept in a context buffer of 32 n_sub bytes), then one plain launch per subcycle reads its own.  Needs a single-grid context with
 * a Dirichlet low x face, state set, and the fused kernels (FP64, or split with RHD_FLAG_SPLIT_FUSED or
 * fewer than 3 dimensions).  Returns without synchronising.  Errors: RHD_ERR_ARG, RHD_ERR_CFL,
 * RHD_ERR_STATE, RHD_ERR_UNSUPPORTED (two-pass split grid), RHD_ERR_OOM, RHD_ERR_CUDA. */
rhd_status rhd_marshak_advance(rhd_ctx* ctx, int n_sub, double chat, double dt, double t0, double tau_rate,
                               double eps, double F_inc, int n_quad);

/* Library identification: ABI version and the compute capability it was built for (e.g. 103). */
int rhd_abi_version(void);
int rhd_built_arch(void);

#ifdef __cplusplus
}
#endif
#endif /* RHD_H */
