/*
 * rhd_oracle.h -- plain, slow FP64 CPU oracle for one subcycle of the gray
 * M1 radiation update under the reduced speed of light approximation
 * (Skinner & Ostriker 2013, Sections 2.3, 3.1, 3.3, 3.4).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this code; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no header, helper or constant with the CUDA
 * path.
 *
 * Conventions (all arrays interior cells only, x fastest: idx = i + nx*(j + ny*k)):
 *   - the radiation state is (E, Fx, Fy, Fz); internally G = F/c is evolved,
 *     so the hyperbolic flux in direction d is chat*(G_d, E*T_dx, E*T_dy, E*T_dz);
 *   - a direction with n_d == 1 is inactive (no transport, no ghost cells);
 *   - absorption coefficients k = rho*kappa are given per cell (kP, kF) or, if
 *     the array is NULL, by the law k = kappa * rho^p with p in {0,1,2}.
 */
#ifndef RHD_ORACLE_H
#define RHD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_OUTFLOW = 1, ORC_BC_REFLECT = 2, ORC_BC_DIRICHLET = 3 };
enum { ORC_EX_FULL = 0, ORC_EX_ABSORB = 1, ORC_EX_EQUILIBRIUM = 2, ORC_EX_FROZEN_T = 3, ORC_EX_LINEAR = 4 };
enum { ORC_LIM_MINMOD = 0, ORC_LIM_MC = 1, ORC_LIM_NONE = 2 };
enum { ORC_CLOSURE_M1 = 0, ORC_CLOSURE_P1 = 1 };
enum { ORC_SPEEDS_M1 = 0, ORC_SPEEDS_FIXED = 1 };

typedef struct {
    int n[3];
    double dx[3];
    int bc_lo[3], bc_hi[3];
    double dirichlet_lo[3][4];   /* (E, Fx, Fy, Fz) held in the ghost cells of a Dirichlet face */
    double dirichlet_hi[3][4];
    double c, a_rad, gamma, mu_over_kB;
    double theta_F, theta_E, E_floor;
    int exchange, beta_tau, limiter, closure, speeds;
    double kappa_P, kappa_F;     /* opacity law used where kP / kF is NULL */
    int kappa_rho_pow;           /* 0, 1 or 2 */
    double linear_eps;           /* ORC_EX_LINEAR: retardation eps = 4 a_R / alpha of c_v = alpha T^3 */
} orc_params;

typedef struct {
    long long n_realizability_fix;   /* cells with |G| > E rescaled (both stages) */
    long long n_face_fallback;       /* (cell, direction) pairs whose PLM slope was zeroed */
    long long n_theta_fallback;      /* quartic solves redone with theta = 1 (c0 > 0) */
    long long n_nonfinite;           /* interior cells with a non-finite result */
    double boundary_E_out;           /* sum over outer faces of dt * area * (energy flux out) */
} orc_stats;

/* M1 Eddington factor chi(f), Eq. (m1:chi). */
double orc_chi(double f);

/* Eddington tensor T (row-major 3x3) of the state (E, G), Eqs. (m1:m1tns), (m1:nhat), (m1:chi).
 * closure = ORC_CLOSURE_M1 or ORC_CLOSURE_P1 (T = I/3). */
void orc_eddington_tensor(double E, const double G[3], int closure, double T[9]);

/* Hyperbolic flux in direction d of the state U = (E, Gx, Gy, Gz): chat*(G_d, E*T_d.). */
void orc_flux(const double U[4], int d, double chat, int closure, double out[4]);

/* Extreme wave speeds lambda_1 (min) and lambda_3 (max) in direction d, Eq. (hyperbolic:evals13),
 * or -+chat/sqrt(3) when speeds = ORC_SPEEDS_FIXED. */
void orc_wave_speeds(const double U[4], int d, double chat, int speeds, double* l1, double* l3);

/* HLL interface flux, Eq. (hyperbolic:hllflux2), with S_R, S_L as defined below it. */
void orc_hll(const double UL[4], const double UR[4], int d, double chat, int closure, int speeds,
             double out[4]);

/* theta-scheme factor [1 - (1-theta) x] / [1 + theta x], Eqs. (source:stiff:radmomentum:soln),
 * (source:stiff:radenergy:soln). */
double orc_theta_factor(double theta, double x);
/* Limited slope from the left and right differences dl = U_i - U_{i-1}, dr = U_{i+1} - U_i: lim =
 * ORC_LIM_MINMOD, ORC_LIM_MC (monotonized central) or ORC_LIM_NONE ((dl + dr)/2). */
double orc_limited_slope(double dl, double dr, int lim);

/* Root in [0, b] of c4 x^4 + c1 x + c0 (c0 <= 0) by bisection to adjacent doubles,
 * b = min(|c0/c1|, |c0/c4|^(1/4)), Section 3.4. */
double orc_quartic_root(double c4, double c1, double c0);

/* One implicit gas-radiation energy exchange (Eqs. source:energyupdate .. source:polynomial) of
 * a single cell over dt.  Updates *E and *T in place.  Returns 1 if the theta = 1 fallback was used. */
int orc_exchange_full(const orc_params* p, double chat, double dt, double rho, double kP,
                      double* E, double* T);

/* Linear exchange of the Pomraning material (Section 4.1.4: c_v = alpha T^3, so v = a_R T^4 is
 * linear in the internal energy) of a single cell over dt, Eqs. (marshak:update) with chat in place
 * of c in the radiation rows (reading): updates *E and *T in place. */
void orc_exchange_linear(const orc_params* p, double chat, double dt, double kP, double* E, double* T);

/* n_sub subcycles of the radiation update.  E, Fx, Fy, Fz (and T in FULL mode) are read and
 * overwritten.  vx, vy, vz, kP, kF, j may be NULL (zero velocity, opacity law, no emissivity).
 * Returns 0 on success, nonzero on bad arguments.  stats may be NULL. */
int orc_subcycles(const orc_params* p, int n_sub, double chat, double dt,
                  double* E, double* Fx, double* Fy, double* Fz, double* T,
                  const double* rho, const double* vx, const double* vy, const double* vz,
                  const double* kP, const double* kF, const double* j, orc_stats* stats);

/* Same, but only the interior box [lo, hi) is advanced and written; every other cell is left
 * as it is.  Used to time a bounded sample of a large grid.  Results inside the box are those
 * of orc_subcycles for n_sub = 1. */
int orc_subcycle_box(const orc_params* p, double chat, double dt, const int lo[3], const int hi[3],
                     double* E, double* Fx, double* Fy, double* Fz, double* T,
                     const double* rho, const double* vx, const double* vy, const double* vz,
                     const double* kP, const double* kF, const double* j, orc_stats* stats);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
