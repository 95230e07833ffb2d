/*
 * rhd_oracle.c -- plain FP64 CPU oracle of the subcycled gray M1 radiation update
 * (Skinner & Ostriker 2013).  TEST INFRASTRUCTURE: only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark use it; the product library never does.
 *
 * It is written to be read against the paper, not to be fast:
 *   - whole-block arrays with explicit ghost layers of width 3, no tiling, no fusion;
 *   - the closure, the wave speeds and the HLL flux in the paper's literal forms
 *     (Eqs. m1:m1tns, m1:nhat, m1:chi, hyperbolic:evals13, hyperbolic:hllflux2);
 *   - the stages of one subcycle in the order of Section 3.1 step 4 and Section 3.4:
 *       ghost fill of U^m -> first-order HLL fluxes -> U^{m+1/2} (predictor, half step,
 *       explicit sources from U^m, direct theta updates over dt/2) -> piecewise-linear
 *       reconstruction of U^{m+1/2} -> HLL fluxes -> U^{m+1} (full step, explicit sources from
 *       U^{m+1/2}, direct theta updates over dt) -> implicit energy exchange -> realizability.
 *   - the quartic of Eq. (source:polynomial) is solved by plain bisection to adjacent doubles,
 *     not by the Newton iteration the CUDA path uses.
 * Where the paper is silent these readings are taken (each is marked "reading" below):
 *   - limiter: componentwise on (E, G); minmod, monotonized central or the unlimited central slope;
 *   - face-state realizability: a reconstructed face value with E <= 0 or |G|^2 > (1 + 1e-12) E^2
 *     zeroes that cell's slope in that direction;
 *   - split order: the predictor takes the explicit O(beta tau) and emissivity sources from U^m and
 *     the theta updates over dt/2; the corrector the explicit sources from U^{m+1/2}, the theta
 *     updates over dt, then the energy exchange once, then E >= E_floor and |G| <= E (rescaling G);
 *   - ghost rule: per direction in the order x, y, z, periodic wraps, outflow clamps, reflect mirrors
 *     (negating the normal G and v), Dirichlet returns the face state.
 *
 * Compile with -ffp-contract=off so that x86-64 and aarch64 give the same bits.
 */
#include "rhd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------
 * Closure, wave speeds, HLL flux (Sections 2.3 and 3.3)
 * ---------------------------------------------------------------------------------------- */

/* Eq. (m1:chi): chi(f) = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)). */
double orc_chi(double f)
{
    return (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
}

/* Eq. (m1:m1tns) with n = F/|F| (Eq. m1:nhat) and f = |F|/(cE) = |G|/E.  At F = 0 the direction
 * is undefined; the limit T = I/3 (chi = 1/3) is used (reading).  f is clamped to 1 (reading). */
void orc_eddington_tensor(double E, const double G[3], int closure, double T[9])
{
    int a, b;
    if (closure == ORC_CLOSURE_P1) {
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b) T[3 * a + b] = (a == b) ? 1.0 / 3.0 : 0.0;
        return;
    }
    double g = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
    double f = g / E;
    if (f > 1.0) f = 1.0;
    double chi = orc_chi(f);
    double n[3] = {0.0, 0.0, 0.0};
    if (g > 0.0) {
        n[0] = G[0] / g;
        n[1] = G[1] / g;
        n[2] = G[2] / g;
    }
    double iso = (1.0 - chi) / 2.0;
    double dir = (3.0 * chi - 1.0) / 2.0;
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) T[3 * a + b] = (a == b ? iso : 0.0) + dir * n[a] * n[b];
}

/* Radiation-subsystem flux in direction d (Eq. algorithm:variables, radiation rows, divided by c
 * in the momentum rows): chat * (G_d, E T_dx, E T_dy, E T_dz). */
void orc_flux(const double U[4], int d, double chat, int closure, double out[4])
{
    double G[3] = {U[1], U[2], U[3]};
    double T[9];
    orc_eddington_tensor(U[0], G, closure, T);
    out[0] = chat * U[1 + d];
    out[1] = chat * U[0] * T[3 * d + 0];
    out[2] = chat * U[0] * T[3 * d + 1];
    out[3] = chat * U[0] * T[3 * d + 2];
}

/* Eq. (hyperbolic:evals13): lambda_{1,3}/chat = { mu f -+ [ (2/3)(4 - 3f^2 - sqrt(4-3f^2))
 *   + 2 mu^2 (2 - f^2 - sqrt(4-3f^2)) ]^{1/2} } / sqrt(4-3f^2),  mu = x_d . n.
 * mu f is taken as 0 at F = 0 and the radicand is clamped at 0 (reading). */
void orc_wave_speeds(const double U[4], int d, double chat, int speeds, double* l1, double* l3)
{
    if (speeds == ORC_SPEEDS_FIXED) {
        *l1 = -chat / sqrt(3.0);
        *l3 = chat / sqrt(3.0);
        return;
    }
    double E = U[0];
    double g = sqrt(U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
    double f = g / E;
    if (f > 1.0) f = 1.0;
    double mu = (g > 0.0) ? U[1 + d] / g : 0.0;
    double s = sqrt(4.0 - 3.0 * f * f);
    double rad = (2.0 / 3.0) * (4.0 - 3.0 * f * f - s) + 2.0 * mu * mu * (2.0 - f * f - s);
    if (rad < 0.0) rad = 0.0;
    *l1 = chat * (mu * f - sqrt(rad)) / s;
    *l3 = chat * (mu * f + sqrt(rad)) / s;
}

/* Eq. (hyperbolic:hllflux2) with S_R = max(l3(L), l3(R)), S_L = min(l1(L), l1(R)),
 * S_R^+ = max(S_R, 0), S_L^- = min(S_L, 0).  If S_R^+ = S_L^- = 0 (both states stream exactly
 * across the interface normal) the flux is the average of the two fluxes (reading). */
void orc_hll(const double UL[4], const double UR[4], int d, double chat, int closure, int speeds,
             double out[4])
{
    double l1L, l3L, l1R, l3R, FL[4], FR[4];
    orc_wave_speeds(UL, d, chat, speeds, &l1L, &l3L);
    orc_wave_speeds(UR, d, chat, speeds, &l1R, &l3R);
    double SR = (l3L > l3R) ? l3L : l3R;
    double SL = (l1L < l1R) ? l1L : l1R;
    double SRp = (SR > 0.0) ? SR : 0.0;
    double SLm = (SL < 0.0) ? SL : 0.0;
    orc_flux(UL, d, chat, closure, FL);
    orc_flux(UR, d, chat, closure, FR);
    double den = SRp - SLm;
    int q;
    if (den <= 0.0) {
        for (q = 0; q < 4; ++q) out[q] = 0.5 * (FL[q] + FR[q]);
        return;
    }
    for (q = 0; q < 4; ++q) out[q] = (SRp * FL[q] - SLm * FR[q] + SRp * SLm * (UR[q] - UL[q])) / den;
}

/* ------------------------------------------------------------------------------------------
 * Source terms (Section 3.4)
 * ---------------------------------------------------------------------------------------- */

double orc_theta_factor(double theta, double x)
{
    return (1.0 - (1.0 - theta) * x) / (1.0 + theta * x);
}

static double quartic(double c4, double c1, double c0, double x)
{
    return c4 * x * x * x * x + c1 * x + c0;
}

/* Section 3.4: f_theta is increasing and convex on x > 0 and, for c0 <= 0, has its root in
 * [0, min(|c0/c1|, |c0/c4|^{1/4})].  Plain bisection until the bracket is two adjacent doubles;
 * the end with the smaller |f| is returned. */
double orc_quartic_root(double c4, double c1, double c0)
{
    double b = fabs(c0 / c1);
    if (c4 > 0.0) {
        double b4 = sqrt(sqrt(fabs(c0 / c4)));
        if (b4 < b) b = b4;
    }
    double lo = 0.0, hi = b;
    double flo = quartic(c4, c1, c0, lo), fhi = quartic(c4, c1, c0, hi);
    if (flo >= 0.0) return lo;
    if (fhi <= 0.0) return hi;
    int it;
    for (it = 0; it < 4000; ++it) {
        double mid = lo + 0.5 * (hi - lo);
        if (mid <= lo || mid >= hi) break;
        double fm = quartic(c4, c1, c0, mid);
        if (fm <= 0.0) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
            fhi = fm;
        }
    }
    return (fabs(flo) <= fabs(fhi)) ? lo : hi;
}

/* Eqs. (source:energyexchange) .. (source:polynomial): one theta-scheme step of the gas-radiation
 * energy exchange with rho fixed.  e = P/(gamma-1), P = rho k_B T / mu (Eq. momenteqns:perfectgas),
 * alpha = a_R [(gamma-1) mu/(rho k_B)]^4, eta = c rho kappa dt, Ebar = e + (c/chat) E is conserved
 * (Eq. source:combinedenergy), x = e^{n+1} solves c4 x^4 + c1 x + c0 = 0 and
 * E^{n+1} = (chat/c)(Ebar - x) (Eq. source:eradupdate).  If c0 > 0 (theta < 1 and stiff) there is
 * no feasible root; the step is redone with theta = 1, which guarantees c0 <= 0 (reading). */
int orc_exchange_full(const orc_params* p, double chat, double dt, double rho, double kP,
                      double* E, double* T)
{
    double c = p->c;
    double q = (p->gamma - 1.0) * p->mu_over_kB / rho;
    double e = (rho * (*T) / p->mu_over_kB) / (p->gamma - 1.0);
    double alpha = p->a_rad * (q * q) * (q * q);
    double eta = c * kP * dt;
    double Ebar = e + (c / chat) * (*E);
    double theta = p->theta_E;
    int fell_back = 0;
    double c4 = alpha * eta * theta;
    double c1 = 1.0 + (chat / c) * eta * theta;
    double c0 = (1.0 - theta) * eta * (alpha * e * e * e * e - (*E)) - (e + (chat / c) * eta * theta * Ebar);
    if (c0 > 0.0) {
        theta = 1.0;
        fell_back = 1;
        c4 = alpha * eta * theta;
        c1 = 1.0 + (chat / c) * eta * theta;
        c0 = -(e + (chat / c) * eta * theta * Ebar);
    }
    double x = orc_quartic_root(c4, c1, c0);
    *E = (chat / c) * (Ebar - x);
    *T = x * q;
    return fell_back;
}

/* ------------------------------------------------------------------------------------------
 * Grid blocks with ghost layers
 * ---------------------------------------------------------------------------------------- */

/* Eqs. (marshak:energyexchange) with c_v = alpha T^3 read in v = a_R T^4:
 *   dv/dt = -eps c kP (v - E),   dE/dt = chat kP (v - E),   eps = 4 a_R / alpha
 * (the paper writes the second row with chat = c).  Eqs. (marshak:update): with
 * dtau = eps c kP dt, the theta-scheme step of v is dv = -(v - E) dtau / (1 + theta (1 + chat/(eps c)) dtau)
 * (the paper's 1 + 1/eps at chat = c), and E changes by -(chat / (eps c)) dv, which keeps
 * v / (eps c) + E / chat fixed (the paper's du = -dv / eps).  T follows from v (reading: v is kept
 * >= 0, which theta < 1 need not do). */
void orc_exchange_linear(const orc_params* p, double chat, double dt, double kP, double* E, double* T)
{
    double eps = p->linear_eps, c = p->c, theta = p->theta_E;
    double v = p->a_rad * (*T) * (*T) * (*T) * (*T);
    double u = *E;
    double dtau = eps * c * kP * dt;
    double dv = -(v - u) * dtau / (1.0 + theta * (1.0 + chat / (eps * c)) * dtau);
    double du = -(chat / (eps * c)) * dv;
    v = v + dv;
    u = u + du;
    if (v < 0.0) v = 0.0;
    *E = u;
    *T = sqrt(sqrt(v / p->a_rad));
}

typedef struct {
    int act[3];          /* direction active (n_d > 1) */
    int g[3];            /* ghost width: 3 in active directions, 0 otherwise */
    int lo[3], hi[3];    /* owned interior box, global cell coordinates */
    int m[3];            /* padded extents */
    long stride[3];
    long size;
} block_t;

static long bidx(const block_t* b, int i, int j, int k)
{
    return (long)(i - b->lo[0] + b->g[0]) + b->stride[1] * (long)(j - b->lo[1] + b->g[1]) +
           b->stride[2] * (long)(k - b->lo[2] + b->g[2]);
}

static long gidx(const orc_params* p, const int ii[3])
{
    return (long)ii[0] + (long)p->n[0] * ((long)ii[1] + (long)p->n[1] * (long)ii[2]);
}

/* Ghost rule (reading): for each direction in the order x, y, z, a coordinate outside [0, n)
 * is mapped by that face's condition -- periodic: wrap; outflow: nearest interior cell; reflect:
 * mirror image with the normal component of G (of v for the gas) negated; Dirichlet: the face's
 * fixed state for the radiation (and the nearest interior cell for the gas).  Returns 1 if a
 * Dirichlet face decided the value (radiation only). */
static int remap(const orc_params* p, int ii[3], double sgn[3], int dirichlet_allowed, int* dface,
                 int* dside)
{
    int d;
    for (d = 0; d < 3; ++d) {
        int n = p->n[d];
        while (ii[d] < 0 || ii[d] >= n) {
            int low = ii[d] < 0;
            int bc = low ? p->bc_lo[d] : p->bc_hi[d];
            if (bc == ORC_BC_DIRICHLET && dirichlet_allowed) {
                *dface = d;
                *dside = low ? 0 : 1;
                return 1;
            }
            if (bc == ORC_BC_PERIODIC) {
                ii[d] = ((ii[d] % n) + n) % n;
            } else if (bc == ORC_BC_OUTFLOW || bc == ORC_BC_DIRICHLET) {
                ii[d] = low ? 0 : n - 1;
            } else { /* reflect */
                ii[d] = low ? (-ii[d] - 1) : (2 * n - 1 - ii[d]);
                sgn[d] = -sgn[d];
            }
        }
    }
    return 0;
}

typedef struct {
    const orc_params* p;
    double chat, dt;
    block_t b;
    /* padded block arrays */
    double* Um[4];      /* U^m = (E, Gx, Gy, Gz) */
    double* Uh[4];      /* U^{m+1/2} */
    double* Fp[3][4];   /* predictor face fluxes, face (cell - e_d | cell) stored at cell */
    double* Fc[3][4];   /* corrector face fluxes */
    double* slope[3][4];
    double *rho, *T, *v[3], *kP, *kF, *jj;
} work_t;

static double kappa_law(double kappa, int pw, double rho)
{
    if (pw == 0) return kappa;
    if (pw == 1) return kappa * rho;
    return (kappa * rho) * rho;
}

static int alloc_work(work_t* w)
{
    long sz = w->b.size;
    int d, q;
    double* all = (double*)calloc((size_t)sz * (4 + 4 + 12 + 12 + 12 + 8), sizeof(double));
    if (!all) return 1;
    double* cur = all;
    for (q = 0; q < 4; ++q) { w->Um[q] = cur; cur += sz; }
    for (q = 0; q < 4; ++q) { w->Uh[q] = cur; cur += sz; }
    for (d = 0; d < 3; ++d)
        for (q = 0; q < 4; ++q) { w->Fp[d][q] = cur; cur += sz; }
    for (d = 0; d < 3; ++d)
        for (q = 0; q < 4; ++q) { w->Fc[d][q] = cur; cur += sz; }
    for (d = 0; d < 3; ++d)
        for (q = 0; q < 4; ++q) { w->slope[d][q] = cur; cur += sz; }
    w->rho = cur; cur += sz;
    w->T = cur; cur += sz;
    for (d = 0; d < 3; ++d) { w->v[d] = cur; cur += sz; }
    w->kP = cur; cur += sz;
    w->kF = cur; cur += sz;
    w->jj = cur; cur += sz;
    return 0;
}

static void free_work(work_t* w) { free(w->Um[0]); }

static void setup_block(block_t* b, const orc_params* p, const int lo[3], const int hi[3])
{
    int d;
    for (d = 0; d < 3; ++d) {
        b->act[d] = p->n[d] > 1;
        b->g[d] = b->act[d] ? 3 : 0;
        b->lo[d] = lo[d];
        b->hi[d] = hi[d];
        b->m[d] = hi[d] - lo[d] + 2 * b->g[d];
    }
    b->stride[0] = 1;
    b->stride[1] = b->m[0];
    b->stride[2] = (long)b->m[0] * b->m[1];
    b->size = b->stride[2] * b->m[2];
}

/* Fill every cell of the padded block (owned box plus ghosts) from the global arrays.  X holds
 * either F (xscale = 1/c) or G = F/c (xscale = 1); the Dirichlet states are always F. */
static void load_block(work_t* w, const double* E, const double* const X[3], double xscale,
                       const double* T, const double* rho, const double* const vin[3],
                       const double* kP, const double* kF, const double* j)
{
    const orc_params* p = w->p;
    const block_t* b = &w->b;
    int k;
#pragma omp parallel for schedule(static)
    for (k = b->lo[2] - b->g[2]; k < b->hi[2] + b->g[2]; ++k) {
        int i, jy, d;
        for (jy = b->lo[1] - b->g[1]; jy < b->hi[1] + b->g[1]; ++jy)
            for (i = b->lo[0] - b->g[0]; i < b->hi[0] + b->g[0]; ++i) {
                long c = bidx(b, i, jy, k);
                /* radiation */
                int ii[3] = {i, jy, k};
                double sgn[3] = {1.0, 1.0, 1.0};
                int dface = 0, dside = 0;
                if (remap(p, ii, sgn, 1, &dface, &dside)) {
                    const double* s = dside ? p->dirichlet_hi[dface] : p->dirichlet_lo[dface];
                    w->Um[0][c] = s[0];
                    for (d = 0; d < 3; ++d) w->Um[1 + d][c] = s[1 + d] / p->c;
                } else {
                    long gi = gidx(p, ii);
                    w->Um[0][c] = E[gi];
                    for (d = 0; d < 3; ++d)
                        w->Um[1 + d][c] = sgn[d] * (xscale == 1.0 ? X[d][gi] : X[d][gi] / p->c);
                }
                /* frozen gas */
                int jj3[3] = {i, jy, k};
                double gs[3] = {1.0, 1.0, 1.0};
                remap(p, jj3, gs, 0, &dface, &dside);
                long gg = gidx(p, jj3);
                double r = rho[gg];
                w->rho[c] = r;
                w->T[c] = T ? T[gg] : 0.0;
                for (d = 0; d < 3; ++d) w->v[d][c] = vin[d] ? gs[d] * vin[d][gg] : 0.0;
                w->kP[c] = kP ? kP[gg] : kappa_law(p->kappa_P, p->kappa_rho_pow, r);
                w->kF[c] = kF ? kF[gg] : kappa_law(p->kappa_F, p->kappa_rho_pow, r);
                w->jj[c] = j ? j[gg] : 0.0;
            }
    }
}

/* Explicit radiation sources S_e,rad other than the absorption of F (Eq. algorithm:source:explicit:rad
 * with Eq. m1:simplifiedsource): E row chat kF (v/c).G, G row chat (4/3) kF E v/c (when the
 * O(beta tau) switch is on), plus the emissivity chat j / c in the E row. */
static void explicit_sources(const work_t* w, long c, const double U[4], double S[4])
{
    const orc_params* p = w->p;
    double chat = w->chat;
    int d;
    for (d = 0; d < 4; ++d) S[d] = 0.0;
    if (p->beta_tau) {
        double kF = w->kF[c];
        double vG = 0.0;
        for (d = 0; d < 3; ++d) vG += (w->v[d][c] / p->c) * U[1 + d];
        S[0] += chat * kF * vG;
        for (d = 0; d < 3; ++d) S[1 + d] += chat * (4.0 / 3.0) * kF * U[0] * (w->v[d][c] / p->c);
    }
    S[0] += chat * w->jj[c] / p->c;
}

/* Direct (non-iterative) theta updates over a stage of length h: absorption of F (Eq.
 * source:stiff:radmomentum:soln), and, by exchange mode, absorption of E (Eq.
 * source:stiff:radenergy:soln) or absorption/emission against the frozen gas temperature. */
static void theta_updates(const work_t* w, long c, double h, double U[4])
{
    const orc_params* p = w->p;
    double chat = w->chat;
    double fF = orc_theta_factor(p->theta_F, chat * w->kF[c] * h);
    U[1] *= fF;
    U[2] *= fF;
    U[3] *= fF;
    if (p->exchange == ORC_EX_ABSORB) {
        U[0] *= orc_theta_factor(p->theta_E, chat * w->kP[c] * h);
    } else if (p->exchange == ORC_EX_FROZEN_T) {
        double x = chat * w->kP[c] * h;
        double T = w->T[c];
        double aT4 = p->a_rad * (T * T) * (T * T);
        U[0] = (U[0] * (1.0 - (1.0 - p->theta_E) * x) + x * aT4) / (1.0 + p->theta_E * x);
    }
}

/* Energy floor and the flux-limiting condition |F| <= cE (Eq. m1:fluxlimit): if |G| > E,
 * G is rescaled onto |G| = E keeping its direction (reading).  Returns 1 if rescaled. */
static int realizability(const orc_params* p, double U[4])
{
    if (U[0] < p->E_floor) U[0] = p->E_floor;
    double g2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    if (g2 > U[0] * U[0]) {
        double s = U[0] / sqrt(g2);
        U[1] *= s;
        U[2] *= s;
        U[3] *= s;
        return 1;
    }
    return 0;
}

/* Is a reconstructed face state outside the realizable set?  E must be positive and
 * |G|^2 <= (1 + 1e-12) E^2; the small allowance keeps exact-streaming states (|G| = E up to
 * rounding) on the realizable side (reading). */
static int face_unrealizable(const double U[4])
{
    double g2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    return !(U[0] > 0.0) || (g2 > (1.0 + 1e-12) * (U[0] * U[0]));
}

/* Limited slope of a cell from its left and right differences (reading r4: componentwise on (E, G);
 * minmod, monotonized central, or the unlimited central difference). */
double orc_limited_slope(double dl, double dr, int lim)
{
    if (lim == ORC_LIM_NONE) return 0.5 * (dl + dr);
    if (dl * dr <= 0.0) return 0.0;
    double s = (dl > 0.0) ? 1.0 : -1.0;
    double a = fabs(dl), b = fabs(dr);
    if (lim == ORC_LIM_MINMOD) return s * (a < b ? a : b);
    /* monotonized central */
    double m = 2.0 * (a < b ? a : b);
    double cen = 0.5 * fabs(dl + dr);
    return s * (m < cen ? m : cen);
}

/* One VL subcycle on the block.  Writes U^{m+1} of the owned box into Eo.. (G form) and T. */
static void run_block(work_t* w, double* Eo, double* Gxo, double* Gyo, double* Gzo, double* To,
                      orc_stats* st)
{
    const orc_params* p = w->p;
    const block_t* b = &w->b;
    double chat = w->chat, dt = w->dt;
    int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    int ext[3];   /* extension of the predictor region beyond the owned box, per direction */
    int d;
    for (d = 0; d < 3; ++d) ext[d] = b->act[d] ? 2 : 0;
    long long n_fix = 0, n_face = 0, n_theta = 0, n_nonfinite = 0;

    /* (1) predictor fluxes: first-order HLL at every face (cell - e_d | cell) with cell in the
     *     owned box extended by 2 in every active direction and by 3 along d on the high side,
     *     L = U^m(cell - e_d), R = U^m(cell) (Eq. hyperbolic:hllflux2, indices (i-1, i)). */
    for (d = 0; d < 3; ++d) {
        if (!b->act[d]) continue;
        int k;
#pragma omp parallel for schedule(static)
        for (k = b->lo[2] - ext[2]; k < b->hi[2] + ext[2] + e[d][2]; ++k) {
            int i, jy, q;
            for (jy = b->lo[1] - ext[1]; jy < b->hi[1] + ext[1] + e[d][1]; ++jy)
                for (i = b->lo[0] - ext[0]; i < b->hi[0] + ext[0] + e[d][0]; ++i) {
                    long c = bidx(b, i, jy, k);
                    long cl = bidx(b, i - e[d][0], jy - e[d][1], k - e[d][2]);
                    double UL[4], UR[4], F[4];
                    for (q = 0; q < 4; ++q) { UL[q] = w->Um[q][cl]; UR[q] = w->Um[q][c]; }
                    orc_hll(UL, UR, d, chat, p->closure, p->speeds, F);
                    for (q = 0; q < 4; ++q) w->Fp[d][q][c] = F[q];
                }
        }
    }

    /* (2) predictor update to the half step on the extended region. */
    {
        int k;
#pragma omp parallel for schedule(static) reduction(+ : n_fix)
        for (k = b->lo[2] - ext[2]; k < b->hi[2] + ext[2]; ++k) {
            int i, jy, q, dd;
            for (jy = b->lo[1] - ext[1]; jy < b->hi[1] + ext[1]; ++jy)
                for (i = b->lo[0] - ext[0]; i < b->hi[0] + ext[0]; ++i) {
                    long c = bidx(b, i, jy, k);
                    double U0[4], U[4], div[4] = {0.0, 0.0, 0.0, 0.0}, S[4];
                    for (q = 0; q < 4; ++q) U0[q] = w->Um[q][c];
                    for (dd = 0; dd < 3; ++dd) {
                        if (!b->act[dd]) continue;
                        long cr = bidx(b, i + e[dd][0], jy + e[dd][1], k + e[dd][2]);
                        for (q = 0; q < 4; ++q) div[q] += (w->Fp[dd][q][cr] - w->Fp[dd][q][c]) / p->dx[dd];
                    }
                    explicit_sources(w, c, U0, S);
                    for (q = 0; q < 4; ++q) U[q] = U0[q] - 0.5 * dt * div[q] + 0.5 * dt * S[q];
                    theta_updates(w, c, 0.5 * dt, U);
                    int fixed = realizability(p, U);
                    int owned = i >= b->lo[0] && i < b->hi[0] && jy >= b->lo[1] && jy < b->hi[1] &&
                                k >= b->lo[2] && k < b->hi[2];
                    if (owned) n_fix += fixed;
                    for (q = 0; q < 4; ++q) w->Uh[q][c] = U[q];
                }
        }
    }

    /* (3) piecewise-linear reconstruction of U^{m+1/2}: limited slopes for every cell within one
     *     cell (along d) of the owned box; a slope whose face values are not realizable is set to
     *     zero for all four components (reading). */
    for (d = 0; d < 3; ++d) {
        if (!b->act[d]) continue;
        int k;
#pragma omp parallel for schedule(static) reduction(+ : n_face)
        for (k = b->lo[2] - e[d][2]; k < b->hi[2] + e[d][2]; ++k) {
            int i, jy, q;
            for (jy = b->lo[1] - e[d][1]; jy < b->hi[1] + e[d][1]; ++jy)
                for (i = b->lo[0] - e[d][0]; i < b->hi[0] + e[d][0]; ++i) {
                    long c = bidx(b, i, jy, k);
                    long cl = bidx(b, i - e[d][0], jy - e[d][1], k - e[d][2]);
                    long cr = bidx(b, i + e[d][0], jy + e[d][1], k + e[d][2]);
                    double s[4], Um_[4], Up_[4];
                    for (q = 0; q < 4; ++q) {
                        s[q] = orc_limited_slope(w->Uh[q][c] - w->Uh[q][cl], w->Uh[q][cr] - w->Uh[q][c],
                                             p->limiter);
                        Um_[q] = w->Uh[q][c] - 0.5 * s[q];
                        Up_[q] = w->Uh[q][c] + 0.5 * s[q];
                    }
                    if (face_unrealizable(Um_) || face_unrealizable(Up_)) {
                        for (q = 0; q < 4; ++q) s[q] = 0.0;
                        int owned = i >= b->lo[0] && i < b->hi[0] && jy >= b->lo[1] && jy < b->hi[1] &&
                                    k >= b->lo[2] && k < b->hi[2];
                        if (owned) n_face += 1;
                    }
                    for (q = 0; q < 4; ++q) w->slope[d][q][c] = s[q];
                }
        }
    }

    /* (4) corrector fluxes at the faces of the owned box: L = U^{m+1/2}(cell - e_d) + slope/2,
     *     R = U^{m+1/2}(cell) - slope/2 (indices (i-1/2, i-1/2)). */
    for (d = 0; d < 3; ++d) {
        if (!b->act[d]) continue;
        int k;
#pragma omp parallel for schedule(static)
        for (k = b->lo[2]; k < b->hi[2] + e[d][2]; ++k) {
            int i, jy, q;
            for (jy = b->lo[1]; jy < b->hi[1] + e[d][1]; ++jy)
                for (i = b->lo[0]; i < b->hi[0] + e[d][0]; ++i) {
                    long c = bidx(b, i, jy, k);
                    long cl = bidx(b, i - e[d][0], jy - e[d][1], k - e[d][2]);
                    double UL[4], UR[4], F[4];
                    for (q = 0; q < 4; ++q) {
                        UL[q] = w->Uh[q][cl] + 0.5 * w->slope[d][q][cl];
                        UR[q] = w->Uh[q][c] - 0.5 * w->slope[d][q][c];
                    }
                    orc_hll(UL, UR, d, chat, p->closure, p->speeds, F);
                    for (q = 0; q < 4; ++q) w->Fc[d][q][c] = F[q];
                }
        }
    }

    /* (5) corrector update, direct theta updates, energy exchange, realizability. */
    {
        int k;
        long nbx = b->hi[0] - b->lo[0], nby = b->hi[1] - b->lo[1];
#pragma omp parallel for schedule(static) reduction(+ : n_fix, n_theta, n_nonfinite)
        for (k = b->lo[2]; k < b->hi[2]; ++k) {
            int i, jy, q, dd;
            for (jy = b->lo[1]; jy < b->hi[1]; ++jy)
                for (i = b->lo[0]; i < b->hi[0]; ++i) {
                    long c = bidx(b, i, jy, k);
                    double Uh_[4], U[4], div[4] = {0.0, 0.0, 0.0, 0.0}, S[4];
                    for (q = 0; q < 4; ++q) Uh_[q] = w->Uh[q][c];
                    for (dd = 0; dd < 3; ++dd) {
                        if (!b->act[dd]) continue;
                        long cr = bidx(b, i + e[dd][0], jy + e[dd][1], k + e[dd][2]);
                        for (q = 0; q < 4; ++q) div[q] += (w->Fc[dd][q][cr] - w->Fc[dd][q][c]) / p->dx[dd];
                    }
                    explicit_sources(w, c, Uh_, S);
                    for (q = 0; q < 4; ++q) U[q] = w->Um[q][c] - dt * div[q] + dt * S[q];
                    theta_updates(w, c, dt, U);
                    double Tn = w->T[c];
                    if (p->exchange == ORC_EX_FULL) {
                        /* the unsplit second-order transport is not positivity preserving; the
                         * exchange acts on E floored at E_floor (reading), which keeps c0 < 0 for
                         * theta = 1 */
                        if (U[0] < p->E_floor) U[0] = p->E_floor;
                        n_theta += orc_exchange_full(p, chat, dt, w->rho[c], w->kP[c], &U[0], &Tn);
                    } else if (p->exchange == ORC_EX_LINEAR) {
                        orc_exchange_linear(p, chat, dt, w->kP[c], &U[0], &Tn);
                    }
                    n_fix += realizability(p, U);
                    if (!(isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]) &&
                          ((p->exchange != ORC_EX_FULL && p->exchange != ORC_EX_LINEAR) || isfinite(Tn))))
                        n_nonfinite += 1;
                    long o = (long)(i - b->lo[0]) + nbx * ((long)(jy - b->lo[1]) + nby * (long)(k - b->lo[2]));
                    Eo[o] = U[0];
                    Gxo[o] = U[1];
                    Gyo[o] = U[2];
                    Gzo[o] = U[3];
                    if (To) To[o] = Tn;
                }
        }
    }

    /* (6) energy leaving through the outer faces of the domain (serial, fixed order). */
    double out = 0.0;
    for (d = 0; d < 3; ++d) {
        if (!b->act[d]) continue;
        double area = 1.0;
        int dd, side;
        for (dd = 0; dd < 3; ++dd)
            if (dd != d && b->act[dd]) area *= p->dx[dd];
        for (side = 0; side < 2; ++side) {
            int face = side ? p->n[d] : 0;
            if (face != (side ? b->hi[d] : b->lo[d])) continue;   /* box does not touch it */
            int lo3[3] = {b->lo[0], b->lo[1], b->lo[2]}, hi3[3] = {b->hi[0], b->hi[1], b->hi[2]};
            lo3[d] = face;
            hi3[d] = face + 1;
            int i, jy, k;
            for (k = lo3[2]; k < hi3[2]; ++k)
                for (jy = lo3[1]; jy < hi3[1]; ++jy)
                    for (i = lo3[0]; i < hi3[0]; ++i)
                        out += (side ? 1.0 : -1.0) * dt * area * w->Fc[d][0][bidx(b, i, jy, k)];
        }
    }

    if (st) {
        st->n_realizability_fix += n_fix;
        st->n_face_fallback += n_face;
        st->n_theta_fallback += n_theta;
        st->n_nonfinite += n_nonfinite;
        st->boundary_E_out += out;
    }
}

static int check_params(const orc_params* p, double chat, double dt)
{
    int d;
    if (!p || !(chat > 0.0) || !(dt >= 0.0) || !(p->c > 0.0)) return 1;
    for (d = 0; d < 3; ++d) {
        if (p->n[d] < 1) return 1;
        if (p->n[d] > 1 && (p->n[d] < 3 || !(p->dx[d] > 0.0))) return 1;
    }
    if (!(p->E_floor > 0.0)) return 1;
    return 0;
}

int orc_subcycle_box(const orc_params* p, double chat, double dt, const int lo[3], const int hi[3],
                     double* E, double* Fx, double* Fy, double* Fz, double* T, const double* rho,
                     const double* vx, const double* vy, const double* vz, const double* kP,
                     const double* kF, const double* j, orc_stats* stats)
{
    if (check_params(p, chat, dt) || !E || !Fx || !Fy || !Fz || !rho) return 1;
    if ((p->exchange == ORC_EX_FULL || p->exchange == ORC_EX_FROZEN_T || p->exchange == ORC_EX_LINEAR) && !T) return 1;
    int d;
    for (d = 0; d < 3; ++d)
        if (lo[d] < 0 || hi[d] > p->n[d] || lo[d] >= hi[d]) return 1;
    work_t w;
    memset(&w, 0, sizeof(w));
    w.p = p;
    w.chat = chat;
    w.dt = dt;
    setup_block(&w.b, p, lo, hi);
    if (alloc_work(&w)) return 2;
    const double* X[3] = {Fx, Fy, Fz};
    const double* vin[3] = {vx, vy, vz};
    load_block(&w, E, X, 1.0 / p->c, T, rho, vin, kP, kF, j);
    long nb = (long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    double* out = (double*)malloc(sizeof(double) * (size_t)nb * 5);
    if (!out) {
        free_work(&w);
        return 2;
    }
    run_block(&w, out, out + nb, out + 2 * nb, out + 3 * nb, out + 4 * nb, stats);
    long o = 0;
    int i, jy, k;
    for (k = lo[2]; k < hi[2]; ++k)
        for (jy = lo[1]; jy < hi[1]; ++jy)
            for (i = lo[0]; i < hi[0]; ++i, ++o) {
                long gi = (long)i + (long)p->n[0] * ((long)jy + (long)p->n[1] * k);
                E[gi] = out[o];
                Fx[gi] = p->c * out[nb + o];
                Fy[gi] = p->c * out[2 * nb + o];
                Fz[gi] = p->c * out[3 * nb + o];
                if (T && (p->exchange == ORC_EX_FULL || p->exchange == ORC_EX_LINEAR)) T[gi] = out[4 * nb + o];
            }
    free(out);
    free_work(&w);
    return 0;
}

int orc_subcycles(const orc_params* p, int n_sub, double chat, double dt, double* E, double* Fx,
                  double* Fy, double* Fz, double* T, const double* rho, const double* vx,
                  const double* vy, const double* vz, const double* kP, const double* kF,
                  const double* j, orc_stats* stats)
{
    if (check_params(p, chat, dt) || n_sub < 0 || !E || !Fx || !Fy || !Fz || !rho) return 1;
    if ((p->exchange == ORC_EX_FULL || p->exchange == ORC_EX_FROZEN_T || p->exchange == ORC_EX_LINEAR) && !T) return 1;
    long n = (long)p->n[0] * p->n[1] * p->n[2];
    int lo[3] = {0, 0, 0};
    int hi[3] = {p->n[0], p->n[1], p->n[2]};
    /* state in G = F/c form for the whole call */
    double* st = (double*)malloc(sizeof(double) * (size_t)n * 10);
    if (!st) return 2;
    double *Ea = st, *Ga[3] = {st + n, st + 2 * n, st + 3 * n}, *Ta = st + 4 * n;
    double *Eb = st + 5 * n, *Gb[3] = {st + 6 * n, st + 7 * n, st + 8 * n}, *Tb = st + 9 * n;
    long i;
    for (i = 0; i < n; ++i) {
        Ea[i] = E[i];
        Ga[0][i] = Fx[i] / p->c;
        Ga[1][i] = Fy[i] / p->c;
        Ga[2][i] = Fz[i] / p->c;
        Ta[i] = T ? T[i] : 0.0;
    }
    const double* vin[3] = {vx, vy, vz};
    int s;
    for (s = 0; s < n_sub; ++s) {
        work_t w;
        memset(&w, 0, sizeof(w));
        w.p = p;
        w.chat = chat;
        w.dt = dt;
        setup_block(&w.b, p, lo, hi);
        if (alloc_work(&w)) {
            free(st);
            return 2;
        }
        const double* X[3] = {Ga[0], Ga[1], Ga[2]};
        load_block(&w, Ea, X, 1.0, Ta, rho, vin, kP, kF, j);
        run_block(&w, Eb, Gb[0], Gb[1], Gb[2], Tb, stats);
        if (p->exchange != ORC_EX_FULL && p->exchange != ORC_EX_LINEAR) memcpy(Tb, Ta, sizeof(double) * (size_t)n);
        free_work(&w);
        /* swap */
        double* t;
        t = Ea; Ea = Eb; Eb = t;
        for (i = 0; i < 3; ++i) { t = Ga[i]; Ga[i] = Gb[i]; Gb[i] = t; }
        t = Ta; Ta = Tb; Tb = t;
    }
    for (i = 0; i < n; ++i) {
        E[i] = Ea[i];
        Fx[i] = p->c * Ga[0][i];
        Fy[i] = p->c * Ga[1][i];
        Fz[i] = p->c * Ga[2][i];
        if (T && (p->exchange == ORC_EX_FULL || p->exchange == ORC_EX_LINEAR)) T[i] = Ta[i];
    }
    free(st);
    return 0;
}
