// subcycle.cuh -- the fused radiation-subcycle kernel (one VL predictor/corrector step of the gray
// M1 radiation subsystem with its source terms, Skinner & Ostriker 2013, Sections 3.1, 3.3, 3.4).
//
// One CTA owns a TX x TY column tile of the grid and marches through a chunk of z planes (2.5D
// blocking).  For each newly loaded plane q of U^m (tile plus a 3-cell halo, boundary conditions
// applied by index remapping at load time) it
//   (b) evaluates the M1 closure once per cell: pressure P = E T (Eq. m1:m1tns written as
//       P = (s-1)E/3 I + 3/(2+s) G G^T / E with s = sqrt(4 - 3 f^2), so that chi = (5 - 2 s)/3) and
//       the wave speeds lambda_1,3 of Eq. (hyperbolic:evals13) per direction;
//   (c) forms the first-order HLL fluxes (Eq. hyperbolic:hllflux2, L/R = cells i-1, i) on x and y
//       faces in shared memory; z faces are formed per column in registers;
//   (d) completes U^{m+1/2} of plane q-1 (half step, explicit O(beta tau) and emissivity sources,
//       theta updates over dt/2, realizability) into a 5-plane ring;
//   (e) runs the corrector for plane q-3: limited piecewise-linear face states of U^{m+1/2}, closure
//       and wave speeds of each face state, HLL fluxes, flux divergence, explicit sources from
//       U^{m+1/2}, theta updates over dt, the energy exchange, realizability, and stores U^{m+1}.
// Every stage follows the order of the CPU oracle; the readings of the paper (limiter, face-state
// fallback, split order, ghost rule) are the same.
//
// Precision: R = double gives the FP64 path.  R = float with SPLIT gives the split path: closure,
// wave speeds, reconstruction and fluxes (and so U^{m+1/2}) in FP32; the update of the FP64 state is
// formed as an FP32 increment (transport + sources + theta terms + exchange change) added once in FP64.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rhd_internal.h"

namespace rhd {

// ------------------------------------------------------------------------------------------------
// precision helpers
// ------------------------------------------------------------------------------------------------
template <typename R>
struct Tol;
template <>
struct Tol<double> {
    // allowance of the face-state realizability test |G|^2 <= (1 + tol) E^2
    static constexpr double face = 1e-12;
};
template <>
struct Tol<float> {
    static constexpr float face = 1e-5f;
};

__device__ __forceinline__ double rsq(double x) { return sqrt(x); }
__device__ __forceinline__ float rsq(float x) { return sqrtf(x); }
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float rmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double rabs(double a) { return fabs(a); }
__device__ __forceinline__ float rabs(float a) { return fabsf(a); }

// ------------------------------------------------------------------------------------------------
// closure, wave speeds, HLL
// ------------------------------------------------------------------------------------------------

// Per-state closure scalars: s = sqrt(4 - 3 f^2) (f clamped to 1), a = isotropic part of P,
// b = coefficient of G G^T in P, invE, inv2ps = 1/(2+s), cs = chat / s.
template <typename R>
struct ClosureScalars {
    R s, a, b, invE, inv2ps, cs;
};

template <typename R>
__device__ __forceinline__ ClosureScalars<R> closure_scalars(R E, R gx, R gy, R gz, R chat, int p1)
{
    ClosureScalars<R> k;
    k.invE = R(1) / E;
    R g2 = gx * gx + gy * gy + gz * gz;
    R f2 = g2 * (k.invE * k.invE);
    f2 = rmin(f2, R(1));
    k.s = rsq(R(4) - R(3) * f2);
    k.inv2ps = R(1) / (R(2) + k.s);
    k.cs = chat / k.s;
    if (p1) {
        k.a = E * R(1.0 / 3.0);
        k.b = R(0);
    } else {
        k.a = (k.s - R(1)) * E * R(1.0 / 3.0);
        k.b = R(3) * k.inv2ps * k.invE;
    }
    return k;
}

// lambda_1, lambda_3 in a direction with flux component gd (Eq. hyperbolic:evals13 rewritten with
// mu f = gd/E and 2 mu^2 (2 - f^2 - s) = (2/3) mu^2 (s-1)(s-2)).
template <typename R>
__device__ __forceinline__ void wave_speeds(const ClosureScalars<R>& k, R gd, R chat, int fixed, R& l1, R& l3)
{
    if (fixed) {
        l3 = chat * R(0.57735026918962576451);
        l1 = -l3;
        return;
    }
    R fd = gd * k.invE;
    R rad = R(2.0 / 3.0) * (k.s - R(1)) * (k.s - R(3) * fd * fd * k.inv2ps);
    rad = rmax(rad, R(0));
    R sr = rsq(rad);
    l1 = (fd - sr) * k.cs;
    l3 = (fd + sr) * k.cs;
}

// Flux chat * (G_d, P_dx, P_dy, P_dz) of a state in direction D.
template <int D, typename R>
__device__ __forceinline__ void dir_flux(const ClosureScalars<R>& k, const R U[4], R chat, R F[4])
{
    R gd = U[1 + D];
    F[0] = chat * gd;
    F[1] = chat * ((D == 0 ? k.a : R(0)) + k.b * gd * U[1]);
    F[2] = chat * ((D == 1 ? k.a : R(0)) + k.b * gd * U[2]);
    F[3] = chat * ((D == 2 ? k.a : R(0)) + k.b * gd * U[3]);
}

// Eq. (hyperbolic:hllflux2); S_R^+ = S_L^- = 0 gives the average (same reading as the oracle).
template <typename R>
__device__ __forceinline__ void hll(const R UL[4], const R UR[4], const R FL[4], const R FR[4], R l1L, R l3L,
                                    R l1R, R l3R, R out[4])
{
    R SR = rmax(l3L, l3R), SL = rmin(l1L, l1R);
    R SRp = rmax(SR, R(0)), SLm = rmin(SL, R(0));
    R den = SRp - SLm;
    if (den > R(0)) {
        R inv = R(1) / den;
        R pr = SRp * SLm;
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = (SRp * FL[q] - SLm * FR[q] + pr * (UR[q] - UL[q])) * inv;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = R(0.5) * (FL[q] + FR[q]);
    }
}

template <typename R>
__device__ __forceinline__ R limited(R dl, R dr, int lim)
{
    if (lim == LIM_NONE) return R(0.5) * (dl + dr);
    bool same = (dl > R(0) && dr > R(0)) || (dl < R(0) && dr < R(0));
    if (!same) return R(0);
    R a = rabs(dl), b = rabs(dr);
    R m = rmin(a, b);
    if (lim == LIM_MC) m = rmin(R(2) * m, R(0.5) * rabs(dl + dr));
    return dl > R(0) ? m : -m;
}

template <typename R>
__device__ __forceinline__ bool face_unrealizable(R E, R gx, R gy, R gz)
{
    R g2 = gx * gx + gy * gy + gz * gz;
    return !(E > R(0)) || (g2 > (R(1) + Tol<R>::face) * (E * E));
}

// Corrector face in direction D: L = plus-state of cell i-1, R = minus-state of cell i, from
// U^{m+1/2} at i-2, i-1, i, i+1 (indices (i-1/2, i-1/2)).  fbL/fbR report a zeroed slope.
template <int D, typename R>
__device__ __forceinline__ void corrector_face(const R um2[4], const R um1[4], const R u0[4], const R up1[4],
                                               R chat, int lim, int p1, int fixed, R F[4], int& fbL, int& fbR)
{
    R sL[4], sR[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        sL[q] = limited(um1[q] - um2[q], u0[q] - um1[q], lim);
        sR[q] = limited(u0[q] - um1[q], up1[q] - u0[q], lim);
    }
    const R h = R(0.5);
    fbL = face_unrealizable(um1[0] - h * sL[0], um1[1] - h * sL[1], um1[2] - h * sL[2], um1[3] - h * sL[3]) ||
          face_unrealizable(um1[0] + h * sL[0], um1[1] + h * sL[1], um1[2] + h * sL[2], um1[3] + h * sL[3]);
    fbR = face_unrealizable(u0[0] - h * sR[0], u0[1] - h * sR[1], u0[2] - h * sR[2], u0[3] - h * sR[3]) ||
          face_unrealizable(u0[0] + h * sR[0], u0[1] + h * sR[1], u0[2] + h * sR[2], u0[3] + h * sR[3]);
    R UL[4], UR[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        UL[q] = fbL ? um1[q] : um1[q] + h * sL[q];
        UR[q] = fbR ? u0[q] : u0[q] - h * sR[q];
    }
    ClosureScalars<R> kL = closure_scalars(UL[0], UL[1], UL[2], UL[3], chat, p1);
    ClosureScalars<R> kR = closure_scalars(UR[0], UR[1], UR[2], UR[3], chat, p1);
    R FL[4], FR[4], l1L, l3L, l1R, l3R;
    dir_flux<D>(kL, UL, chat, FL);
    dir_flux<D>(kR, UR, chat, FR);
    wave_speeds(kL, UL[1 + D], chat, fixed, l1L, l3L);
    wave_speeds(kR, UR[1 + D], chat, fixed, l1R, l3R);
    hll(UL, UR, FL, FR, l1L, l3L, l1R, l3R, F);
}

// ------------------------------------------------------------------------------------------------
// boundary remapping (ghost rule identical to the oracle's)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool inside(const GridParams& g, int x, int y, int z)
{
    return (unsigned)x < (unsigned)g.n[0] && (unsigned)y < (unsigned)g.n[1] && (unsigned)z < (unsigned)g.n[2];
}

// Maps (x, y, z) into the domain; returns the Dirichlet face (0..5) that decides the value, or -1.
static __device__ __noinline__ int remap_cell(const GridParams& g, int pos[3], int sg[3], bool dirichlet_allowed)
{
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
        int n = g.n[d];
#pragma unroll 1
        for (int guard = 0; guard < 64 && (pos[d] < 0 || pos[d] >= n); ++guard) {
            bool low = pos[d] < 0;
            int bc = low ? g.bc_lo[d] : g.bc_hi[d];
            if (bc == BC_DIRICHLET && dirichlet_allowed) return 2 * d + (low ? 0 : 1);
            if (bc == BC_PERIODIC) {
                pos[d] = ((pos[d] % n) + n) % n;
            } else if (bc == BC_OUTFLOW || bc == BC_DIRICHLET) {
                pos[d] = low ? 0 : n - 1;
            } else {
                pos[d] = low ? (-pos[d] - 1) : (2 * n - 1 - pos[d]);
                sg[d] = -sg[d];
            }
        }
        pos[d] = min(max(pos[d], 0), n - 1);  // never leave the array, even if the loop gave up
    }
    return -1;
}

__device__ __forceinline__ long long lin(const GridParams& g, int x, int y, int z)
{
    return (long long)x + (long long)g.n[0] * ((long long)y + (long long)g.n[1] * (long long)z);
}

// U^m = (E, Gx, Gy, Gz) at any cell, ghosts by the boundary rule.
__device__ __forceinline__ void load_U(const GridParams& g, const GridArrays& a, int x, int y, int z, double U[4])
{
    int sg[3] = {1, 1, 1};
    if (!inside(g, x, y, z)) {
        int pos[3] = {x, y, z};
        int df = remap_cell(g, pos, sg, true);
        if (df >= 0) {
            const double* s = (df & 1) ? g.dir_hi[df >> 1] : g.dir_lo[df >> 1];
            U[0] = s[0];
            U[1] = s[1];
            U[2] = s[2];
            U[3] = s[3];
            return;
        }
        x = pos[0];
        y = pos[1];
        z = pos[2];
    }
    long long i = lin(g, x, y, z);
    U[0] = __ldg(a.E + i);
    U[1] = sg[0] < 0 ? -__ldg(a.G[0] + i) : __ldg(a.G[0] + i);
    U[2] = sg[1] < 0 ? -__ldg(a.G[1] + i) : __ldg(a.G[1] + i);
    U[3] = sg[2] < 0 ? -__ldg(a.G[2] + i) : __ldg(a.G[2] + i);
}

// Frozen gas seen by the source terms of one cell (ghosts: nearest interior cell, mirrored
// velocity for reflecting faces).
template <typename R>
struct GasCell {
    R kP, kF, v[3], j;
    double T, rho;
};

__device__ __forceinline__ double kappa_law(double kappa, int p, double rho)
{
    return p == 0 ? kappa : (p == 1 ? kappa * rho : (kappa * rho) * rho);
}
__device__ __forceinline__ float kappa_law_f(float kappa, int p, float rho)
{
    return p == 0 ? kappa : (p == 1 ? kappa * rho : (kappa * rho) * rho);
}

template <typename R, bool SPLIT>
__device__ __forceinline__ GasCell<R> load_gas(const GridParams& g, const GridArrays& a, int x, int y, int z,
                                               bool need_T, bool need_rho64)
{
    int sg[3] = {1, 1, 1};
    if (!inside(g, x, y, z)) {
        int pos[3] = {x, y, z};
        remap_cell(g, pos, sg, false);
        x = pos[0];
        y = pos[1];
        z = pos[2];
    }
    long long i = lin(g, x, y, z);
    GasCell<R> c;
    c.T = need_T ? __ldg(a.T + i) : 0.0;
    if (SPLIT) {
        float r = __ldg(a.rho32 + i);
        c.rho = need_rho64 ? __ldg(a.rho + i) : 0.0;
        c.kP = a.kP32 ? __ldg(a.kP32 + i) : kappa_law_f(g.f_kappa_P, g.kpow, r);
        c.kF = a.kF32 ? __ldg(a.kF32 + i) : kappa_law_f(g.f_kappa_F, g.kpow, r);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            R v = a.v32[d] ? (R)__ldg(a.v32[d] + i) : R(0);
            c.v[d] = sg[d] < 0 ? -v : v;
        }
        c.j = a.j32 ? __ldg(a.j32 + i) : 0.0f;
    } else {
        double r = __ldg(a.rho + i);
        c.rho = r;
        c.kP = a.kP ? __ldg(a.kP + i) : kappa_law(g.kappa_P, g.kpow, r);
        c.kF = a.kF ? __ldg(a.kF + i) : kappa_law(g.kappa_F, g.kpow, r);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            R v = a.v[d] ? (R)__ldg(a.v[d] + i) : R(0);
            c.v[d] = sg[d] < 0 ? -v : v;
        }
        c.j = a.j ? (R)__ldg(a.j + i) : R(0);
    }
    return c;
}

// Explicit sources other than the absorption of F (Eq. algorithm:source:explicit:rad with
// Eq. m1:simplifiedsource): E row chat kF (v/c).G, G row chat (4/3) kF E v/c, plus chat j / c.
template <typename R>
__device__ __forceinline__ void explicit_sources(const GridParams& g, const GasCell<R>& gc, const R U[4], R chat,
                                                 R S[4])
{
    const R inv_c = sizeof(R) == 8 ? (R)g.inv_c : (R)g.f_inv_c;
    S[0] = chat * gc.j * inv_c;
    S[1] = S[2] = S[3] = R(0);
    if (g.beta_tau) {
        R b0 = gc.v[0] * inv_c, b1 = gc.v[1] * inv_c, b2 = gc.v[2] * inv_c;
        R vG = b0 * U[1] + b1 * U[2] + b2 * U[3];
        S[0] += chat * gc.kF * vG;
        R w = chat * R(4.0 / 3.0) * gc.kF * U[0];
        S[1] += w * b0;
        S[2] += w * b1;
        S[3] += w * b2;
    }
}

// Direct theta updates over a stage of length h (Eqs. source:stiff:radmomentum:soln,
// source:stiff:radenergy:soln, and the frozen-temperature variant).
template <typename R>
__device__ __forceinline__ void theta_updates(const GridParams& g, const GasCell<R>& gc, R chat, R h, R U[4])
{
    const R thF = sizeof(R) == 8 ? (R)g.theta_F : (R)g.f_theta_F;
    const R thE = sizeof(R) == 8 ? (R)g.theta_E : (R)g.f_theta_E;
    R xF = chat * gc.kF * h;
    R fF = (R(1) - (R(1) - thF) * xF) / (R(1) + thF * xF);
    U[1] *= fF;
    U[2] *= fF;
    U[3] *= fF;
    if (g.exchange == EX_ABSORB) {
        R xP = chat * gc.kP * h;
        U[0] *= (R(1) - (R(1) - thE) * xP) / (R(1) + thE * xP);
    } else if (g.exchange == EX_FROZEN_T) {
        R xP = chat * gc.kP * h;
        R T = (R)gc.T;
        R aT4 = (sizeof(R) == 8 ? (R)g.a_rad : (R)g.f_a_rad) * (T * T) * (T * T);
        U[0] = (U[0] * (R(1) - (R(1) - thE) * xP) + xP * aT4) / (R(1) + thE * xP);
    }
}

// Energy floor and |G| <= E (Eq. m1:fluxlimit); returns 1 if G was rescaled.
template <typename R>
__device__ __forceinline__ int realize(R U[4], R E_floor)
{
    if (U[0] < E_floor) U[0] = E_floor;
    R g2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    if (g2 > U[0] * U[0]) {
        R s = U[0] / rsq(g2);
        U[1] *= s;
        U[2] *= s;
        U[3] *= s;
        return 1;
    }
    return 0;
}

// ------------------------------------------------------------------------------------------------
// implicit energy exchange (Eqs. source:energyexchange - source:polynomial), solved for
// delta = e^{n+1} - e^n: the paper's quartic c4 x^4 + c1 x + c0 with x = e + delta reads
//   g(delta) = eta theta alpha (e + delta)^4 + (1 + (chat/c) eta theta) delta
//              + eta [(1 - theta) alpha e^4 - E] = 0,
// then E^{n+1} = E - (chat/c) delta (Eq. source:eradupdate) and T^{n+1} = (e + delta) q.
// g is increasing and convex, so Newton from delta = 0 lands at or above the root after one step
// and then decreases monotonically; it stops when an iterate no longer decreases (a fixed point
// to rounding).  The step is clamped to the paper's bracket x <= min(|c0/c1|, |c0/c4|^{1/4}), and
// bisection on that bracket finishes any solve that has not converged after 100 iterations.
// c0 > 0 (no feasible root for theta < 1, Section 3.4) redoes the step with theta = 1.
// ------------------------------------------------------------------------------------------------
struct ExchangeOut {
    int theta_fb, newton_fb, iters;
};

__device__ __forceinline__ ExchangeOut exchange_fp64(const GridParams& g, double chat, double dt, double rho,
                                                     double kP, double& E, double& T)
{
    ExchangeOut o = {0, 0, 0};
    const double c = g.c;
    const double q = (g.gamma - 1.0) * g.mu_over_kB / rho;
    const double e = (rho * T / g.mu_over_kB) / (g.gamma - 1.0);
    const double alpha = g.a_rad * (q * q) * (q * q);
    const double eta = c * kP * dt;
    const double r = chat / c;
    double th = g.theta_E;
    double Ebar = e + (c / chat) * E;
    double e4 = (e * e) * (e * e);
    double c0 = (1.0 - th) * eta * (alpha * e4 - E) - (e + r * eta * th * Ebar);
    if (c0 > 0.0) {
        th = 1.0;
        o.theta_fb = 1;
        c0 = -(e + r * eta * th * Ebar);
    }
    const double A = eta * th * alpha;
    const double B = 1.0 + r * eta * th;
    const double C = eta * ((1.0 - th) * alpha * e4 - E);
    double b = fabs(c0 / B);
    if (A > 0.0) b = fmin(b, sqrt(sqrt(fabs(c0 / A))));
    const double dhi = b - e;   // delta upper bound
    const double dlo = -e;      // x >= 0
    double d = 0.0;
    bool conv = false;
    int it;
    for (it = 0; it < 100; ++it) {
        double x = e + d;
        double x2 = x * x;
        double gv = A * x2 * x2 + B * d + C;
        double gp = 4.0 * A * x2 * x + B;
        double dn = d - gv / gp;
        if (dn > dhi) dn = dhi;
        if (dn < dlo) dn = dlo;
        if (it > 0 && !(dn < d)) {
            conv = true;
            break;
        }
        d = dn;
    }
    o.iters = it;
    if (!conv) {
        // bisection to adjacent doubles on [dlo, dhi]
        o.newton_fb = 1;
        double lo = dlo, hi = dhi;
        for (int k = 0; k < 2200; ++k) {
            double mid = lo + 0.5 * (hi - lo);
            if (!(mid > lo && mid < hi)) break;
            double x = e + mid;
            double x2 = x * x;
            double gv = A * x2 * x2 + B * mid + C;
            if (gv <= 0.0) lo = mid; else hi = mid;
        }
        d = lo;
    }
    E = E - r * d;
    T = (e + d) * q;
    return o;
}

// FP32 Newton for delta with the same iteration; the caller applies E - (chat/c) delta and
// T + q delta to the FP64 state.
__device__ __forceinline__ float exchange_delta_fp32(const GridParams& g, float chat, float dt, float rho, float kP,
                                                     float E, float T, ExchangeOut& o, float& qout)
{
    o.theta_fb = o.newton_fb = o.iters = 0;
    const float c = g.f_c;
    const float q = g.f_gm1_mu / rho;
    const float e = rho * T / g.f_gm1_mu;
    const float alpha = g.f_a_rad * (q * q) * (q * q);
    const float eta = c * kP * dt;
    const float r = chat * g.f_inv_c;
    float th = g.f_theta_E;
    float e4 = (e * e) * (e * e);
    float Ebar = e + E / r;
    float c0 = (1.0f - th) * eta * (alpha * e4 - E) - (e + r * eta * th * Ebar);
    if (c0 > 0.0f) {
        th = 1.0f;
        o.theta_fb = 1;
        c0 = -(e + r * eta * th * Ebar);
    }
    const float A = eta * th * alpha;
    const float B = 1.0f + r * eta * th;
    const float C = eta * ((1.0f - th) * alpha * e4 - E);
    float b = fabsf(c0 / B);
    if (A > 0.0f) b = fminf(b, sqrtf(sqrtf(fabsf(c0 / A))));
    const float dhi = b - e, dlo = -e;
    float d = 0.0f;
    bool conv = false;
    int it;
    for (it = 0; it < 60; ++it) {
        float x = e + d;
        float x2 = x * x;
        float gv = A * x2 * x2 + B * d + C;
        float gp = 4.0f * A * x2 * x + B;
        float dn = d - gv / gp;
        dn = fminf(fmaxf(dn, dlo), dhi);
        if (it > 0 && !(dn < d)) {
            conv = true;
            break;
        }
        d = dn;
    }
    o.iters = it;
    if (!conv) {
        o.newton_fb = 1;
        float lo = dlo, hi = dhi;
        for (int k = 0; k < 300; ++k) {
            float mid = lo + 0.5f * (hi - lo);
            if (!(mid > lo && mid < hi)) break;
            float x = e + mid;
            float x2 = x * x;
            float gv = A * x2 * x2 + B * mid + C;
            if (gv <= 0.0f) lo = mid; else hi = mid;
        }
        d = lo;
    }
    qout = q;
    return d;
}

// ------------------------------------------------------------------------------------------------
// geometry of a tile
// ------------------------------------------------------------------------------------------------
template <int TX, int TY, int DIM>
struct Geo {
    static constexpr int NT = TX * TY;
    static constexpr int HY = DIM >= 2 ? 1 : 0;
    static constexpr int W3 = TX + 6, H3 = TY + 6 * HY;
    static constexpr int W2 = TX + 4, H2 = TY + 4 * HY;
    static constexpr int N3 = W3 * H3, N2 = W2 * H2;
    static constexpr int NR2 = (N2 + NT - 1) / NT;
    static constexpr int NR3 = (N3 + NT - 1) / NT;
    static constexpr int NFX = (W2 + 1) * H2;
    static constexpr int NFY = HY ? W2 * (H2 + 1) : 1;
    static constexpr int NCX = (TX + 1) * TY;
    static constexpr int NCY = HY ? TX * (TY + 1) : 1;
    static constexpr int RING = DIM == 3 ? 5 : 1;
    // shared-memory layout in units of R
    static constexpr int OFF_UM = 0;                      // 4 x N3
    static constexpr int OFF_CC = OFF_UM + 4 * N3;        // 9 x N3 closure data
    static constexpr int OFF_FX = OFF_CC + 9 * N3;        // 4 x NFX
    static constexpr int OFF_FY = OFF_FX + 4 * NFX;       // 4 x NFY
    static constexpr int OFF_UH = OFF_FY + 4 * NFY;       // RING x 4 x N2
    static constexpr int TOTAL = OFF_UH + RING * 4 * N2;

    __device__ static __forceinline__ int i3(int lx, int ly) { return (lx + 3) + W3 * (ly + 3 * HY); }
    __device__ static __forceinline__ int i2(int lx, int ly) { return (lx + 2) + W2 * (ly + 2 * HY); }
    // enumeration of R3 cells: the R2 cells first, then the outer ring
    __device__ static __forceinline__ void cell_of(int c, int& lx, int& ly)
    {
        if (c < N2) {
            lx = c % W2 - 2;
            ly = c / W2 - 2 * HY;
            return;
        }
        int o = c - N2;
        if (!HY) {
            lx = o == 0 ? -3 : TX + 2;
            ly = 0;
            return;
        }
        if (o < H3) {
            lx = -3;
            ly = o - 3;
        } else if (o < 2 * H3) {
            lx = TX + 2;
            ly = o - H3 - 3;
        } else if (o < 2 * H3 + W2) {
            lx = o - 2 * H3 - 2;
            ly = -3;
        } else {
            lx = o - 2 * H3 - W2 - 2;
            ly = TY + 2;
        }
    }
};

// warp-aggregated counter update
__device__ __forceinline__ void add_counter(unsigned long long* dst, unsigned v)
{
    unsigned s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}
__device__ __forceinline__ void max_counter(unsigned* dst, unsigned v)
{
    unsigned s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = max(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0 && s) atomicMax(dst, s);
}

struct Counters {
    unsigned fix, face, theta, newton_fb, nonfinite, iter_max;
};

// ------------------------------------------------------------------------------------------------
// one tile of one subcycle: planes [z0, z1) of the column tile at (x0, y0)
// ------------------------------------------------------------------------------------------------
template <typename R, int TX, int TY, int DIM, bool SPLIT>
__device__ __forceinline__ void subcycle_tile(const GridParams& g, const GridArrays& a, double chat_d, double dt_d,
                                              int x0, int y0, int z0, int z1, R* sm, Counters& cnt)
{
    using G = Geo<TX, TY, DIM>;
    const int t = threadIdx.x;
    R* Um = sm + G::OFF_UM;
    R* Cc = sm + G::OFF_CC;
    R* Fx = sm + G::OFF_FX;
    R* Fy = sm + G::OFF_FY;
    R* Uh = sm + G::OFF_UH;
    const R chat = (R)chat_d;
    const R dt = (R)dt_d;
    const R hdt = R(0.5) * dt;
    const R idx = (R)g.inv_dx[0], idy = (R)g.inv_dx[1], idz = (R)g.inv_dx[2];
    const int p1 = g.closure == 1, fixed = g.speeds == 1, lim = g.limiter;
    const R E_floor = sizeof(R) == 8 ? (R)g.E_floor : (R)g.f_E_floor;
    const bool needT_pred = g.exchange == EX_FROZEN_T;

    // per-thread z pipeline of the predictor (own R2 cells: c = t + r * NT)
    R zU[G::NR2][4], zP[G::NR2][3], zl[G::NR2][2], dxy[G::NR2][4], zfl[G::NR2][4];
    // corrector: lower z face of the own tile column
    R cfl[4];
    const int tlx = t % TX, tly = t / TX;   // own tile cell

    const int qbeg = (DIM == 3) ? z0 - 3 : 0;
    const int qend = (DIM == 3) ? z1 + 3 : 1;
#pragma unroll 1
    for (int qz = qbeg; qz < qend; ++qz) {
        // (a) U^m of plane qz on the tile plus 3-cell halo
#pragma unroll
        for (int r = 0; r < G::NR3; ++r) {
            int c = t + r * G::NT;
            if (c < G::N3) {
                int lx, ly;
                G::cell_of(c, lx, ly);
                double U[4];
                load_U(g, a, x0 + lx, y0 + ly, qz, U);
                int i = G::i3(lx, ly);
                Um[0 * G::N3 + i] = (R)U[0];
                Um[1 * G::N3 + i] = (R)U[1];
                Um[2 * G::N3 + i] = (R)U[2];
                Um[3 * G::N3 + i] = (R)U[3];
            }
        }
        __syncthreads();
        // (b) closure once per cell: P and the x, y wave speeds to shared memory; z data of the
        //     own R2 cells to registers
        R nU[G::NR2][4], nP[G::NR2][3], nl[G::NR2][2];
#pragma unroll
        for (int r = 0; r < G::NR3; ++r) {
            int c = t + r * G::NT;
            if (c < G::N3) {
                int lx, ly;
                G::cell_of(c, lx, ly);
                int i = G::i3(lx, ly);
                R U[4] = {Um[i], Um[G::N3 + i], Um[2 * G::N3 + i], Um[3 * G::N3 + i]};
                ClosureScalars<R> k = closure_scalars(U[0], U[1], U[2], U[3], chat, p1);
                R Pxx = k.a + k.b * U[1] * U[1], Pxy = k.b * U[1] * U[2], Pxz = k.b * U[1] * U[3];
                R Pyy = k.a + k.b * U[2] * U[2], Pyz = k.b * U[2] * U[3];
                R l1x, l3x, l1y = R(0), l3y = R(0);
                wave_speeds(k, U[1], chat, fixed, l1x, l3x);
                if (G::HY) wave_speeds(k, U[2], chat, fixed, l1y, l3y);
                Cc[0 * G::N3 + i] = Pxx;
                Cc[1 * G::N3 + i] = Pxy;
                Cc[2 * G::N3 + i] = Pxz;
                Cc[3 * G::N3 + i] = Pyy;
                Cc[4 * G::N3 + i] = Pyz;
                Cc[5 * G::N3 + i] = l1x;
                Cc[6 * G::N3 + i] = l3x;
                Cc[7 * G::N3 + i] = l1y;
                Cc[8 * G::N3 + i] = l3y;
                if (r < G::NR2 && c < G::N2) {
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) nU[r][qq] = U[qq];
                    if (DIM == 3) {
                        nP[r][0] = Pxz;
                        nP[r][1] = Pyz;
                        nP[r][2] = k.a + k.b * U[3] * U[3];
                        wave_speeds(k, U[3], chat, fixed, nl[r][0], nl[r][1]);
                    }
                }
            }
        }
        __syncthreads();
        // (c) first-order HLL fluxes on the x and y faces of the R2 rows / columns
        for (int f = t; f < G::NFX; f += G::NT) {
            int row = f / (G::W2 + 1);
            int lx = f % (G::W2 + 1) - 2;
            int ly = row - 2 * G::HY;
            int iL = G::i3(lx - 1, ly), iR = G::i3(lx, ly);
            R UL[4], UR[4], FL[4], FR[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                UL[qq] = Um[qq * G::N3 + iL];
                UR[qq] = Um[qq * G::N3 + iR];
            }
            FL[0] = chat * UL[1];
            FL[1] = chat * Cc[0 * G::N3 + iL];
            FL[2] = chat * Cc[1 * G::N3 + iL];
            FL[3] = chat * Cc[2 * G::N3 + iL];
            FR[0] = chat * UR[1];
            FR[1] = chat * Cc[0 * G::N3 + iR];
            FR[2] = chat * Cc[1 * G::N3 + iR];
            FR[3] = chat * Cc[2 * G::N3 + iR];
            R F[4];
            hll(UL, UR, FL, FR, Cc[5 * G::N3 + iL], Cc[6 * G::N3 + iL], Cc[5 * G::N3 + iR], Cc[6 * G::N3 + iR], F);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) Fx[qq * G::NFX + f] = F[qq];
        }
        if (G::HY) {
            for (int f = t; f < G::NFY; f += G::NT) {
                int fy = f / G::W2;
                int lx = f % G::W2 - 2;
                int ly = fy - 2;
                int iL = G::i3(lx, ly - 1), iR = G::i3(lx, ly);
                R UL[4], UR[4], FL[4], FR[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    UL[qq] = Um[qq * G::N3 + iL];
                    UR[qq] = Um[qq * G::N3 + iR];
                }
                FL[0] = chat * UL[2];
                FL[1] = chat * Cc[1 * G::N3 + iL];
                FL[2] = chat * Cc[3 * G::N3 + iL];
                FL[3] = chat * Cc[4 * G::N3 + iL];
                FR[0] = chat * UR[2];
                FR[1] = chat * Cc[1 * G::N3 + iR];
                FR[2] = chat * Cc[3 * G::N3 + iR];
                FR[3] = chat * Cc[4 * G::N3 + iR];
                R F[4];
                hll(UL, UR, FL, FR, Cc[7 * G::N3 + iL], Cc[8 * G::N3 + iL], Cc[7 * G::N3 + iR], Cc[8 * G::N3 + iR],
                    F);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) Fy[qq * G::NFY + f] = F[qq];
            }
        }
        __syncthreads();
        // (d) x/y divergence of plane qz; z face (qz-1 | qz); U^{m+1/2} of plane p = qz - 1 (3D) or qz
        const int p = (DIM == 3) ? qz - 1 : qz;
        const bool do_pred = (DIM == 3) ? (qz >= z0 - 1) : true;
#pragma unroll
        for (int r = 0; r < G::NR2; ++r) {
            int c = t + r * G::NT;
            if (c < G::N2) {
                int lx = c % G::W2 - 2, ly = c / G::W2 - 2 * G::HY;
                R nd[4];
                int fl = (ly + 2 * G::HY) * (G::W2 + 1) + (lx + 2);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) nd[qq] = (Fx[qq * G::NFX + fl + 1] - Fx[qq * G::NFX + fl]) * idx;
                if (G::HY) {
                    int fb = (ly + 2) * G::W2 + (lx + 2);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        nd[qq] = nd[qq] + (Fy[qq * G::NFY + fb + G::W2] - Fy[qq * G::NFY + fb]) * idy;
                }
                R zfh[4] = {R(0), R(0), R(0), R(0)};
                if (DIM == 3 && qz > qbeg) {
                    // z face between plane qz-1 (stored) and qz (new)
                    R FL[4] = {chat * zU[r][3], chat * zP[r][0], chat * zP[r][1], chat * zP[r][2]};
                    R FR[4] = {chat * nU[r][3], chat * nP[r][0], chat * nP[r][1], chat * nP[r][2]};
                    hll(zU[r], nU[r], FL, FR, zl[r][0], zl[r][1], nl[r][0], nl[r][1], zfh);
                }
                if (do_pred && (DIM != 3 || qz > qbeg + 1)) {
                    R U0[4], div[4];
                    if (DIM == 3) {
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            U0[qq] = zU[r][qq];
                            div[qq] = dxy[r][qq] + (zfh[qq] - zfl[r][qq]) * idz;
                        }
                    } else {
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            U0[qq] = nU[r][qq];
                            div[qq] = nd[qq];
                        }
                    }
                    GasCell<R> gc = load_gas<R, SPLIT>(g, a, x0 + lx, y0 + ly, p, needT_pred, false);
                    R S[4];
                    explicit_sources(g, gc, U0, chat, S);
                    R U[4];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) U[qq] = U0[qq] - hdt * div[qq] + hdt * S[qq];
                    theta_updates(g, gc, chat, hdt, U);
                    int fx_ = realize(U, E_floor);
                    bool owned = lx >= 0 && lx < TX && ly >= 0 && ly < TY && x0 + lx < g.n[0] &&
                                 y0 + ly < g.n[1] && p >= z0 && p < z1;
                    if (owned) cnt.fix += fx_;
                    int slot = (DIM == 3) ? ((p + 10) % 5) : 0;
                    R* dst = Uh + slot * 4 * G::N2;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) dst[qq * G::N2 + c] = U[qq];
                }
                if (DIM == 3) {
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        zfl[r][qq] = zfh[qq];
                        zU[r][qq] = nU[r][qq];
                        dxy[r][qq] = nd[qq];
                    }
#pragma unroll
                    for (int qq = 0; qq < 3; ++qq) zP[r][qq] = nP[r][qq];
                    zl[r][0] = nl[r][0];
                    zl[r][1] = nl[r][1];
                }
            }
        }
        __syncthreads();
        // (e) corrector for plane k
        const int k = (DIM == 3) ? qz - 3 : qz;
        if (DIM == 3 && qz == z0 + 2) {
            // lower z face of the first plane: (z0 - 1 | z0) from U^{m+1/2} at z0-2 .. z0+1
            const R* s0 = Uh + ((z0 - 2 + 10) % 5) * 4 * G::N2;
            const R* s1 = Uh + ((z0 - 1 + 10) % 5) * 4 * G::N2;
            const R* s2 = Uh + ((z0 + 10) % 5) * 4 * G::N2;
            const R* s3 = Uh + ((z0 + 1 + 10) % 5) * 4 * G::N2;
            int i = G::i2(tlx, tly);
            R a0[4], a1[4], a2[4], a3[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                a0[qq] = s0[qq * G::N2 + i];
                a1[qq] = s1[qq * G::N2 + i];
                a2[qq] = s2[qq * G::N2 + i];
                a3[qq] = s3[qq * G::N2 + i];
            }
            int fbL, fbR;
            corrector_face<2>(a0, a1, a2, a3, chat, lim, p1, fixed, cfl, fbL, fbR);
            if (fbR && x0 + tlx < g.n[0] && y0 + tly < g.n[1]) cnt.face += 1;
        }
        const bool do_corr = (DIM == 3) ? (k >= z0 && k < z1) : true;
        if (do_corr) {
            const R* Uk = Uh + ((DIM == 3) ? ((k + 10) % 5) : 0) * 4 * G::N2;
            // x faces of the tile rows
            for (int f = t; f < G::NCX; f += G::NT) {
                int ly = f / (TX + 1), lx = f % (TX + 1);
                R u[4][4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    int i = G::i2(lx - 2 + m, ly);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) u[m][qq] = Uk[qq * G::N2 + i];
                }
                R F[4];
                int fbL, fbR;
                corrector_face<0>(u[0], u[1], u[2], u[3], chat, lim, p1, fixed, F, fbL, fbR);
                if (fbR && lx < TX && x0 + lx < g.n[0] && y0 + ly < g.n[1]) cnt.face += 1;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) Fx[qq * G::NFX + f] = F[qq];
            }
            if (G::HY) {
                for (int f = t; f < G::NCY; f += G::NT) {
                    int ly = f / TX, lx = f % TX;
                    R u[4][4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        int i = G::i2(lx, ly - 2 + m);
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) u[m][qq] = Uk[qq * G::N2 + i];
                    }
                    R F[4];
                    int fbL, fbR;
                    corrector_face<1>(u[0], u[1], u[2], u[3], chat, lim, p1, fixed, F, fbL, fbR);
                    if (fbR && ly < TY && x0 + lx < g.n[0] && y0 + ly < g.n[1]) cnt.face += 1;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) Fy[qq * G::NFY + f] = F[qq];
                }
            }
            // z face (k | k+1) of the own column
            R cfh[4] = {R(0), R(0), R(0), R(0)};
            if (DIM == 3) {
                int i = G::i2(tlx, tly);
                R a0[4], a1[4], a2[4], a3[4];
                const R* s0 = Uh + ((k - 1 + 10) % 5) * 4 * G::N2;
                const R* s1 = Uk;
                const R* s2 = Uh + ((k + 1 + 10) % 5) * 4 * G::N2;
                const R* s3 = Uh + ((k + 2 + 10) % 5) * 4 * G::N2;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    a0[qq] = s0[qq * G::N2 + i];
                    a1[qq] = s1[qq * G::N2 + i];
                    a2[qq] = s2[qq * G::N2 + i];
                    a3[qq] = s3[qq * G::N2 + i];
                }
                int fbL, fbR;
                corrector_face<2>(a0, a1, a2, a3, chat, lim, p1, fixed, cfh, fbL, fbR);
                if (fbR && k + 1 < z1 && x0 + tlx < g.n[0] && y0 + tly < g.n[1]) cnt.face += 1;
            }
            __syncthreads();
            // accumulation for the own tile cell
            const int gx = x0 + tlx, gy = y0 + tly;
            if (gx < g.n[0] && gy < g.n[1]) {
                R div[4];
                int fl = tly * (TX + 1) + tlx;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) div[qq] = (Fx[qq * G::NFX + fl + 1] - Fx[qq * G::NFX + fl]) * idx;
                if (G::HY) {
                    int fb = tly * TX + tlx;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        div[qq] = div[qq] + (Fy[qq * G::NFY + fb + TX] - Fy[qq * G::NFY + fb]) * idy;
                }
                if (DIM == 3) {
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) div[qq] = div[qq] + (cfh[qq] - cfl[qq]) * idz;
                }
                R Uhk[4];
                int ih = G::i2(tlx, tly);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) Uhk[qq] = Uk[qq * G::N2 + ih];
                const bool full = g.exchange == EX_FULL;
                GasCell<R> gc = load_gas<R, SPLIT>(g, a, gx, gy, k, full || needT_pred, full);
                R S[4];
                explicit_sources(g, gc, Uhk, chat, S);
                long long li = lin(g, gx, gy, k);
                double U0[4] = {a.E[li], a.G[0][li], a.G[1][li], a.G[2][li]};
                double Un[4];
                double Tn = gc.T;
                if constexpr (!SPLIT) {
                    double U[4];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) U[qq] = U0[qq] - dt_d * (double)div[qq] + dt_d * (double)S[qq];
                    GasCell<double> gd;
                    gd.kP = (double)gc.kP;
                    gd.kF = (double)gc.kF;
                    gd.T = gc.T;
                    gd.rho = gc.rho;
                    gd.j = (double)gc.j;
                    gd.v[0] = (double)gc.v[0];
                    gd.v[1] = (double)gc.v[1];
                    gd.v[2] = (double)gc.v[2];
                    theta_updates(g, gd, chat_d, dt_d, U);
                    if (full) {
                        // transport can leave E <= 0 (not positivity preserving); exchange on E >= E_floor
                        if (U[0] < g.E_floor) U[0] = g.E_floor;
                        ExchangeOut o = exchange_fp64(g, chat_d, dt_d, gc.rho, (double)gc.kP, U[0], Tn);
                        cnt.theta += o.theta_fb;
                        cnt.newton_fb += o.newton_fb;
                        cnt.iter_max = max(cnt.iter_max, (unsigned)o.iters);
                    }
                    cnt.fix += realize(U, g.E_floor);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) Un[qq] = U[qq];
                } else {
                    // FP32 increment relative to the FP64 state
                    float u0f[4] = {(float)U0[0], (float)U0[1], (float)U0[2], (float)U0[3]};
                    float d[4];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) d[qq] = (float)(-dt * div[qq] + dt * S[qq]);
                    const float thF = g.f_theta_F, thE = g.f_theta_E;
                    float xF = (float)chat * (float)gc.kF * (float)dt;
                    float wF = xF / (1.0f + thF * xF);
#pragma unroll
                    for (int qq = 1; qq < 4; ++qq) d[qq] -= (u0f[qq] + d[qq]) * wF;
                    if (g.exchange == EX_ABSORB) {
                        float xP = (float)chat * (float)gc.kP * (float)dt;
                        d[0] -= (u0f[0] + d[0]) * (xP / (1.0f + thE * xP));
                    } else if (g.exchange == EX_FROZEN_T) {
                        float xP = (float)chat * (float)gc.kP * (float)dt;
                        float Tf = (float)gc.T;
                        float aT4 = g.f_a_rad * (Tf * Tf) * (Tf * Tf);
                        d[0] += xP * (aT4 - (u0f[0] + d[0])) / (1.0f + thE * xP);
                    }
                    double Etr = U0[0] + (double)d[0];
                    if (full) {
                        // exchange on E >= E_floor; its change is applied to the FP64 energy
                        if (Etr < g.E_floor) Etr = g.E_floor;
                        ExchangeOut o;
                        float qv;
                        float del = exchange_delta_fp32(g, (float)chat, (float)dt, (float)gc.rho, (float)gc.kP,
                                                        (float)Etr, (float)gc.T, o, qv);
                        Etr -= (double)(((float)chat * g.f_inv_c) * del);
                        d[0] = (float)(Etr - U0[0]);
                        Tn = gc.T + (double)(qv * del);
                        cnt.theta += o.theta_fb;
                        cnt.newton_fb += o.newton_fb;
                        cnt.iter_max = max(cnt.iter_max, (unsigned)o.iters);
                    }
                    Un[0] = Etr;
#pragma unroll
                    for (int qq = 1; qq < 4; ++qq) Un[qq] = U0[qq] + (double)d[qq];
                    // realizability: cheap FP32 screen, exact FP64 test only near the limit
                    float ef = u0f[0] + d[0];
                    float g2f = 0.f;
#pragma unroll
                    for (int qq = 1; qq < 4; ++qq) {
                        float gq = u0f[qq] + d[qq];
                        g2f += gq * gq;
                    }
                    if (!(ef > g.f_E_floor * 1.001f) || g2f > 0.9999f * ef * ef) cnt.fix += realize(Un, g.E_floor);
                }
                bool bad = !(isfinite(Un[0]) && isfinite(Un[1]) && isfinite(Un[2]) && isfinite(Un[3]) &&
                             (!full || isfinite(Tn)));
                cnt.nonfinite += bad;
                a.Eo[li] = Un[0];
                a.Go[0][li] = Un[1];
                a.Go[1][li] = Un[2];
                a.Go[2][li] = Un[3];
                if (full) a.T[li] = Tn;
            }
            if (DIM == 3) {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) cfl[qq] = cfh[qq];
            }
        }
        __syncthreads();
    }
}

template <typename R, int TX, int TY, int DIM, bool SPLIT>
__global__ void __launch_bounds__(TX* TY, 2) subcycle_kernel(const __grid_constant__ StepParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    const int tile = blockIdx.x;
    const int x0 = (tile % P.tiles_x) * TX;
    const int y0 = (tile / P.tiles_x) * TY;
    int z0 = 0, z1 = 1;
    if (DIM == 3) {
        z0 = blockIdx.y * P.z_chunk;
        z1 = min(z0 + P.z_chunk, P.g.n[2]);
    }
    Counters cnt = {0, 0, 0, 0, 0, 0};
    subcycle_tile<R, TX, TY, DIM, SPLIT>(P.g, P.a, P.chat, P.dt, x0, y0, z0, z1, sm, cnt);
    add_counter(&P.stats->n_fix, cnt.fix);
    add_counter(&P.stats->n_face, cnt.face);
    add_counter(&P.stats->n_theta, cnt.theta);
    add_counter(&P.stats->n_newton_fb, cnt.newton_fb);
    add_counter(&P.stats->n_nonfinite, cnt.nonfinite);
    max_counter(&P.stats->newton_iter_max, cnt.iter_max);
}

// Persistent ensemble kernel: CTAs pull (grid, tile) items from a global counter until the queue is
// empty; the item-to-grid map is a prefix sum over the grids' tile counts (binary search).
template <typename R, int TX, int TY, bool SPLIT>
__global__ void __launch_bounds__(TX* TY, 2) ensemble_kernel(const __grid_constant__ EnsembleParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    __shared__ long long item_s;
    __shared__ __align__(16) EnsembleGrid eg_s;
    Counters cnt = {0, 0, 0, 0, 0, 0};
#pragma unroll 1
    while (true) {
        if (threadIdx.x == 0) item_s = (long long)atomicAdd(P.counter, 1ull);
        __syncthreads();
        long long item = item_s;
        __syncthreads();
        if (item >= P.n_items) break;
        int lo = 0, hi = P.n_grids - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (P.grids[mid].first_item <= item) lo = mid; else hi = mid - 1;
        }
        {
            const int* src = reinterpret_cast<const int*>(P.grids + lo);
            int* dst = reinterpret_cast<int*>(&eg_s);
            for (int w = threadIdx.x; w < (int)(sizeof(EnsembleGrid) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
        }
        __syncthreads();
        const EnsembleGrid& eg = eg_s;
        long long local = item - eg.first_item;
        int txy = (int)(local % ((long long)eg.tiles_x * eg.tiles_y));
        int tz = (int)(local / ((long long)eg.tiles_x * eg.tiles_y));
        int x0 = (txy % eg.tiles_x) * TX, y0 = (txy / eg.tiles_x) * TY;
        int z0 = tz * P.z_chunk, z1 = min(z0 + P.z_chunk, eg.g.n[2]);
        subcycle_tile<R, TX, TY, 3, SPLIT>(eg.g, eg.a, P.chat, eg.dt, x0, y0, z0, z1, sm, cnt);
        __syncthreads();
    }
    add_counter(&P.stats->n_fix, cnt.fix);
    add_counter(&P.stats->n_face, cnt.face);
    add_counter(&P.stats->n_theta, cnt.theta);
    add_counter(&P.stats->n_newton_fb, cnt.newton_fb);
    add_counter(&P.stats->n_nonfinite, cnt.nonfinite);
    max_counter(&P.stats->newton_iter_max, cnt.iter_max);
}

}  // namespace rhd
