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

#include "dfloat.cuh"
#include "fp_convert.cuh"
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

// Index checks of the debug build (-DRHD_BOUNDS_CHECK, librhd_debug.so): chk(i, n) compares an index
// with its array's extent; an index outside it is counted in this translation unit's device record
// (with the source line, index and extent of the first one) and replaced by 0, so the access stays
// inside the array (no trap, no fault) and the host reports it (rhd_stats.bounds_violations,
// RHD_ERR_BOUNDS).  In the release build chk is the identity.
#ifdef RHD_BOUNDS_CHECK
static __device__ OobRecord g_oob;
__device__ __forceinline__ void oob_note(long long i, long long n, int line)
{
    if (atomicAdd(&g_oob.count, 1ull) == 0ull) {
        g_oob.line = line;
        g_oob.index = i;
        g_oob.extent = n;
    }
}
template <typename I>
__device__ __forceinline__ I chk_at(I i, long long n, int line)
{
    if ((unsigned long long)(long long)i >= (unsigned long long)n) {
        oob_note((long long)i, n, line);
        return I(0);
    }
    return i;
}
#define chk(i, n) chk_at((i), (long long)(n), __LINE__)
#else
#define chk(i, n) (i)
#endif
// Asynchronous global->shared copies (cp.async): the next plane is fetched while the current one
// is being computed; completion is awaited with cp.async.wait_all before the data are read.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ bool finite_d(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff; }
template <typename R>
__device__ __forceinline__ R to_r(double x);
template <>
__device__ __forceinline__ double to_r<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_r<float>(double x) { return d2f_trunc(x); }

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
    R invE = rcp(E);
    R f2 = xmul(xfma(gz, gz, xfma(gy, gy, xmul(gx, gx))), xmul(invE, invE));
    R invEb = invE;
    if (f2 > R(1)) {
        // |G| > E (a state outside the realizable set, e.g. an input U^m): the closure is that of
        // f = 1 along n = G/|G|, i.e. of the state (E, G/f), so mu f = gd/(E f) in the wave speeds and
        // b G G^T = E n n^T with b = 1/(E f^2).  Face states of the corrector have passed the
        // realizability test and never take this branch beyond its rounding allowance.
        const R q = rcp(sqrt_fast(f2));
        invE = xmul(invE, q);
        invEb = xmul(invE, q);
        f2 = R(1);
    }
    k.invE = invE;
    const R x4 = xfma(R(-3), f2, R(4));  // in [1, 4]
    R inv_s;
    if constexpr (sizeof(R) == 8) {
        inv_s = rsqrt_nr(x4);  // s and 1/s from one refined inverse square root
        k.s = xmul(x4, inv_s);
    } else {
        k.s = sqrt_fast(x4);
        inv_s = rcp(k.s);
    }
    k.inv2ps = rcp(xadd(R(2), k.s));
    k.cs = xmul(chat, inv_s);
    if (p1) {
        k.a = xmul(E, R(1.0 / 3.0));
        k.b = R(0);
    } else {
        k.a = xmul(xmul(xadd(k.s, R(-1)), E), R(1.0 / 3.0));
        k.b = xmul(xmul(R(3), k.inv2ps), invEb);
    }
    return k;
}

// lambda_1, lambda_3 in a direction with flux component gd (Eq. hyperbolic:evals13 rewritten with
// mu f = gd/E and 2 mu^2 (2 - f^2 - s) = (2/3) mu^2 (s-1)(s-2)).  The closure and the wave speeds use
// explicitly rounded operations (xmul / xadd / xfma): a tile evaluates them for its own cells and for
// its halo cells, which are other tiles' own cells, and both must get the same bits.
template <typename R>
__device__ __forceinline__ void wave_speeds(const ClosureScalars<R>& k, R gd, R chat, int fixed, R& l1, R& l3)
{
    if (fixed) {
        l3 = xmul(chat, R(0.57735026918962576451));
        l1 = -l3;
        return;
    }
    const R fd = xmul(gd, k.invE);
    R rad = xmul(xmul(R(2.0 / 3.0), xadd(k.s, R(-1))), xfma(-xmul(xmul(R(3), fd), fd), k.inv2ps, k.s));
    rad = rmax(rad, R(0));
    const R sr = sqrt_fast(rad);
    l1 = xmul(xadd(fd, -sr), k.cs);
    l3 = xmul(xadd(fd, sr), k.cs);
}

// Flux chat * (G_d, P_dx, P_dy, P_dz) of a state in direction D.
template <int D, typename R>
__device__ __forceinline__ void dir_flux(const ClosureScalars<R>& k, const R U[4], R chat, R F[4])
{
    const R gd = U[1 + D], bg = xmul(k.b, gd);
    F[0] = xmul(chat, gd);
    F[1] = xmul(chat, xfma(bg, U[1], D == 0 ? k.a : R(0)));
    F[2] = xmul(chat, xfma(bg, U[2], D == 1 ? k.a : R(0)));
    F[3] = xmul(chat, xfma(bg, U[3], D == 2 ? k.a : R(0)));
}

// Eq. (hyperbolic:hllflux2); S_R^+ = S_L^- = 0 gives the average (same reading as the oracle).
template <typename R>
__device__ __forceinline__ void hll(const R UL[4], const R UR[4], const R FL[4], const R FR[4], R l1L, R l3L,
                                    R l1R, R l3R, R out[4])
{
    R SR = rmax(l3L, l3R), SL = rmin(l1L, l1R);
    R SRp = rmax(SR, R(0)), SLm = rmin(SL, R(0));
    R den = xadd(SRp, -SLm);
    if (den > R(0)) {
        R inv = rcp(den);
        R pr = xmul(SRp, SLm);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            out[q] = xmul(xfma(pr, xadd(UR[q], -UL[q]), xfma(SRp, FL[q], xmul(-SLm, FR[q]))), inv);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = xmul(R(0.5), xadd(FL[q], FR[q]));
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
    const R g2 = xfma(gz, gz, xfma(gy, gy, xmul(gx, gx)));
    return !(E > R(0)) || (g2 > xmul(R(1) + Tol<R>::face, xmul(E, E)));
}

// Face states of one cell in direction D for the corrector: the limited slope of U^{m+1/2} from
// cells i-1, i, i+1, the two face values U -/+ slope/2 (zero slope if either is not realizable),
// and for each face value the flux in direction D and the wave speeds lambda_1, lambda_3.
// Layout of out[20]: minus state (4), its flux (4), l1, l3, plus state (4), its flux (4), l1, l3.
template <int D, typename R>
__device__ __forceinline__ int face_states(const R um[4], const R u0[4], const R up[4], R chat, int lim, int p1,
                                           int fixed, R out[20])
{
    R sl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sl[q] = limited(u0[q] - um[q], up[q] - u0[q], lim);
    const R h = R(0.5);
    R Sm[4], Sp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        Sm[q] = u0[q] - h * sl[q];
        Sp[q] = u0[q] + h * sl[q];
    }
    int fb = face_unrealizable(Sm[0], Sm[1], Sm[2], Sm[3]) || face_unrealizable(Sp[0], Sp[1], Sp[2], Sp[3]);
    if (fb) {
#pragma unroll
        for (int q = 0; q < 4; ++q) Sm[q] = Sp[q] = u0[q];
    }
    ClosureScalars<R> km = closure_scalars(Sm[0], Sm[1], Sm[2], Sm[3], chat, p1);
    ClosureScalars<R> kp = closure_scalars(Sp[0], Sp[1], Sp[2], Sp[3], chat, p1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        out[q] = Sm[q];
        out[10 + q] = Sp[q];
    }
    dir_flux<D>(km, Sm, chat, out + 4);
    dir_flux<D>(kp, Sp, chat, out + 14);
    wave_speeds(km, Sm[1 + D], chat, fixed, out[8], out[9]);
    wave_speeds(kp, Sp[1 + D], chat, fixed, out[18], out[19]);
    return fb;
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
#ifdef RHD_BOUNDS_CHECK
    if ((unsigned)x >= (unsigned)g.n[0] || (unsigned)y >= (unsigned)g.n[1] || (unsigned)z >= (unsigned)g.n[2]) {
        // the coordinates packed into one number: x + 2^20 (y + 2^20 z), offset by 2^19 each
        oob_note((long long)(x + (1 << 19)) + ((long long)(y + (1 << 19)) << 20) + ((long long)(z + (1 << 19)) << 40),
                 -1, __LINE__);
        return 0;
    }
#endif
    return (long long)x + (long long)g.n[0] * ((long long)y + (long long)g.n[1] * (long long)z);
}
// cells of the interior arrays and of the stored U^{m+1/2} of the two-pass path (grid plus its ghost
// layers in the directions that are not periodic on both faces)
__device__ __forceinline__ long long n_cells(const GridParams& g) { return (long long)g.n[0] * g.n[1] * g.n[2]; }
__device__ __forceinline__ long long n_padded(const GridParams& g)
{
    return (long long)upad_extent(g, 0) * upad_extent(g, 1) * upad_extent(g, 2);
}

// U^m = (E, Gx, Gy, Gz) at any cell, ghosts by the boundary rule.
__device__ __forceinline__ void load_U(const GridParams& g, const GridArrays& a, int x, int y, int z, double U[4])
{
    int sg[3] = {1, 1, 1};
    if (!inside(g, x, y, z)) {
        int pos[3] = {x, y, z};
        int df = remap_cell(g, pos, sg, true);
        if (df >= 0) {
            const double* s = (df == 0 && a.dir_dev) ? a.dir_dev : ((df & 1) ? g.dir_hi[df >> 1] : g.dir_lo[df >> 1]);
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
    double T, rho;  // rho in FP64 is loaded only where the FP64 exchange needs it
    float rho32;
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
        c.rho32 = r;
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
        c.rho32 = 0.0f;
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
    R fF = (R(1) - (R(1) - thF) * xF) * rcp(R(1) + thF * xF);
    U[1] *= fF;
    U[2] *= fF;
    U[3] *= fF;
    if (g.exchange == EX_ABSORB) {
        R xP = chat * gc.kP * h;
        U[0] *= (R(1) - (R(1) - thE) * xP) * rcp(R(1) + thE * xP);
    } else if (g.exchange == EX_FROZEN_T) {
        R xP = chat * gc.kP * h;
        R T = (R)gc.T;
        R aT4 = (sizeof(R) == 8 ? (R)g.a_rad : (R)g.f_a_rad) * (T * T) * (T * T);
        U[0] = (U[0] * (R(1) - (R(1) - thE) * xP) + xP * aT4) * rcp(R(1) + thE * xP);
    }
}

// Energy floor and |G| <= E (Eq. m1:fluxlimit); returns 1 if G was rescaled.
template <typename R>
__device__ __forceinline__ int realize(R U[4], R E_floor)
{
    if (U[0] < E_floor) U[0] = E_floor;
    R g2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    if (g2 > U[0] * U[0]) {
        R s = U[0] / sqrt(g2);
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

__device__ __forceinline__ float exchange_delta_fp32(const GridParams& g, float chat, float dt, float rho, float kP,
                                                     float E, float T, ExchangeOut& o, float& qout);

__device__ __forceinline__ ExchangeOut exchange_fp64(const GridParams& g, double chat, double dt, double rho,
                                                     double kP, double& E, double& T)
{
    ExchangeOut o = {0, 0, 0};
    // divisions as Newton-refined reciprocals times the numerator (within an ulp or two; the iteration
    // below converges to its own rounding fixed point either way)
    const double c = g.c;
    const double q = g.gm1_mu * rcp(rho);
    const double e = rho * T * g.inv_gm1_mu;
    const double alpha = g.a_rad * (q * q) * (q * q);
    const double eta = c * kP * dt;
    const double r = chat * g.inv_c;
    double th = g.theta_E;
    double Ebar = e + E * rcp(r);
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
    double b = fabs(c0 * rcp(B));
    if (A > 0.0) b = fmin(b, sqrt(sqrt(fabs(c0 * rcp(A)))));
    const double dhi = b - e;   // delta upper bound
    const double dlo = -e;      // x >= 0
    // start from the same iteration in FP32 (within 2^-25 of the root, on the FP32 pipe; values outside
    // the FP32 range give a non-finite seed and the start d = 0): one or two FP64 steps then reach the
    // FP64 rounding fixed point, against up to about fifteen from d = 0 on states far from equilibrium
    double d = 0.0;
    {
        ExchangeOut o32;
        float q32;
        const float d32 = exchange_delta_fp32(g, (float)chat, (float)dt, (float)rho, (float)kP, (float)E, (float)T,
                                              o32, q32);
        if (isfinite(d32) && !o32.newton_fb) d = fmin(fmax((double)d32, dlo), dhi);
    }
    bool conv = false;
    int it;
    for (it = 0; it < 100; ++it) {
        double x = e + d;
        double x2 = x * x;
        double gv = A * x2 * x2 + B * d + C;
        double gp = 4.0 * A * x2 * x + B;
        double dn = d - gv * rcp(gp);
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

// Linear exchange of the Pomraning material (c_v = alpha T^3, Section 4.1.4): Eqs. (marshak:update)
// in v = a_R T^4 with dtau = eps c kP dt, dv = -(v - E) dtau / (1 + theta (1 + chat/(eps c)) dtau),
// dE = -(chat / (eps c)) dv (the paper's chat = c gives 1 + 1/eps and -dv/eps), so v/(eps c) + E/chat
// is kept; v is kept >= 0 and T follows from it.
__device__ __forceinline__ void exchange_linear_fp64(const GridParams& g, double chat, double dt, double kP, double& E,
                                                     double& T)
{
    const double eps = g.linear_eps, c = g.c;
    const double T2 = T * T;
    double v = g.a_rad * T2 * T2;
    const double dtau = eps * c * kP * dt;
    const double r = chat * g.inv_eps_c;  // chat / (eps c), 1/(eps c) from the host
    const double dv = -(v - E) * dtau * rcp(1.0 + g.theta_E * (1.0 + r) * dtau);
    E = E + (-r * dv);
    v = v + dv;
    if (v < 0.0) v = 0.0;
    T = sqrt(sqrt(v * g.inv_a_rad));
}

// FP32 Newton for delta with the same iteration, which also stops once a step is small enough that
// the next could not change the FP32 result; the caller applies E - (chat/c) delta and T + q delta
// to the FP64 state.
__device__ __forceinline__ float exchange_delta_fp32(const GridParams& g, float chat, float dt, float rho, float kP,
                                                     float E, float T, ExchangeOut& o, float& qout)
{
    o.theta_fb = o.newton_fb = o.iters = 0;
    const float c = g.f_c;
    const float q = g.f_gm1_mu * rcp(rho);
    const float e = rho * T * rcp(g.f_gm1_mu);
    const float alpha = g.f_a_rad * (q * q) * (q * q);
    const float eta = c * kP * dt;
    const float r = chat * g.f_inv_c;
    float th = g.f_theta_E;
    float e4 = (e * e) * (e * e);
    float Ebar = e + E * rcp(r);
    float c0 = (1.0f - th) * eta * (alpha * e4 - E) - (e + r * eta * th * Ebar);
    if (c0 > 0.0f) {
        th = 1.0f;
        o.theta_fb = 1;
        c0 = -(e + r * eta * th * Ebar);
    }
    const float A = eta * th * alpha;
    const float B = 1.0f + r * eta * th;
    const float C = eta * ((1.0f - th) * alpha * e4 - E);
    float b = fabsf(c0 * rcp(B));
    if (A > 0.0f) b = fminf(b, sqrt_fast(sqrt_fast(fabsf(c0 * rcp(A)))));
    const float dhi = b - e, dlo = -e;
    float d = 0.0f;
    bool conv = false;
    int it;
    for (it = 0; it < 60; ++it) {
        float x = e + d;
        float x2 = x * x;
        float gv = A * x2 * x2 + B * d + C;
        float gp = 4.0f * A * x2 * x + B;
        float dn = d - gv * rcp(gp);
        dn = fminf(fmaxf(dn, dlo), dhi);
        if (it > 0 && !(dn < d)) {
            conv = true;
            break;
        }
        // a step below 2^-13 x: Newton's error after it is at most (g''/2g') step^2 <= 1.5 step^2 / x
        // (g'' = 12 A x^2, g' >= 4 A x^3), i.e. under 2^-25 x, below half an FP32 ulp of x, so the
        // iterate is final without the extra iteration that would find the fixed point
        if (fabsf(dn - d) <= 1.220703125e-4f * x) {
            d = dn;
            conv = true;
            ++it;
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
    // threads of the CTA: one per tile cell in 2D and 3D; in 1D one per cell of the widest per-phase set
    // (the 3-cell halo on each side: TX + 6 predictor cells, TX + 5 faces), so no phase takes a second
    // round.  A 1D subcycle on a short grid is bound by its longest dependent chain, and each FP64
    // instruction occupies a warp's pipe for as long with 2 active lanes as with 32, so a second round
    // for the halo would nearly double the kernel's time.
    static constexpr int NT = DIM == 1 ? ((TX + 6 + 31) / 32) * 32 : TX * TY;
    static constexpr int HY = DIM >= 2 ? 1 : 0;
    static constexpr int W3 = TX + 6, H3 = TY + 6 * HY;
    static constexpr int W2 = TX + 4, H2 = TY + 4 * HY;
    static constexpr int N3 = W3 * H3, N2 = W2 * H2;
    static constexpr int NR2 = (N2 + NT - 1) / NT;
    static constexpr int NR3 = (N3 + NT - 1) / NT;
    // predictor faces
    static constexpr int NFX = (W2 + 1) * H2;
    static constexpr int NFY = HY ? W2 * (H2 + 1) : 0;
    // corrector: cells with face states, and faces
    static constexpr int NSX = (TX + 2) * TY;
    static constexpr int NSY = HY ? TX * (TY + 2) : 0;
    static constexpr int NCX = (TX + 1) * TY;
    static constexpr int NCY = HY ? TX * (TY + 1) : 0;
    static constexpr int RING = DIM == 3 ? 3 : 1;
    // shared memory (units of R): predictor buffers and corrector buffers share one region
    static constexpr int P_UM = 0;                 // 4 x N3 U^m
    static constexpr int P_CC = P_UM + 4 * N3;     // 9 x N3 closure data
    static constexpr int P_FX = P_CC + 9 * N3;     // 4 x NFX
    static constexpr int P_FY = P_FX + 4 * NFX;    // 4 x NFY
    static constexpr int P_END = P_FY + 4 * NFY;
    static constexpr int C_SX = 0;                 // 20 x NSX face states (x)
    static constexpr int C_SY = C_SX + 20 * NSX;   // 20 x NSY face states (y)
    static constexpr int C_FX = C_SY + 20 * NSY;   // 4 x NCX fluxes
    static constexpr int C_FY = C_FX + 4 * NCX;    // 4 x NCY fluxes
    static constexpr int C_END = C_FY + 4 * NCY;
    static constexpr int UNION = P_END > C_END ? P_END : C_END;
    static constexpr int OFF_UH = UNION;           // RING x 4 x N2
    static constexpr int END_R = OFF_UH + RING * 4 * N2;
    // FP64 staging (offsets in doubles from the 8-byte aligned end of the R region):
    // U^m of the next plane on R3, and U^m, T of the corrector plane on the tile
    static constexpr int ST_U = 0;                 // 4 x N3
    static constexpr int ST_C = ST_U + 4 * N3;     // 5 x NT
    static constexpr int ST_END = ST_C + 5 * NT;
    __host__ __device__ static constexpr size_t r_bytes(size_t rsize) { return ((END_R * rsize + 15) / 16) * 16; }
    __host__ __device__ static constexpr size_t bytes(size_t rsize) { return r_bytes(rsize) + 8 * (size_t)ST_END; }

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
    unsigned fix, face, theta, newton_fb, nonfinite, iter_max, timeout;
};

// ------------------------------------------------------------------------------------------------
// Stiff sources of a split-path cell (a8, a9) at FP64 accuracy.  Reconstruction, closure, fluxes and
// the explicit O(beta tau) and emissivity sources give an FP32 increment d of the cell; the stiff
// sources then act on the FP64 state U0 + d (U0 the state at t^m) exactly as in the FP64 path, with the
// FP32 copies of the gas inputs as their inputs (the density exact; an absorption coefficient is the
// FP32 copy of its array, or the opacity law evaluated at that density).  The FP64 pipe of this part
// runs at a small fraction of the FP32 rate and with a long latency, so the arithmetic is double-float
// on the FP32 pipe (dfloat.cuh: about 48 bits, a few 2^-48 relative per operation), and FP64
// operations are spent only on splitting the FP64 state into double-floats and adding the results back
// to it (about ten per cell in FULL mode):
//   - theta updates of G (Eq. source:stiff:radmomentum:soln) and of E in ABSORB (Eq.
//     source:stiff:radenergy:soln): x = chat k dt and the factor (1 - (1 - theta) x)/(1 + theta x) in
//     double-float, then (U0 + d) f as one FP64 FMA per component; FROZEN_T's a_R T^4 term likewise;
//   - the FULL exchange (Eqs. source:energyupdate - source:polynomial): the paper's quartic written
//     for the temperature change t = T^{n+1} - T^n (t = q delta with delta = e^{n+1} - e^n and
//     q = (gamma - 1) mu/(k_B rho)) and multiplied by x = chat kP dt > 0,
//       R(t) = sigma (1 + theta x) t + x (a_R [theta (T + t)^4 + (1 - theta) T^4] - E) = 0,
//     sigma = (chat/c)/q, after which E^{n+1} = E - sigma t (Eq. source:eradupdate: E - (chat/c) delta).
//     The FP32 Newton iteration on delta (exchange_delta_fp32) gives the seed t0 = q delta, within a
//     few 2^-24 T of the root; R(t0) is evaluated in double-float (its two terms cancel near the root)
//     and one step with Halley's second-order term, t = t0 - c - (R''/2R') c^2 with c = R/R', follows,
//     R' and R'' in FP32: the step's error is of order c^3/T^2 plus the FP32 relative error of R' times
//     c, a few 2^-48 T in all, and the E error (sigma times that) a few 2^-48 max(E, a_R T^4),
//     independent of the ratio of gas to radiation energy.  E^{n+1} and T^{n+1} are the FP64 state plus
//     double-float increments.  A cell whose seed or step is not finite, or whose step exceeds 2^-20 T
//     (a seed the FP32 iteration got wrong, e.g. in units that leave its range), is solved instead by
//     FP64 Newton steps from the seed (R is convex and increasing in t for T + t >= 0, so the iterates
//     decrease monotonically after the first; the first iterate that does not decrease is the answer).
// The theta fallback (c0 > 0, Section 3.4) is decided by the FP32 iteration.  E is floored at E_floor
// before the exchange, as in the FP64 path.
// ------------------------------------------------------------------------------------------------
struct SplitStiffConsts {
    dfl cdt;         // chat dt (absorption-coefficient arrays)
    dfl KP, KF;      // chat dt kappa_P, chat dt kappa_F (the opacity law's factor)
    dfl aR, thF, omF, thE, omE;  // a_R, theta, 1 - theta
    dfl sig1;        // (chat/c) / ((gamma - 1) mu/k_B): sigma = sig1 rho
    dfl Efl;         // E_floor
    double chat, dt, sig1d;
};

__device__ __forceinline__ SplitStiffConsts split_stiff_consts(const GridParams& g, double chat, double dt)
{
    SplitStiffConsts k;
    const double cdt = chat * dt;
    k.cdt = dconst(cdt);
    k.KP = dconst(cdt * g.kappa_P);
    k.KF = dconst(cdt * g.kappa_F);
    k.sig1d = chat * g.inv_c / g.gm1_mu;
    k.sig1 = dconst(k.sig1d);
    k.Efl = dconst(g.E_floor);
    k.aR = dconst(g.a_rad);
    k.thF = dconst(g.theta_F);
    k.omF = dconst(1.0 - g.theta_F);
    k.thE = dconst(g.theta_E);
    k.omE = dconst(1.0 - g.theta_E);
    k.chat = chat;
    k.dt = dt;
    return k;
}

// chat dt k of a split-path cell: k the FP32 copy of its array, or the opacity law K rho^p with
// K = chat dt kappa
__device__ __forceinline__ dfl split_x(const SplitStiffConsts& k, const float* karr, float kv, dfl K, int p, float rho)
{
    if (karr) return dmul(k.cdt, kv);
    return p == 0 ? K : (p == 1 ? dmul(K, rho) : dmul(dmul(K, rho), rho));
}
__device__ __forceinline__ bool is_one(dfl t) { return t.hi == 1.0f && t.lo == 0.0f; }
// (1 - (1 - theta) x)/(1 + theta x)
__device__ __forceinline__ dfl theta_factor(dfl x, dfl th, dfl om)
{
    if (is_one(th)) return drcp(dadd(x, 1.0f));
    return dmul(dadd(dneg(dmul(om, x)), 1.0f), drcp(dadd(dmul(th, x), 1.0f)));
}
// (U0 + d) f in FP64 for a double-float factor f: U0 (f_hi + f_lo) + d f_hi (d is an FP32 quantity, so
// its product is rounded in FP32); f_hi + f_lo is exact in FP64
__device__ __forceinline__ double scale_state(double U0, float d, double f64, float fhi)
{
    return fma(U0, f64, f2d_exact(__fmul_rn(d, fhi)));
}

// U0: the FP64 state at t^m; d: the FP32 increment (transport and explicit sources over dt); T: the gas
// temperature (read for FROZEN_T, read and updated for FULL and LINEAR).  Writes Un = U^{m+1} before
// realizability.
__device__ __forceinline__ void split_stiff(const GridParams& g, const GridArrays& a, const SplitStiffConsts& k,
                                            float chat, float dt, const GasCell<float>& gc, const double U0[4],
                                            const float d[4], double& T, double Un[4], Counters& cnt)
{
    const float rho = gc.rho32;
    {
        const dfl fF = theta_factor(split_x(k, a.kF32, gc.kF, k.KF, g.kpow, rho), k.thF, k.omF);
        const double f64 = df2d(fF);
#pragma unroll
        for (int q = 1; q < 4; ++q) Un[q] = scale_state(U0[q], d[q], f64, fF.hi);
    }
    const int ex = g.exchange;
    if (ex == EX_EQUILIBRIUM) {
        Un[0] = U0[0] + f2d_exact(d[0]);
        return;
    }
    if (ex == EX_LINEAR) {
        double E = U0[0] + f2d_exact(d[0]);
        const double kP = a.kP32 ? f2d_exact(gc.kP) : kappa_law(g.kappa_P, g.kpow, f2d_exact(rho));
        exchange_linear_fp64(g, k.chat, k.dt, kP, E, T);
        Un[0] = E;
        return;
    }
    const dfl xP = split_x(k, a.kP32, gc.kP, k.KP, g.kpow, rho);
    if (ex == EX_ABSORB) {
        const dfl fE = theta_factor(xP, k.thE, k.omE);
        Un[0] = scale_state(U0[0], d[0], df2d(fE), fE.hi);
        return;
    }
    if (ex == EX_FROZEN_T) {
        // (E (1 - (1 - theta) x) + x a_R T^4)/(1 + theta x) = (U0 + d) fE + x a_R T^4 / (1 + theta x)
        const dfl rD = drcp(dadd(dmul(k.thE, xP), 1.0f));
        const dfl fE = dmul(dadd(dneg(dmul(k.omE, xP)), 1.0f), rD);
        const dfl W = dmul(dmul(xP, dmul(k.aR, dsqr(dsqr(d2df(T))))), rD);
        const dfl Z = dadd(W, __fmaf_rn(d2f_rn(U0[0]), fE.lo, __fmul_rn(d[0], fE.hi)));
        Un[0] = fma(U0[0], f2d_exact(fE.hi), f2d_exact(Z.hi)) + f2d_exact(Z.lo);
        return;
    }
    // FULL.  E_in = U0 + d, floored (transport is not positivity preserving)
    dfl Ein = dadd(d2df_fast(U0[0]), d[0]);
    const bool floored = Ein.hi < k.Efl.hi || (Ein.hi == k.Efl.hi && Ein.lo < k.Efl.lo);
    if (floored) Ein = k.Efl;
    const dfl Td = d2df_fast(T);
    ExchangeOut o;
    float qv;
    const float del = exchange_delta_fp32(g, chat, dt, rho, gc.kP, Ein.hi, Td.hi, o, qv);
    const float t0 = qv * del;
    const bool thone = o.theta_fb || is_one(k.thE);
    const dfl th = o.theta_fb ? dfl{1.0f, 0.0f} : k.thE;
    const dfl sig = dmul(k.sig1, rho);
    const dfl sD = dmul(sig, dadd(thone ? xP : dmul(th, xP), 1.0f));  // sigma (1 + theta x)
    // R(t0) in double-float
    const dfl T1 = dadd(Td, t0);
    const dfl T1s = dsqr(T1);
    dfl M = dsqr(T1s);
    if (!thone) M = dadd_same(dmul(th, M), dmul(k.omE, dsqr(dsqr(Td))));
    const dfl R = dadd(dmul(sD, t0), dmul(xP, dadd(dmul(k.aR, M), dneg(Ein))));
    // the step with Halley's term: R' = sigma (1 + theta x) + 4 theta x a_R T1^3, R''/2R' = 6 theta x a_R T1^2 / R'
    const float T1h = T1.hi;
    const float q4 = 4.0f * th.hi * xP.hi * k.aR.hi * T1h * T1h;
    const float Rp = __fmaf_rn(q4, T1h, sD.hi);
    const float iRp = rcp(Rp);
    const float ch = R.hi * iRp;
    const float cl = __fmaf_rn(1.5f * q4 * iRp * ch, ch, (__fmaf_rn(-ch, Rp, R.hi) + R.lo) * iRp);
    dfl t = two_sum(t0, -ch);
    t = fast_two_sum(t.hi, t.lo - cl);
    o.iters += 1;
    const bool ok = isfinite(t.hi) && isfinite(t.lo) && isfinite(sD.hi) && fabsf(ch) <= 9.5367431640625e-7f * fabsf(T1h);
    if (ok) {
        const dfl sigt = dmul(sig, t);
        const dfl inc = floored ? dneg(sigt) : dadd(dneg(sigt), d[0]);
        Un[0] = ((floored ? g.E_floor : U0[0]) + f2d_exact(inc.hi)) + f2d_exact(inc.lo);
        T = (T + f2d_exact(t.hi)) + f2d_exact(t.lo);
    } else {
        // FP64 Newton steps from the seed (or from t = 0 if the seed is not finite)
        const double E = floored ? g.E_floor : U0[0] + f2d_exact(d[0]);
        const double rhod = f2d_exact(rho);
        const double kPd = a.kP32 ? f2d_exact(gc.kP) : kappa_law(g.kappa_P, g.kpow, rhod);
        const double xPd = k.chat * k.dt * kPd, thd = o.theta_fb ? 1.0 : g.theta_E, sigd = k.sig1d * rhod;
        const double sDd = sigd * fma(thd, xPd, 1.0);
        double ts = isfinite(t0) ? f2d_exact(t0) : 0.0;
        bool settled = false;
#pragma unroll 1
        for (int s = 0; s < 64; ++s) {
            const double T1d = T + ts, T1sd = T1d * T1d;
            double Md = T1sd * T1sd;
            if (thd != 1.0) {
                const double T2 = T * T, T4 = T2 * T2;
                Md = fma(thd, Md - T4, T4);
            }
            const double Rv = fma(sDd, ts, xPd * fma(g.a_rad, Md, -E));
            const double tn = ts - Rv / fma(4.0 * thd * xPd * g.a_rad * T1sd, T1d, sDd);
            if (s > 0 && !(tn < ts)) {
                settled = true;
                o.iters += s;
                break;
            }
            ts = tn;
        }
        if (!settled) {
            o.newton_fb = 1;
            o.iters += 64;
        }
        Un[0] = fma(-sigd, ts, E);
        T = T + ts;
    }
    cnt.theta += o.theta_fb;
    cnt.newton_fb += o.newton_fb;
    cnt.iter_max = max(cnt.iter_max, (unsigned)o.iters);
}

template <typename R>
__device__ __forceinline__ void store20(R* base, int stride, int idx, const R v[20])
{
#pragma unroll
    for (int q = 0; q < 20; ++q) base[q * stride + idx] = v[q];
}

// HLL from stored face states: L = plus part of cell iL, R = minus part of cell iR
template <typename R>
__device__ __forceinline__ void hll_stored(const R* base, int stride, int iL, int iR, R F[4])
{
    R UL[4], UR[4], FL[4], FR[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        UL[q] = base[(10 + q) * stride + iL];
        FL[q] = base[(14 + q) * stride + iL];
        UR[q] = base[q * stride + iR];
        FR[q] = base[(4 + q) * stride + iR];
    }
    hll(UL, UR, FL, FR, base[18 * stride + iL], base[19 * stride + iL], base[8 * stride + iR], base[9 * stride + iR],
        F);
}

// ------------------------------------------------------------------------------------------------
// one tile of one subcycle: planes [z0, z1) of the column tile at (x0, y0)
// ------------------------------------------------------------------------------------------------
template <typename R, int TX, int TY, int DIM, bool SPLIT>
__device__ __forceinline__ void subcycle_tile(const GridParams& g, const GridArrays& a, double chat_d, double dt_d,
                                              int x0, int y0, int z0, int z1, R* sm, Counters& cnt)
{
    using G = Geo<TX, TY, DIM>;
    const int t = threadIdx.x;
    R* Um = sm + G::P_UM;
    R* Cc = sm + G::P_CC;
    R* Fx = sm + G::P_FX;
    R* Fy = sm + G::P_FY;
    R* Sx = sm + G::C_SX;
    R* Sy = sm + G::C_SY;
    R* Cx = sm + G::C_FX;
    R* Cy = sm + G::C_FY;
    R* Uh = sm + G::OFF_UH;
    double* stU = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(sm) + G::r_bytes(sizeof(R)));
    double* stC = stU + G::ST_C;
    const R chat = (R)chat_d;
    const R dt = (R)dt_d;
    const R hdt = R(0.5) * dt;
    const SplitStiffConsts sk = split_stiff_consts(g, chat_d, dt_d);
    const R idx = (R)g.inv_dx[0], idy = (R)g.inv_dx[1], idz = (R)g.inv_dx[2];
    const int p1 = g.closure == 1, fixed = g.speeds == 1, lim = g.limiter;
    const R E_floor = sizeof(R) == 8 ? (R)g.E_floor : (R)g.f_E_floor;
    const bool needT_pred = g.exchange == EX_FROZEN_T;
    const long long nxy = (long long)g.n[0] * g.n[1];

    // cells of the R3 region handled by this thread, fixed for all planes
    int c_i3[G::NR3], c_off[G::NR3];
    // the tile's halo lies inside the domain in x and y: loads need no boundary remap there
    const bool xy_inside = x0 - 3 >= 0 && x0 + TX + 3 <= g.n[0] &&
                           (G::HY == 0 || (y0 - 3 >= 0 && y0 + TY + 3 <= g.n[1]));
#pragma unroll
    for (int r = 0; r < G::NR3; ++r) {
        int c = t + r * G::NT;
        int lx = 0, ly = 0;
        if (c < G::N3) G::cell_of(c, lx, ly);
        c_i3[r] = G::i3(lx, ly);
        c_off[r] = (x0 + lx) + g.n[0] * (y0 + ly);
    }

    const int tlx0 = t % TX, tly0 = t / TX;
    // fetch U^m of plane q on R3 into the staging buffer (asynchronously where no remap is needed)
    auto issue_plane = [&](int q) {
        const bool fast = xy_inside && (unsigned)q < (unsigned)g.n[2];
        const long long zoff = (long long)q * nxy;
#pragma unroll
        for (int r = 0; r < G::NR3; ++r) {
            int c = t + r * G::NT;
            if (c < G::N3) {
                if (fast) {
                    long long i = chk(zoff + c_off[r], n_cells(g));
                    cp_async8(stU + 0 * G::N3 + c, a.E + i);
                    cp_async8(stU + 1 * G::N3 + c, a.G[0] + i);
                    cp_async8(stU + 2 * G::N3 + c, a.G[1] + i);
                    cp_async8(stU + 3 * G::N3 + c, a.G[2] + i);
                } else {
                    int lx, ly;
                    G::cell_of(c, lx, ly);
                    double U[4];
                    load_U(g, a, x0 + lx, y0 + ly, q, U);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) stU[qq * G::N3 + c] = U[qq];
                }
            }
        }
    };
    // fetch the FP64 state (and T) of the own tile cell of corrector plane k
    const bool needT_corr = g.exchange == EX_FULL || g.exchange == EX_FROZEN_T || g.exchange == EX_LINEAR;
    auto issue_corr = [&](int k) {
        if (x0 + tlx0 < g.n[0] && y0 + tly0 < g.n[1] && (unsigned)k < (unsigned)g.n[2]) {
            long long i = lin(g, x0 + tlx0, y0 + tly0, k);
            cp_async8(stC + 0 * G::NT + t, a.E + i);
            cp_async8(stC + 1 * G::NT + t, a.G[0] + i);
            cp_async8(stC + 2 * G::NT + t, a.G[1] + i);
            cp_async8(stC + 3 * G::NT + t, a.G[2] + i);
            if (needT_corr) cp_async8(stC + 4 * G::NT + t, a.T + i);
        }
    };

    // per-thread z pipeline of the predictor (own R2 cells: c = t + r * NT)
    R zU[G::NR2][4], zP[G::NR2][3], zl[G::NR2][2], dxy[G::NR2][4], zfl[G::NR2][4];
    // corrector: lower z face and the plus face state (z) of the previous plane, own tile column
    R cfl[4], zplus[10];
    const int tlx = tlx0, tly = tly0;

    const int qbeg = (DIM == 3) ? z0 - 3 : 0;
    const int qend = (DIM == 3) ? z1 + 3 : 1;
    issue_plane(qbeg);
    cp_async_commit();
#pragma unroll 1
    for (int qz = qbeg; qz < qend; ++qz) {
        // (a) U^m of plane qz on the tile plus 3-cell halo: staged copy -> R (each thread converts
        //     the cells it fetched itself, so its own wait suffices)
        cp_async_wait_all();
#pragma unroll
        for (int r = 0; r < G::NR3; ++r) {
            int c = t + r * G::NT;
            if (c < G::N3) {
                int i = c_i3[r];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) Um[qq * G::N3 + i] = to_r<R>(stU[qq * G::N3 + c]);
            }
        }
        __syncthreads();
        // prefetch the next plane and the FP64 state of this iteration's corrector plane
        if (qz + 1 < qend) issue_plane(qz + 1);
        if (DIM == 3) issue_corr(qz - 3); else issue_corr(qz);
        cp_async_commit();
        // (b) closure once per cell: P and the x, y wave speeds to shared memory; z data of the
        //     own R2 cells to registers
        R nU[G::NR2][4], nP[G::NR2][3], nl[G::NR2][2];
#pragma unroll
        for (int r = 0; r < G::NR3; ++r) {
            int c = t + r * G::NT;
            if (c < G::N3) {
                int i = c_i3[r];
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
        for (int f = t; f < G::NFX + G::NFY; f += G::NT) {
            R UL[4], UR[4], FL[4], FR[4], F[4];
            if (f < G::NFX) {
                int row = f / (G::W2 + 1);
                int lx = f % (G::W2 + 1) - 2;
                int ly = row - 2 * G::HY;
                int iL = G::i3(lx - 1, ly), iR = G::i3(lx, ly);
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
                hll(UL, UR, FL, FR, Cc[5 * G::N3 + iL], Cc[6 * G::N3 + iL], Cc[5 * G::N3 + iR], Cc[6 * G::N3 + iR],
                    F);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) Fx[qq * G::NFX + f] = F[qq];
            } else {
                int fy = (f - G::NFX) / G::W2;
                int lx = (f - G::NFX) % G::W2 - 2;
                int ly = fy - 2;
                int iL = G::i3(lx, ly - 1), iR = G::i3(lx, ly);
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
                hll(UL, UR, FL, FR, Cc[7 * G::N3 + iL], Cc[8 * G::N3 + iL], Cc[7 * G::N3 + iR], Cc[8 * G::N3 + iR],
                    F);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) Fy[qq * G::NFY + (f - G::NFX)] = F[qq];
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
                    int slot = (DIM == 3) ? ((p + 3) % 3) : 0;
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
        const bool own_col = x0 + tlx < g.n[0] && y0 + tly < g.n[1];
        if (DIM == 3 && qz == z0 + 1) {
            // plus face state (z) of cell z0-1, from U^{m+1/2} at z0-2, z0-1, z0
            const int i = G::i2(tlx, tly);
            R u[3][4], fs[20];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const R* sl = Uh + ((z0 - 2 + m + 3) % 3) * 4 * G::N2;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) u[m][qq] = sl[qq * G::N2 + i];
            }
            face_states<2>(u[0], u[1], u[2], chat, lim, p1, fixed, fs);
#pragma unroll
            for (int qq = 0; qq < 10; ++qq) zplus[qq] = fs[10 + qq];
        }
        if (DIM == 3 && qz == z0 + 2) {
            // face states (z) of cell z0 and the lower face (z0 - 1 | z0)
            const int i = G::i2(tlx, tly);
            R u[3][4], fs[20];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const R* sl = Uh + ((z0 - 1 + m + 3) % 3) * 4 * G::N2;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) u[m][qq] = sl[qq * G::N2 + i];
            }
            int fb = face_states<2>(u[0], u[1], u[2], chat, lim, p1, fixed, fs);
            if (fb && own_col) cnt.face += 1;
            R UL[4], UR[4], FL[4], FR[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                UL[qq] = zplus[qq];
                FL[qq] = zplus[4 + qq];
                UR[qq] = fs[qq];
                FR[qq] = fs[4 + qq];
            }
            hll(UL, UR, FL, FR, zplus[8], zplus[9], fs[8], fs[9], cfl);
#pragma unroll
            for (int qq = 0; qq < 10; ++qq) zplus[qq] = fs[10 + qq];
        }
        const bool do_corr = (DIM == 3) ? (k >= z0 && k < z1) : true;
        if (do_corr) {
            const R* Uk = Uh + ((DIM == 3) ? ((k + 3) % 3) : 0) * 4 * G::N2;
            // (e1) face states of the tile cells and their neighbours along x and y
            for (int c = t; c < G::NSX + G::NSY; c += G::NT) {
                R fs[20];
                if (c < G::NSX) {
                    int ly = c / (TX + 2), lx = c % (TX + 2) - 1;
                    R u[3][4];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        int i = G::i2(lx - 1 + m, ly);
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) u[m][qq] = Uk[qq * G::N2 + i];
                    }
                    int fb = face_states<0>(u[0], u[1], u[2], chat, lim, p1, fixed, fs);
                    if (fb && lx >= 0 && lx < TX && x0 + lx < g.n[0] && y0 + ly < g.n[1]) cnt.face += 1;
                    store20(Sx, G::NSX, c, fs);
                } else {
                    int cy = c - G::NSX;
                    int ly = cy / TX - 1, lx = cy % TX;
                    R u[3][4];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        int i = G::i2(lx, ly - 1 + m);
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) u[m][qq] = Uk[qq * G::N2 + i];
                    }
                    int fb = face_states<1>(u[0], u[1], u[2], chat, lim, p1, fixed, fs);
                    if (fb && ly >= 0 && ly < TY && x0 + lx < g.n[0] && y0 + ly < g.n[1]) cnt.face += 1;
                    store20(Sy, G::NSY, cy, fs);
                }
            }
            // z face (k | k+1) of the own column: face states of cell k+1, plus state of cell k kept
            R cfh[4] = {R(0), R(0), R(0), R(0)};
            if (DIM == 3) {
                const int i = G::i2(tlx, tly);
                R u[3][4], fs[20];
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const R* sl = Uh + ((k + m + 3) % 3) * 4 * G::N2;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) u[m][qq] = sl[qq * G::N2 + i];
                }
                int fb = face_states<2>(u[0], u[1], u[2], chat, lim, p1, fixed, fs);
                if (fb && k + 1 < z1 && own_col) cnt.face += 1;
                R FL[4], FR[4], UL[4], UR[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    UL[qq] = zplus[qq];
                    FL[qq] = zplus[4 + qq];
                    UR[qq] = fs[qq];
                    FR[qq] = fs[4 + qq];
                }
                hll(UL, UR, FL, FR, zplus[8], zplus[9], fs[8], fs[9], cfh);
#pragma unroll
                for (int qq = 0; qq < 10; ++qq) zplus[qq] = fs[10 + qq];
            }
            __syncthreads();
            // (e2) HLL fluxes on the tile's x and y faces
            for (int f = t; f < G::NCX + G::NCY; f += G::NT) {
                R F[4];
                if (f < G::NCX) {
                    int ly = f / (TX + 1), lx = f % (TX + 1);
                    int iL = lx + (TX + 2) * ly;   // cell lx-1
                    hll_stored(Sx, G::NSX, iL, iL + 1, F);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) Cx[qq * G::NCX + f] = F[qq];
                } else {
                    int fc = f - G::NCX;
                    int ly = fc / TX, lx = fc % TX;
                    int iL = lx + TX * ly;         // cell ly-1
                    hll_stored(Sy, G::NSY, iL, iL + TX, F);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) Cy[qq * G::NCY + fc] = F[qq];
                }
            }
            __syncthreads();
            // (e3) accumulation for the own tile cell
            if (own_col) {
                const int gx = x0 + tlx, gy = y0 + tly;
                R div[4];
                int fl = tly * (TX + 1) + tlx;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) div[qq] = (Cx[qq * G::NCX + fl + 1] - Cx[qq * G::NCX + fl]) * idx;
                if (G::HY) {
                    int fb = tly * TX + tlx;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        div[qq] = div[qq] + (Cy[qq * G::NCY + fb + TX] - Cy[qq * G::NCY + fb]) * idy;
                }
                if (DIM == 3) {
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) div[qq] = div[qq] + (cfh[qq] - cfl[qq]) * idz;
                }
                R Uhk[4];
                int ih = G::i2(tlx, tly);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) Uhk[qq] = Uk[qq * G::N2 + ih];
                const bool full = g.exchange == EX_FULL, linear = g.exchange == EX_LINEAR;
                GasCell<R> gc = load_gas<R, SPLIT>(g, a, gx, gy, k, false, full && !SPLIT);
                R S[4];
                explicit_sources(g, gc, Uhk, chat, S);
                long long li = lin(g, gx, gy, k);
                cp_async_wait_all();  // own staged copies of U^m and T for this cell
                double U0[4] = {stC[t], stC[G::NT + t], stC[2 * G::NT + t], stC[3 * G::NT + t]};
                double Un[4];
                double Tn = needT_corr ? stC[4 * G::NT + t] : 0.0;
                gc.T = Tn;
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
                    } else if (linear) {
                        exchange_linear_fp64(g, chat_d, dt_d, (double)gc.kP, U[0], Tn);
                    }
                    cnt.fix += realize(U, g.E_floor);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) Un[qq] = U[qq];
                } else {
                    // FP32 increment relative to the FP64 state; the stiff sources in FP64
                    float d[4];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) d[qq] = -dt * div[qq] + dt * S[qq];
                    split_stiff(g, a, sk, (float)chat, (float)dt, gc, U0, d, Tn, Un, cnt);
                    // realizability: cheap FP32 screen, exact FP64 test only near the limit
                    const float ef = d2f_trunc(Un[0]);
                    float g2f = 0.f;
#pragma unroll
                    for (int qq = 1; qq < 4; ++qq) {
                        const float gq = d2f_trunc(Un[qq]);
                        g2f += gq * gq;
                    }
                    if (!(ef > g.f_E_floor * 1.001f) || g2f > 0.9999f * ef * ef) cnt.fix += realize(Un, g.E_floor);
                }
                bool bad = !(finite_d(Un[0]) && finite_d(Un[1]) && finite_d(Un[2]) && finite_d(Un[3]) &&
                             (!(full || linear) || finite_d(Tn)));
                cnt.nonfinite += bad;
                a.Eo[li] = Un[0];
                a.Go[0][li] = Un[1];
                a.Go[1][li] = Un[2];
                a.Go[2][li] = Un[3];
                if (full || linear) a.T[li] = Tn;
            }
            if (DIM == 3) {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) cfl[qq] = cfh[qq];
            }
        }
        __syncthreads();
    }
    cp_async_wait_all();  // no copy may outlive the tile
}

}  // namespace rhd

#include "subcycle_pair.cuh"
#include "subcycle_twopass.cuh"

namespace rhd {

// shared-memory bytes of a tile routine
template <typename R, int TX, int TY, int DIM, bool SPLIT>
constexpr size_t tile_smem_bytes()
{
    return Geo<TX, TY, DIM>::bytes(sizeof(R));
}

template <typename R, int TX, int TY, int DIM, bool SPLIT>
__global__ void __launch_bounds__(Geo<TX, TY, DIM>::NT,
                                  (Geo<TX, TY, DIM>::NT > 256 || (sizeof(R) == 8 && Geo<TX, TY, DIM>::NT >= 256)) ? 1 : 2)
    subcycle_kernel(const __grid_constant__ StepParams P)
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
__global__ void __launch_bounds__(TX* TY, (TX * TY > 256 || (sizeof(R) == 8 && TX * TY >= 256)) ? 1 : 2)
    ensemble_kernel(const __grid_constant__ EnsembleParams P)
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
