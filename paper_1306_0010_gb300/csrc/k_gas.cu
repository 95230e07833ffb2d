// k_gas.cu -- the gas step around the radiation subcycles (Section 3.1 steps 3 and 6, Section 3.4):
// the Euler equations for (rho, rho v, E_gas) with the explicit gas sources S_e,gas of
// Eq. (algorithm:source:explicit:gas) (no gravity), advanced by one van Leer predictor / corrector step:
//
//   predictor: first-order HLLC fluxes of the ghost-filled state at t^n on the faces of the grid
//              extended by two ghost layers, then W^{n+1/2} on that extended grid (half step; sources
//              from the gas and the radiation at t^n);
//   corrector: limited piecewise-linear primitives of W^{n+1/2}, HLLC fluxes on the interior faces,
//              then the full step (sources from the gas at t^{n+1/2} and the radiation at t^n);
//   correction (after the subcycles): dt/2 [S_e,gas(W^{n+1/2}, U_rad^{n+1}) - S_e,gas(W^{n+1/2}, U_rad^n)].
//
// Each face flux is computed once, by one thread, and stored (the face arrays of one direction); the
// update kernels take the flux differences.  The HLLC solver (Toro, Riemann Solvers and Numerical
// Methods for Fluid Dynamics, Sec. 10.4) uses the Davis wave-speed estimates; the left star state when
// S* = 0; HLL where the contact speed's denominator is not negative.
//
// Precision: the kernels are templates on the arithmetic type R.  FP64 grids: R = double throughout.
// Split grids: R = float for reconstruction, wave speeds and HLLC (inputs truncated to FP32 by integer
// bit operations, FP32 fluxes stored), the flux differences and the sources; the half step W^{n+1/2} is
// an FP32 intermediate; the state (rho, v, T) accumulates FP32 increments in FP64, the pattern of the
// radiation's split path.  The increments of the primitive variables follow from those of the conserved
// ones (d rho, dM, dE) without cancellation: with rho' = rho + d rho,
//     dv = (dM - v d rho) / rho',   dK = (M.dv + dM.v') / 2   (the kinetic energy's change),
//     dT = ((gamma - 1) mu/k_B (dE - dK) - T d rho) / rho',
// so each is accurate relative to the increment itself, whatever the ratio of kinetic to internal
// energy, and the FP64 state gains FP64 additions only.  Divisions are reciprocals (FP64: the hardware
// approximation refined by Newton-Raphson; FP32: the hardware approximation) times the numerator.
#include <cuda_runtime.h>
#include <math.h>

#include "fp_convert.cuh"
#include "gas_index.h"
#include "gas_internal.h"

namespace rhd {

namespace {

constexpr int GAS_THREADS = 256;

template <typename R>
struct Prim {
    R r, v[3], P;
};

template <typename R>
__device__ __forceinline__ R flip(R x, int s)
{
    return s < 0 ? -x : x;
}

// physical constants in R
template <typename R>
struct Consts {
    R gamma, inv_gm1, inv_mu;
};
template <typename R>
__device__ __forceinline__ Consts<R> consts(const GasParams& p);
template <>
__device__ __forceinline__ Consts<double> consts<double>(const GasParams& p)
{
    return {p.gamma, p.inv_gm1, p.inv_mu};
}
template <>
__device__ __forceinline__ Consts<float> consts<float>(const GasParams& p)
{
    return {p.f_gamma, p.f_inv_gm1, p.f_inv_mu};
}

// the gas state at t^n of interior cell i, with the normal velocity components of a mirrored ghost
// cell flipped (s)
__device__ __forceinline__ Prim<double> load_prim(const GasParams& p, const GasArrays& a, long long i, const int s[3])
{
    Prim<double> w;
    w.r = a.rho[i];
    for (int d = 0; d < 3; ++d) w.v[d] = flip(a.v[d][i], s[d]);
    w.P = w.r * a.T[i] * p.inv_mu;
    return w;
}

template <typename R>
__device__ __forceinline__ Prim<R> load_prim_t(const GasParams& p, const GasArrays& a, long long i, const int s[3]);
template <>
__device__ __forceinline__ Prim<double> load_prim_t<double>(const GasParams& p, const GasArrays& a, long long i,
                                                            const int s[3])
{
    return load_prim(p, a, i, s);
}
template <>
__device__ __forceinline__ Prim<float> load_prim_t<float>(const GasParams& p, const GasArrays& a, long long i,
                                                          const int s[3])
{
    Prim<float> w;
    w.r = a.rho32[i];
    for (int d = 0; d < 3; ++d) w.v[d] = flip(a.v32[d][i], s[d]);
    w.P = w.r * d2f_trunc(a.T[i]) * p.f_inv_mu;
    return w;
}

template <typename R>
__device__ __forceinline__ R kin2(const Prim<R>& w)
{
    return w.v[0] * w.v[0] + w.v[1] * w.v[1] + w.v[2] * w.v[2];
}

// (rho, Mx, My, Mz, E_gas) of a primitive state (FP64)
__device__ __forceinline__ void to_cons(const GasParams& p, const Prim<double>& w, double U[5])
{
    U[0] = w.r;
    for (int d = 0; d < 3; ++d) U[1 + d] = w.r * w.v[d];
    U[4] = w.P * p.inv_gm1 + 0.5 * w.r * kin2(w);
}

// primitive state of U (FP64); a negative internal energy is floored to zero (returns true then).
// inv_r receives 1/rho.
__device__ __forceinline__ bool to_prim(const GasParams& p, const double U[5], Prim<double>& w, double& inv_r)
{
    w.r = U[0];
    inv_r = rcp(U[0]);
    for (int d = 0; d < 3; ++d) w.v[d] = U[1 + d] * inv_r;
    double e = U[4] - 0.5 * (U[1] * w.v[0] + U[2] * w.v[1] + U[3] * w.v[2]);
    const bool neg = e < 0.0;
    if (neg) e = 0.0;
    w.P = p.gm1 * e;
    return neg;
}

template <typename R, int D>
__device__ __forceinline__ void euler_flux(const Consts<R>& k, const Prim<R>& w, R F[5], R& E)
{
    const R u = w.v[D];
    E = w.P * k.inv_gm1 + R(0.5) * w.r * kin2(w);
    F[0] = w.r * u;
    for (int q = 0; q < 3; ++q) F[1 + q] = w.r * w.v[q] * u;
    F[1 + D] += w.P;
    F[4] = (E + w.P) * u;
}

template <typename R, int D>
__device__ void hllc(const Consts<R>& k, const Prim<R>& L, const Prim<R>& Rt, R F[5])
{
    const R irL = rcp(L.r), irR = rcp(Rt.r);
    const R aL = sqrt_fast(k.gamma * L.P * irL), aR = sqrt_fast(k.gamma * Rt.P * irR);
    const R uL = L.v[D], uR = Rt.v[D];
    const R SL = fmin(uL - aL, uR - aR), SR = fmax(uL + aL, uR + aR);
    R FL[5], FR[5], EL, ER;
    if (SL >= R(0)) {
        euler_flux<R, D>(k, L, F, EL);
        return;
    }
    if (SR <= R(0)) {
        euler_flux<R, D>(k, Rt, F, ER);
        return;
    }
    euler_flux<R, D>(k, L, FL, EL);
    euler_flux<R, D>(k, Rt, FR, ER);
    const R den = L.r * (SL - uL) - Rt.r * (SR - uR);
    if (den < R(0)) {
        const R Ss = (Rt.P - L.P + L.r * uL * (SL - uL) - Rt.r * uR * (SR - uR)) * rcp(den);
        const bool left = Ss >= R(0);
        const Prim<R>& K = left ? L : Rt;
        const R S = left ? SL : SR, EK = left ? EL : ER, uK = K.v[D], irK = left ? irL : irR;
        const R* FK = left ? FL : FR;
        const R chi = K.r * (S - uK) * rcp(S - Ss);
        R Us[5];
        Us[0] = chi;
        for (int q = 0; q < 3; ++q) Us[1 + q] = chi * K.v[q];
        Us[1 + D] = chi * Ss;
        Us[4] = chi * (EK * irK + (Ss - uK) * (Ss + K.P * irK * rcp(S - uK)));
        const R UK[5] = {K.r, K.r * K.v[0], K.r * K.v[1], K.r * K.v[2], EK};
        for (int q = 0; q < 5; ++q) F[q] = FK[q] + S * (Us[q] - UK[q]);
    } else {
        const R UL[5] = {L.r, L.r * L.v[0], L.r * L.v[1], L.r * L.v[2], EL};
        const R UR[5] = {Rt.r, Rt.r * Rt.v[0], Rt.r * Rt.v[1], Rt.r * Rt.v[2], ER};
        const R iw = rcp(SR - SL);
        for (int q = 0; q < 5; ++q) F[q] = (SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) * iw;
    }
}

template <typename R>
__device__ __forceinline__ R limited_slope(R dl, R dr, int lim)
{
    if (lim == 2) return R(0.5) * (dl + dr);  // no limiter
    if (dl * dr <= R(0)) return R(0);
    const R s = dl > R(0) ? R(1) : R(-1);
    const R m = fmin(fabs(dl), fabs(dr));
    if (lim == 0) return s * m;                          // minmod
    return s * fmin(R(2) * m, R(0.5) * fabs(dl + dr));  // monotonized central
}

__device__ __forceinline__ double absorption(const GasParams& p, const double* kF, long long i, double rho)
{
    if (kF) return kF[i];
    return p.kpow == 0 ? p.kappa_F : (p.kpow == 1 ? p.kappa_F * rho : (p.kappa_F * rho) * rho);
}

// S_e,gas rows of rho v and E_gas: k (G - (4/3) v E / c) and -k v.G (the terms with v only when beta tau is on)
__device__ __forceinline__ void gas_source(const GasParams& p, double k, const double v[3], double E, const double G[3],
                                           double S[5])
{
    S[0] = 0.0;
    if (p.beta_tau) {
        for (int d = 0; d < 3; ++d) S[1 + d] = k * (G[d] - (4.0 / 3.0) * v[d] * E * p.inv_c);
        S[4] = -k * (v[0] * G[0] + v[1] * G[1] + v[2] * G[2]);
    } else {
        for (int d = 0; d < 3; ++d) S[1 + d] = k * G[d];
        S[4] = 0.0;
    }
}

// split grids: the same sources in FP32 (k from the FP64 array truncated, or the law in FP32)
__device__ __forceinline__ float absorption32(const GasParams& p, const double* kF, long long i, float rho)
{
    if (kF) return d2f_trunc(kF[i]);
    return p.kpow == 0 ? p.f_kappa_F : (p.kpow == 1 ? p.f_kappa_F * rho : (p.f_kappa_F * rho) * rho);
}
__device__ __forceinline__ void gas_source32(const GasParams& p, float k, const float v[3], float E, const float G[3],
                                             float S[5])
{
    S[0] = 0.0f;
    if (p.beta_tau) {
        for (int d = 0; d < 3; ++d) S[1 + d] = k * (G[d] - (4.0f / 3.0f) * v[d] * E * p.f_inv_c);
        S[4] = -k * (v[0] * G[0] + v[1] * G[1] + v[2] * G[2]);
    } else {
        for (int d = 0; d < 3; ++d) S[1 + d] = k * G[d];
        S[4] = 0.0f;
    }
}

// Tests of FP64 values by their bits, on the integer pipes (an FP64 comparison occupies the FP64 pipe,
// which the split kernels otherwise leave to the accumulation): finite, and below zero (not -0, not NaN)
__device__ __forceinline__ bool finite_bits(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff; }
__device__ __forceinline__ bool below_zero_bits(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 && b != (long long)0x8000000000000000ull && finite_bits(x);
}

// Increments of the primitive variables from those of the conserved ones, D = (d rho, dMx, dMy, dMz,
// dE), at a state (r, v, T) in FP32: dv, dT and rho' = r + d rho (see the precision note above).
struct PrimInc {
    float r1, dv[3], dT;
};
__device__ __forceinline__ PrimInc prim_increment(const GasParams& p, float r, const float v[3], float T,
                                                  const float D[5])
{
    PrimInc o;
    o.r1 = r + D[0];
    const float inv = rcp(o.r1);
    float dK2 = 0.0f;  // 2 dK = M.dv + dM.v'
    for (int d = 0; d < 3; ++d) {
        o.dv[d] = (D[1 + d] - v[d] * D[0]) * inv;
        dK2 += r * v[d] * o.dv[d] + D[1 + d] * (v[d] + o.dv[d]);
    }
    o.dT = (p.f_gm1_mu * (D[4] - 0.5f * dK2) - T * D[0]) * inv;
    return o;
}

__device__ __forceinline__ bool finite_prim(const Prim<double>& w)
{
    return isfinite(w.r) && isfinite(w.v[0]) && isfinite(w.v[1]) && isfinite(w.v[2]) && isfinite(w.P);
}

__device__ __forceinline__ long long first_index() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long index_stride() { return (long long)gridDim.x * blockDim.x; }

// minus the divergence of the stored FP64 face fluxes (FP64 grids)
template <typename R>
__device__ __forceinline__ void flux_divergence(const GasParams& p, const GasArrays& a, const long long lo[3],
                                                const long long hi[3], double dU[5]);
template <>
__device__ __forceinline__ void flux_divergence<double>(const GasParams& p, const GasArrays& a, const long long lo[3],
                                                        const long long hi[3], double dU[5])
{
    for (int q = 0; q < 5; ++q) dU[q] = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (p.n[d] <= 1) continue;
        for (int q = 0; q < 5; ++q) dU[q] -= (a.flux[d][q][hi[d]] - a.flux[d][q][lo[d]]) * p.inv_dx[d];
    }
}

// split grids: minus the divergence of the stored FP32 face fluxes, in FP32
__device__ __forceinline__ void flux_divergence32(const GasParams& p, const GasArrays& a, const long long lo[3],
                                                  const long long hi[3], float dU[5])
{
    for (int q = 0; q < 5; ++q) dU[q] = 0.0f;
    for (int d = 0; d < 3; ++d) {
        if (p.n[d] <= 1) continue;
        for (int q = 0; q < 5; ++q) {
            const float* F = reinterpret_cast<const float*>(a.flux[d][q]);
            dU[q] -= (F[hi[d]] - F[lo[d]]) * p.f_inv_dx[d];
        }
    }
}

// ---------------------------------------------------------------------------------------- predictor

template <typename R, int D>
__global__ void __launch_bounds__(GAS_THREADS) gas_pred_flux_kernel(GasParams p, GasArrays a)
{
    int fe[3];
    gas_pred_faces(p, D, fe);
    const long long nf = gas_count(fe);
    const Consts<R> k = consts<R>(p);
    for (long long f = first_index(); f < nf; f += index_stride()) {
        long long iL, iR;
        int sL[3], sR[3];
        gas_pred_flux_cells(p, D, f, &iL, sL, &iR, sR);
        const Prim<R> WL = load_prim_t<R>(p, a, iL, sL), WR = load_prim_t<R>(p, a, iR, sR);
        R F[5];
        hllc<R, D>(k, WL, WR, F);
        for (int q = 0; q < 5; ++q) reinterpret_cast<R*>(a.flux[D][q])[f] = F[q];
    }
}

// split grids (R = float): memory-bound, so more resident warps (6 and 5 CTAs of 256 per SM) keep more loads
// in flight than the few registers they cost; FP64 grids: bound by the FP64 pipe
template <typename R>
__global__ void __launch_bounds__(GAS_THREADS, sizeof(R) == 4 ? 6 : 1) gas_pred_update_kernel(GasParams p, GasArrays a)
{
    const long long ne = gas_count(p.m);
    const double hdt = 0.5 * p.dt;
    unsigned long long floors = 0;
    if constexpr (sizeof(R) == 4) {
        // split grids: W^{n+1/2} in FP32 from the FP32 copies of W^n and FP32 increments
        const float fh = (float)hdt;
        for (long long i = first_index(); i < ne; i += index_stride()) {
            long long k, lo[3], hi[3];
            int s[3];
            bool inside;
            gas_pred_update_cells(p, i, &k, s, &inside, lo, hi);
            const float r = a.rho32[k], T = d2f_trunc(a.T[k]);
            const float v[3] = {flip(a.v32[0][k], s[0]), flip(a.v32[1][k], s[1]), flip(a.v32[2][k], s[2])};
            float dU[5], S[5];
            flux_divergence32(p, a, lo, hi, dU);
            const float G[3] = {flip(d2f_trunc(a.G[0][k]), s[0]), flip(d2f_trunc(a.G[1][k]), s[1]),
                                flip(d2f_trunc(a.G[2][k]), s[2])};
            gas_source32(p, absorption32(p, a.kF, k, r), v, d2f_trunc(a.E[k]), G, S);
            float D[5];
            for (int q = 0; q < 5; ++q) D[q] = fh * (dU[q] + S[q]);
            const PrimInc o = prim_increment(p, r, v, T, D);
            float Th = T + o.dT;
            if (Th < 0.0f) {
                Th = 0.0f;
                if (inside) ++floors;
            }
            a.wh32[0][i] = o.r1;
            for (int d = 0; d < 3; ++d) a.wh32[1 + d][i] = v[d] + o.dv[d];
            a.wh32[4][i] = o.r1 * Th * p.f_inv_mu;
        }
        if (floors) atomicAdd(&a.counters[0], floors);
    } else {
        for (long long i = first_index(); i < ne; i += index_stride()) {
            long long k, lo[3], hi[3];
            int s[3];
            bool inside;
            gas_pred_update_cells(p, i, &k, s, &inside, lo, hi);
            const Prim<double> W = load_prim(p, a, k, s);
            double U[5], dU[5];
            to_cons(p, W, U);
            flux_divergence<R>(p, a, lo, hi, dU);
            const double G[3] = {flip(a.G[0][k], s[0]), flip(a.G[1][k], s[1]), flip(a.G[2][k], s[2])};
            double S[5];
            gas_source(p, absorption(p, a.kF, k, W.r), W.v, a.E[k], G, S);
            double Uh[5], inv_r;
            for (int q = 0; q < 5; ++q) Uh[q] = U[q] + hdt * dU[q] + hdt * S[q];
            Prim<double> Wh;
            if (to_prim(p, Uh, Wh, inv_r) && inside) ++floors;
            const double w5[5] = {Wh.r, Wh.v[0], Wh.v[1], Wh.v[2], Wh.P};
            for (int q = 0; q < 5; ++q) a.wh[q][i] = w5[q];
        }
        if (floors) atomicAdd(&a.counters[0], floors);
    }
}

// ---------------------------------------------------------------------------------------- corrector

template <typename R>
__device__ __forceinline__ R load_half(const GasArrays& a, int q, long long x);
template <>
__device__ __forceinline__ double load_half<double>(const GasArrays& a, int q, long long x)
{
    return a.wh[q][x];
}
template <>
__device__ __forceinline__ float load_half<float>(const GasArrays& a, int q, long long x)
{
    return a.wh32[q][x];
}

template <typename R, int D>
__global__ void __launch_bounds__(GAS_THREADS) gas_corr_flux_kernel(GasParams p, GasArrays a)
{
    int fe[3];
    gas_corr_faces(p, D, fe);
    const long long nf = gas_count(fe);
    const Consts<R> k = consts<R>(p);
    for (long long f = first_index(); f < nf; f += index_stride()) {
        // W^{n+1/2} of the cells f - 2 e_D .. f + e_D
        long long x[4];
        gas_corr_flux_cells(p, D, f, x);
        R w[4][5];
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 5; ++q) w[j][q] = load_half<R>(a, q, x[j]);
        // limited slopes of the cells on each side of the face; a slope whose face values have
        // rho <= 0 or P <= 0 is zeroed (all components)
        Prim<R> WL, WR;
        for (int side = 0; side < 2; ++side) {
            const R* wm = w[side];
            const R* w0 = w[side + 1];
            const R* wp = w[side + 2];
            R sl[5];
            for (int q = 0; q < 5; ++q) sl[q] = limited_slope<R>(w0[q] - wm[q], wp[q] - w0[q], p.limiter);
            bool bad = false;
            for (int hs = 0; hs < 2; ++hs) {
                const R sg = hs ? R(0.5) : R(-0.5);
                bad = bad || !(w0[0] + sg * sl[0] > R(0)) || !(w0[4] + sg * sl[4] > R(0));
            }
            if (bad)
                for (int q = 0; q < 5; ++q) sl[q] = R(0);
            Prim<R>& W = side ? WR : WL;
            const R h = side ? R(-0.5) : R(0.5);  // cell f - e_D: its high face; cell f: its low face
            W.r = w0[0] + h * sl[0];
            for (int q = 0; q < 3; ++q) W.v[q] = w0[1 + q] + h * sl[1 + q];
            W.P = w0[4] + h * sl[4];
        }
        R F[5];
        hllc<R, D>(k, WL, WR, F);
        for (int q = 0; q < 5; ++q) reinterpret_cast<R*>(a.flux[D][q])[f] = F[q];
    }
}

template <typename R>
__global__ void __launch_bounds__(GAS_THREADS, sizeof(R) == 4 ? 5 : 1) gas_corr_update_kernel(GasParams p, GasArrays a)
{
    const long long nc = gas_count(p.n);
    unsigned long long floors = 0, bad = 0;
    if constexpr (sizeof(R) == 4) {
        // split grids: FP32 increments (fluxes, sources at W^{n+1/2}) accumulated into the FP64 state
        const float fdt = (float)p.dt;
        for (long long i = first_index(); i < nc; i += index_stride()) {
            long long x, lo[3], hi[3];
            gas_corr_update_cells(p, i, &x, lo, hi);
            const double rho = a.rho[i], T = a.T[i];
            const double v[3] = {a.v[0][i], a.v[1][i], a.v[2][i]};
            const float v32[3] = {d2f_trunc(v[0]), d2f_trunc(v[1]), d2f_trunc(v[2])};
            float dU[5], S[5];
            flux_divergence32(p, a, lo, hi, dU);
            const float rh = a.wh32[0][x];
            const float vh[3] = {a.wh32[1][x], a.wh32[2][x], a.wh32[3][x]};
            const float kh = absorption32(p, a.kF, i, rh);
            const double E = a.E[i];
            const double G[3] = {a.G[0][i], a.G[1][i], a.G[2][i]};
            const float G32[3] = {d2f_trunc(G[0]), d2f_trunc(G[1]), d2f_trunc(G[2])};
            gas_source32(p, kh, vh, d2f_trunc(E), G32, S);
            float D[5];
            for (int q = 0; q < 5; ++q) D[q] = fdt * (dU[q] + S[q]);
            const PrimInc o = prim_increment(p, d2f_trunc(rho), v32, d2f_trunc(T), D);
            const double rho1 = rho + f2d_exact(D[0]);
            double T1 = T + f2d_exact(o.dT);
            if (below_zero_bits(T1)) {
                T1 = 0.0;
                ++floors;
            }
            double v1[3];
            for (int d = 0; d < 3; ++d) v1[d] = v[d] + f2d_exact(o.dv[d]);
            if (!(finite_bits(rho1) && finite_bits(v1[0]) && finite_bits(v1[1]) && finite_bits(v1[2]) &&
                  finite_bits(T1)))
                ++bad;
            a.rho[i] = rho1;
            for (int d = 0; d < 3; ++d) a.v[d][i] = v1[d];
            a.T[i] = T1;
            a.pend[0][i] = f2d_exact(kh);
            for (int d = 0; d < 3; ++d) a.pend[1 + d][i] = f2d_exact(vh[d]);
            a.pend[4][i] = E;
            for (int d = 0; d < 3; ++d) a.pend[5 + d][i] = G[d];
        }
        if (floors) atomicAdd(&a.counters[0], floors);
        if (bad) atomicAdd(&a.counters[1], bad);
    } else {
        for (long long i = first_index(); i < nc; i += index_stride()) {
            long long x, lo[3], hi[3];
            gas_corr_update_cells(p, i, &x, lo, hi);
            const int one[3] = {1, 1, 1};
            const Prim<double> W = load_prim(p, a, i, one);
            double U[5], dU[5];
            to_cons(p, W, U);
            flux_divergence<R>(p, a, lo, hi, dU);
            const double rh = a.wh[0][x];
            const double vh[3] = {a.wh[1][x], a.wh[2][x], a.wh[3][x]};
            const double kh = absorption(p, a.kF, i, rh);
            const double E = a.E[i];
            const double G[3] = {a.G[0][i], a.G[1][i], a.G[2][i]};
            double S[5];
            gas_source(p, kh, vh, E, G, S);
            double U1[5], inv_r;
            for (int q = 0; q < 5; ++q) U1[q] = U[q] + p.dt * dU[q] + p.dt * S[q];
            Prim<double> W1;
            if (to_prim(p, U1, W1, inv_r)) ++floors;
            if (!finite_prim(W1)) ++bad;
            a.rho[i] = W1.r;
            for (int d = 0; d < 3; ++d) a.v[d][i] = W1.v[d];
            a.T[i] = W1.P * p.mu_over_kB * inv_r;
            a.pend[0][i] = kh;
            for (int d = 0; d < 3; ++d) a.pend[1 + d][i] = vh[d];
            a.pend[4][i] = E;
            for (int d = 0; d < 3; ++d) a.pend[5 + d][i] = G[d];
        }
        if (floors) atomicAdd(&a.counters[0], floors);
        if (bad) atomicAdd(&a.counters[1], bad);
    }
}

// ---------------------------------------------------------------------------------------- correction

template <bool SPLIT>
__global__ void __launch_bounds__(GAS_THREADS) gas_correct_kernel(GasParams p, GasArrays a)
{
    const long long nc = gas_count(p.n);
    const double hdt = 0.5 * p.dt;
    unsigned long long floors = 0, bad = 0;
    if constexpr (SPLIT) {
        // split grids: the change of the sources in FP32 (the radiation's change as the difference of its
        // FP32 copies: its error is that of the FP32 sources themselves), its momentum and energy
        // increments accumulated into the FP64 state
        const float fh = (float)hdt;
        for (long long i = first_index(); i < nc; i += index_stride()) {
            const double rho = a.rho[i], T = a.T[i];
            const double v[3] = {a.v[0][i], a.v[1][i], a.v[2][i]};
            const float v32[3] = {d2f_trunc(v[0]), d2f_trunc(v[1]), d2f_trunc(v[2])};
            const float kh = d2f_trunc(a.pend[0][i]);
            const float vh[3] = {d2f_trunc(a.pend[1][i]), d2f_trunc(a.pend[2][i]), d2f_trunc(a.pend[3][i])};
            float dG[3];
            for (int d = 0; d < 3; ++d) dG[d] = d2f_trunc(a.G[d][i]) - d2f_trunc(a.pend[5 + d][i]);
            float dS[5];
            gas_source32(p, kh, vh, d2f_trunc(a.E[i]) - d2f_trunc(a.pend[4][i]), dG, dS);
            const float D[5] = {0.0f, fh * dS[1], fh * dS[2], fh * dS[3], fh * dS[4]};
            const PrimInc o = prim_increment(p, d2f_trunc(rho), v32, d2f_trunc(T), D);
            double T1 = T + f2d_exact(o.dT);
            if (below_zero_bits(T1)) {
                T1 = 0.0;
                ++floors;
            }
            double v1[3];
            for (int d = 0; d < 3; ++d) v1[d] = v[d] + f2d_exact(o.dv[d]);
            if (!(finite_bits(v1[0]) && finite_bits(v1[1]) && finite_bits(v1[2]) && finite_bits(T1))) ++bad;
            for (int d = 0; d < 3; ++d) a.v[d][i] = v1[d];
            a.T[i] = T1;
        }
        if (floors) atomicAdd(&a.counters[0], floors);
        if (bad) atomicAdd(&a.counters[1], bad);
    } else {
        for (long long i = first_index(); i < nc; i += index_stride()) {
            const int one[3] = {1, 1, 1};
            const Prim<double> W = load_prim(p, a, i, one);
            double U[5];
            to_cons(p, W, U);
            // S_e,gas is linear in the radiation state: S(W^{n+1/2}, U_rad^{n+1}) - S(W^{n+1/2}, U_rad^n) is S of
            // the radiation's change
            const double kh = a.pend[0][i];
            const double vh[3] = {a.pend[1][i], a.pend[2][i], a.pend[3][i]};
            const double dG[3] = {a.G[0][i] - a.pend[5][i], a.G[1][i] - a.pend[6][i], a.G[2][i] - a.pend[7][i]};
            double dS[5];
            gas_source(p, kh, vh, a.E[i] - a.pend[4][i], dG, dS);
            for (int q = 1; q < 5; ++q) U[q] = U[q] + hdt * dS[q];
            Prim<double> W1;
            double inv_r;
            if (to_prim(p, U, W1, inv_r)) ++floors;
            if (!finite_prim(W1)) ++bad;
            for (int d = 0; d < 3; ++d) a.v[d][i] = W1.v[d];
            a.T[i] = W1.P * p.mu_over_kB * inv_r;
        }
        if (floors) atomicAdd(&a.counters[0], floors);
        if (bad) atomicAdd(&a.counters[1], bad);
    }
}

int blocks_for(long long n)
{
    const long long b = (n + GAS_THREADS - 1) / GAS_THREADS;
    return (int)(b < 1 ? 1 : (b > (1LL << 30) ? (1LL << 30) : b));
}

template <typename R>
void pred_flux(const GasParams& p, const GasArrays& a, int d, int nb, cudaStream_t s)
{
    if (d == 0) gas_pred_flux_kernel<R, 0><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else if (d == 1) gas_pred_flux_kernel<R, 1><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else gas_pred_flux_kernel<R, 2><<<nb, GAS_THREADS, 0, s>>>(p, a);
}

template <typename R>
void corr_flux(const GasParams& p, const GasArrays& a, int d, int nb, cudaStream_t s)
{
    if (d == 0) gas_corr_flux_kernel<R, 0><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else if (d == 1) gas_corr_flux_kernel<R, 1><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else gas_corr_flux_kernel<R, 2><<<nb, GAS_THREADS, 0, s>>>(p, a);
}

}  // namespace

cudaError_t launch_gas_pred_flux(const GasParams& p, const GasArrays& a, int d, cudaStream_t s)
{
    int e[3];
    gas_pred_faces(p, d, e);
    const int nb = blocks_for(gas_count(e));
    if (p.split) pred_flux<float>(p, a, d, nb, s);
    else pred_flux<double>(p, a, d, nb, s);
    return cudaGetLastError();
}

cudaError_t launch_gas_pred_update(const GasParams& p, const GasArrays& a, cudaStream_t s)
{
    const int nb = blocks_for(gas_count(p.m));
    if (p.split) gas_pred_update_kernel<float><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else gas_pred_update_kernel<double><<<nb, GAS_THREADS, 0, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_gas_corr_flux(const GasParams& p, const GasArrays& a, int d, cudaStream_t s)
{
    int e[3];
    gas_corr_faces(p, d, e);
    const int nb = blocks_for(gas_count(e));
    if (p.split) corr_flux<float>(p, a, d, nb, s);
    else corr_flux<double>(p, a, d, nb, s);
    return cudaGetLastError();
}

cudaError_t launch_gas_corr_update(const GasParams& p, const GasArrays& a, cudaStream_t s)
{
    const int nb = blocks_for(gas_count(p.n));
    if (p.split) gas_corr_update_kernel<float><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else gas_corr_update_kernel<double><<<nb, GAS_THREADS, 0, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_gas_correct(const GasParams& p, const GasArrays& a, cudaStream_t s)
{
    if (p.split) gas_correct_kernel<true><<<blocks_for(gas_count(p.n)), GAS_THREADS, 0, s>>>(p, a);
    else gas_correct_kernel<false><<<blocks_for(gas_count(p.n)), GAS_THREADS, 0, s>>>(p, a);
    return cudaGetLastError();
}

}  // namespace rhd
