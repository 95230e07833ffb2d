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
// update kernels take the flux differences.  Everything is FP64.  The HLLC solver (Toro, Riemann
// Solvers and Numerical Methods for Fluid Dynamics, Sec. 10.4) uses the Davis wave-speed estimates; the
// left star state when S* = 0; HLL where the contact speed's denominator is not negative.
#include <cuda_runtime.h>
#include <math.h>

#include "gas_index.h"
#include "gas_internal.h"

namespace rhd {

namespace {

constexpr int GAS_THREADS = 256;

struct Prim {
    double r, v[3], P;
};

__device__ __forceinline__ Prim load_prim(const GasParams& p, const GasArrays& a, long long i, const double s[3])
{
    Prim w;
    w.r = a.rho[i];
    for (int d = 0; d < 3; ++d) w.v[d] = a.v[d][i] * s[d];
    w.P = w.r * a.T[i] * p.inv_mu;
    return w;
}

__device__ __forceinline__ double kin2(const Prim& w)
{
    return w.v[0] * w.v[0] + w.v[1] * w.v[1] + w.v[2] * w.v[2];
}

// (rho, Mx, My, Mz, E_gas) of a primitive state
__device__ __forceinline__ void to_cons(const GasParams& p, const Prim& w, double U[5])
{
    U[0] = w.r;
    for (int d = 0; d < 3; ++d) U[1 + d] = w.r * w.v[d];
    U[4] = w.P * p.inv_gm1 + 0.5 * w.r * kin2(w);
}

// primitive state of U; a negative internal energy is floored to zero (returns true then)
__device__ __forceinline__ bool to_prim(const GasParams& p, const double U[5], Prim& w)
{
    w.r = U[0];
    for (int d = 0; d < 3; ++d) w.v[d] = U[1 + d] / U[0];
    double e = U[4] - 0.5 * (U[1] * w.v[0] + U[2] * w.v[1] + U[3] * w.v[2]);
    const bool neg = e < 0.0;
    if (neg) e = 0.0;
    w.P = p.gm1 * e;
    return neg;
}

template <int D>
__device__ __forceinline__ void euler_flux(const GasParams& p, const Prim& w, double F[5], double& E)
{
    const double u = w.v[D];
    E = w.P * p.inv_gm1 + 0.5 * w.r * kin2(w);
    F[0] = w.r * u;
    for (int k = 0; k < 3; ++k) F[1 + k] = w.r * w.v[k] * u;
    F[1 + D] += w.P;
    F[4] = (E + w.P) * u;
}

template <int D>
__device__ void hllc(const GasParams& p, const Prim& L, const Prim& R, double F[5])
{
    const double aL = sqrt(p.gamma * L.P / L.r), aR = sqrt(p.gamma * R.P / R.r);
    const double uL = L.v[D], uR = R.v[D];
    const double SL = fmin(uL - aL, uR - aR), SR = fmax(uL + aL, uR + aR);
    double FL[5], FR[5], EL, ER;
    if (SL >= 0.0) {
        euler_flux<D>(p, L, F, EL);
        return;
    }
    if (SR <= 0.0) {
        euler_flux<D>(p, R, F, ER);
        return;
    }
    euler_flux<D>(p, L, FL, EL);
    euler_flux<D>(p, R, FR, ER);
    const double den = L.r * (SL - uL) - R.r * (SR - uR);
    if (den < 0.0) {
        const double Ss = (R.P - L.P + L.r * uL * (SL - uL) - R.r * uR * (SR - uR)) / den;
        const bool left = Ss >= 0.0;
        const Prim& K = left ? L : R;
        const double S = left ? SL : SR, EK = left ? EL : ER, uK = K.v[D];
        const double* FK = left ? FL : FR;
        const double chi = K.r * (S - uK) / (S - Ss);
        double Us[5];
        Us[0] = chi;
        for (int k = 0; k < 3; ++k) Us[1 + k] = chi * K.v[k];
        Us[1 + D] = chi * Ss;
        Us[4] = chi * (EK / K.r + (Ss - uK) * (Ss + K.P / (K.r * (S - uK))));
        const double UK[5] = {K.r, K.r * K.v[0], K.r * K.v[1], K.r * K.v[2], EK};
        for (int q = 0; q < 5; ++q) F[q] = FK[q] + S * (Us[q] - UK[q]);
    } else {
        const double UL[5] = {L.r, L.r * L.v[0], L.r * L.v[1], L.r * L.v[2], EL};
        const double UR[5] = {R.r, R.r * R.v[0], R.r * R.v[1], R.r * R.v[2], ER};
        for (int q = 0; q < 5; ++q) F[q] = (SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) / (SR - SL);
    }
}

__device__ __forceinline__ double limited_slope(double dl, double dr, int lim)
{
    if (lim == 2) return 0.5 * (dl + dr);  // no limiter
    if (dl * dr <= 0.0) return 0.0;
    const double s = dl > 0.0 ? 1.0 : -1.0;
    const double x = fabs(dl), y = fabs(dr);
    const double m = fmin(x, y);
    if (lim == 0) return s * m;            // minmod
    return s * fmin(2.0 * m, 0.5 * fabs(dl + dr));  // monotonized central
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

__device__ __forceinline__ bool finite_prim(const Prim& w)
{
    return isfinite(w.r) && isfinite(w.v[0]) && isfinite(w.v[1]) && isfinite(w.v[2]) && isfinite(w.P);
}

__device__ __forceinline__ long long first_index() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long index_stride() { return (long long)gridDim.x * blockDim.x; }

// ---------------------------------------------------------------------------------------- predictor

template <int D>
__global__ void __launch_bounds__(GAS_THREADS) gas_pred_flux_kernel(GasParams p, GasArrays a)
{
    int fe[3];
    gas_pred_faces(p, D, fe);
    const long long nf = gas_count(fe);
    for (long long f = first_index(); f < nf; f += index_stride()) {
        long long iL, iR;
        double sL[3], sR[3];
        gas_pred_flux_cells(p, D, f, &iL, sL, &iR, sR);
        const Prim WL = load_prim(p, a, iL, sL), WR = load_prim(p, a, iR, sR);
        double F[5];
        hllc<D>(p, WL, WR, F);
        for (int q = 0; q < 5; ++q) a.flux[D][q][f] = F[q];
    }
}

__global__ void __launch_bounds__(GAS_THREADS) gas_pred_update_kernel(GasParams p, GasArrays a)
{
    const long long ne = gas_count(p.m);
    const double hdt = 0.5 * p.dt;
    unsigned long long floors = 0;
    for (long long i = first_index(); i < ne; i += index_stride()) {
        long long k, lo[3], hi[3];
        double s[3];
        bool inside;
        gas_pred_update_cells(p, i, &k, s, &inside, lo, hi);
        const Prim W = load_prim(p, a, k, s);
        double U[5], dU[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        to_cons(p, W, U);
        for (int d = 0; d < 3; ++d) {
            if (p.n[d] <= 1) continue;
            for (int q = 0; q < 5; ++q) dU[q] -= (a.flux[d][q][hi[d]] - a.flux[d][q][lo[d]]) * p.inv_dx[d];
        }
        const double G[3] = {a.G[0][k] * s[0], a.G[1][k] * s[1], a.G[2][k] * s[2]};
        double S[5];
        gas_source(p, absorption(p, a.kF, k, W.r), W.v, a.E[k], G, S);
        double Uh[5];
        for (int q = 0; q < 5; ++q) Uh[q] = U[q] + hdt * dU[q] + hdt * S[q];
        Prim Wh;
        if (to_prim(p, Uh, Wh) && inside) ++floors;
        a.wh[0][i] = Wh.r;
        for (int d = 0; d < 3; ++d) a.wh[1 + d][i] = Wh.v[d];
        a.wh[4][i] = Wh.P;
    }
    if (floors) atomicAdd(&a.counters[0], floors);
}

// ---------------------------------------------------------------------------------------- corrector

template <int D>
__global__ void __launch_bounds__(GAS_THREADS) gas_corr_flux_kernel(GasParams p, GasArrays a)
{
    int fe[3];
    gas_corr_faces(p, D, fe);
    const long long nf = gas_count(fe);
    for (long long f = first_index(); f < nf; f += index_stride()) {
        // W^{n+1/2} of the cells f - 2 e_D .. f + e_D
        long long x[4];
        gas_corr_flux_cells(p, D, f, x);
        double w[4][5];
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 5; ++q) w[j][q] = a.wh[q][x[j]];
        // limited slopes of the cells on each side of the face; a slope whose face values have
        // rho <= 0 or P <= 0 is zeroed (all components)
        Prim WL, WR;
        for (int side = 0; side < 2; ++side) {
            const double* wm = w[side];
            const double* w0 = w[side + 1];
            const double* wp = w[side + 2];
            double sl[5];
            for (int q = 0; q < 5; ++q) sl[q] = limited_slope(w0[q] - wm[q], wp[q] - w0[q], p.limiter);
            bool bad = false;
            for (int h = 0; h < 2; ++h) {
                const double sg = h ? 0.5 : -0.5;
                bad = bad || !(w0[0] + sg * sl[0] > 0.0) || !(w0[4] + sg * sl[4] > 0.0);
            }
            if (bad)
                for (int q = 0; q < 5; ++q) sl[q] = 0.0;
            Prim& W = side ? WR : WL;
            const double h = side ? -0.5 : 0.5;  // cell A - e_D: its high face; cell A: its low face
            W.r = w0[0] + h * sl[0];
            for (int k = 0; k < 3; ++k) W.v[k] = w0[1 + k] + h * sl[1 + k];
            W.P = w0[4] + h * sl[4];
        }
        double F[5];
        hllc<D>(p, WL, WR, F);
        for (int q = 0; q < 5; ++q) a.flux[D][q][f] = F[q];
    }
}

__global__ void __launch_bounds__(GAS_THREADS) gas_corr_update_kernel(GasParams p, GasArrays a)
{
    const long long nc = gas_count(p.n);
    unsigned long long floors = 0, bad = 0;
    for (long long i = first_index(); i < nc; i += index_stride()) {
        long long x, lo[3], hi[3];
        gas_corr_update_cells(p, i, &x, lo, hi);
        const double one[3] = {1.0, 1.0, 1.0};
        const Prim W = load_prim(p, a, i, one);
        double U[5], dU[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        to_cons(p, W, U);
        for (int d = 0; d < 3; ++d) {
            if (p.n[d] <= 1) continue;
            for (int q = 0; q < 5; ++q) dU[q] -= (a.flux[d][q][hi[d]] - a.flux[d][q][lo[d]]) * p.inv_dx[d];
        }
        const double rh = a.wh[0][x];
        const double vh[3] = {a.wh[1][x], a.wh[2][x], a.wh[3][x]};
        const double kh = absorption(p, a.kF, i, rh);
        const double E = a.E[i];
        const double G[3] = {a.G[0][i], a.G[1][i], a.G[2][i]};
        double S[5];
        gas_source(p, kh, vh, E, G, S);
        double U1[5];
        for (int q = 0; q < 5; ++q) U1[q] = U[q] + p.dt * dU[q] + p.dt * S[q];
        Prim W1;
        if (to_prim(p, U1, W1)) ++floors;
        if (!finite_prim(W1)) ++bad;
        a.rho[i] = W1.r;
        for (int d = 0; d < 3; ++d) a.v[d][i] = W1.v[d];
        a.T[i] = W1.P * p.mu_over_kB / W1.r;
        a.pend[0][i] = kh;
        for (int d = 0; d < 3; ++d) a.pend[1 + d][i] = vh[d];
        a.pend[4][i] = E;
        for (int d = 0; d < 3; ++d) a.pend[5 + d][i] = G[d];
    }
    if (floors) atomicAdd(&a.counters[0], floors);
    if (bad) atomicAdd(&a.counters[1], bad);
}

// ---------------------------------------------------------------------------------------- correction

__global__ void __launch_bounds__(GAS_THREADS) gas_correct_kernel(GasParams p, GasArrays a)
{
    const long long nc = gas_count(p.n);
    const double hdt = 0.5 * p.dt;
    unsigned long long floors = 0, bad = 0;
    for (long long i = first_index(); i < nc; i += index_stride()) {
        const double one[3] = {1.0, 1.0, 1.0};
        const Prim W = load_prim(p, a, i, one);
        double U[5];
        to_cons(p, W, U);
        const double kh = a.pend[0][i];
        const double vh[3] = {a.pend[1][i], a.pend[2][i], a.pend[3][i]};
        const double G1[3] = {a.G[0][i], a.G[1][i], a.G[2][i]};
        const double G0[3] = {a.pend[5][i], a.pend[6][i], a.pend[7][i]};
        double S1[5], S0[5];
        gas_source(p, kh, vh, a.E[i], G1, S1);
        gas_source(p, kh, vh, a.pend[4][i], G0, S0);
        for (int q = 1; q < 5; ++q) U[q] = U[q] + hdt * (S1[q] - S0[q]);
        Prim W1;
        if (to_prim(p, U, W1)) ++floors;
        if (!finite_prim(W1)) ++bad;
        for (int d = 0; d < 3; ++d) a.v[d][i] = W1.v[d];
        a.T[i] = W1.P * p.mu_over_kB / W1.r;
    }
    if (floors) atomicAdd(&a.counters[0], floors);
    if (bad) atomicAdd(&a.counters[1], bad);
}

int blocks_for(long long n)
{
    const long long b = (n + GAS_THREADS - 1) / GAS_THREADS;
    return (int)(b < 1 ? 1 : (b > (1LL << 30) ? (1LL << 30) : b));
}

}  // namespace

cudaError_t launch_gas_pred_flux(const GasParams& p, const GasArrays& a, int d, cudaStream_t s)
{
    int e[3];
    gas_pred_faces(p, d, e);
    const int nb = blocks_for(gas_count(e));
    if (d == 0) gas_pred_flux_kernel<0><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else if (d == 1) gas_pred_flux_kernel<1><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else gas_pred_flux_kernel<2><<<nb, GAS_THREADS, 0, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_gas_pred_update(const GasParams& p, const GasArrays& a, cudaStream_t s)
{
    gas_pred_update_kernel<<<blocks_for(gas_count(p.m)), GAS_THREADS, 0, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_gas_corr_flux(const GasParams& p, const GasArrays& a, int d, cudaStream_t s)
{
    int e[3];
    gas_corr_faces(p, d, e);
    const int nb = blocks_for(gas_count(e));
    if (d == 0) gas_corr_flux_kernel<0><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else if (d == 1) gas_corr_flux_kernel<1><<<nb, GAS_THREADS, 0, s>>>(p, a);
    else gas_corr_flux_kernel<2><<<nb, GAS_THREADS, 0, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_gas_corr_update(const GasParams& p, const GasArrays& a, cudaStream_t s)
{
    gas_corr_update_kernel<<<blocks_for(gas_count(p.n)), GAS_THREADS, 0, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_gas_correct(const GasParams& p, const GasArrays& a, cudaStream_t s)
{
    gas_correct_kernel<<<blocks_for(gas_count(p.n)), GAS_THREADS, 0, s>>>(p, a);
    return cudaGetLastError();
}

}  // namespace rhd
