// gas_internal.h -- device-side parameters and launchers of the gas step (k_gas.cu), shared with the
// host runtime (rhd_api.cu).  Not part of the public C ABI.
//
// The gas step advances (rho, rho v, E_gas) of the Euler equations with the explicit gas sources
// S_e,gas (Eq. algorithm:source:explicit:gas, no gravity) by one van Leer predictor / corrector step
// (Section 3.1 step 3, Section 3.4), and later corrects those sources to second order with the
// radiation at t^{n+1} (Section 3.1 step 6).
#pragma once

#include <cuda_runtime.h>

namespace rhd {

constexpr int GAS_GHOST = 2;  // ghost layers of W^{n+1/2} (the corrector's stencil spans i-2 .. i+1)

struct GasParams {
    int n[3];                 // interior cells per direction
    int g[3];                 // ghost layers of W^{n+1/2}: GAS_GHOST in active directions (n > 1), else 0
    int m[3];                 // extents of W^{n+1/2}: n + 2 g
    int bc_lo[3], bc_hi[3];   // rhd_bc of each face
    double inv_dx[3];
    double gamma, gm1, inv_gm1;   // gamma, gamma - 1, 1 / (gamma - 1)
    double mu_over_kB, inv_mu;    // P = rho T / (mu/k_B)
    double inv_c;
    double kappa_F;           // opacity law k_F = kappa_F rho^kpow where no kF array is given
    int kpow, beta_tau, limiter;
    double dt;
    // split grids: the face fluxes (reconstruction, wave speeds, HLLC), the sources and the increments
    // in FP32 with these FP32 copies; the state (rho, v, T) accumulates them in FP64
    int split;
    float f_gamma, f_inv_gm1, f_inv_mu, f_inv_dx[3];
    float f_gm1, f_gm1_mu, f_inv_gm1_mu, f_inv_c, f_kappa_F;  // gamma - 1, (gamma - 1) mu/k_B, its inverse
};

struct GasArrays {
    double* rho;              // gas at t^n (read), overwritten with t^{n+1} by the corrector
    double* T;
    double* v[3];             // all three components present
    const float* rho32;       // split grids: FP32 copies of rho and v (current with the FP64 state)
    const float* v32[3];
    const double* kF;         // NULL: the opacity law
    const double* E;          // radiation at t^n (step) or t^{n+1} (correction), G = F/c
    const double* G[3];
    double* wh[5];            // W^{n+1/2} = (rho, vx, vy, vz, P) on the extended grid m[0] x m[1] x m[2]
                              // (FP64 grids; NULL on split grids)
    float* wh32[5];           // split grids: W^{n+1/2} in FP32 (an intermediate of the step, like the
                              // radiation's U^{m+1/2})
    double* flux[3][5];       // face fluxes of direction d (predictor layout (m_d + 1) x m_e, corrector
                              // layout (n_d + 1) x n_e), components (rho, Mx, My, Mz, E_gas); FP32 values
                              // (the first half of each buffer) on split grids
    double* pend[8];          // kept for the correction: k_F(rho^{n+1/2}), v^{n+1/2} (3), E^n, G^n (3)
    unsigned long long* counters;  // [0] cells whose internal energy was floored to 0, [1] non-finite cells
};

// one gas step over p.dt is: launch_gas_pred_flux for each active direction, launch_gas_pred_update,
// launch_gas_corr_flux for each active direction, launch_gas_corr_update (all on one stream)
cudaError_t launch_gas_pred_flux(const GasParams& p, const GasArrays& a, int d, cudaStream_t s);
cudaError_t launch_gas_pred_update(const GasParams& p, const GasArrays& a, cudaStream_t s);
cudaError_t launch_gas_corr_flux(const GasParams& p, const GasArrays& a, int d, cudaStream_t s);
cudaError_t launch_gas_corr_update(const GasParams& p, const GasArrays& a, cudaStream_t s);
// the second-order source correction with the radiation in a.E, a.G (t^{n+1}) over p.dt
cudaError_t launch_gas_correct(const GasParams& p, const GasArrays& a, cudaStream_t s);

}  // namespace rhd
