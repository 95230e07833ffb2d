// rhd_internal.h -- types shared by the host runtime and the kernels of librhd.so (not public).
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (types only; the library does not link libcuda)
#include <cuda_runtime.h>

#include <mutex>

namespace rhd {

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2, BC_DIRICHLET = 3 };
enum { EX_FULL = 0, EX_ABSORB = 1, EX_EQUILIBRIUM = 2, EX_FROZEN_T = 3, EX_LINEAR = 4 };
enum { LIM_MINMOD = 0, LIM_MC = 1, LIM_NONE = 2 };

// Device-side event counters of the subcycles (zeroed by a reset).
struct DevStats {
    unsigned long long n_fix;
    unsigned long long n_face;
    unsigned long long n_theta;
    unsigned long long n_newton_fb;
    unsigned long long n_nonfinite;
    unsigned int newton_iter_max;
    unsigned int n_timeout;     // bounded waits that ran out (the tile's work was abandoned)
};

// Per-grid constants of one subcycle launch.
struct GridParams {
    int n[3];
    int nact;                   // number of active directions (they are x, then y, then z)
    double inv_dx[3];
    int bc_lo[3], bc_hi[3];
    double dir_lo[3][4];        // Dirichlet states (E, Gx, Gy, Gz), G = F/c
    double dir_hi[3][4];
    double c, a_rad, gamma, mu_over_kB;
    double theta_F, theta_E, E_floor;
    double kappa_P, kappa_F;
    double linear_eps;          // EX_LINEAR: retardation eps = 4 a_R / alpha of the material c_v = alpha T^3
    int kpow;
    int exchange, beta_tau, limiter, closure, speeds;
    // derived on the host: 1/c, (gamma - 1) mu/k_B and its inverse, 1/(eps c) and 1/a_R of the linear
    // exchange, and FP32 copies used by the split path
    double inv_c, gm1_mu, inv_gm1_mu, inv_eps_c, inv_a_rad;
    float f_inv_c, f_gm1_mu, f_c, f_a_rad, f_theta_F, f_theta_E, f_E_floor, f_kappa_P, f_kappa_F;
    float f_inv_dx[3];
    // two-pass split path: ghost layers of U^{m+1/2} stored per direction, 2, or 0 where both faces are
    // periodic (a periodic ghost value is the wrapped interior value, computed from the same cells)
    int pad[3];
};

// extent of the stored U^{m+1/2} in direction d (two-pass split path)
__host__ __device__ inline int upad_extent(const GridParams& g, int d) { return g.n[d] + 2 * g.pad[d]; }

// Device arrays of one grid.  FP32 copies of the frozen inputs are used by the split path.
struct GridArrays {
    const double* E;            // U^m
    const double* G[3];
    double* Eo;                 // U^{m+1}
    double* Go[3];
    double* T;                  // gas temperature: read (FROZEN_T), read+write in place (FULL)
    const double* rho;
    const double* v[3];         // NULL: zero velocity
    const double* kP;           // NULL: opacity law
    const double* kF;
    const double* j;            // NULL: no emissivity
    const float* rho32;
    const float* v32[3];
    const float* kP32;
    const float* kF32;
    const float* j32;
    // two-pass split path only (else NULL):
    float4* um32;               // U^m as FP32 (each component truncated toward zero): read by the predictor,
                                // rewritten with U^{m+1} by the corrector
    const float4* gas4;         // (rho, vx, vy, vz) as FP32 per cell (the FP32 gas copies interleaved)
    const double* dir_dev;      // non-NULL: the low x face's Dirichlet state (E, Gx, Gy, Gz) in device memory,
                                // written by a kernel before each subcycle (fused kernels; else NULL)
};

struct StepParams {
    GridParams g;
    GridArrays a;
    double chat, dt;
    float f_chat, f_dt;         // FP32 copies: FP32 code reads them as constant operands (no conversion)
    float4* uhalf;              // two-pass split path: U^{m+1/2} on the grid plus its ghost layers (pad[])
    int z_chunk;                // planes per CTA
    int tx, ty;                 // tile shape (selects the kernel instantiation)
    int tiles_x, tiles_y;       // tile grid in x, y
    int staging;                // two-pass corrector: 0 per-thread cp.async, 1 one TMA tile copy per plane
    unsigned wait_polls;        // TMA staging: polls of each plane's mbarrier wait before the tile gives up
    DevStats* stats;
    CUtensorMap uh_map;         // staging 1: tensor map of uhalf as floats {4 (n0+4), n1+4, n2+4}, box {4 (32+4), 8+4, 1}
};

// The exchange once per gas step (rhd_gas_exchange): the current state and the gas, updated in place.
struct GasExchangeParams {
    GridParams g;               // exchange parameters (theta_E, a_rad, gamma, mu_over_kB, E_floor, kappa law)
    double* E;
    double* G[3];
    double* T;
    const double* rho;
    const double* kP;           // NULL: the opacity law
    double chat, dt;
    long long n;
    DevStats* stats;
};

// Ensemble work items: (grid, tile) pairs handed out by a global counter.
struct EnsembleGrid {
    GridParams g;
    GridArrays a;
    double dt;
    float f_dt;
    int tiles_x, tiles_y, tiles_z;
    long long first_item;       // prefix sum of tiles over the grids before this one
    // two-pass ensembles: U^{m+1/2} of this grid (with its ghost layers, pad[]) and the
    // predictor's tiles over that array, with their prefix sum
    float4* uhalf;
    int ptiles_x, ptiles_y, ptiles_z;
    long long first_pitem;
};

struct EnsembleParams {
    const EnsembleGrid* grids;  // device array
    int n_grids;
    long long n_items;          // corrector (or fused) work items
    long long n_pitems;         // predictor work items (two-pass)
    double chat;
    float f_chat;
    int z_chunk;
    int limiter;                // shared by all grids (the two-pass corrector is instantiated per limiter)
    unsigned long long* counter;  // work-queue head, reset before each launch
    DevStats* stats;
};

// Raises a kernel's dynamic shared-memory limit once per (kernel, device) (a driver call, so not on every
// launch).  One instance per launch site, which may choose among a few kernels of one size.
struct SmemLimitOnce {
    std::mutex m;
    const void* fn[16] = {};
    int dev_of[16] = {};
    int n = 0;
    template <typename K>
    cudaError_t set(K k, size_t smem)
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
        const void* f = reinterpret_cast<const void*>(k);
        std::lock_guard<std::mutex> lock(m);
        for (int i = 0; i < n; ++i)
            if (fn[i] == f && dev_of[i] == dev) return cudaSuccess;
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && dev >= 0 && n < 16) {
            fn[n] = f;
            dev_of[n] = dev;
            ++n;
        }
        return e;
    }
};

// Launch wrappers (defined in the kernel translation units).
cudaError_t launch_subcycle_fp64(const StepParams& p, cudaStream_t s);
cudaError_t launch_subcycle_split(const StepParams& p, cudaStream_t s);
cudaError_t launch_twopass_split(const StepParams& p, cudaStream_t s);
cudaError_t launch_twopass_predictor(const StepParams& p, cudaStream_t s);
cudaError_t launch_twopass_corrector(const StepParams& p, cudaStream_t s);
bool tma_available();  // tensor-map staging of the two-pass corrector can be used on this device
// FP32 mirror of the FP64 state (E, G): dst[i] = truncation toward zero of each component
cudaError_t launch_to_um32(float4* dst, const double* E, const double* G0, const double* G1, const double* G2,
                           long long n, cudaStream_t s);
// interleaved FP32 gas: dst[i] = (rho32[i], vx[i], vy[i], vz[i]), absent velocity components zero
cudaError_t launch_to_gas4(float4* dst, const float* rho32, const float* vx, const float* vy, const float* vz,
                           long long n, cudaStream_t s);
// Encode the corrector's tensor map over a stored U^{m+1/2} array (ghost layers in x and y); false if the driver entry point is
// missing or the encoding is refused.
bool encode_uhalf_map(CUtensorMap* map, float4* uhalf, const GridParams& g);
cudaError_t launch_ensemble_fp64(const EnsembleParams& p, int n_ctas, cudaStream_t s);
cudaError_t launch_gas_exchange(const GasExchangeParams& p, int num_sms, cudaStream_t s);
cudaError_t launch_ensemble_split(const EnsembleParams& p, int n_ctas, cudaStream_t s);
int ensemble_ctas_per_sm_fp64();
int ensemble_ctas_per_sm_split();
cudaError_t launch_ensemble_predictor(const EnsembleParams& p, int n_ctas, cudaStream_t s);
cudaError_t launch_ensemble_corrector(const EnsembleParams& p, int n_ctas, cudaStream_t s);
int ensemble_ctas_per_sm_predictor();
int ensemble_ctas_per_sm_corrector();

// Tile geometry: the default per precision and dimensionality, and the shapes compiled for 3D.
void tile_shape(int precision, int nact, int* tx, int* ty);
void ensemble_tile_shape(int precision, int* tx, int* ty);  // the fused ensemble kernels' tile (3D)
bool tile_supported(int precision, int nact, int tx, int ty);

// Auxiliary kernels (k_aux.cu).
cudaError_t launch_scale_copy(double* dst, const double* src, double scale, long long n, cudaStream_t s);
cudaError_t launch_to_float(float* dst, const double* src, long long n, cudaStream_t s);
cudaError_t launch_reduce_state(const double* E, const double* G0, const double* G1, const double* G2,
                                long long n, double* partials, int n_blocks, cudaStream_t s);
cudaError_t launch_reduce_finish(const double* partials, int n_blocks, double* out5, cudaStream_t s);
// out-of-range index records of the kernel modules (nonzero only in the debug build, RHD_BOUNDS_CHECK):
// the count and the source line, index and extent (-1: grid coordinates packed by lin) of the first
struct OobRecord {
    unsigned long long count;
    int line, pad;
    long long index, extent;
};
cudaError_t oob_read_fp64(OobRecord* out, int reset, cudaStream_t s);
cudaError_t oob_read_split(OobRecord* out, int reset, cudaStream_t s);
bool bounds_checked_fp64();
bool bounds_checked_split();
// Marshak boundary (k_aux.cu): block m writes (E, F/c, 0, 0) of the low x face at
// tau = tau_rate (t0 + (m + 1/2) dt) into out[4 m .. 4 m + 3], m < n_steps
cudaError_t launch_marshak_boundary(double t0, double dt, double tau_rate, double eps, double F_inc, double c,
                                    int n_quad, int n_steps, double* out, cudaStream_t s);
// reduced-speed-of-light helpers (k_rsla.cu): maxima over the grid into partial[nb] (partial holds nb + 1)
int rsla_blocks(int num_sms);
cudaError_t launch_signal_speed(const GridParams& g, const double* rho, const double* T, const double* E,
                                const double* const v[3], const double* kF, double dx_min, long long n, int nb,
                                double* partial, cudaStream_t s);
cudaError_t launch_max_optical_depth(const GridParams& g, const double* kF, const double* rho, const double dx[3],
                                     int nb, double* partial, cudaStream_t s);
int reduce_blocks_for(long long n);

}  // namespace rhd
