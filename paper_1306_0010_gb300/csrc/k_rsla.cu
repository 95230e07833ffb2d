// k_rsla.cu -- grid reductions behind the reduced-speed-of-light helpers of librhd.so
// (Sections 3.1 and 3.2): the maximum gas signal speed v_max = max(|v| + c_eff) of
// Eq. algorithm:ceff, and the largest optical depth of the domain along the grid axes, which set
// Delta t_gas (Eq. algorithm:gastimestep) and the choice of chat (Eq. rsla:staticdiffreq).
//
// Every block reduces a fixed set of cells (or lines) to its maximum and a one-block kernel takes
// the maximum of the block results: the result does not depend on timing.  A NaN anywhere is
// carried to the result (the comparisons below keep it), so the host can report it.
#include <cuda_runtime.h>
#include <math.h>

#include "fp_convert.cuh"
#include "rhd_internal.h"

namespace rhd {

constexpr int RS_THREADS = 256;

// the larger of a, b, a NaN in either winning
__device__ __forceinline__ double max_nan(double a, double b) { return (b > a || b != b) ? b : a; }

// k_F of cell i: the per-cell array if given, else the opacity law kappa_F rho^p
__device__ __forceinline__ double flux_absorption(const GridParams& g, const double* kF, const double* rho,
                                                  long long i)
{
    if (kF) return kF[i];
    const double r = rho[i];
    return g.kpow == 0 ? g.kappa_F : (g.kpow == 1 ? g.kappa_F * r : (g.kappa_F * r) * r);
}

// block maximum of v into out[blockIdx.x]
__device__ __forceinline__ void block_max(double v, double* out)
{
    __shared__ double sh[RS_THREADS];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = RS_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = max_nan(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// v_max over the cells: |v| + sqrt((gamma P + (4/9) E (1 - exp(-k_F dx))) / rho) with P = rho T / (mu/k_B).
// The FP64 value (the result) costs an exponential, two square roots and two divisions on the FP64
// pipe; only the maximum matters, so each cell is first screened in FP32 (inputs truncated, relative
// error about 1e-6) and evaluated in FP64 only if its FP32 value is not below the thread's running FP32
// maximum by more than 2^-12, or is NaN or inf.  The cell holding the FP64 maximum always passes the
// screen, so the result is the FP64 maximum itself; FP32 underflow or overflow only sends more cells
// to the FP64 evaluation.
__global__ void __launch_bounds__(RS_THREADS) signal_speed_kernel(GridParams g, const double* rho, const double* T,
                                                                  const double* E, const double* v0, const double* v1,
                                                                  const double* v2, const double* kF, double dx_min,
                                                                  long long n, double* partial)
{
    const float gam = (float)g.gamma, inv_mu = (float)(1.0 / g.mu_over_kB), dxf = (float)dx_min;
    double m = 0.0;
    float m32 = 0.0f;
    for (long long i = (long long)blockIdx.x * RS_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * RS_THREADS) {
        const double r = rho[i], Ti = T[i], Ei = E[i], kFi = kF ? kF[i] : 0.0;
        const double a = v0 ? v0[i] : 0.0, b = v1 ? v1[i] : 0.0, c = v2 ? v2[i] : 0.0;
        const float rf = d2f_trunc(r), af = d2f_trunc(a), bf = d2f_trunc(b), cf = d2f_trunc(c);
        const float kf = kF ? d2f_trunc(kFi) : (g.kpow == 0 ? g.f_kappa_F : (g.kpow == 1 ? g.f_kappa_F * rf : (g.f_kappa_F * rf) * rf));
        const float Pf = rf * d2f_trunc(Ti) * inv_mu;
        const float radf = (4.0f / 9.0f) * d2f_trunc(Ei) * (-expm1f(-kf * dxf));
        const float s32 = sqrtf(af * af + bf * bf + cf * cf) + sqrtf((gam * Pf + radf) / rf);
        if (!(s32 < m32 * 0.999755859375f)) {
            m32 = fmaxf(m32, s32);
            const double k = kF ? kFi : flux_absorption(g, nullptr, rho, i);
            const double P = r * Ti / g.mu_over_kB;
            const double rad = (4.0 / 9.0) * Ei * (-expm1(-k * dx_min));
            m = max_nan(m, sqrt(a * a + b * b + c * c) + sqrt((g.gamma * P + rad) / r));
        }
    }
    block_max(m, partial);
}

// the largest sum of k_F dx_axis along the grid lines parallel to `axis` (cells indexed
// x + nx (y + ny z)); lines along y or z: one thread per line, consecutive threads on consecutive x;
// lines along x: one warp per line, lanes on strided x, then a fixed shuffle tree
__global__ void __launch_bounds__(RS_THREADS) line_depth_kernel(GridParams g, const double* kF, const double* rho,
                                                                int axis, double dx, double* partial)
{
    const long long nx = g.n[0], ny = g.n[1], nz = g.n[2];
    double m = 0.0;
    if (axis == 0) {
        const long long lines = ny * nz;
        const int lane = threadIdx.x & 31;
        const long long warp0 = ((long long)blockIdx.x * RS_THREADS + threadIdx.x) >> 5;
        const long long nwarps = ((long long)gridDim.x * RS_THREADS) >> 5;
        for (long long l = warp0; l < lines; l += nwarps) {
            double s = 0.0;
            for (long long x = lane; x < nx; x += 32) s += flux_absorption(g, kF, rho, l * nx + x);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            m = max_nan(m, s * dx);
        }
    } else {
        const long long lines = axis == 1 ? nx * nz : nx * ny;
        const long long len = axis == 1 ? ny : nz, step = axis == 1 ? nx : nx * ny;
        for (long long l = (long long)blockIdx.x * RS_THREADS + threadIdx.x; l < lines;
             l += (long long)gridDim.x * RS_THREADS) {
            const long long x = l % nx, o = l / nx;  // o: z (axis y) or y (axis z)
            long long i = axis == 1 ? x + nx * ny * o : x + nx * o;
            double s = 0.0;
            for (long long k = 0; k < len; ++k, i += step) s += flux_absorption(g, kF, rho, i);
            m = max_nan(m, s * dx);
        }
    }
    block_max(m, partial);
}

__global__ void max_finish_kernel(const double* partial, int nb, double* out)
{
    double m = 0.0;
    for (int i = threadIdx.x; i < nb; i += RS_THREADS) m = max_nan(m, partial[i]);
    __shared__ double sh[RS_THREADS];
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = RS_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = max_nan(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = max_nan(*out, sh[0]);
}

// blocks of every reduction launch (the partial buffer holds this many doubles + 1 for the result)
int rsla_blocks(int num_sms) { return num_sms * 4; }

cudaError_t launch_signal_speed(const GridParams& g, const double* rho, const double* T, const double* E,
                                const double* const v[3], const double* kF, double dx_min, long long n, int nb,
                                double* partial, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(partial + nb, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    signal_speed_kernel<<<nb, RS_THREADS, 0, s>>>(g, rho, T, E, v[0], v[1], v[2], kF, dx_min, n, partial);
    max_finish_kernel<<<1, RS_THREADS, 0, s>>>(partial, nb, partial + nb);
    return cudaGetLastError();
}

cudaError_t launch_max_optical_depth(const GridParams& g, const double* kF, const double* rho, const double dx[3],
                                     int nb, double* partial, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(partial + nb, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    for (int axis = 0; axis < 3; ++axis) {
        if (g.n[axis] <= 1) continue;
        line_depth_kernel<<<nb, RS_THREADS, 0, s>>>(g, kF, rho, axis, dx[axis], partial);
        max_finish_kernel<<<1, RS_THREADS, 0, s>>>(partial, nb, partial + nb);
    }
    return cudaGetLastError();
}

}  // namespace rhd
