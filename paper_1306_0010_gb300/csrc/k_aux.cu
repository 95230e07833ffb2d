// k_aux.cu -- auxiliary kernels of librhd.so: F <-> G = F/c conversion, FP32 copies of the frozen
// inputs for the split path, and a deterministic reduction of the state for the statistics.
#include <cuda_runtime.h>
#include <math.h>

#include "rhd_internal.h"

namespace rhd {

// dst = src / c (divide = 1) or dst = src * c (divide = 0); dst may alias src.
__global__ void scale_copy_kernel(double* dst, const double* src, double c, int divide, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = divide ? src[i] / c : src[i] * c;
}

cudaError_t launch_scale_copy(double* dst, const double* src, double scale, long long n, cudaStream_t s)
{
    // scale > 0: divide by scale; scale < 0: multiply by -scale
    if (n <= 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    scale_copy_kernel<<<blocks, 256, 0, s>>>(dst, src, scale > 0 ? scale : -scale, scale > 0 ? 1 : 0, n);
    return cudaGetLastError();
}

__global__ void to_float_kernel(float* dst, const double* src, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = (float)src[i];
}

cudaError_t launch_to_float(float* dst, const double* src, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    to_float_kernel<<<blocks, 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

// Block b sums the fixed range [b*chunk, (b+1)*chunk) in a fixed order (per-thread strided sums,
// then a fixed tree), so the result does not depend on timing.
constexpr int RED_THREADS = 256;

__global__ void reduce_state_kernel(const double* E, const double* G0, const double* G1, const double* G2,
                                    long long n, long long chunk, double* partials)
{
    __shared__ double sh[5][RED_THREADS];
    long long beg = (long long)blockIdx.x * chunk;
    long long end = beg + chunk < n ? beg + chunk : n;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    double mf = 0.0;
    for (long long i = beg + threadIdx.x; i < end; i += RED_THREADS) {
        double e = E[i], a = G0[i], b = G1[i], c = G2[i];
        s[0] += e;
        s[1] += a;
        s[2] += b;
        s[3] += c;
        double f = sqrt(a * a + b * b + c * c) / e;
        mf = f > mf ? f : mf;
    }
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = s[q];
    sh[4][threadIdx.x] = mf;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 5) partials[(long long)blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void reduce_finish_kernel(const double* partials, int nb, double* out5)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0}, mf = 0.0;
    for (int b = 0; b < nb; ++b) {
        for (int q = 0; q < 4; ++q) s[q] += partials[b * 5 + q];
        mf = fmax(mf, partials[b * 5 + 4]);
    }
    for (int q = 0; q < 4; ++q) out5[q] = s[q];
    out5[4] = mf;
}

int reduce_blocks_for(long long n)
{
    long long b = (n + (1 << 16) - 1) >> 16;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

cudaError_t launch_reduce_state(const double* E, const double* G0, const double* G1, const double* G2, long long n,
                                double* partials, int n_blocks, cudaStream_t s)
{
    long long chunk = (n + n_blocks - 1) / n_blocks;
    reduce_state_kernel<<<n_blocks, RED_THREADS, 0, s>>>(E, G0, G1, G2, n, chunk, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce_finish(const double* partials, int n_blocks, double* out5, cudaStream_t s)
{
    reduce_finish_kernel<<<1, 32, 0, s>>>(partials, n_blocks, out5);
    return cudaGetLastError();
}

// Low x face of the non-equilibrium Marshak wave (Section 4.1.4) for a run of subcycles, one block per
// subcycle m at tau = tau_rate (t0 + (m + 1/2) dt): the Su & Olson surface value u(0, tau) of
// Eq. (marshak:suolson) at chi = 0, its two integrals by the midpoint rule over n points (thread-strided
// partial sums, then a fixed tree), E = 4 F_inc u / c and F from c E + 2 F = 4 F_inc (Eq. marshak:bc_ix1);
// out[4 m ..] = (E, F / c, 0, 0), the solver's (E, G) of the Dirichlet ghost cells of that subcycle.
__global__ void marshak_boundary_kernel(double t0, double dt, double tau_rate, double eps, double F_inc, double c,
                                        int n, double* out_all)
{
    const double tau = tau_rate * (t0 + (blockIdx.x + 0.5) * dt);
    double* out = out_all + 4 * (long long)blockIdx.x;
    __shared__ double sh1[RED_THREADS], sh2[RED_THREADS];
    double s1 = 0.0, s2 = 0.0;
    for (int k = threadIdx.x; k < n; k += RED_THREADS) {
        const double eta = (k + 0.5) / n;
        const double g1 = eta * sqrt(eps + 1.0 / (1.0 - eta * eta));
        const double q1 = 3.0 + 4.0 * g1 * g1;
        s1 += exp(-tau * eta * eta) * sin(acos(sqrt(3.0 / q1))) / (eta * sqrt(q1));
        const double g2 = sqrt((1.0 - eta) * (eps + 1.0 / eta));
        const double q2 = 3.0 + 4.0 * g2 * g2;
        s2 += exp(-tau / (eps * eta)) * sin(acos(sqrt(3.0 / q2))) / (eta * (1.0 + eps * eta) * sqrt(q2));
    }
    sh1[threadIdx.x] = s1;
    sh2[threadIdx.x] = s2;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh1[threadIdx.x] += sh1[threadIdx.x + w];
            sh2[threadIdx.x] += sh2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double r3 = sqrt(3.0), pi = 3.14159265358979323846;
        const double u = 1.0 - (2.0 * r3 / pi) * sh1[0] / n - (r3 / pi) * exp(-tau) * sh2[0] / n;
        const double E = 4.0 * F_inc * u / c;
        out[0] = E;
        out[1] = ((4.0 * F_inc - c * E) / 2.0) / c;
        out[2] = 0.0;
        out[3] = 0.0;
    }
}

cudaError_t launch_marshak_boundary(double t0, double dt, double tau_rate, double eps, double F_inc, double c,
                                    int n_quad, int n_steps, double* out, cudaStream_t s)
{
    if (n_steps <= 0) return cudaSuccess;
    marshak_boundary_kernel<<<n_steps, RED_THREADS, 0, s>>>(t0, dt, tau_rate, eps, F_inc, c, n_quad, out);
    return cudaGetLastError();
}

}  // namespace rhd
