// The FP64 reciprocal of the kernels (Newton-Raphson on the hardware approximation) against CUDA's
// correctly rounded 1.0 / x: prints the largest distance in units in the last place over random
// values with exponents in [-1000, 1000] (reciprocals in the normal range) and a few exact cases.
// Built and run by tests/test_gpu_fp64_rcp.py.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "fp_convert.cuh"

__global__ void rcp_kernel(const double* x, double* mine, double* ieee, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        mine[i] = rhd::rcp(x[i]);
        ieee[i] = 1.0 / x[i];
    }
}

static int64_t bits(double v)
{
    int64_t b;
    std::memcpy(&b, &v, sizeof b);
    return b;
}

int main()
{
    const int n = 1 << 20;
    std::vector<double> x(n);
    std::mt19937_64 rng(1306);
    std::uniform_real_distribution<double> mant(1.0, 2.0);
    std::uniform_int_distribution<int> ex(-1000, 1000);
    for (int i = 0; i < n; ++i) x[i] = (i & 1 ? -1.0 : 1.0) * std::ldexp(mant(rng), ex(rng));
    const double exact[] = {1.0, 2.0, 0.5, 3.0, 0.1, 1.0 / 3.0, 7.0, 1e-300, 1e300, 1.5, 0.75};
    for (int i = 0; i < (int)(sizeof exact / sizeof exact[0]); ++i) x[i] = exact[i];
    double *dx, *dm, *di;
    if (cudaMalloc(&dx, n * sizeof(double)) || cudaMalloc(&dm, n * sizeof(double)) || cudaMalloc(&di, n * sizeof(double)))
        return 2;
    cudaMemcpy(dx, x.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    rcp_kernel<<<(n + 255) / 256, 256>>>(dx, dm, di, n);
    std::vector<double> m(n), r(n);
    if (cudaMemcpy(m.data(), dm, n * sizeof(double), cudaMemcpyDeviceToHost) ||
        cudaMemcpy(r.data(), di, n * sizeof(double), cudaMemcpyDeviceToHost))
        return 3;
    int64_t worst = 0, exact_misses = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t d = bits(m[i]) > bits(r[i]) ? bits(m[i]) - bits(r[i]) : bits(r[i]) - bits(m[i]);
        if (d > worst) worst = d;
        if (i < (int)(sizeof exact / sizeof exact[0]) && d != 0) ++exact_misses;
    }
    std::printf("max_ulp %lld exact_cases_off %lld\n", (long long)worst, (long long)exact_misses);
    cudaFree(dx);
    cudaFree(dm);
    cudaFree(di);
    return 0;
}
