// The FP64 reciprocal and inverse square root of the kernels (Newton-Raphson on the hardware
// approximations) against CUDA's correctly rounded 1.0 / x and 1.0 / sqrt(x): prints the largest
// distance in units in the last place over random values with exponents in [-1000, 1000] (results in
// the normal range) and a few exact cases, and that of x rsqrt(x) from sqrt(x) on [1, 4] (the range in
// which the closure uses it).  Built and run by tests/test_gpu_fp64_rcp.py.
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

// ax = |x|: 1/sqrt(ax) both ways; y = 1 + 3 frac(ax) in [1, 4): y rsqrt(y) against sqrt(y)
__global__ void rsqrt_kernel(const double* x, double* mine, double* ieee, double* mine_s, double* ieee_s, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double ax = fabs(x[i]);
        mine[i] = rhd::rsqrt_nr(ax);
        ieee[i] = 1.0 / sqrt(ax);
        const double y = 1.0 + 3.0 * (ax / exp2(floor(log2(ax))) - 1.0);
        mine_s[i] = y * rhd::rsqrt_nr(y);
        ieee_s[i] = sqrt(y);
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
    double *dms, *dis;
    if (cudaMalloc(&dms, n * sizeof(double)) || cudaMalloc(&dis, n * sizeof(double))) return 2;
    rsqrt_kernel<<<(n + 255) / 256, 256>>>(dx, dm, di, dms, dis, n);
    std::vector<double> ms(n), rs(n);
    if (cudaMemcpy(m.data(), dm, n * sizeof(double), cudaMemcpyDeviceToHost) ||
        cudaMemcpy(r.data(), di, n * sizeof(double), cudaMemcpyDeviceToHost) ||
        cudaMemcpy(ms.data(), dms, n * sizeof(double), cudaMemcpyDeviceToHost) ||
        cudaMemcpy(rs.data(), dis, n * sizeof(double), cudaMemcpyDeviceToHost))
        return 3;
    int64_t worst_rsqrt = 0, worst_sqrt = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t d = bits(m[i]) > bits(r[i]) ? bits(m[i]) - bits(r[i]) : bits(r[i]) - bits(m[i]);
        const int64_t e = bits(ms[i]) > bits(rs[i]) ? bits(ms[i]) - bits(rs[i]) : bits(rs[i]) - bits(ms[i]);
        if (d > worst_rsqrt) worst_rsqrt = d;
        if (e > worst_sqrt) worst_sqrt = e;
    }
    std::printf("max_ulp %lld exact_cases_off %lld max_ulp_rsqrt %lld max_ulp_sqrt14 %lld\n", (long long)worst,
                (long long)exact_misses, (long long)worst_rsqrt, (long long)worst_sqrt);
    cudaFree(dx);
    cudaFree(dm);
    cudaFree(di);
    cudaFree(dms);
    cudaFree(dis);
    return 0;
}
