// The double-float operations of the split path's stiff sources (dfloat.cuh) against FP64: prints, per
// operation, the largest relative error over random operands in units of u^2 = 2^-48, and the number of
// FP64 -> FP32 roundings (d2f_rn, integer bit operations) that differ from CUDA's __double2float_rn.
// Built and run by tests/test_gpu_dfloat.py.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "dfloat.cuh"

using rhd::dfl;

enum { OP_D2DF, OP_ADDF, OP_ADD, OP_ADDSAME, OP_MULF, OP_MUL, OP_SQR, OP_RCP, N_OPS };

__device__ double val(dfl x) { return (double)x.hi + (double)x.lo; }

// a: operand pairs as FP64 values (each turned into a double-float first); out[op * n + i]: relative error
__global__ void check_kernel(const double* a, const double* b, const float* f, double* err, unsigned* rn_miss, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dfl x = rhd::d2df(a[i]), y = rhd::d2df(b[i]);
    const double X = val(x), Y = val(y), F = (double)f[i];
    auto rel = [](double got, double ref) { return ref == 0.0 ? fabs(got) : fabs(got - ref) / fabs(ref); };
    err[OP_D2DF * n + i] = rel(X, a[i]);
    err[OP_ADDF * n + i] = rel(val(rhd::dadd(x, f[i])), X + F);
    err[OP_ADD * n + i] = rel(val(rhd::dadd(x, y)), X + Y);
    err[OP_ADDSAME * n + i] = rel(val(rhd::dadd_same(x, rhd::dfl{fabsf(y.hi) * (x.hi < 0 ? -1.f : 1.f), 0.f})),
                                  X + fabs((double)y.hi) * (x.hi < 0 ? -1.0 : 1.0));
    err[OP_MULF * n + i] = rel(val(rhd::dmul(x, f[i])), X * F);
    err[OP_MUL * n + i] = rel(val(rhd::dmul(x, y)), X * Y);
    err[OP_SQR * n + i] = rel(val(rhd::dsqr(x)), X * X);
    const dfl ax = rhd::dadd(rhd::dfl{fabsf(x.hi), x.hi < 0 ? -x.lo : x.lo}, 1.0f);  // >= 1
    err[OP_RCP * n + i] = rel(val(rhd::drcp(ax)), 1.0 / val(ax));
    if (rhd::d2f_rn(a[i]) != __double2float_rn(a[i])) atomicAdd(rn_miss, 1u);
}

int main()
{
    const int n = 1 << 20;
    std::vector<double> a(n), b(n);
    std::vector<float> f(n);
    std::mt19937_64 rng(13060010);
    std::uniform_real_distribution<double> mant(1.0, 2.0);
    std::uniform_int_distribution<int> ex(-40, 40);
    for (int i = 0; i < n; ++i) {
        a[i] = (i & 1 ? -1.0 : 1.0) * std::ldexp(mant(rng), ex(rng));
        // every fourth pair nearly cancels (b close to -a), to exercise the accurate sum
        b[i] = (i % 4 == 0) ? -a[i] * (1.0 + std::ldexp(mant(rng), -30 + (int)(rng() % 25)))
                            : (i & 2 ? -1.0 : 1.0) * std::ldexp(mant(rng), ex(rng));
        f[i] = (float)((i & 4 ? -1.0 : 1.0) * std::ldexp(mant(rng), ex(rng)));
    }
    double *da, *db, *de;
    float* df;
    unsigned* dm;
    if (cudaMalloc(&da, n * sizeof(double)) || cudaMalloc(&db, n * sizeof(double)) || cudaMalloc(&df, n * sizeof(float)) ||
        cudaMalloc(&de, (size_t)N_OPS * n * sizeof(double)) || cudaMalloc(&dm, sizeof(unsigned)))
        return 2;
    cudaMemcpy(da, a.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(db, b.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(df, f.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(dm, 0, sizeof(unsigned));
    check_kernel<<<(n + 255) / 256, 256>>>(da, db, df, de, dm, n);
    std::vector<double> e((size_t)N_OPS * n);
    unsigned miss = 0;
    if (cudaMemcpy(e.data(), de, e.size() * sizeof(double), cudaMemcpyDeviceToHost) ||
        cudaMemcpy(&miss, dm, sizeof miss, cudaMemcpyDeviceToHost))
        return 3;
    const char* names[N_OPS] = {"d2df", "add_fp", "add", "add_same", "mul_fp", "mul", "sqr", "rcp"};
    const double u2 = std::ldexp(1.0, -48);
    for (int op = 0; op < N_OPS; ++op) {
        double w = 0.0;
        for (int i = 0; i < n; ++i) w = std::fmax(w, e[(size_t)op * n + i]);
        std::printf("%s %.4f\n", names[op], w / u2);
    }
    std::printf("rn_miss %u\n", miss);
    cudaFree(da);
    cudaFree(db);
    cudaFree(df);
    cudaFree(de);
    cudaFree(dm);
    return 0;
}
