// rhd_noalloc.cu -- the subcycle entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: for example code that runs while another component owns the
// device memory through its own pool allocator (a foreign cudaMalloc there can fail or break that
// pool's accounting), or an application that must keep a device-memory footprint fixed when the
// library is loaded.  rhd_subcycle_noalloc serves them: the caller passes device inputs and outputs,
// and the only scratch the FP64 subcycle kernel needs (the working copy of the state in G = F/c form
// and the event counters) lives in the static device array below, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "rhd.h"
#include "rhd_internal.h"

namespace rhd {
rhd_status noalloc_prepare(const rhd_grid_desc* d, GridParams* gp, int* tiles_x, int* tiles_y, int* z_chunk);
rhd_status noalloc_fail(rhd_status st, const std::string& msg);
}  // namespace rhd

using namespace rhd;

namespace {

constexpr long long kMaxCells = RHD_NOALLOC_MAX_CELLS;
constexpr size_t kStateBytes = sizeof(double) * 4 * (size_t)kMaxCells;  // E, Gx, Gy, Gz
constexpr size_t kScratchBytes = kStateBytes + 256;                     // + the event counters

}  // namespace

// The scratch memory.  In host code this name is only a stand-in for the symbol: the device address
// is obtained with cudaGetSymbolAddress on each device (see scratch_address) and passed to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mutex;
void* g_scratch_ptr[256] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
rhd_status scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= 256) return noalloc_fail(RHD_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(RHD_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return RHD_OK;
}

#define NA_CUDA(call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return noalloc_fail(RHD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" rhd_status rhd_subcycle_noalloc(const rhd_grid_desc* d, const double dirichlet[24], int n_sub,
                                           double chat, double dt, const double* E, const double* Fx,
                                           const double* Fy, const double* Fz, const double* rho, const double* T,
                                           const double* vx, const double* vy, const double* vz, const double* kP,
                                           const double* kF, const double* j, double* E_out, double* Fx_out,
                                           double* Fy_out, double* Fz_out, double* T_out, rhd_stats* stats)
{
    if (!d) return noalloc_fail(RHD_ERR_ARG, "descriptor is NULL");
    if (!E || !Fx || !Fy || !Fz || !rho || !T || !E_out || !Fx_out || !Fy_out || !Fz_out || !T_out)
        return noalloc_fail(RHD_ERR_ARG, "E, Fx, Fy, Fz, rho, T and all outputs are required (device pointers)");
    if (n_sub < 0) return noalloc_fail(RHD_ERR_ARG, "n_sub must be >= 0");
    if (d->precision != RHD_FP64) return noalloc_fail(RHD_ERR_ARG, "the no-allocation entry point runs the FP64 path only");
    GridParams gp;
    int tiles_x = 0, tiles_y = 0, z_chunk = 1;
    rhd_status st = noalloc_prepare(d, &gp, &tiles_x, &tiles_y, &z_chunk);
    if (st) return st;
    const long long n = (long long)d->n[0] * d->n[1] * d->n[2];
    if (n > kMaxCells)
        return noalloc_fail(RHD_ERR_ARG, "grid has " + std::to_string(n) + " cells; the no-allocation entry point holds at most " +
                                             std::to_string(kMaxCells));
    if (!(std::isfinite(chat) && chat > 0.0) || !(std::isfinite(dt) && dt >= 0.0))
        return noalloc_fail(RHD_ERR_ARG, "chat must be positive and dt non-negative");
    if (chat > d->c * (1.0 + 1e-12)) return noalloc_fail(RHD_ERR_CFL, "chat must not exceed c");
    double dxmin = INFINITY;
    for (int k = 0; k < 3; ++k)
        if (d->n[k] > 1) dxmin = std::fmin(dxmin, d->dx[k]);
    if (std::isfinite(dxmin) && dt > d->cfl * dxmin / chat * (1.0 + 1e-12))
        return noalloc_fail(RHD_ERR_CFL, "dt exceeds cfl * min(dx) / chat");
    if (dirichlet) {
        for (int f = 0; f < 6; ++f) {
            double* dst = (f & 1) ? gp.dir_hi[f >> 1] : gp.dir_lo[f >> 1];
            dst[0] = dirichlet[4 * f];
            for (int q = 1; q < 4; ++q) dst[q] = dirichlet[4 * f + q] / d->c;
        }
    }

    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    unsigned char* scratch = nullptr;
    if ((st = scratch_address(dev, &scratch))) return st;
    double* A[4];
    for (int q = 0; q < 4; ++q) A[q] = reinterpret_cast<double*>(scratch) + (size_t)q * (size_t)n;
    DevStats* dstats = reinterpret_cast<DevStats*>(scratch + kStateBytes);
    double* B[4] = {E_out, Fx_out, Fy_out, Fz_out};
    cudaStream_t s = (cudaStream_t)d->cuda_stream;
    const size_t bytes = sizeof(double) * (size_t)n;

    // counters start at zero on every call; the state starts from the inputs (G = F/c)
    NA_CUDA(cudaMemsetAsync(dstats, 0, sizeof(DevStats), s));
    NA_CUDA(cudaMemcpyAsync(A[0], E, bytes, cudaMemcpyDeviceToDevice, s));
    NA_CUDA(launch_scale_copy(A[1], Fx, d->c, n, s));
    NA_CUDA(launch_scale_copy(A[2], Fy, d->c, n, s));
    NA_CUDA(launch_scale_copy(A[3], Fz, d->c, n, s));
    if (T_out != T) NA_CUDA(cudaMemcpyAsync(T_out, T, bytes, cudaMemcpyDeviceToDevice, s));

    StepParams p;
    std::memset(&p, 0, sizeof(p));
    p.g = gp;
    p.chat = chat;
    p.dt = dt;
    p.f_chat = (float)chat;
    p.f_dt = (float)dt;
    p.z_chunk = z_chunk;
    p.tx = 16;
    p.ty = 8;
    p.tiles_x = tiles_x;
    p.tiles_y = tiles_y;
    p.stats = dstats;
    GridArrays& a = p.a;
    a.T = T_out;
    a.rho = rho;
    a.v[0] = vx;
    a.v[1] = vy;
    a.v[2] = vz;
    a.kP = kP;
    a.kF = kF;
    a.j = j;
    // ping-pong between the scratch state (A) and the caller's outputs (B, holding G until the end)
    for (int step = 0; step < n_sub; ++step) {
        double** src = (step & 1) ? B : A;
        double** dst = (step & 1) ? A : B;
        a.E = src[0];
        a.Eo = dst[0];
        for (int q = 0; q < 3; ++q) {
            a.G[q] = src[1 + q];
            a.Go[q] = dst[1 + q];
        }
        NA_CUDA(launch_subcycle_fp64(p, s));
    }
    if ((n_sub & 1) == 0) {
        NA_CUDA(cudaMemcpyAsync(E_out, A[0], bytes, cudaMemcpyDeviceToDevice, s));
        for (int q = 0; q < 3; ++q) NA_CUDA(launch_scale_copy(B[1 + q], A[1 + q], -d->c, n, s));
    } else {
        for (int q = 0; q < 3; ++q) NA_CUDA(launch_scale_copy(B[1 + q], B[1 + q], -d->c, n, s));
    }
    // the counters come back on every call, so that non-finite results are never reported as success
    DevStats h;
    NA_CUDA(cudaMemcpyAsync(&h, dstats, sizeof(h), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->n_subcycles = n_sub;
        stats->n_realizability_fix = (int64_t)h.n_fix;
        stats->n_face_fallback = (int64_t)h.n_face;
        stats->n_theta_fallback = (int64_t)h.n_theta;
        stats->n_newton_fallback = (int64_t)h.n_newton_fb;
        stats->n_nonfinite = (int64_t)h.n_nonfinite;
        stats->newton_iter_max = (int32_t)h.newton_iter_max;
    }
    if (h.n_nonfinite) return noalloc_fail(RHD_ERR_NONFINITE, "non-finite values were produced");
    return RHD_OK;
}
