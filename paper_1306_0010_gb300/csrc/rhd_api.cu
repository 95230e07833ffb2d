// rhd_api.cu -- host runtime of librhd.so: contexts, device buffers, argument checks, stream
// ordering, the CUDA-graph cache of the subcycle loop, statistics, and the batched ensemble.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>  // header-only: ranges are recorded only when a profiler is attached

#include "rhd.h"
#include "rhd_internal.h"
#include "gas_index.h"
#include "gas_internal.h"

using namespace rhd;

namespace {

thread_local std::string g_init_error;

// RHD_LOG: 0 (default) silent; 1 error messages to stderr; 2 also the launch configurations chosen
int log_level()
{
    static const int lv = [] {
        const char* v = std::getenv("RHD_LOG");
        return v ? std::atoi(v) : 0;
    }();
    return lv;
}

// NVTX range around one API call (visible in Nsight tools; a no-op otherwise)
struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
};

struct GraphEntry {
    int n_sub;
    int start;
    double chat, dt;
    cudaGraphExec_t exec;
    unsigned long long stamp;
};

// Device state of one grid.
struct GridState {
    rhd_grid_desc desc;
    GridParams gp;
    long long ncell = 0;
    int tx = 0, ty = 0, tiles_x = 0, tiles_y = 0, z_chunk = 1;
    double* U[2][4] = {{nullptr}};
    double* T = nullptr;
    double* rho = nullptr;
    double* v[3] = {nullptr, nullptr, nullptr};
    double* kP = nullptr;
    double* kF = nullptr;
    double* j = nullptr;
    float* rho32 = nullptr;
    float* v32[3] = {nullptr, nullptr, nullptr};
    float* kP32 = nullptr;
    float* kF32 = nullptr;
    float* j32 = nullptr;
    bool has_v = false, has_kP = false, has_kF = false, has_j = false;
    bool has_moments = false, has_gas = false;
    int variant = 0;              // RHD_VARIANT_FUSED / RHD_VARIANT_TWOPASS
    int staging = 0;              // RHD_STAGING_*
    float4* uhalf = nullptr;      // two-pass: U^{m+1/2} with its ghost layers
    float4* um32 = nullptr;       // two-pass: FP32 mirror of the current state (valid when um32_ok)
    float4* gas4 = nullptr;       // two-pass: interleaved FP32 (rho, v) (valid when gas4_ok)
    bool um32_ok = false, gas4_ok = false;
    CUtensorMap uh_map;           // its tensor map (staging RHD_STAGING_TMA), valid when uh_map_ok
    bool uh_map_ok = false;
    const double* dir_dev = nullptr;  // low x Dirichlet state in device memory (rhd_marshak_advance only)
    bool tuned = false;           // RHD_FLAG_AUTOTUNE handled
    double tuned_ms = -1.0;       // time per subcycle measured by the last tuning
    // gas step scratch (allocated by the first rhd_gas_step): W^{n+1/2} on the extended grid, the face
    // fluxes of each active direction, and what rhd_gas_correct needs
    double* gas_wh[5] = {nullptr};
    float* gas_wh32[5] = {nullptr};  // split grids: FP32 copy of W^{n+1/2}
    double* gas_flux[3][5] = {{nullptr}};  // FP32 values on split grids
    double* gas_pend[8] = {nullptr};
    bool gas_pending = false;     // a gas step waits for its source correction
    double gas_dt = 0.0;
};

}  // namespace

struct rhd_ctx {
    bool ensemble = false;
    int device = 0;
    int num_sms = 152;
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;  // the caller's stream when it is not the legacy default stream
    bool own_stream = false;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<GridState> grids;
    int cur = 0;  // buffer index holding the current state (shared by all grids)
    unsigned wait_polls = 1u << 22;  // polls of the two-pass corrector's TMA plane waits (rhd_set_wait_limit)
    DevStats* dstats = nullptr;
    double* red_partials = nullptr;
    double* rsla_partial = nullptr;  // reduced-speed-of-light reductions: rsla_blocks() + 1 doubles
    double* marshak_state = nullptr;  // rhd_marshak_advance: low x Dirichlet states, 4 doubles per subcycle
    unsigned long long* gas_counters = nullptr;  // gas step: [0] internal-energy floors, [1] non-finite cells
    int marshak_cap = 0;              // subcycles it holds
    double* red_out = nullptr;
    int red_blocks = 1;
    long long n_subcycles = 0;
    std::vector<GraphEntry> graphs;
    unsigned long long stamp = 0;
    std::string err;
    // RHD_DEVICE_MEMORY_LIMIT (bytes, read at creation): cap on the context's cumulative device
    // allocations, a test hook that forces RHD_ERR_OOM without exhausting the device
    size_t mem_limit = 0, mem_used = 0;
    // kernel timing: events recorded around each kernel launch (plain launches while enabled)
    bool ktiming = false;
    std::vector<cudaEvent_t> kev;          // event pool, reused after each read
    size_t kev_used = 0;
    struct KRec { int kernel; size_t e0, e1; double alg_bytes; };
    std::vector<KRec> krec;
    // ensemble
    EnsembleGrid* d_egrids[2] = {nullptr, nullptr};
    unsigned long long* d_counter = nullptr;
    long long n_items = 0, n_pitems = 0;
    int ens_ctas = 0, ens_pctas = 0, ens_cctas = 0;  // fused / predictor / corrector persistent CTAs
};

namespace {

rhd_status fail(rhd_ctx* ctx, rhd_status st, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    else g_init_error = msg;
    if (log_level() >= 1) std::fprintf(stderr, "rhd: status %d: %s\n", (int)st, msg.c_str());
    return st;
}

#define RHD_CUDA(ctx, call)                                                                          \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? RHD_ERR_OOM : RHD_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

// With the legacy default stream the work runs on a library stream (CUDA graphs cannot be captured
// on the legacy stream) ordered after the caller's stream, and the caller's stream after the work.
// Any other stream is used directly.
rhd_status enter(rhd_ctx* ctx)
{
    RHD_CUDA(ctx, cudaSetDevice(ctx->device));
    if (!ctx->own_stream) return RHD_OK;
    RHD_CUDA(ctx, cudaEventRecord(ctx->ev_in, ctx->user_stream));
    RHD_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
    return RHD_OK;
}
rhd_status leave(rhd_ctx* ctx)
{
    if (!ctx->own_stream) return RHD_OK;
    RHD_CUDA(ctx, cudaEventRecord(ctx->ev_out, ctx->stream));
    RHD_CUDA(ctx, cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
    return RHD_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

rhd_status validate_desc(rhd_ctx* ctx, const rhd_grid_desc* d)
{
    if (!d) return fail(ctx, RHD_ERR_ARG, "descriptor is NULL");
    int nact = 0;
    bool seen_inactive = false;
    for (int k = 0; k < 3; ++k) {
        if (d->n[k] < 1) return fail(ctx, RHD_ERR_ARG, "n[" + std::to_string(k) + "] must be >= 1");
        if (d->n[k] > 1) {
            if (seen_inactive) return fail(ctx, RHD_ERR_ARG, "inactive directions (n = 1) must be the trailing ones");
            if (d->n[k] < 3) return fail(ctx, RHD_ERR_ARG, "active directions need n >= 3");
            if (!finite_pos(d->dx[k])) return fail(ctx, RHD_ERR_ARG, "dx must be positive and finite");
            for (int s = 0; s < 2; ++s) {
                int bc = s ? d->bc_hi[k] : d->bc_lo[k];
                if (bc < 0 || bc > 3) return fail(ctx, RHD_ERR_ARG, "unknown boundary condition");
            }
            ++nact;
        } else {
            seen_inactive = true;
        }
    }
    if (nact == 0) nact = 0;
    long long ncell = (long long)d->n[0] * d->n[1] * d->n[2];
    if (ncell > (1LL << 34)) return fail(ctx, RHD_ERR_ARG, "grid too large");
    if (!finite_pos(d->c)) return fail(ctx, RHD_ERR_ARG, "c must be positive");
    if (!(std::isfinite(d->a_rad) && d->a_rad >= 0)) return fail(ctx, RHD_ERR_ARG, "a_rad must be >= 0");
    if (!(std::isfinite(d->gamma) && d->gamma > 1.0)) return fail(ctx, RHD_ERR_ARG, "gamma must be > 1");
    if (!finite_pos(d->mu_over_kB)) return fail(ctx, RHD_ERR_ARG, "mu_over_kB must be positive");
    if (!(d->theta_F > 0 && d->theta_F <= 1) || !(d->theta_E > 0 && d->theta_E <= 1))
        return fail(ctx, RHD_ERR_ARG, "theta must lie in (0, 1]");
    if (!finite_pos(d->E_floor)) return fail(ctx, RHD_ERR_ARG, "E_floor must be positive");
    // the kernels' reciprocals flush subnormal inputs: E >= E_floor must be a normal number of the
    // arithmetic that divides by it (FP64; FP32 on split grids)
    if (d->E_floor < DBL_MIN) return fail(ctx, RHD_ERR_ARG, "E_floor must be at least the smallest normal FP64 number");
    if (d->precision == RHD_SPLIT && d->E_floor < (double)FLT_MIN)
        return fail(ctx, RHD_ERR_ARG, "E_floor must be at least the smallest normal FP32 number (1.2e-38) on split grids");
    if (!(d->cfl > 0 && d->cfl <= 1)) return fail(ctx, RHD_ERR_ARG, "cfl must lie in (0, 1]");
    if (d->exchange < 0 || d->exchange > 4) return fail(ctx, RHD_ERR_ARG, "unknown exchange mode");
    if (d->exchange == RHD_EX_LINEAR && !finite_pos(d->linear_eps))
        return fail(ctx, RHD_ERR_ARG, "the linear exchange needs linear_eps > 0");
    if ((d->flags & RHD_FLAG_EXCHANGE_ON_GAS_STEP) && d->exchange != RHD_EX_FULL)
        return fail(ctx, RHD_ERR_ARG, "RHD_FLAG_EXCHANGE_ON_GAS_STEP needs exchange = RHD_EX_FULL");
    if (d->limiter < 0 || d->limiter > 2) return fail(ctx, RHD_ERR_ARG, "unknown limiter");
    if (d->closure < 0 || d->closure > 1) return fail(ctx, RHD_ERR_ARG, "unknown closure");
    if (d->speeds < 0 || d->speeds > 1) return fail(ctx, RHD_ERR_ARG, "unknown wave-speed option");
    if (d->precision < 0 || d->precision > 1) return fail(ctx, RHD_ERR_ARG, "unknown precision");
    if (d->z_chunk < 0) return fail(ctx, RHD_ERR_ARG, "z_chunk must be >= 0");
    if (!(std::isfinite(d->kappa_P) && d->kappa_P >= 0) || !(std::isfinite(d->kappa_F) && d->kappa_F >= 0))
        return fail(ctx, RHD_ERR_ARG, "kappa must be >= 0");
    if (d->kappa_rho_pow < 0 || d->kappa_rho_pow > 2) return fail(ctx, RHD_ERR_ARG, "kappa_rho_pow must be 0, 1 or 2");
    return RHD_OK;
}

int count_active(const rhd_grid_desc& d)
{
    int n = 0;
    for (int k = 0; k < 3; ++k) n += d.n[k] > 1;
    return n;
}

void fill_params(GridState& gs)
{
    const rhd_grid_desc& d = gs.desc;
    GridParams& g = gs.gp;
    std::memset(&g, 0, sizeof(g));
    for (int k = 0; k < 3; ++k) {
        g.n[k] = d.n[k];
        g.inv_dx[k] = d.n[k] > 1 ? 1.0 / d.dx[k] : 0.0;
        g.bc_lo[k] = d.bc_lo[k];
        g.bc_hi[k] = d.bc_hi[k];
    }
    g.nact = count_active(d);
    g.c = d.c;
    g.a_rad = d.a_rad;
    g.gamma = d.gamma;
    g.mu_over_kB = d.mu_over_kB;
    g.theta_F = d.theta_F;
    g.theta_E = d.theta_E;
    g.E_floor = d.E_floor;
    g.kappa_P = d.kappa_P;
    g.kappa_F = d.kappa_F;
    g.kpow = d.kappa_rho_pow;
    // the paper's placement of the exchange: none in the subcycles (rhd_gas_exchange runs it once per gas step)
    g.exchange = (d.flags & RHD_FLAG_EXCHANGE_ON_GAS_STEP) ? RHD_EX_EQUILIBRIUM : d.exchange;
    g.linear_eps = d.linear_eps;
    g.beta_tau = d.beta_tau ? 1 : 0;
    g.limiter = d.limiter;
    g.closure = d.closure;
    g.speeds = d.speeds;
    g.inv_c = 1.0 / d.c;
    g.gm1_mu = (d.gamma - 1.0) * d.mu_over_kB;
    g.inv_gm1_mu = 1.0 / g.gm1_mu;
    g.inv_eps_c = 1.0 / (d.linear_eps * d.c);
    g.inv_a_rad = 1.0 / d.a_rad;
    g.f_inv_c = (float)g.inv_c;
    g.f_gm1_mu = (float)g.gm1_mu;
    g.f_c = (float)d.c;
    g.f_a_rad = (float)d.a_rad;
    g.f_theta_F = (float)d.theta_F;
    g.f_theta_E = (float)d.theta_E;
    g.f_E_floor = (float)d.E_floor;
    g.f_kappa_P = (float)d.kappa_P;
    g.f_kappa_F = (float)d.kappa_F;
    for (int k = 0; k < 3; ++k) g.f_inv_dx[k] = (float)g.inv_dx[k];
    for (int k = 0; k < 3; ++k) g.pad[k] = (d.bc_lo[k] == RHD_BC_PERIODIC && d.bc_hi[k] == RHD_BC_PERIODIC) ? 0 : 2;
    tile_shape(d.precision, g.nact, &gs.tx, &gs.ty);
    if (const char* ov = std::getenv("RHD_TILE")) {  // "TXxTY": measurement override of the tile shape
        int tx = 0, ty = 0;
        if (std::sscanf(ov, "%dx%d", &tx, &ty) == 2 && tile_supported(d.precision, g.nact, tx, ty)) {
            gs.tx = tx;
            gs.ty = ty;
        }
    }
    gs.tiles_x = (d.n[0] + gs.tx - 1) / gs.tx;
    gs.tiles_y = (d.n[1] + gs.ty - 1) / gs.ty;
    int zc = d.z_chunk;
    if (zc <= 0) {
        // enough CTAs to fill the GPU several times over, but long enough z runs to amortise the
        // 6-plane pipeline start-up of each chunk
        long long tiles = (long long)gs.tiles_x * gs.tiles_y;
        zc = d.n[2];
        while (zc > 32 && tiles * ((d.n[2] + zc - 1) / zc) < 152LL * 8) zc = (zc + 1) / 2;
    }
    gs.z_chunk = std::max(1, std::min(zc, d.n[2]));
}

rhd_status dalloc(rhd_ctx* ctx, void** p, size_t bytes)
{
    if (ctx && ctx->mem_limit && ctx->mem_used + bytes > ctx->mem_limit) {
        *p = nullptr;
        return fail(ctx, RHD_ERR_OOM, "RHD_DEVICE_MEMORY_LIMIT reached (" + std::to_string(ctx->mem_used + bytes) +
                                          " bytes requested in total)");
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? RHD_ERR_OOM : RHD_ERR_CUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    if (ctx) ctx->mem_used += bytes;
    return RHD_OK;
}

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void free_grid(GridState& gs)
{
    for (int b = 0; b < 2; ++b)
        for (int q = 0; q < 4; ++q) dfree(gs.U[b][q]);
    dfree(gs.T);
    dfree(gs.rho);
    for (int d = 0; d < 3; ++d) {
        dfree(gs.v[d]);
        dfree(gs.v32[d]);
    }
    dfree(gs.kP);
    dfree(gs.kF);
    dfree(gs.j);
    dfree(gs.rho32);
    dfree(gs.kP32);
    dfree(gs.kF32);
    dfree(gs.j32);
    dfree(gs.uhalf);
    dfree(gs.um32);
    dfree(gs.gas4);
    for (int q = 0; q < 5; ++q) {
        dfree(gs.gas_wh[q]);
        dfree(gs.gas_wh32[q]);
    }
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 5; ++q) dfree(gs.gas_flux[d][q]);
    for (int q = 0; q < 8; ++q) dfree(gs.gas_pend[q]);
    gs.gas_pending = false;
}

void clear_graphs(rhd_ctx* ctx)
{
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
}

// Buffers of the two-pass split path: U^{m+1/2} with its ghost layers, the FP32 state mirror and the
// interleaved FP32 gas (allocated once, kept until the variant changes).
rhd_status alloc_twopass(rhd_ctx* ctx, GridState& gs)
{
    rhd_status st;
    if (!gs.uhalf) {
        size_t np = (size_t)upad_extent(gs.gp, 0) * upad_extent(gs.gp, 1) * upad_extent(gs.gp, 2);
        if ((st = dalloc(ctx, (void**)&gs.uhalf, sizeof(float4) * np))) return st;
    }
    if (!gs.um32) {
        if ((st = dalloc(ctx, (void**)&gs.um32, sizeof(float4) * (size_t)gs.ncell))) return st;
        gs.um32_ok = false;
    }
    if (!gs.gas4) {
        if ((st = dalloc(ctx, (void**)&gs.gas4, sizeof(float4) * (size_t)gs.ncell))) return st;
        gs.gas4_ok = false;
    }
    return RHD_OK;
}

void free_twopass(GridState& gs)
{
    dfree(gs.uhalf);
    dfree(gs.um32);
    dfree(gs.gas4);
    gs.um32_ok = gs.gas4_ok = false;
}

rhd_status alloc_grid(rhd_ctx* ctx, GridState& gs)
{
    size_t bytes = sizeof(double) * (size_t)gs.ncell;
    for (int b = 0; b < 2; ++b)
        for (int q = 0; q < 4; ++q) {
            rhd_status st = dalloc(ctx, (void**)&gs.U[b][q], bytes);
            if (st) return st;
        }
    rhd_status st = dalloc(ctx, (void**)&gs.T, bytes);
    if (st) return st;
    st = dalloc(ctx, (void**)&gs.rho, bytes);
    if (st) return st;
    if (gs.desc.precision == RHD_SPLIT) {
        st = dalloc(ctx, (void**)&gs.rho32, sizeof(float) * (size_t)gs.ncell);
        if (st) return st;
    }
    if (gs.variant == RHD_VARIANT_TWOPASS) return alloc_twopass(ctx, gs);
    return RHD_OK;
}

rhd_status common_init(rhd_ctx* ctx)
{
    if (const char* lim = std::getenv("RHD_DEVICE_MEMORY_LIMIT")) ctx->mem_limit = (size_t)std::strtoull(lim, nullptr, 10);
    RHD_CUDA(ctx, cudaGetDevice(&ctx->device));
    RHD_CUDA(ctx, cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    if (ctx->user_stream == nullptr || ctx->user_stream == cudaStreamLegacy || ctx->user_stream == cudaStreamPerThread) {
        RHD_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    } else {
        ctx->stream = ctx->user_stream;
    }
    RHD_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
    RHD_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));
    rhd_status st = dalloc(ctx, (void**)&ctx->dstats, sizeof(DevStats));
    if (st) return st;
    RHD_CUDA(ctx, cudaMemset(ctx->dstats, 0, sizeof(DevStats)));
    if ((st = dalloc(ctx, (void**)&ctx->gas_counters, 2 * sizeof(unsigned long long)))) return st;
    RHD_CUDA(ctx, cudaMemset(ctx->gas_counters, 0, 2 * sizeof(unsigned long long)));
    return RHD_OK;
}

void destroy_ctx(rhd_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    clear_graphs(ctx);
    for (auto& gs : ctx->grids) free_grid(gs);
    dfree(ctx->dstats);
    dfree(ctx->red_partials);
    dfree(ctx->red_out);
    dfree(ctx->rsla_partial);
    dfree(ctx->marshak_state);
    dfree(ctx->gas_counters);
    dfree(ctx->d_egrids[0]);
    dfree(ctx->d_egrids[1]);
    dfree(ctx->d_counter);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    for (auto e : ctx->kev) cudaEventDestroy(e);
    if (ctx->stream && ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

// copy a host or device FP64 array into a device buffer (on the library stream)
rhd_status put(rhd_ctx* ctx, double* dst, const double* src, long long n, int on_device)
{
    RHD_CUDA(ctx, cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    return RHD_OK;
}

rhd_status set_optional(rhd_ctx* ctx, GridState& gs, double*& buf, float*& buf32, bool& has, const double* src,
                        int on_device)
{
    if (!src) {
        has = false;
        return RHD_OK;
    }
    size_t bytes = sizeof(double) * (size_t)gs.ncell;
    if (!buf) {
        rhd_status st = dalloc(ctx, (void**)&buf, bytes);
        if (st) return st;
    }
    rhd_status st = put(ctx, buf, src, gs.ncell, on_device);
    if (st) return st;
    if (gs.desc.precision == RHD_SPLIT) {
        if (!buf32) {
            st = dalloc(ctx, (void**)&buf32, sizeof(float) * (size_t)gs.ncell);
            if (st) return st;
        }
        RHD_CUDA(ctx, launch_to_float(buf32, buf, gs.ncell, ctx->stream));
    }
    has = true;
    return RHD_OK;
}

rhd_status set_gas(rhd_ctx* ctx, GridState& gs, const double* rho, const double* T, const double* vx,
                   const double* vy, const double* vz, const double* kP, const double* kF, const double* j,
                   int on_device)
{
    if (!rho || !T) return fail(ctx, RHD_ERR_ARG, "rho and T are required");
    rhd_status st = enter(ctx);
    if (st) return st;
    // the arrays the captured subcycle graphs point at, and which of them are present: the graphs stay
    // valid when a new state arrives in the same arrays
    auto layout = [&gs] {
        return std::vector<const void*>{gs.v[0], gs.v[1], gs.v[2], gs.v32[0], gs.v32[1], gs.v32[2], gs.kP, gs.kP32,
                                        gs.kF, gs.kF32, gs.j, gs.j32,
                                        (const void*)(uintptr_t)(gs.has_v | gs.has_kP << 1 | gs.has_kF << 2 |
                                                                 gs.has_j << 3 | gs.has_gas << 4)};
    };
    const std::vector<const void*> before = layout();
    if ((st = put(ctx, gs.rho, rho, gs.ncell, on_device))) return st;
    if ((st = put(ctx, gs.T, T, gs.ncell, on_device))) return st;
    if (gs.desc.precision == RHD_SPLIT) RHD_CUDA(ctx, launch_to_float(gs.rho32, gs.rho, gs.ncell, ctx->stream));
    const double* vin[3] = {vx, vy, vz};
    bool hv[3];
    for (int d = 0; d < 3; ++d)
        if ((st = set_optional(ctx, gs, gs.v[d], gs.v32[d], hv[d], vin[d], on_device))) return st;
    gs.has_v = hv[0] || hv[1] || hv[2];
    // velocity components that were not given are zero: keep them as absent
    for (int d = 0; d < 3; ++d)
        if (!hv[d]) {
            dfree(gs.v[d]);
            dfree(gs.v32[d]);
        }
    if ((st = set_optional(ctx, gs, gs.kP, gs.kP32, gs.has_kP, kP, on_device))) return st;
    if ((st = set_optional(ctx, gs, gs.kF, gs.kF32, gs.has_kF, kF, on_device))) return st;
    if ((st = set_optional(ctx, gs, gs.j, gs.j32, gs.has_j, j, on_device))) return st;
    gs.has_gas = true;
    gs.gas4_ok = false;
    gs.gas_pending = false;  // a pending source correction belongs to the replaced state
    if (layout() != before) clear_graphs(ctx);  // the kernels' array pointers changed
    return leave(ctx);
}

// conserved = false: (E, F) with G = F / c formed on the device; true: (E, G) copied as they are
rhd_status set_moments(rhd_ctx* ctx, GridState& gs, const double* E, const double* Fx, const double* Fy,
                       const double* Fz, int on_device, bool conserved = false)
{
    if (!E || !Fx || !Fy || !Fz) return fail(ctx, RHD_ERR_ARG, "E and the three flux components are required");
    rhd_status st = enter(ctx);
    if (st) return st;
    double** U = gs.U[ctx->cur];
    if ((st = put(ctx, U[0], E, gs.ncell, on_device))) return st;
    const double* F[3] = {Fx, Fy, Fz};
    for (int d = 0; d < 3; ++d) {
        if (conserved) {
            if ((st = put(ctx, U[1 + d], F[d], gs.ncell, on_device))) return st;
        } else if (on_device) {
            RHD_CUDA(ctx, launch_scale_copy(U[1 + d], F[d], gs.desc.c, gs.ncell, ctx->stream));
        } else {
            if ((st = put(ctx, U[1 + d], F[d], gs.ncell, 0))) return st;
            RHD_CUDA(ctx, launch_scale_copy(U[1 + d], U[1 + d], gs.desc.c, gs.ncell, ctx->stream));
        }
    }
    gs.has_moments = true;
    gs.um32_ok = false;
    return leave(ctx);
}

// conserved = false: (E, F = c G); true: (E, G) as the solver holds them
rhd_status get_moments(rhd_ctx* ctx, GridState& gs, double* E, double* Fx, double* Fy, double* Fz, int on_device,
                       bool conserved = false)
{
    if (!E || !Fx || !Fy || !Fz) return fail(ctx, RHD_ERR_ARG, "E and the three flux components are required");
    if (!gs.has_moments) return fail(ctx, RHD_ERR_STATE, "moments were never set");
    rhd_status st = enter(ctx);
    if (st) return st;
    double** U = gs.U[ctx->cur];
    double** W = gs.U[1 - ctx->cur];  // scratch: the other half of the ping-pong pair
    size_t bytes = sizeof(double) * (size_t)gs.ncell;
    double* F[3] = {Fx, Fy, Fz};
    if (conserved) {
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        for (int q = 0; q < 4; ++q)
            RHD_CUDA(ctx, cudaMemcpyAsync(q ? F[q - 1] : E, U[q], bytes, kind, ctx->stream));
    } else if (on_device) {
        RHD_CUDA(ctx, cudaMemcpyAsync(E, U[0], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        for (int d = 0; d < 3; ++d) RHD_CUDA(ctx, launch_scale_copy(F[d], U[1 + d], -gs.desc.c, gs.ncell, ctx->stream));
    } else {
        for (int d = 0; d < 3; ++d) RHD_CUDA(ctx, launch_scale_copy(W[1 + d], U[1 + d], -gs.desc.c, gs.ncell, ctx->stream));
        RHD_CUDA(ctx, cudaMemcpyAsync(E, U[0], bytes, cudaMemcpyDeviceToHost, ctx->stream));
        for (int d = 0; d < 3; ++d) RHD_CUDA(ctx, cudaMemcpyAsync(F[d], W[1 + d], bytes, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if ((st = leave(ctx))) return st;
    RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RHD_OK;
}

rhd_status get_T(rhd_ctx* ctx, GridState& gs, double* T, int on_device)
{
    if (!T) return fail(ctx, RHD_ERR_ARG, "T is required");
    if (!gs.has_gas) return fail(ctx, RHD_ERR_STATE, "gas state was never set");
    rhd_status st = enter(ctx);
    if (st) return st;
    RHD_CUDA(ctx, cudaMemcpyAsync(T, gs.T, sizeof(double) * (size_t)gs.ncell,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if ((st = leave(ctx))) return st;
    RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RHD_OK;
}

StepParams step_params(rhd_ctx* ctx, GridState& gs, int src, double chat, double dt)
{
    StepParams p;
    std::memset(&p, 0, sizeof(p));
    p.g = gs.gp;
    GridArrays& a = p.a;
    a.E = gs.U[src][0];
    for (int d = 0; d < 3; ++d) a.G[d] = gs.U[src][1 + d];
    a.Eo = gs.U[1 - src][0];
    for (int d = 0; d < 3; ++d) a.Go[d] = gs.U[1 - src][1 + d];
    a.T = gs.T;
    a.dir_dev = gs.dir_dev;
    a.rho = gs.rho;
    for (int d = 0; d < 3; ++d) {
        a.v[d] = gs.v[d];
        a.v32[d] = gs.v32[d];
    }
    a.kP = gs.has_kP ? gs.kP : nullptr;
    a.kF = gs.has_kF ? gs.kF : nullptr;
    a.j = gs.has_j ? gs.j : nullptr;
    a.rho32 = gs.rho32;
    a.kP32 = gs.has_kP ? gs.kP32 : nullptr;
    a.kF32 = gs.has_kF ? gs.kF32 : nullptr;
    a.j32 = gs.has_j ? gs.j32 : nullptr;
    const bool twopass = gs.variant == RHD_VARIANT_TWOPASS;
    a.um32 = twopass ? gs.um32 : nullptr;
    a.gas4 = twopass ? gs.gas4 : nullptr;
    p.chat = chat;
    p.dt = dt;
    p.f_chat = (float)chat;
    p.f_dt = (float)dt;
    p.uhalf = gs.uhalf;
    p.staging = gs.staging;
    p.wait_polls = ctx->wait_polls;
    if (gs.staging == RHD_STAGING_TMA) p.uh_map = gs.uh_map;
    p.z_chunk = gs.z_chunk;
    p.tx = gs.tx;
    p.ty = gs.ty;
    p.tiles_x = gs.tiles_x;
    p.tiles_y = gs.tiles_y;
    p.stats = ctx->dstats;
    return p;
}

rhd_status check_dt(rhd_ctx* ctx, const GridState& gs, double chat, double dt)
{
    if (!finite_pos(chat)) return fail(ctx, RHD_ERR_ARG, "chat must be positive and finite");
    if (!(std::isfinite(dt) && dt >= 0.0)) return fail(ctx, RHD_ERR_ARG, "dt must be finite and >= 0");
    if (chat > gs.desc.c * (1.0 + 1e-12)) return fail(ctx, RHD_ERR_CFL, "chat must not exceed c");
    double dxmin = INFINITY;
    for (int k = 0; k < 3; ++k)
        if (gs.desc.n[k] > 1) dxmin = std::min(dxmin, gs.desc.dx[k]);
    if (std::isfinite(dxmin) && dt > gs.desc.cfl * dxmin / chat * (1.0 + 1e-12))
        return fail(ctx, RHD_ERR_CFL, "dt exceeds cfl * min(dx) / chat");
    return RHD_OK;
}

// kernels reported by the kernel timer
enum KernelId {
    K_FUSED_FP64 = 0, K_FUSED_SPLIT, K_PREDICTOR, K_CORRECTOR, K_ENS_FP64, K_ENS_SPLIT, K_ENS_PRED, K_ENS_CORR,
    K_GAS_PRED_FLUX, K_GAS_PRED_UPDATE, K_GAS_CORR_FLUX, K_GAS_CORR_UPDATE, K_GAS_CORRECT, K_GAS_EXCHANGE,
    K_COUNT
};
const char* const kKernelNames[K_COUNT] = {"subcycle_fused_fp64", "subcycle_fused_split", "twopass_predictor_split",
                                           "twopass_corrector_split", "ensemble_fp64", "ensemble_split",
                                           "ensemble_predictor_split", "ensemble_corrector_split",
                                           "gas_predictor_flux", "gas_predictor_update", "gas_corrector_flux",
                                           "gas_corrector_update", "gas_source_correction", "gas_step_exchange"};

// Algorithmic bytes per interior cell of one launch of kernel k: every array the kernel reads, read
// once, and every array it writes, written once.  Fused kernels: U^m and U^{m+1} (4 FP64 each), the
// gas arrays in the kernel's precision, T.  Two-pass kernels: the predictor reads the FP32 state
// mirror (16 B) and the interleaved FP32 gas (16 B) and writes U^{m+1/2} (16 B); the corrector reads
// U^{m+1/2}, U^m (FP64), the gas and T, and writes U^{m+1} (FP64), T and the new mirror.
double alg_bytes_per_cell(const GridState& gs, int k)
{
    const bool split = gs.desc.precision == RHD_SPLIT;
    const double w = split ? 4.0 : 8.0;
    const double opt = w * ((gs.has_kP ? 1 : 0) + (gs.has_kF ? 1 : 0) + (gs.has_j ? 1 : 0));
    const double gas = w * (1 + (gs.has_v ? 3 : 0)) + opt;
    const int ex = gs.gp.exchange;  // the subcycles' exchange (none with RHD_FLAG_EXCHANGE_ON_GAS_STEP)
    const bool tw = ex == RHD_EX_FULL || ex == RHD_EX_LINEAR;
    const double Tr = (tw || ex == RHD_EX_FROZEN_T) ? 8.0 : 0.0, Tw = tw ? 8.0 : 0.0;
    switch (k) {
    case K_PREDICTOR: return 16.0 + 16.0 + opt + (ex == RHD_EX_FROZEN_T ? 8.0 : 0.0) + 16.0;
    case K_CORRECTOR: return 16.0 + 32.0 + 16.0 + opt + Tr + 32.0 + Tw + 16.0;
    default: return 32.0 + gas + Tr + 32.0 + Tw;
    }
}

rhd_status kev_record(rhd_ctx* ctx, size_t* idx)
{
    if (ctx->kev_used == ctx->kev.size()) {
        cudaEvent_t e = nullptr;
        RHD_CUDA(ctx, cudaEventCreate(&e));
        ctx->kev.push_back(e);
    }
    *idx = ctx->kev_used++;
    RHD_CUDA(ctx, cudaEventRecord(ctx->kev[*idx], ctx->stream));
    return RHD_OK;
}

// Launch fn, bracketed by timing events when the kernel timer is on.
template <typename Fn>
rhd_status timed_launch(rhd_ctx* ctx, int kernel, double alg_bytes, Fn&& fn)
{
    size_t e0 = 0, e1 = 0;
    rhd_status st;
    if (ctx->ktiming && (st = kev_record(ctx, &e0))) return st;
    cudaError_t e = fn();
    if (e != cudaSuccess)
        return fail(ctx, RHD_ERR_CUDA, std::string(kKernelNames[kernel]) + " launch: " + cudaGetErrorString(e));
    if (ctx->ktiming) {
        if ((st = kev_record(ctx, &e1))) return st;
        ctx->krec.push_back({kernel, e0, e1, alg_bytes});
    }
    return RHD_OK;
}

// Before two-pass subcycles: rebuild the FP32 state mirror (from buffer cur) and the interleaved FP32
// gas if they may be stale.  Each two-pass subcycle's corrector rewrites the mirror with U^{m+1}.
rhd_status prepare_twopass(rhd_ctx* ctx, GridState& gs)
{
    if (gs.variant != RHD_VARIANT_TWOPASS) return RHD_OK;
    if (!gs.gas4_ok && gs.has_gas) {
        RHD_CUDA(ctx, launch_to_gas4(gs.gas4, gs.rho32, gs.v32[0], gs.v32[1], gs.v32[2], gs.ncell, ctx->stream));
        gs.gas4_ok = true;
    }
    if (!gs.um32_ok && gs.has_moments) {
        double** U = gs.U[ctx->cur];
        RHD_CUDA(ctx, launch_to_um32(gs.um32, U[0], U[1], U[2], U[3], gs.ncell, ctx->stream));
        gs.um32_ok = true;
    }
    return RHD_OK;
}

rhd_status launch_one(rhd_ctx* ctx, GridState& gs, int src, double chat, double dt)
{
    StepParams p = step_params(ctx, gs, src, chat, dt);
    cudaStream_t s = ctx->stream;
    const double nc = (double)gs.ncell;
    if (gs.desc.precision != RHD_SPLIT)
        return timed_launch(ctx, K_FUSED_FP64, nc * alg_bytes_per_cell(gs, K_FUSED_FP64),
                            [&] { return launch_subcycle_fp64(p, s); });
    if (gs.variant != RHD_VARIANT_TWOPASS) {
        gs.um32_ok = false;
        return timed_launch(ctx, K_FUSED_SPLIT, nc * alg_bytes_per_cell(gs, K_FUSED_SPLIT),
                            [&] { return launch_subcycle_split(p, s); });
    }
    rhd_status st = timed_launch(ctx, K_PREDICTOR, nc * alg_bytes_per_cell(gs, K_PREDICTOR),
                                 [&] { return launch_twopass_predictor(p, s); });
    if (st) return st;
    return timed_launch(ctx, K_CORRECTOR, nc * alg_bytes_per_cell(gs, K_CORRECTOR),
                        [&] { return launch_twopass_corrector(p, s); });
}

// Run n_sub steps: replay a cached graph (or issue the launches directly).
template <typename LaunchFn>
rhd_status run_steps(rhd_ctx* ctx, int n_sub, double chat, double dt, bool use_graph, LaunchFn&& launch)
{
    if (!use_graph) {
        for (int s = 0; s < n_sub; ++s) {
            rhd_status st = launch((ctx->cur + s) & 1);
            if (st) return st;
        }
        return RHD_OK;
    }
    for (auto& g : ctx->graphs)
        if (g.n_sub == n_sub && g.start == ctx->cur && g.chat == chat && g.dt == dt) {
            g.stamp = ++ctx->stamp;
            RHD_CUDA(ctx, cudaGraphLaunch(g.exec, ctx->stream));
            return RHD_OK;
        }
    cudaGraph_t graph = nullptr;
    RHD_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    rhd_status st = RHD_OK;
    for (int s = 0; s < n_sub && st == RHD_OK; ++s) st = launch((ctx->cur + s) & 1);
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess) return fail(ctx, RHD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(ctx, RHD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    if (ctx->graphs.size() >= 6) {
        auto it = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                   [](const GraphEntry& a, const GraphEntry& b) { return a.stamp < b.stamp; });
        cudaGraphExecDestroy(it->exec);
        ctx->graphs.erase(it);
    }
    ctx->graphs.push_back({n_sub, ctx->cur, chat, dt, exec, ++ctx->stamp});
    RHD_CUDA(ctx, cudaGraphLaunch(exec, ctx->stream));
    return RHD_OK;
}

rhd_status ensure_reduce(rhd_ctx* ctx, long long n)
{
    int nb = reduce_blocks_for(n);
    if (ctx->red_partials && ctx->red_blocks >= nb) return RHD_OK;
    dfree(ctx->red_partials);
    dfree(ctx->red_out);
    rhd_status st = dalloc(ctx, (void**)&ctx->red_partials, sizeof(double) * 5 * (size_t)nb);
    if (st) return st;
    st = dalloc(ctx, (void**)&ctx->red_out, sizeof(double) * 5);
    if (st) return st;
    ctx->red_blocks = nb;
    return RHD_OK;
}

// ---------------------------------------------------------------------------------------------
// ensemble launch helpers
// ---------------------------------------------------------------------------------------------

// Per-parity grid tables (src = 0 / 1) and the work-item count for the current z chunk.
rhd_status ens_prepare(rhd_ctx* ctx, double chat, const double* dt_per_grid, double* dt_sig)
{
    const int ng = (int)ctx->grids.size();
    std::vector<EnsembleGrid> eg(ng);
    *dt_sig = 0.0;
    for (int src = 0; src < 2; ++src) {
        long long first = 0, pfirst = 0;
        for (int i = 0; i < ng; ++i) {
            GridState& gs = ctx->grids[i];
            const bool twopass = gs.variant == RHD_VARIANT_TWOPASS;
            StepParams p = step_params(ctx, gs, src, chat, dt_per_grid[i]);
            std::memset(&eg[i], 0, sizeof(EnsembleGrid));
            eg[i].g = p.g;
            eg[i].a = p.a;
            eg[i].dt = dt_per_grid[i];
            eg[i].f_dt = (float)dt_per_grid[i];
            // corrector (two-pass) or fused items: tiles of the interior; the two-pass kernels use 32 x 8,
            // the fused ensemble kernels their own tile
            int etx = 32, ety = 8;
            if (!twopass) ensemble_tile_shape(gs.desc.precision == RHD_SPLIT ? 1 : 0, &etx, &ety);
            eg[i].tiles_x = (gs.desc.n[0] + etx - 1) / etx;
            eg[i].tiles_y = (gs.desc.n[1] + ety - 1) / ety;
            eg[i].tiles_z = (gs.desc.n[2] + gs.z_chunk - 1) / gs.z_chunk;
            eg[i].first_item = first;
            first += (long long)eg[i].tiles_x * eg[i].tiles_y * eg[i].tiles_z;
            if (twopass) {  // predictor items: 32 x 8 tiles of the stored U^{m+1/2} (ghost layers included)
                eg[i].uhalf = gs.uhalf;
                eg[i].ptiles_x = (upad_extent(gs.gp, 0) + 31) / 32;
                eg[i].ptiles_y = (upad_extent(gs.gp, 1) + 7) / 8;
                eg[i].ptiles_z = (upad_extent(gs.gp, 2) + gs.z_chunk - 1) / gs.z_chunk;
                eg[i].first_pitem = pfirst;
                pfirst += (long long)eg[i].ptiles_x * eg[i].ptiles_y * eg[i].ptiles_z;
            }
            if (src == 0) *dt_sig = *dt_sig * 1.000000119 + dt_per_grid[i];
        }
        ctx->n_items = first;
        ctx->n_pitems = pfirst;
        RHD_CUDA(ctx, cudaMemcpyAsync(ctx->d_egrids[src], eg.data(), sizeof(EnsembleGrid) * (size_t)ng,
                                      cudaMemcpyHostToDevice, ctx->stream));
    }
    return RHD_OK;
}

// One subcycle of every grid reading buffer src: one persistent launch (fused), or a persistent
// predictor launch followed by a persistent corrector launch (two-pass).
rhd_status ens_launch(rhd_ctx* ctx, double chat, int src)
{
    const bool split = ctx->grids[0].desc.precision == RHD_SPLIT;
    const bool twopass = ctx->grids[0].variant == RHD_VARIANT_TWOPASS;
    EnsembleParams ep;
    std::memset(&ep, 0, sizeof(ep));
    ep.grids = ctx->d_egrids[src];
    ep.n_grids = (int)ctx->grids.size();
    ep.n_items = ctx->n_items;
    ep.n_pitems = ctx->n_pitems;
    ep.chat = chat;
    ep.f_chat = (float)chat;
    ep.z_chunk = ctx->grids[0].z_chunk;
    ep.limiter = ctx->grids[0].desc.limiter;
    ep.stats = ctx->dstats;
    if (!twopass) {
        double bytes = 0.0;
        for (auto& gs : ctx->grids) {
            bytes += (double)gs.ncell * alg_bytes_per_cell(gs, K_FUSED_FP64);
            gs.um32_ok = false;
        }
        ep.counter = ctx->d_counter;
        RHD_CUDA(ctx, cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned long long), ctx->stream));
        return timed_launch(ctx, split ? K_ENS_SPLIT : K_ENS_FP64, bytes, [&] {
            return split ? launch_ensemble_split(ep, ctx->ens_ctas, ctx->stream)
                         : launch_ensemble_fp64(ep, ctx->ens_ctas, ctx->stream);
        });
    }
    double pbytes = 0.0, cbytes = 0.0;
    for (auto& gs : ctx->grids) {
        pbytes += (double)gs.ncell * alg_bytes_per_cell(gs, K_PREDICTOR);
        cbytes += (double)gs.ncell * alg_bytes_per_cell(gs, K_CORRECTOR);
    }
    RHD_CUDA(ctx, cudaMemsetAsync(ctx->d_counter, 0, 2 * sizeof(unsigned long long), ctx->stream));
    ep.counter = ctx->d_counter;
    rhd_status st = timed_launch(ctx, K_ENS_PRED, pbytes,
                                 [&] { return launch_ensemble_predictor(ep, ctx->ens_pctas, ctx->stream); });
    if (st) return st;
    ep.counter = ctx->d_counter + 1;
    return timed_launch(ctx, K_ENS_CORR, cbytes,
                        [&] { return launch_ensemble_corrector(ep, ctx->ens_cctas, ctx->stream); });
}

// ---------------------------------------------------------------------------------------------
// launch configurations and the autotuner
// ---------------------------------------------------------------------------------------------

rhd_launch_config current_config(const GridState& gs)
{
    rhd_launch_config c;
    c.variant = gs.variant;
    c.tile_x = gs.variant == RHD_VARIANT_TWOPASS ? 32 : gs.tx;
    c.tile_y = gs.variant == RHD_VARIANT_TWOPASS ? 8 : gs.ty;
    c.z_chunk = gs.z_chunk;
    c.staging = gs.staging;
    c.ms_per_subcycle = gs.tuned_ms;
    return c;
}

bool config_supported(const GridState& gs, const rhd_launch_config& c)
{
    const int nact = gs.gp.nact, prec = gs.desc.precision;
    if (c.z_chunk < 1) return false;
    if (c.variant == RHD_VARIANT_TWOPASS)
        // TMA copies one box per plane, which cannot wrap around a periodic x or y; the linear
        // exchange runs in the fused kernels only
        return prec == RHD_SPLIT && nact == 3 && gs.desc.exchange != RHD_EX_LINEAR && c.tile_x == 32 && c.tile_y == 8 &&
               (c.staging == RHD_STAGING_CPASYNC ||
                (c.staging == RHD_STAGING_TMA && tma_available() && gs.gp.pad[0] && gs.gp.pad[1]));
    if (c.variant != RHD_VARIANT_FUSED || c.staging != RHD_STAGING_CPASYNC) return false;
    return tile_supported(prec, nact, c.tile_x, c.tile_y);
}

// Make c the configuration of gs (c must be supported); allocates or frees the U^{m+1/2} buffer.
rhd_status apply_config(rhd_ctx* ctx, GridState& gs, const rhd_launch_config& c)
{
    if (c.variant == RHD_VARIANT_TWOPASS) {
        rhd_status st = alloc_twopass(ctx, gs);
        if (st) return st;
    } else {
        free_twopass(gs);
    }
    gs.um32_ok = false;
    if (c.staging == RHD_STAGING_TMA) {
        gs.uh_map_ok = encode_uhalf_map(&gs.uh_map, gs.uhalf, gs.gp);
        if (!gs.uh_map_ok) return fail(ctx, RHD_ERR_CUDA, "tensor map of U^{m+1/2} could not be encoded");
    } else {
        gs.uh_map_ok = false;
    }
    gs.variant = c.variant;
    gs.staging = c.staging;
    gs.tx = c.tile_x;
    gs.ty = c.tile_y;
    gs.tiles_x = (gs.desc.n[0] + gs.tx - 1) / gs.tx;
    gs.tiles_y = (gs.desc.n[1] + gs.ty - 1) / gs.ty;
    gs.z_chunk = std::max(1, std::min(c.z_chunk, gs.desc.n[2]));
    clear_graphs(ctx);
    return RHD_OK;
}

std::vector<rhd_launch_config> grid_candidates(const GridState& gs)
{
    std::vector<rhd_launch_config> v;
    auto add = [&](int variant, int tx, int ty, int zc, int staging) {
        rhd_launch_config c = {variant, tx, ty, std::max(1, std::min(zc, gs.desc.n[2])), staging, -1.0};
        if (!config_supported(gs, c)) return;
        for (auto& o : v)
            if (o.variant == c.variant && o.tile_x == c.tile_x && o.tile_y == c.tile_y && o.z_chunk == c.z_chunk &&
                o.staging == c.staging)
                return;
        v.push_back(c);
    };
    if (gs.gp.nact < 3) {
        rhd_launch_config c = current_config(gs);
        add(c.variant, c.tile_x, c.tile_y, c.z_chunk, c.staging);
    } else if (gs.desc.precision == RHD_FP64) {
        for (int zc : {8, 16, 32, 64, 128, 256, 512}) add(RHD_VARIANT_FUSED, 16, 16, zc, RHD_STAGING_CPASYNC);
    } else {
        for (int stg : {RHD_STAGING_CPASYNC, RHD_STAGING_TMA})
            for (int zc : {16, 32, 64, 128}) add(RHD_VARIANT_TWOPASS, 32, 8, zc, stg);
        const int tiles[3][2] = {{32, 8}, {32, 16}, {64, 8}};
        for (auto& t : tiles)
            for (int zc : {32, 64, 128}) add(RHD_VARIANT_FUSED, t[0], t[1], zc, RHD_STAGING_CPASYNC);
    }
    return v;
}

// Copies of what a timed candidate run overwrites: the temperature (updated in place by the FULL
// exchange) of every grid, and the statistics.
struct TuneBackup {
    std::vector<double*> T;
    DevStats* stats = nullptr;
};

rhd_status tune_backup(rhd_ctx* ctx, TuneBackup& b)
{
    b.T.assign(ctx->grids.size(), nullptr);
    for (size_t i = 0; i < ctx->grids.size(); ++i) {
        GridState& gs = ctx->grids[i];
        if (gs.desc.exchange != RHD_EX_FULL && gs.desc.exchange != RHD_EX_LINEAR) continue;
        rhd_status st = dalloc(ctx, (void**)&b.T[i], sizeof(double) * (size_t)gs.ncell);
        if (st) return st;
        RHD_CUDA(ctx, cudaMemcpyAsync(b.T[i], gs.T, sizeof(double) * (size_t)gs.ncell, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    }
    rhd_status st = dalloc(ctx, (void**)&b.stats, sizeof(DevStats));
    if (st) return st;
    RHD_CUDA(ctx, cudaMemcpyAsync(b.stats, ctx->dstats, sizeof(DevStats), cudaMemcpyDeviceToDevice, ctx->stream));
    return RHD_OK;
}

rhd_status tune_restore(rhd_ctx* ctx, TuneBackup& b)
{
    for (size_t i = 0; i < ctx->grids.size(); ++i)
        if (b.T[i])
            RHD_CUDA(ctx, cudaMemcpyAsync(ctx->grids[i].T, b.T[i], sizeof(double) * (size_t)ctx->grids[i].ncell,
                                          cudaMemcpyDeviceToDevice, ctx->stream));
    if (b.stats)
        RHD_CUDA(ctx, cudaMemcpyAsync(ctx->dstats, b.stats, sizeof(DevStats), cudaMemcpyDeviceToDevice, ctx->stream));
    return RHD_OK;
}

void tune_free(TuneBackup& b)
{
    for (auto& p : b.T) dfree(p);
    dfree(b.stats);
}

// Mean milliseconds per launch of reps launches of fn (after one warm-up), on the context's stream;
// every launch reads the current buffer, so the state does not advance.
template <typename Fn>
rhd_status time_launches(rhd_ctx* ctx, int reps, Fn&& fn, double* ms)
{
    *ms = -1.0;
    rhd_status st = fn();
    if (st) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RHD_CUDA(ctx, cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, RHD_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
    }
    ce = cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < reps && ce == cudaSuccess && st == RHD_OK; ++r) st = fn();
    if (ce == cudaSuccess && st == RHD_OK) ce = cudaEventRecord(e1, ctx->stream);
    if (ce == cudaSuccess && st == RHD_OK) ce = cudaEventSynchronize(e1);
    float f = 0.0f;
    if (ce == cudaSuccess && st == RHD_OK) ce = cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (ce != cudaSuccess) return fail(ctx, RHD_ERR_CUDA, std::string("tuning timer: ") + cudaGetErrorString(ce));
    *ms = (double)f / reps;
    return RHD_OK;
}

void report(const std::vector<rhd_launch_config>& all, const rhd_launch_config& best, rhd_launch_config* table,
            int capacity, int* n_entries, rhd_launch_config* chosen)
{
    if (table)
        for (int i = 0; i < (int)all.size() && i < capacity; ++i) table[i] = all[i];
    if (n_entries) *n_entries = (int)all.size();
    if (chosen) *chosen = best;
}

// Choices already made in this process, by grid shape and mode.
std::mutex g_tune_mutex;
std::map<std::string, rhd_launch_config> g_tune_cache;

std::string tune_key(rhd_ctx* ctx)
{
    std::string k = std::to_string(ctx->device) + (ctx->ensemble ? "E" : "G");
    for (auto& gs : ctx->grids) {
        const rhd_grid_desc& d = gs.desc;
        k += ":" + std::to_string(d.n[0]) + "x" + std::to_string(d.n[1]) + "x" + std::to_string(d.n[2]) + "/" +
             std::to_string(d.precision) + std::to_string(gs.gp.exchange) + std::to_string(d.beta_tau) +
             std::to_string(d.limiter) + std::to_string(d.closure) + std::to_string(d.speeds) +
             std::to_string(gs.has_v) + std::to_string(gs.has_kP) + std::to_string(gs.has_kF) +
             std::to_string(gs.has_j);
    }
    return k;
}

rhd_status grid_autotune(rhd_ctx* ctx, double chat, double dt, int reps, rhd_launch_config* table, int capacity,
                         int* n_entries, rhd_launch_config* chosen)
{
    GridState& gs = ctx->grids[0];
    std::vector<rhd_launch_config> cand = grid_candidates(gs);
    const rhd_launch_config before = current_config(gs);
    rhd_status st = enter(ctx);
    if (st) return st;
    TuneBackup b;
    if ((st = tune_backup(ctx, b))) {
        tune_free(b);
        return st;
    }
    int best = -1;
    for (size_t i = 0; i < cand.size() && !st; ++i) {
        if ((st = apply_config(ctx, gs, cand[i]))) {
            if (st != RHD_ERR_OOM) break;
            st = RHD_OK;  // e.g. no room for the U^{m+1/2} buffer: the candidate is skipped
            continue;
        }
        double ms = -1.0;
        st = prepare_twopass(ctx, gs);
        if (!st) st = time_launches(ctx, reps, [&] { return launch_one(ctx, gs, ctx->cur, chat, dt); }, &ms);
        gs.um32_ok = false;  // the timed correctors rewrote the mirror with the next state
        if (!st) st = tune_restore(ctx, b);
        cand[i].ms_per_subcycle = ms;
        if (!st && ms >= 0.0 && (best < 0 || ms < cand[best].ms_per_subcycle)) best = (int)i;
    }
    rhd_status st2 = RHD_OK;
    if (!st) st2 = apply_config(ctx, gs, best >= 0 ? cand[best] : before);
    if (!st && !st2) st2 = tune_restore(ctx, b);
    cudaError_t ce = cudaStreamSynchronize(ctx->stream);
    tune_free(b);
    if (st) return st;
    if (st2) return st2;
    if (ce != cudaSuccess) return fail(ctx, RHD_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
    gs.tuned = true;
    gs.tuned_ms = best >= 0 ? cand[best].ms_per_subcycle : -1.0;
    report(cand, current_config(gs), table, capacity, n_entries, chosen);
    if (log_level() >= 2) {
        const rhd_launch_config c = current_config(gs);
        std::fprintf(stderr, "rhd: tuned %dx%dx%d: variant %d tile %dx%d z %d staging %d, %.3f ms per subcycle\n",
                     gs.desc.n[0], gs.desc.n[1], gs.desc.n[2], c.variant, c.tile_x, c.tile_y, c.z_chunk, c.staging,
                     c.ms_per_subcycle);
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[tune_key(ctx)] = current_config(gs);
    }
    return leave(ctx);
}

rhd_status grid_tune_once(rhd_ctx* ctx, double chat, double dt)
{
    GridState& gs = ctx->grids[0];
    rhd_launch_config c;
    bool hit = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(tune_key(ctx));
        if (it != g_tune_cache.end()) {
            c = it->second;
            hit = true;
        }
    }
    if (hit && config_supported(gs, c)) {
        rhd_status st = apply_config(ctx, gs, c);
        if (st) return st;
        gs.tuned = true;
        gs.tuned_ms = c.ms_per_subcycle;
        return RHD_OK;
    }
    return grid_autotune(ctx, chat, dt, 3, nullptr, 0, nullptr, nullptr);
}

// Make every grid of an ensemble use variant v with z chunk zc (allocating or freeing U^{m+1/2}).
rhd_status ens_apply(rhd_ctx* ctx, int v, int zc)
{
    for (auto& gs : ctx->grids) {
        if (v == RHD_VARIANT_TWOPASS) {
            rhd_status st = alloc_twopass(ctx, gs);
            if (st) return st;
        }
    }
    for (auto& gs : ctx->grids) {
        if (v != RHD_VARIANT_TWOPASS) free_twopass(gs);
        gs.um32_ok = false;
        gs.variant = v;
        gs.z_chunk = zc;  // one chunk length for all grids, as at creation
    }
    clear_graphs(ctx);
    return RHD_OK;
}

rhd_status ensemble_autotune(rhd_ctx* ctx, double chat, const double* dt_per_grid, int reps,
                             rhd_launch_config* table, int capacity, int* n_entries, rhd_launch_config* chosen)
{
    GridState& g0 = ctx->grids[0];
    const bool split = g0.desc.precision == RHD_SPLIT;
    int max_nz = 1;
    for (auto& gs : ctx->grids) max_nz = std::max(max_nz, gs.desc.n[2]);
    std::vector<rhd_launch_config> cand;
    auto add = [&](int v, int zc) {
        if (zc > max_nz && zc != 8) return;
        if (v == RHD_VARIANT_TWOPASS) cand.push_back({v, 32, 8, zc, RHD_STAGING_CPASYNC, -1.0});
        else cand.push_back({v, g0.tx, g0.ty, zc, RHD_STAGING_CPASYNC, -1.0});
    };
    if (split && g0.desc.exchange != RHD_EX_LINEAR)
        for (int zc : {16, 32, 64}) add(RHD_VARIANT_TWOPASS, zc);
    for (int zc : {8, 16, 32, 64, 128}) add(RHD_VARIANT_FUSED, zc);
    const int v_before = g0.variant, zc_before = g0.z_chunk;
    rhd_status st = enter(ctx);
    if (st) return st;
    TuneBackup b;
    if ((st = tune_backup(ctx, b))) {
        tune_free(b);
        return st;
    }
    int best = -1;
    for (size_t i = 0; i < cand.size() && !st; ++i) {
        if ((st = ens_apply(ctx, cand[i].variant, cand[i].z_chunk))) {
            if (st != RHD_ERR_OOM) break;
            st = RHD_OK;  // no room for the U^{m+1/2} buffers: skipped
            continue;
        }
        double dt_sig = 0.0, ms = -1.0;
        for (auto& gs : ctx->grids)
            if (!st) st = prepare_twopass(ctx, gs);
        if (!st) st = ens_prepare(ctx, chat, dt_per_grid, &dt_sig);
        if (!st) st = time_launches(ctx, reps, [&] { return ens_launch(ctx, chat, ctx->cur); }, &ms);
        for (auto& gs : ctx->grids) gs.um32_ok = false;
        if (!st) st = tune_restore(ctx, b);
        cand[i].ms_per_subcycle = ms;
        if (!st && ms >= 0.0 && (best < 0 || ms < cand[best].ms_per_subcycle)) best = (int)i;
    }
    rhd_status st2 = RHD_OK;
    if (!st) st2 = best >= 0 ? ens_apply(ctx, cand[best].variant, cand[best].z_chunk) : ens_apply(ctx, v_before, zc_before);
    if (!st && !st2) st2 = tune_restore(ctx, b);
    cudaError_t ce = cudaStreamSynchronize(ctx->stream);
    tune_free(b);
    if (st) return st;
    if (st2) return st2;
    if (ce != cudaSuccess) return fail(ctx, RHD_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
    g0.tuned = true;
    g0.tuned_ms = best >= 0 ? cand[best].ms_per_subcycle : -1.0;
    rhd_launch_config cur = current_config(g0);
    report(cand, cur, table, capacity, n_entries, chosen);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[tune_key(ctx)] = cur;
    }
    return leave(ctx);
}

rhd_status ensemble_tune_once(rhd_ctx* ctx, double chat, const double* dt_per_grid)
{
    GridState& g0 = ctx->grids[0];
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(tune_key(ctx));
        if (it != g_tune_cache.end()) {
            rhd_status st = ens_apply(ctx, it->second.variant, it->second.z_chunk);
            if (st) return st;
            g0.tuned = true;
            g0.tuned_ms = it->second.ms_per_subcycle;
            return RHD_OK;
        }
    }
    return ensemble_autotune(ctx, chat, dt_per_grid, 3, nullptr, 0, nullptr, nullptr);
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
// ---------------------------------------------------------------------------------------------
// reduced-speed-of-light helpers (Sections 3.1, 3.2)
// ---------------------------------------------------------------------------------------------
namespace {

double active_dx_min(const rhd_grid_desc& d)
{
    double m = INFINITY;
    for (int k = 0; k < 3; ++k)
        if (d.n[k] > 1) m = std::min(m, d.dx[k]);
    return std::isfinite(m) ? m : d.dx[0];
}

// one grid-wide maximum: the single grid of a context with its state set, the reduction buffer,
// the launch (fill), the result copied back
template <class Fill>
rhd_status grid_maximum(rhd_ctx* ctx, double* out, bool need_moments, const char* what, Fill fill)
{
    if (!ctx || !out) return fail(ctx, RHD_ERR_ARG, "ctx and the output are required");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "not available on an ensemble context");
    GridState& gs = ctx->grids[0];
    if (!gs.has_gas || (need_moments && !gs.has_moments))
        return fail(ctx, RHD_ERR_STATE, need_moments ? "set the moments and the gas state first" : "set the gas state first");
    rhd_status st = enter(ctx);
    if (st) return st;
    const int nb = rsla_blocks(ctx->num_sms);
    if (!ctx->rsla_partial && (st = dalloc(ctx, (void**)&ctx->rsla_partial, sizeof(double) * (size_t)(nb + 1))))
        return st;
    RHD_CUDA(ctx, fill(gs, nb, ctx->rsla_partial));
    double h = 0.0;
    RHD_CUDA(ctx, cudaMemcpyAsync(&h, ctx->rsla_partial + nb, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if ((st = leave(ctx))) return st;
    RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *out = h;
    if (!std::isfinite(h)) return fail(ctx, RHD_ERR_NONFINITE, std::string(what) + " is not finite");
    return RHD_OK;
}

}  // namespace

extern "C" {

int rhd_abi_version(void) { return RHD_ABI_VERSION; }
int rhd_built_arch(void) { return 103; }
int rhd_bounds_checked(void) { return (bounds_checked_fp64() && bounds_checked_split()) ? 1 : 0; }

const char* rhd_last_error(const rhd_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

rhd_status rhd_init_grid(rhd_ctx** out, const rhd_grid_desc* d)
{
    ApiRange range_("rhd_init_grid");
    if (!out) return fail(nullptr, RHD_ERR_ARG, "out is NULL");
    rhd_status st = validate_desc(nullptr, d);
    if (st) return st;
    rhd_ctx* ctx = new (std::nothrow) rhd_ctx();
    if (!ctx) return fail(nullptr, RHD_ERR_OOM, "host allocation failed");
    ctx->user_stream = (cudaStream_t)d->cuda_stream;
    st = common_init(ctx);
    if (!st) {
        ctx->grids.resize(1);
        GridState& gs = ctx->grids[0];
        gs.desc = *d;
        gs.ncell = (long long)d->n[0] * d->n[1] * d->n[2];
        fill_params(gs);
        // split 3D grids: the two-pass kernels unless the fused kernel is asked for
        if (d->precision == RHD_SPLIT && gs.gp.nact == 3 && d->exchange != RHD_EX_LINEAR) {
            gs.variant = (d->flags & RHD_FLAG_SPLIT_FUSED) ? 0 : 1;
            if (const char* v = std::getenv("RHD_VARIANT")) gs.variant = std::strcmp(v, "fused") == 0 ? 0 : 1;
            // the two kernels recompute nothing across z chunks but two predictor planes: short chunks
            // cost little and fill the GPU evenly
            if (gs.variant == 1 && d->z_chunk == 0) gs.z_chunk = std::min(32, d->n[2]);
        }
        st = alloc_grid(ctx, gs);
    }
    if (st) {
        g_init_error = ctx->err;
        destroy_ctx(ctx);
        return st;
    }
    *out = ctx;
    return RHD_OK;
}

rhd_status rhd_destroy(rhd_ctx* ctx)
{
    destroy_ctx(ctx);
    return RHD_OK;
}

rhd_status rhd_set_gas_state(rhd_ctx* ctx, const double* rho, const double* T, const double* vx, const double* vy,
                             const double* vz, const double* kP, const double* kF, const double* j, int on_device)
{
    ApiRange range_("rhd_set_gas_state");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "use rhd_ensemble_set_gas_state on an ensemble");
    return set_gas(ctx, ctx->grids[0], rho, T, vx, vy, vz, kP, kF, j, on_device);
}

rhd_status rhd_set_moments(rhd_ctx* ctx, const double* E, const double* Fx, const double* Fy, const double* Fz,
                           int on_device)
{
    ApiRange range_("rhd_set_moments");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "use rhd_ensemble_set_moments on an ensemble");
    return set_moments(ctx, ctx->grids[0], E, Fx, Fy, Fz, on_device);
}

rhd_status rhd_set_conserved(rhd_ctx* ctx, const double* E, const double* Gx, const double* Gy, const double* Gz,
                             int on_device)
{
    ApiRange range_("rhd_set_conserved");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "not available on an ensemble context");
    return set_moments(ctx, ctx->grids[0], E, Gx, Gy, Gz, on_device, true);
}

rhd_status rhd_get_conserved(rhd_ctx* ctx, double* E, double* Gx, double* Gy, double* Gz, int on_device)
{
    ApiRange range_("rhd_get_conserved");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "not available on an ensemble context");
    return get_moments(ctx, ctx->grids[0], E, Gx, Gy, Gz, on_device, true);
}

rhd_status rhd_set_dirichlet(rhd_ctx* ctx, int face, const double state[4])
{
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (face < 0 || face > 5 || !state) return fail(ctx, RHD_ERR_ARG, "face must be in [0, 5] and state non-NULL");
    for (int q = 0; q < 4; ++q)
        if (!std::isfinite(state[q])) return fail(ctx, RHD_ERR_ARG, "Dirichlet state must be finite");
    for (auto& gs : ctx->grids) {
        double* dst = (face & 1) ? gs.gp.dir_hi[face >> 1] : gs.gp.dir_lo[face >> 1];
        dst[0] = state[0];
        for (int q = 1; q < 4; ++q) dst[q] = state[q] / gs.desc.c;
    }
    clear_graphs(ctx);
    return RHD_OK;
}

rhd_status rhd_radiation_subcycle(rhd_ctx* ctx, int n_sub, double chat, double dt)
{
    ApiRange range_("rhd_radiation_subcycle");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "use rhd_ensemble_subcycle on an ensemble");
    if (n_sub < 0) return fail(ctx, RHD_ERR_ARG, "n_sub must be >= 0");
    GridState& gs = ctx->grids[0];
    rhd_status st = check_dt(ctx, gs, chat, dt);
    if (st) return st;
    if (!gs.has_moments || !gs.has_gas) return fail(ctx, RHD_ERR_STATE, "set the moments and the gas state first");
    if (n_sub == 0) return RHD_OK;
    if ((gs.desc.flags & RHD_FLAG_AUTOTUNE) && !gs.tuned && (st = grid_tune_once(ctx, chat, dt))) return st;
    if ((st = enter(ctx))) return st;
    if ((st = prepare_twopass(ctx, gs))) return st;
    bool use_graph = !(gs.desc.flags & RHD_FLAG_NO_GRAPH) && !ctx->ktiming;
    st = run_steps(ctx, n_sub, chat, dt, use_graph, [&](int src) { return launch_one(ctx, gs, src, chat, dt); });
    if (st) return st;
    ctx->cur = (ctx->cur + n_sub) & 1;
    ctx->n_subcycles += n_sub;
    return leave(ctx);
}

rhd_status rhd_marshak_advance(rhd_ctx* ctx, int n_sub, double chat, double dt, double t0, double tau_rate, double eps,
                               double F_inc, int n_quad)
{
    ApiRange range_("rhd_marshak_advance");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "not available on an ensemble context");
    if (n_sub < 0 || n_quad < 1 || !std::isfinite(t0) || !finite_pos(tau_rate) || !finite_pos(eps) ||
        !(std::isfinite(F_inc) && F_inc >= 0.0))
        return fail(ctx, RHD_ERR_ARG, "need n_sub >= 0, n_quad >= 1, finite t0, tau_rate > 0, eps > 0, F_inc >= 0");
    GridState& gs = ctx->grids[0];
    rhd_status st = check_dt(ctx, gs, chat, dt);
    if (st) return st;
    if (!gs.has_moments || !gs.has_gas) return fail(ctx, RHD_ERR_STATE, "set the moments and the gas state first");
    if (gs.desc.bc_lo[0] != RHD_BC_DIRICHLET) return fail(ctx, RHD_ERR_ARG, "the low x face must be Dirichlet");
    if (gs.desc.precision == RHD_SPLIT && gs.variant == RHD_VARIANT_TWOPASS)
        return fail(ctx, RHD_ERR_UNSUPPORTED, "the device boundary state is read by the fused kernels only");
    if (n_sub == 0) return RHD_OK;
    if ((st = enter(ctx))) return st;
    if (ctx->marshak_cap < n_sub) {
        // the stream may still read the old states: wait before replacing them
        RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(ctx->marshak_state);
        ctx->marshak_cap = 0;
        if ((st = dalloc(ctx, (void**)&ctx->marshak_state, 4 * sizeof(double) * (size_t)n_sub))) return st;
        ctx->marshak_cap = n_sub;
    }
    // every subcycle's boundary state at once (one block each), then the subcycles, each reading its own
    RHD_CUDA(ctx, launch_marshak_boundary(t0, dt, tau_rate, eps, F_inc, gs.desc.c, n_quad, n_sub, ctx->marshak_state,
                                          ctx->stream));
    for (int m = 0; m < n_sub && !st; ++m) {
        gs.dir_dev = ctx->marshak_state + 4 * (size_t)m;
        st = launch_one(ctx, gs, (ctx->cur + m) & 1, chat, dt);
    }
    gs.dir_dev = nullptr;
    if (st) return st;
    ctx->cur = (ctx->cur + n_sub) & 1;
    ctx->n_subcycles += n_sub;
    return leave(ctx);
}

namespace {

GasParams gas_params(const GridState& gs, double dt)
{
    GasParams p;
    std::memset(&p, 0, sizeof(p));
    gas_set_geometry(p, gs.desc.n, gs.desc.bc_lo, gs.desc.bc_hi);
    for (int d = 0; d < 3; ++d) p.inv_dx[d] = gs.desc.n[d] > 1 ? 1.0 / gs.desc.dx[d] : 0.0;
    p.gamma = gs.desc.gamma;
    p.gm1 = gs.desc.gamma - 1.0;
    p.inv_gm1 = 1.0 / p.gm1;
    p.mu_over_kB = gs.desc.mu_over_kB;
    p.inv_mu = 1.0 / gs.desc.mu_over_kB;
    p.inv_c = 1.0 / gs.desc.c;
    p.kappa_F = gs.desc.kappa_F;
    p.kpow = gs.desc.kappa_rho_pow;
    p.beta_tau = gs.desc.beta_tau;
    p.limiter = gs.desc.limiter;
    p.dt = dt;
    p.split = gs.desc.precision == RHD_SPLIT;
    p.f_gamma = (float)p.gamma;
    p.f_inv_gm1 = (float)p.inv_gm1;
    p.f_inv_mu = (float)p.inv_mu;
    for (int d = 0; d < 3; ++d) p.f_inv_dx[d] = (float)p.inv_dx[d];
    p.f_gm1 = (float)p.gm1;
    p.f_gm1_mu = (float)(p.gm1 * p.mu_over_kB);
    p.f_inv_gm1_mu = (float)(1.0 / (p.gm1 * p.mu_over_kB));
    p.f_inv_c = (float)p.inv_c;
    p.f_kappa_F = (float)p.kappa_F;
    return p;
}

GasArrays gas_arrays(rhd_ctx* ctx, GridState& gs)
{
    GasArrays a;
    std::memset(&a, 0, sizeof(a));
    a.rho = gs.rho;
    a.T = gs.T;
    for (int d = 0; d < 3; ++d) a.v[d] = gs.v[d];
    a.rho32 = gs.rho32;
    for (int d = 0; d < 3; ++d) a.v32[d] = gs.v32[d];
    a.kF = gs.has_kF ? gs.kF : nullptr;
    a.E = gs.U[ctx->cur][0];
    for (int d = 0; d < 3; ++d) a.G[d] = gs.U[ctx->cur][1 + d];
    for (int q = 0; q < 5; ++q) {
        a.wh[q] = gs.gas_wh[q];
        a.wh32[q] = gs.gas_wh32[q];
    }
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 5; ++q) a.flux[d][q] = gs.gas_flux[d][q];
    for (int q = 0; q < 8; ++q) a.pend[q] = gs.gas_pend[q];
    a.counters = ctx->gas_counters;
    return a;
}

// The gas step's scratch, and all three velocity components (a component that was never given starts
// at zero: the radiation force and the fluxes make it nonzero).
rhd_status gas_prepare(rhd_ctx* ctx, GridState& gs, const GasParams& p)
{
    rhd_status st;
    if (!gs.gas_wh[0] && !gs.gas_wh32[0]) {
        const size_t fb = p.split ? sizeof(float) : sizeof(double);
        for (int q = 0; q < 5; ++q) {
            if (!p.split && (st = dalloc(ctx, (void**)&gs.gas_wh[q], sizeof(double) * (size_t)gas_count(p.m))))
                return st;
            if (p.split && (st = dalloc(ctx, (void**)&gs.gas_wh32[q], sizeof(float) * (size_t)gas_count(p.m))))
                return st;
        }
        for (int d = 0; d < 3; ++d) {
            if (gs.desc.n[d] <= 1) continue;
            for (int q = 0; q < 5; ++q)
                if ((st = dalloc(ctx, (void**)&gs.gas_flux[d][q], fb * (size_t)gas_face_capacity(p, d)))) return st;
        }
        for (int q = 0; q < 8; ++q)
            if ((st = dalloc(ctx, (void**)&gs.gas_pend[q], sizeof(double) * (size_t)gs.ncell))) return st;
    }
    bool added = false;
    for (int d = 0; d < 3; ++d) {
        if (gs.v[d]) continue;
        if ((st = dalloc(ctx, (void**)&gs.v[d], sizeof(double) * (size_t)gs.ncell))) return st;
        RHD_CUDA(ctx, cudaMemsetAsync(gs.v[d], 0, sizeof(double) * (size_t)gs.ncell, ctx->stream));
        if (gs.desc.precision == RHD_SPLIT) {
            if (!gs.v32[d] && (st = dalloc(ctx, (void**)&gs.v32[d], sizeof(float) * (size_t)gs.ncell))) return st;
            RHD_CUDA(ctx, cudaMemsetAsync(gs.v32[d], 0, sizeof(float) * (size_t)gs.ncell, ctx->stream));
        }
        added = true;
    }
    if (added) {
        gs.has_v = true;
        clear_graphs(ctx);  // the subcycle kernels' velocity pointers changed
    }
    return RHD_OK;
}

// After the gas changed: the FP32 copies the split subcycles read
rhd_status gas_refresh_copies(rhd_ctx* ctx, GridState& gs)
{
    if (gs.desc.precision == RHD_SPLIT) {
        RHD_CUDA(ctx, launch_to_float(gs.rho32, gs.rho, gs.ncell, ctx->stream));
        for (int d = 0; d < 3; ++d) RHD_CUDA(ctx, launch_to_float(gs.v32[d], gs.v[d], gs.ncell, ctx->stream));
    }
    gs.gas4_ok = false;
    return RHD_OK;
}

// bytes per cell of each gas kernel (each array read or written once per launch): the gas state is
// 40 B (rho, T, v; on split grids the predictor reads the FP32 rho, v and the FP64 T, 24 B), W^{n+1/2}
// 40 B (20 B in FP32 on split grids), one face-flux array 40 B per cell (20 B split), the radiation
// 32 B, the correction's record 64 B
double gas_alg_bytes(const GridState& gs, int k, int nact)
{
    const bool split = gs.desc.precision == RHD_SPLIT;
    const double kf = gs.has_kF ? 8.0 : 0.0, fl = split ? 20.0 : 40.0;
    switch (k) {
    case K_GAS_PRED_FLUX: return (split ? 24.0 : 40.0) + fl;
    case K_GAS_PRED_UPDATE: return (split ? 24.0 : 40.0) + 32.0 + kf + fl * nact + (split ? 20.0 : 40.0);
    case K_GAS_CORR_FLUX: return (split ? 20.0 : 40.0) + fl;
    case K_GAS_CORR_UPDATE: return 40.0 + fl * nact + (split ? 16.0 : 32.0) + 32.0 + kf + 40.0 + 64.0;
    default: return 40.0 + 64.0 + 32.0 + 32.0;  // K_GAS_CORRECT
    }
}

rhd_status single_grid(rhd_ctx* ctx, const char* what)
{
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, std::string(what) + " runs on single grids, not ensembles");
    const GridState& gs = ctx->grids[0];
    if (!gs.has_gas || !gs.has_moments) return fail(ctx, RHD_ERR_STATE, "set the gas state and the moments first");
    return RHD_OK;
}

}  // namespace

rhd_status rhd_gas_step(rhd_ctx* ctx, double dt_gas)
{
    ApiRange range_("rhd_gas_step");
    rhd_status st = single_grid(ctx, "rhd_gas_step");
    if (st) return st;
    if (!(std::isfinite(dt_gas) && dt_gas >= 0.0)) return fail(ctx, RHD_ERR_ARG, "dt_gas must be finite and >= 0");
    GridState& gs = ctx->grids[0];
    if ((st = enter(ctx))) return st;
    const GasParams p = gas_params(gs, dt_gas);
    if ((st = gas_prepare(ctx, gs, p))) return st;
    const GasArrays a = gas_arrays(ctx, gs);
    const double ext = (double)gas_count(p.m), nc = (double)gs.ncell;
    int nact = 0;
    for (int d = 0; d < 3; ++d) nact += gs.desc.n[d] > 1;
    cudaStream_t s = ctx->stream;
    for (int d = 0; d < 3; ++d) {
        if (gs.desc.n[d] <= 1) continue;
        if ((st = timed_launch(ctx, K_GAS_PRED_FLUX, ext * gas_alg_bytes(gs, K_GAS_PRED_FLUX, nact),
                               [&] { return launch_gas_pred_flux(p, a, d, s); })))
            return st;
    }
    if ((st = timed_launch(ctx, K_GAS_PRED_UPDATE, ext * gas_alg_bytes(gs, K_GAS_PRED_UPDATE, nact),
                           [&] { return launch_gas_pred_update(p, a, s); })))
        return st;
    for (int d = 0; d < 3; ++d) {
        if (gs.desc.n[d] <= 1) continue;
        if ((st = timed_launch(ctx, K_GAS_CORR_FLUX, nc * gas_alg_bytes(gs, K_GAS_CORR_FLUX, nact),
                               [&] { return launch_gas_corr_flux(p, a, d, s); })))
            return st;
    }
    if ((st = timed_launch(ctx, K_GAS_CORR_UPDATE, nc * gas_alg_bytes(gs, K_GAS_CORR_UPDATE, nact),
                           [&] { return launch_gas_corr_update(p, a, s); })))
        return st;
    if ((st = gas_refresh_copies(ctx, gs))) return st;
    gs.gas_pending = true;
    gs.gas_dt = dt_gas;
    return leave(ctx);
}

rhd_status rhd_gas_correct(rhd_ctx* ctx)
{
    ApiRange range_("rhd_gas_correct");
    rhd_status st = single_grid(ctx, "rhd_gas_correct");
    if (st) return st;
    GridState& gs = ctx->grids[0];
    if (!gs.gas_pending) return fail(ctx, RHD_ERR_STATE, "no gas step waits for its source correction");
    if ((st = enter(ctx))) return st;
    const GasParams p = gas_params(gs, gs.gas_dt);
    const GasArrays a = gas_arrays(ctx, gs);
    if ((st = timed_launch(ctx, K_GAS_CORRECT, (double)gs.ncell * gas_alg_bytes(gs, K_GAS_CORRECT, 0),
                           [&] { return launch_gas_correct(p, a, ctx->stream); })))
        return st;
    if ((st = gas_refresh_copies(ctx, gs))) return st;
    gs.gas_pending = false;
    return leave(ctx);
}

rhd_status rhd_gas_exchange(rhd_ctx* ctx, double dt_gas, double chat)
{
    ApiRange range_("rhd_gas_exchange");
    rhd_status st = single_grid(ctx, "rhd_gas_exchange");
    if (st) return st;
    GridState& gs = ctx->grids[0];
    if (!(gs.desc.flags & RHD_FLAG_EXCHANGE_ON_GAS_STEP))
        return fail(ctx, RHD_ERR_STATE, "the grid exchanges in its subcycles (no RHD_FLAG_EXCHANGE_ON_GAS_STEP)");
    if (!(std::isfinite(dt_gas) && dt_gas >= 0.0)) return fail(ctx, RHD_ERR_ARG, "dt_gas must be finite and >= 0");
    if (!(chat > 0.0 && chat <= gs.desc.c)) return fail(ctx, RHD_ERR_ARG, "chat must lie in (0, c]");
    if (!gs.has_moments || !gs.has_gas) return fail(ctx, RHD_ERR_STATE, "set the moments and the gas state first");
    if ((st = enter(ctx))) return st;
    GasExchangeParams p;
    std::memset(&p, 0, sizeof(p));
    p.g = gs.gp;
    p.g.exchange = RHD_EX_FULL;
    double** U = gs.U[ctx->cur];
    p.E = U[0];
    for (int q = 0; q < 3; ++q) p.G[q] = U[1 + q];
    p.T = gs.T;
    p.rho = gs.rho;
    p.kP = gs.has_kP ? gs.kP : nullptr;
    p.chat = chat;
    p.dt = dt_gas;
    p.n = gs.ncell;
    p.stats = ctx->dstats;
    // E, G, T: read 40 B and written 40 B per cell; rho (and kP) read
    const double bytes = (double)gs.ncell * (80.0 + 8.0 + (gs.has_kP ? 8.0 : 0.0));
    if ((st = timed_launch(ctx, K_GAS_EXCHANGE, bytes, [&] { return launch_gas_exchange(p, ctx->num_sms, ctx->stream); })))
        return st;
    gs.um32_ok = false;  // the state changed: the two-pass path's FP32 mirror is rebuilt before the next subcycle
    return leave(ctx);
}

rhd_status rhd_get_gas(rhd_ctx* ctx, double* rho, double* vx, double* vy, double* vz, double* T, int on_device)
{
    ApiRange range_("rhd_get_gas");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "rhd_get_gas runs on single grids, not ensembles");
    GridState& gs = ctx->grids[0];
    if (!gs.has_gas) return fail(ctx, RHD_ERR_STATE, "the gas state is not set");
    rhd_status st = enter(ctx);
    if (st) return st;
    const size_t bytes = sizeof(double) * (size_t)gs.ncell;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    double* out[5] = {rho, vx, vy, vz, T};
    const double* src[5] = {gs.rho, gs.v[0], gs.v[1], gs.v[2], gs.T};
    for (int q = 0; q < 5; ++q) {
        if (!out[q]) continue;
        if (src[q]) RHD_CUDA(ctx, cudaMemcpyAsync(out[q], src[q], bytes, kind, ctx->stream));
        else if (on_device) RHD_CUDA(ctx, cudaMemsetAsync(out[q], 0, bytes, ctx->stream));
        else std::memset(out[q], 0, bytes);
    }
    if ((st = leave(ctx))) return st;
    RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RHD_OK;
}

rhd_status rhd_get_moments(rhd_ctx* ctx, double* E, double* Fx, double* Fy, double* Fz, int on_device)
{
    ApiRange range_("rhd_get_moments");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "use rhd_ensemble_get_moments on an ensemble");
    return get_moments(ctx, ctx->grids[0], E, Fx, Fy, Fz, on_device);
}

rhd_status rhd_get_gas_state(rhd_ctx* ctx, double* T, int on_device)
{
    ApiRange range_("rhd_get_gas_state");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "use rhd_ensemble_get_gas_state on an ensemble");
    return get_T(ctx, ctx->grids[0], T, on_device);
}

rhd_status rhd_max_signal_speed(rhd_ctx* ctx, double* v_max)
{
    ApiRange range_("rhd_max_signal_speed");
    return grid_maximum(ctx, v_max, true, "v_max", [&](GridState& gs, int nb, double* part) {
        const double* v[3] = {gs.v[0], gs.v[1], gs.v[2]};
        return launch_signal_speed(gs.gp, gs.rho, gs.T, gs.U[ctx->cur][0], v, gs.has_kF ? gs.kF : nullptr,
                                   active_dx_min(gs.desc), gs.ncell, nb, part, ctx->stream);
    });
}

rhd_status rhd_max_optical_depth(rhd_ctx* ctx, double* tau_max)
{
    ApiRange range_("rhd_max_optical_depth");
    return grid_maximum(ctx, tau_max, false, "tau_max", [&](GridState& gs, int nb, double* part) {
        return launch_max_optical_depth(gs.gp, gs.has_kF ? gs.kF : nullptr, gs.rho, gs.desc.dx, nb, part, ctx->stream);
    });
}

rhd_status rhd_suggest_chat(double c, double v_max, double tau_max, double ratio, double* chat)
{
    if (!chat) return fail(nullptr, RHD_ERR_ARG, "chat is NULL");
    if (!finite_pos(c) || !finite_pos(v_max) || !finite_pos(ratio) || !(std::isfinite(tau_max) && tau_max >= 0.0))
        return fail(nullptr, RHD_ERR_ARG, "c, v_max and ratio must be positive and finite, tau_max finite and >= 0");
    *chat = std::min(c, ratio * v_max * std::max(1.0, tau_max));
    return RHD_OK;
}

// the fewest subcycles of length <= dmax spanning dg (Eq. algorithm:radtimestep)
static rhd_status span_subcycles(double dg, double dmax, double* dt_rad, int* n_sub)
{
    const double q = std::ceil(dg / dmax);
    if (!(q < 2147483647.0)) return fail(nullptr, RHD_ERR_ARG, "more than 2^31 subcycles per gas step");
    int n = std::max(1, (int)q);
    while (dg / n > dmax) ++n;
    *dt_rad = dg / n;
    *n_sub = n;
    return RHD_OK;
}

rhd_status rhd_time_steps(double cfl, double dx_min, double v_max, double chat, double* dt_gas, double* dt_rad,
                          int* n_sub)
{
    if (!dt_gas || !dt_rad || !n_sub) return fail(nullptr, RHD_ERR_ARG, "dt_gas, dt_rad and n_sub are required");
    if (!finite_pos(cfl) || !finite_pos(dx_min) || !finite_pos(v_max) || !finite_pos(chat))
        return fail(nullptr, RHD_ERR_ARG, "cfl, dx_min, v_max and chat must be positive and finite");
    const double dg = cfl * dx_min / v_max;
    const rhd_status st = span_subcycles(dg, cfl * dx_min / chat, dt_rad, n_sub);
    if (st == RHD_OK) *dt_gas = dg;
    return st;
}

rhd_status rhd_subcycle_steps(double cfl, double dx_min, double chat, double dt_gas, double* dt_rad, int* n_sub)
{
    if (!dt_rad || !n_sub) return fail(nullptr, RHD_ERR_ARG, "dt_rad and n_sub are required");
    if (!finite_pos(cfl) || !finite_pos(dx_min) || !finite_pos(chat) || !finite_pos(dt_gas))
        return fail(nullptr, RHD_ERR_ARG, "cfl, dx_min, chat and dt_gas must be positive and finite");
    return span_subcycles(dt_gas, cfl * dx_min / chat, dt_rad, n_sub);
}

rhd_status rhd_marshak_boundary(double tau, double eps, double F_inc, double c, int n_quad, double state[4])
{
    if (!state) return fail(nullptr, RHD_ERR_ARG, "state is NULL");
    if (!(std::isfinite(tau) && tau >= 0.0) || !finite_pos(eps) || !(std::isfinite(F_inc) && F_inc >= 0.0) ||
        !finite_pos(c) || n_quad < 1)
        return fail(nullptr, RHD_ERR_ARG, "need tau >= 0, eps > 0, F_inc >= 0, c > 0, n_quad >= 1 (finite)");
    // at chi = 0: sin(Theta) = 2 Gamma / sqrt(3 + 4 Gamma^2) since cos(Theta) = sqrt(3 / (3 + 4 Gamma^2))
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < n_quad; ++k) {
        const double eta = (k + 0.5) / n_quad;
        const double g1 = eta * std::sqrt(eps + 1.0 / (1.0 - eta * eta));
        const double q1 = 3.0 + 4.0 * g1 * g1;
        s1 += std::exp(-tau * eta * eta) * std::sin(std::acos(std::sqrt(3.0 / q1))) / (eta * std::sqrt(q1));
        const double g2 = std::sqrt((1.0 - eta) * (eps + 1.0 / eta));
        const double q2 = 3.0 + 4.0 * g2 * g2;
        s2 += std::exp(-tau / (eps * eta)) * std::sin(std::acos(std::sqrt(3.0 / q2))) /
              (eta * (1.0 + eps * eta) * std::sqrt(q2));
    }
    const double r3 = std::sqrt(3.0), pi = 3.14159265358979323846;
    const double u = 1.0 - (2.0 * r3 / pi) * s1 / n_quad - (r3 / pi) * std::exp(-tau) * s2 / n_quad;
    const double E = 4.0 * F_inc * u / c;
    state[0] = E;
    state[1] = (4.0 * F_inc - c * E) / 2.0;
    state[2] = state[3] = 0.0;
    return RHD_OK;
}

rhd_status rhd_reset_stats(rhd_ctx* ctx)
{
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    rhd_status st = enter(ctx);
    if (st) return st;
    RHD_CUDA(ctx, cudaMemsetAsync(ctx->dstats, 0, sizeof(DevStats), ctx->stream));
    RHD_CUDA(ctx, cudaMemsetAsync(ctx->gas_counters, 0, 2 * sizeof(unsigned long long), ctx->stream));
    RHD_CUDA(ctx, oob_read_fp64(nullptr, 1, ctx->stream));
    RHD_CUDA(ctx, oob_read_split(nullptr, 1, ctx->stream));
    ctx->n_subcycles = 0;
    return leave(ctx);
}

rhd_status rhd_get_stats(rhd_ctx* ctx, rhd_stats* out)
{
    ApiRange range_("rhd_get_stats");
    if (!ctx || !out) return fail(ctx, RHD_ERR_ARG, "ctx and out are required");
    std::memset(out, 0, sizeof(*out));
    rhd_status st = enter(ctx);
    if (st) return st;
    DevStats hs;
    RHD_CUDA(ctx, cudaMemcpyAsync(&hs, ctx->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, ctx->stream));
    unsigned long long gas_counts[2] = {0, 0};
    RHD_CUDA(ctx, cudaMemcpyAsync(gas_counts, ctx->gas_counters, sizeof(gas_counts), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    double sums[5] = {0, 0, 0, 0, 0};
    for (auto& gs : ctx->grids) {
        if (!gs.has_moments) continue;
        if ((st = ensure_reduce(ctx, gs.ncell))) return st;
        double** U = gs.U[ctx->cur];
        int nb = reduce_blocks_for(gs.ncell);
        RHD_CUDA(ctx, launch_reduce_state(U[0], U[1], U[2], U[3], gs.ncell, ctx->red_partials, nb, ctx->stream));
        RHD_CUDA(ctx, launch_reduce_finish(ctx->red_partials, nb, ctx->red_out, ctx->stream));
        double h[5];
        RHD_CUDA(ctx, cudaMemcpyAsync(h, ctx->red_out, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
        RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        sums[0] += h[0];
        for (int d = 0; d < 3; ++d) sums[1 + d] += gs.desc.c * h[1 + d];
        sums[4] = std::max(sums[4], h[4]);
    }
    OobRecord oob[2];
    RHD_CUDA(ctx, oob_read_fp64(&oob[0], 0, ctx->stream));
    RHD_CUDA(ctx, oob_read_split(&oob[1], 0, ctx->stream));
    if ((st = leave(ctx))) return st;
    RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    out->bounds_violations = (int64_t)(oob[0].count + oob[1].count);
    out->n_subcycles = ctx->n_subcycles;
    out->n_realizability_fix = (int64_t)hs.n_fix;
    out->n_face_fallback = (int64_t)hs.n_face;
    out->n_theta_fallback = (int64_t)hs.n_theta;
    out->n_newton_fallback = (int64_t)hs.n_newton_fb;
    out->n_nonfinite = (int64_t)hs.n_nonfinite;
    out->newton_iter_max = (int32_t)hs.newton_iter_max;
    out->wait_timeouts = (int32_t)hs.n_timeout;
    out->sum_E = sums[0];
    for (int d = 0; d < 3; ++d) out->sum_F[d] = sums[1 + d];
    out->max_f = sums[4];
    out->gas_energy_floors = (int64_t)gas_counts[0];
    out->gas_nonfinite = (int64_t)gas_counts[1];
    if (out->bounds_violations) {
        const OobRecord& r = oob[0].count ? oob[0] : oob[1];
        return fail(ctx, RHD_ERR_BOUNDS,
                    std::to_string(out->bounds_violations) + " out-of-range array indices; first in the " +
                        (oob[0].count ? "FP64" : "split") + " kernels at source line " + std::to_string(r.line) +
                        ": index " + std::to_string(r.index) + " of extent " + std::to_string(r.extent));
    }
    if (out->wait_timeouts) return fail(ctx, RHD_ERR_TIMEOUT, "a device-side wait ran out; some tiles were not updated");
    if (out->n_nonfinite)
        return fail(ctx, RHD_ERR_NONFINITE,
                    std::to_string(out->n_nonfinite) + " non-finite values were produced since the last reset");
    if (out->gas_nonfinite)
        return fail(ctx, RHD_ERR_NONFINITE,
                    std::to_string(out->gas_nonfinite) + " cells of the gas step became non-finite since the last reset");
    return RHD_OK;
}

rhd_status rhd_synchronize(rhd_ctx* ctx, int timeout_ms)
{
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    auto t0 = std::chrono::steady_clock::now();
    while (true) {
        cudaError_t e = cudaStreamQuery(ctx->stream);
        if (e == cudaSuccess) return RHD_OK;
        if (e != cudaErrorNotReady) return fail(ctx, RHD_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
        if (timeout_ms >= 0) {
            auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms) return fail(ctx, RHD_ERR_TIMEOUT, "stream still busy after the timeout");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

// ---------------------------------------------------------------------------------------------
// ensemble
// ---------------------------------------------------------------------------------------------
rhd_status rhd_ensemble_create(rhd_ctx** out, int n_grids, const rhd_grid_desc* descs)
{
    ApiRange range_("rhd_ensemble_create");
    if (descs && n_grids > 0)
        for (int g = 0; g < n_grids; ++g)
            if (descs[g].flags & RHD_FLAG_EXCHANGE_ON_GAS_STEP)
                return fail(nullptr, RHD_ERR_ARG, "RHD_FLAG_EXCHANGE_ON_GAS_STEP needs a single grid (ensembles have no gas step)");
    if (!out || !descs || n_grids < 1) return fail(nullptr, RHD_ERR_ARG, "out, descs and n_grids >= 1 are required");
    for (int i = 0; i < n_grids; ++i) {
        rhd_status st = validate_desc(nullptr, descs + i);
        if (st) return st;
        if (count_active(descs[i]) != 3) return fail(nullptr, RHD_ERR_ARG, "ensemble grids must be 3D");
        const rhd_grid_desc& a = descs[0];
        const rhd_grid_desc& b = descs[i];
        if (a.precision != b.precision || a.exchange != b.exchange || a.limiter != b.limiter ||
            a.closure != b.closure || a.speeds != b.speeds)
            return fail(nullptr, RHD_ERR_ARG, "ensemble grids must share precision, exchange, limiter, closure, speeds");
    }
    rhd_ctx* ctx = new (std::nothrow) rhd_ctx();
    if (!ctx) return fail(nullptr, RHD_ERR_OOM, "host allocation failed");
    ctx->ensemble = true;
    ctx->user_stream = (cudaStream_t)descs[0].cuda_stream;
    rhd_status st = common_init(ctx);
    if (!st) {
        ctx->grids.resize(n_grids);
        long long items = 0;
        for (int i = 0; i < n_grids && !st; ++i) {
            GridState& gs = ctx->grids[i];
            gs.desc = descs[i];
            gs.ncell = (long long)descs[i].n[0] * descs[i].n[1] * descs[i].n[2];
            fill_params(gs);
            // split ensembles run the two-pass kernels unless descs[0] asks for the fused kernel (the
            // linear exchange runs in the fused kernels only)
            gs.variant = (descs[0].precision == RHD_SPLIT && !(descs[0].flags & RHD_FLAG_SPLIT_FUSED) &&
                          descs[0].exchange != RHD_EX_LINEAR)
                             ? RHD_VARIANT_TWOPASS
                             : RHD_VARIANT_FUSED;
            st = alloc_grid(ctx, gs);
        }
        // one z chunk for all grids (the largest grid's automatic choice)
        int zc = descs[0].z_chunk > 0 ? descs[0].z_chunk : 32;
        for (auto& gs : ctx->grids) gs.z_chunk = zc;
        for (auto& gs : ctx->grids)
            items += (long long)gs.tiles_x * gs.tiles_y * ((gs.desc.n[2] + zc - 1) / zc);
        ctx->n_items = items;
        if (!st) st = dalloc(ctx, (void**)&ctx->d_egrids[0], sizeof(EnsembleGrid) * (size_t)n_grids);
        if (!st) st = dalloc(ctx, (void**)&ctx->d_egrids[1], sizeof(EnsembleGrid) * (size_t)n_grids);
        if (!st) st = dalloc(ctx, (void**)&ctx->d_counter, 2 * sizeof(unsigned long long));
        if (!st) {
            int per_sm = descs[0].precision == RHD_SPLIT ? ensemble_ctas_per_sm_split() : ensemble_ctas_per_sm_fp64();
            ctx->ens_ctas = per_sm * ctx->num_sms;
            if (descs[0].precision == RHD_SPLIT) {
                ctx->ens_pctas = ensemble_ctas_per_sm_predictor() * ctx->num_sms;
                ctx->ens_cctas = ensemble_ctas_per_sm_corrector() * ctx->num_sms;
            }
        }
    }
    if (st) {
        g_init_error = ctx->err;
        destroy_ctx(ctx);
        return st;
    }
    *out = ctx;
    return RHD_OK;
}

static rhd_status ens_grid(rhd_ctx* ctx, int grid, GridState** gs)
{
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (!ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "not an ensemble context");
    if (grid < 0 || grid >= (int)ctx->grids.size()) return fail(ctx, RHD_ERR_ARG, "grid index out of range");
    *gs = &ctx->grids[grid];
    return RHD_OK;
}

rhd_status rhd_ensemble_set_gas_state(rhd_ctx* ctx, int grid, const double* rho, const double* T, const double* vx,
                                      const double* vy, const double* vz, const double* kP, const double* kF,
                                      const double* j, int on_device)
{
    GridState* gs;
    rhd_status st = ens_grid(ctx, grid, &gs);
    if (st) return st;
    return set_gas(ctx, *gs, rho, T, vx, vy, vz, kP, kF, j, on_device);
}

rhd_status rhd_ensemble_set_moments(rhd_ctx* ctx, int grid, const double* E, const double* Fx, const double* Fy,
                                    const double* Fz, int on_device)
{
    GridState* gs;
    rhd_status st = ens_grid(ctx, grid, &gs);
    if (st) return st;
    return set_moments(ctx, *gs, E, Fx, Fy, Fz, on_device);
}

rhd_status rhd_ensemble_get_moments(rhd_ctx* ctx, int grid, double* E, double* Fx, double* Fy, double* Fz,
                                    int on_device)
{
    GridState* gs;
    rhd_status st = ens_grid(ctx, grid, &gs);
    if (st) return st;
    return get_moments(ctx, *gs, E, Fx, Fy, Fz, on_device);
}

rhd_status rhd_ensemble_get_gas_state(rhd_ctx* ctx, int grid, double* T, int on_device)
{
    GridState* gs;
    rhd_status st = ens_grid(ctx, grid, &gs);
    if (st) return st;
    return get_T(ctx, *gs, T, on_device);
}

rhd_status rhd_ensemble_subcycle(rhd_ctx* ctx, int n_sub, double chat, const double* dt_per_grid)
{
    ApiRange range_("rhd_ensemble_subcycle");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (!ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "not an ensemble context");
    if (n_sub < 0 || !dt_per_grid) return fail(ctx, RHD_ERR_ARG, "n_sub >= 0 and dt_per_grid are required");
    int ng = (int)ctx->grids.size();
    for (int i = 0; i < ng; ++i) {
        rhd_status st = check_dt(ctx, ctx->grids[i], chat, dt_per_grid[i]);
        if (st) return st;
        if (!ctx->grids[i].has_moments || !ctx->grids[i].has_gas)
            return fail(ctx, RHD_ERR_STATE, "set the moments and gas state of every grid first");
    }
    if (n_sub == 0) return RHD_OK;
    rhd_status st = RHD_OK;
    if ((ctx->grids[0].desc.flags & RHD_FLAG_AUTOTUNE) && !ctx->grids[0].tuned &&
        (st = ensemble_tune_once(ctx, chat, dt_per_grid)))
        return st;
    if ((st = enter(ctx))) return st;
    for (auto& gs : ctx->grids)
        if ((st = prepare_twopass(ctx, gs))) return st;
    double dt_sig = 0.0;
    if ((st = ens_prepare(ctx, chat, dt_per_grid, &dt_sig))) return st;
    bool use_graph = !(ctx->grids[0].desc.flags & RHD_FLAG_NO_GRAPH) && !ctx->ktiming;
    st = run_steps(ctx, n_sub, chat, dt_sig, use_graph, [&](int src) { return ens_launch(ctx, chat, src); });
    if (st) return st;
    ctx->cur = (ctx->cur + n_sub) & 1;
    ctx->n_subcycles += n_sub;
    return leave(ctx);
}

// ---------------------------------------------------------------------------------------------
// launch configuration and autotuner
// ---------------------------------------------------------------------------------------------
rhd_status rhd_autotune(rhd_ctx* ctx, double chat, double dt, int reps, rhd_launch_config* table, int capacity,
                        int* n_entries, rhd_launch_config* chosen)
{
    ApiRange range_("rhd_autotune");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "use rhd_ensemble_autotune on an ensemble");
    if (reps < 1 || capacity < 0) return fail(ctx, RHD_ERR_ARG, "reps >= 1 and capacity >= 0 are required");
    GridState& gs = ctx->grids[0];
    rhd_status st = check_dt(ctx, gs, chat, dt);
    if (st) return st;
    if (!gs.has_moments || !gs.has_gas) return fail(ctx, RHD_ERR_STATE, "set the moments and the gas state first");
    return grid_autotune(ctx, chat, dt, reps, table, capacity, n_entries, chosen);
}

rhd_status rhd_ensemble_autotune(rhd_ctx* ctx, double chat, const double* dt_per_grid, int reps,
                                 rhd_launch_config* table, int capacity, int* n_entries, rhd_launch_config* chosen)
{
    ApiRange range_("rhd_ensemble_autotune");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (!ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "not an ensemble context");
    if (reps < 1 || capacity < 0 || !dt_per_grid)
        return fail(ctx, RHD_ERR_ARG, "reps >= 1, capacity >= 0 and dt_per_grid are required");
    for (size_t i = 0; i < ctx->grids.size(); ++i) {
        rhd_status st = check_dt(ctx, ctx->grids[i], chat, dt_per_grid[i]);
        if (st) return st;
        if (!ctx->grids[i].has_moments || !ctx->grids[i].has_gas)
            return fail(ctx, RHD_ERR_STATE, "set the moments and gas state of every grid first");
    }
    return ensemble_autotune(ctx, chat, dt_per_grid, reps, table, capacity, n_entries, chosen);
}

rhd_status rhd_set_kernel_timing(rhd_ctx* ctx, int enable)
{
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->ktiming = enable != 0;
    ctx->kev_used = 0;
    ctx->krec.clear();
    return RHD_OK;
}

rhd_status rhd_get_kernel_times(rhd_ctx* ctx, rhd_kernel_time* out, int capacity, int* n_entries)
{
    if (!ctx || capacity < 0 || (capacity > 0 && !out)) return fail(ctx, RHD_ERR_ARG, "ctx and out are required");
    RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    long long launches[K_COUNT] = {0};
    double ms[K_COUNT] = {0.0}, bytes[K_COUNT] = {0.0};
    for (auto& r : ctx->krec) {
        float f = 0.0f;
        RHD_CUDA(ctx, cudaEventElapsedTime(&f, ctx->kev[r.e0], ctx->kev[r.e1]));
        launches[r.kernel] += 1;
        ms[r.kernel] += f;
        bytes[r.kernel] = r.alg_bytes;
    }
    ctx->kev_used = 0;
    ctx->krec.clear();
    int n = 0;
    for (int k = 0; k < K_COUNT; ++k) {
        if (!launches[k]) continue;
        if (n < capacity) {
            rhd_kernel_time& o = out[n];
            std::memset(&o, 0, sizeof(o));
            std::snprintf(o.name, sizeof(o.name), "%s", kKernelNames[k]);
            o.launches = launches[k];
            o.total_ms = ms[k];
            o.alg_bytes_per_launch = bytes[k];
        }
        ++n;
    }
    if (n_entries) *n_entries = n;
    return RHD_OK;
}

rhd_status rhd_get_launch_config(rhd_ctx* ctx, rhd_launch_config* out)
{
    if (!ctx || !out) return fail(ctx, RHD_ERR_ARG, "ctx and out are required");
    *out = current_config(ctx->grids[0]);
    return RHD_OK;
}

rhd_status rhd_set_wait_limit(rhd_ctx* ctx, long long polls)
{
    ApiRange range_("rhd_set_wait_limit");
    if (!ctx) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
    if (polls > 0xffffffffLL) return fail(ctx, RHD_ERR_ARG, "polls must be below 2^32");
    ctx->wait_polls = polls < 0 ? (1u << 22) : (unsigned)polls;
    clear_graphs(ctx);  // the captured launches carry the limit
    return RHD_OK;
}

rhd_status rhd_set_launch_config(rhd_ctx* ctx, const rhd_launch_config* cfg)
{
    if (!ctx || !cfg) return fail(ctx, RHD_ERR_ARG, "ctx and cfg are required");
    if (ctx->ensemble) return fail(ctx, RHD_ERR_STATE, "not available on an ensemble context");
    GridState& gs = ctx->grids[0];
    if (!config_supported(gs, *cfg)) return fail(ctx, RHD_ERR_ARG, "launch configuration not supported for this grid");
    rhd_status st = enter(ctx);  // frees / allocates device memory: order after the caller's work
    if (st) return st;
    RHD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if ((st = apply_config(ctx, gs, *cfg))) return st;
    gs.tuned_ms = -1.0;
    return leave(ctx);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// helpers shared with the no-allocation entry point (rhd_noalloc.cu)
// ---------------------------------------------------------------------------------------------
namespace rhd {

// Validate a descriptor and derive the launch parameters of one grid (no allocation).
rhd_status noalloc_prepare(const rhd_grid_desc* d, GridParams* gp, int* tiles_x, int* tiles_y, int* z_chunk)
{
    rhd_status st = validate_desc(nullptr, d);
    if (st) return st;
    GridState gs;
    gs.desc = *d;
    gs.ncell = (long long)d->n[0] * d->n[1] * d->n[2];
    fill_params(gs);
    *gp = gs.gp;
    *tiles_x = gs.tiles_x;
    *tiles_y = gs.tiles_y;
    *z_chunk = gs.z_chunk;
    return RHD_OK;
}

// Record the message returned by rhd_last_error(NULL) and pass the status through.
rhd_status noalloc_fail(rhd_status st, const std::string& msg) { return fail(nullptr, st, msg); }

}  // namespace rhd
