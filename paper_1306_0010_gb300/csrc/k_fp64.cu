// k_fp64.cu -- FP64 instantiations of the fused subcycle kernel and of the ensemble kernel.
#include <algorithm>

#include "subcycle.cuh"

namespace rhd {

template <typename R, int TX, int TY, int DIM, bool SPLIT>
static cudaError_t launch_tile_kernel(const StepParams& p, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes<R, TX, TY, DIM, SPLIT>();
    auto k = subcycle_kernel<R, TX, TY, DIM, SPLIT>;
    static SmemLimitOnce smem_once;
    cudaError_t e = smem_once.set(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(p.tiles_x * p.tiles_y), DIM == 3 ? (unsigned)((p.g.n[2] + p.z_chunk - 1) / p.z_chunk) : 1u);
    k<<<grid, Geo<TX, TY, DIM>::NT, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, int TX, int TY, bool SPLIT>
static cudaError_t launch_ens_kernel(const EnsembleParams& p, int n_ctas, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes<R, TX, TY, 3, SPLIT>();
    auto k = ensemble_kernel<R, TX, TY, SPLIT>;
    static SmemLimitOnce smem_once;
    cudaError_t e = smem_once.set(k, smem);
    if (e != cudaSuccess) return e;
    k<<<n_ctas, TX * TY, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, int TX, int TY, bool SPLIT>
static int ens_occupancy()
{
    const size_t smem = tile_smem_bytes<R, TX, TY, 3, SPLIT>();
    auto k = ensemble_kernel<R, TX, TY, SPLIT>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, TX * TY, smem) != cudaSuccess || n < 1) return 1;
    return n;
}

void tile_shape(int precision, int nact, int* tx, int* ty)
{
    if (nact == 1) {
        *tx = 122;  // 128 threads: the tile and its 3-cell halo on each side
        *ty = 1;
    } else if (precision == 0) {
        // one CTA of 256 threads per SM (255 registers each): against 16x8 tiles (two CTAs of 128) it
        // recomputes the predictor on 1.89 instead of 2.41 times the tile's cells, which the FP64 pipe pays
        *tx = 16;
        *ty = 16;
    } else {
        *tx = 32;
        *ty = 8;
    }
}

void ensemble_tile_shape(int precision, int* tx, int* ty)
{
    // the tiles ensemble_kernel is instantiated with (launch_ensemble_fp64, launch_ensemble_split)
    *tx = precision == 0 ? 16 : 32;
    *ty = precision == 0 ? 16 : 8;
}

bool tile_supported(int precision, int nact, int tx, int ty)
{
    int dx, dy;
    tile_shape(precision, nact, &dx, &dy);
    if (tx == dx && ty == dy) return true;
    if (nact != 3) return false;
    if (precision == 0) return false;
    return (tx == 32 && ty == 16) || (tx == 64 && ty == 8);
}

cudaError_t launch_subcycle_fp64(const StepParams& p, cudaStream_t s)
{
    switch (p.g.nact) {
    case 1: return launch_tile_kernel<double, 122, 1, 1, false>(p, s);
    case 2: return launch_tile_kernel<double, 16, 16, 2, false>(p, s);
    default: return launch_tile_kernel<double, 16, 16, 3, false>(p, s);
    }
}

cudaError_t launch_ensemble_fp64(const EnsembleParams& p, int n_ctas, cudaStream_t s)
{
    return launch_ens_kernel<double, 16, 16, false>(p, n_ctas, s);
}

int ensemble_ctas_per_sm_fp64() { return ens_occupancy<double, 16, 16, false>(); }

// The stiff exchange integrated once per gas step (Section 3.1 step 2, the paper's placement of S_i): in
// every cell, E floored at E_floor, then the FULL quartic theta scheme of the subcycles (exchange_fp64,
// Eqs. source:energyupdate - source:polynomial) over dt = Delta t_gas, then |G| <= E by rescaling G.
// FP64 on every grid: it runs once per gas step, not per subcycle.  One thread per cell, grid-stride.
__global__ void __launch_bounds__(256) gas_exchange_kernel(const __grid_constant__ GasExchangeParams P)
{
    Counters cnt = {0, 0, 0, 0, 0, 0, 0};
    const GridParams& g = P.g;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += (long long)gridDim.x * blockDim.x) {
        double E = P.E[i], T = P.T[i];
        const double rho = P.rho[i];
        const double kP = P.kP ? P.kP[i] : kappa_law(g.kappa_P, g.kpow, rho);
        if (E < g.E_floor) E = g.E_floor;
        const ExchangeOut o = exchange_fp64(g, P.chat, P.dt, rho, kP, E, T);
        cnt.theta += o.theta_fb;
        cnt.newton_fb += o.newton_fb;
        cnt.iter_max = max(cnt.iter_max, (unsigned)o.iters);
        double G[3] = {P.G[0][i], P.G[1][i], P.G[2][i]};
        const double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
        if (g2 > E * E) {
            const double sc = E / sqrt(g2);
            G[0] *= sc;
            G[1] *= sc;
            G[2] *= sc;
            cnt.fix += 1;
        }
        cnt.nonfinite += !(finite_d(E) && finite_d(T) && finite_d(G[0]) && finite_d(G[1]) && finite_d(G[2]));
        P.E[i] = E;
        P.T[i] = T;
        P.G[0][i] = G[0];
        P.G[1][i] = G[1];
        P.G[2][i] = G[2];
    }
    add_counter(&P.stats->n_fix, cnt.fix);
    add_counter(&P.stats->n_theta, cnt.theta);
    add_counter(&P.stats->n_newton_fb, cnt.newton_fb);
    add_counter(&P.stats->n_nonfinite, cnt.nonfinite);
    max_counter(&P.stats->newton_iter_max, cnt.iter_max);
}

cudaError_t launch_gas_exchange(const GasExchangeParams& p, int num_sms, cudaStream_t s)
{
    const long long blocks = std::min<long long>((p.n + 255) / 256, (long long)num_sms * 8);
    gas_exchange_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(p);
    return cudaGetLastError();
}

// Out-of-range index record of this module's kernels (debug builds; the release build has none and
// reports 0): copied to *out on stream s and, with reset, zeroed after the copy.
cudaError_t oob_read_fp64(OobRecord* out, int reset, cudaStream_t s)
{
#ifdef RHD_BOUNDS_CHECK
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_oob);
    if (e != cudaSuccess) return e;
    if (out && (e = cudaMemcpyAsync(out, p, sizeof(OobRecord), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    return reset ? cudaMemsetAsync(p, 0, sizeof(OobRecord), s) : cudaSuccess;
#else
    (void)reset;
    (void)s;
    if (out) *out = OobRecord{0, 0, 0, 0, 0};
    return cudaSuccess;
#endif
}
bool bounds_checked_fp64()
{
#ifdef RHD_BOUNDS_CHECK
    return true;
#else
    return false;
#endif
}

}  // namespace rhd
