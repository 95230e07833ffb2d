// k_fp64.cu -- Split-precision (FP32 fluxes, FP64 state) instantiations of the fused subcycle kernel and of the ensemble kernel.
#include <type_traits>

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


cudaError_t launch_subcycle_split(const StepParams& p, cudaStream_t s)
{
    switch (p.g.nact) {
    case 1: return launch_tile_kernel<float, 122, 1, 1, true>(p, s);
    case 2: return launch_tile_kernel<float, 32, 8, 2, true>(p, s);
    default:
        if (p.ty == 16) return launch_tile_kernel<float, 32, 16, 3, true>(p, s);
        if (p.tx == 64) return launch_tile_kernel<float, 64, 8, 3, true>(p, s);
        return launch_tile_kernel<float, 32, 8, 3, true>(p, s);
    }
}

cudaError_t launch_ensemble_split(const EnsembleParams& p, int n_ctas, cudaStream_t s)
{
    return launch_ens_kernel<float, 32, 8, true>(p, n_ctas, s);
}

// Two-pass split subcycle (3D): predictor over the grid and its stored ghost layers, then corrector.
cudaError_t launch_twopass_predictor(const StepParams& p, cudaStream_t s)
{
    constexpr int TX = 32, TY = 8;
    const int zc = p.z_chunk;
    StepParams pp = p;
    pp.tiles_x = (upad_extent(p.g, 0) + TX - 1) / TX;
    pp.tiles_y = (upad_extent(p.g, 1) + TY - 1) / TY;
    auto k = predictor_kernel<TX, TY>;
    const size_t smem = GeoPred<TX, TY>::bytes();
    static SmemLimitOnce smem_once;
    cudaError_t e = smem_once.set(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(pp.tiles_x * pp.tiles_y), (unsigned)((upad_extent(p.g, 2) + zc - 1) / zc));
    k<<<grid, TX * TY, smem, s>>>(pp);
    return cudaGetLastError();
}

cudaError_t launch_twopass_corrector(const StepParams& p, cudaStream_t s)
{
    constexpr int TX = 32, TY = 8;
    const int zc = p.z_chunk;
    StepParams pc = p;
    pc.tiles_x = (p.g.n[0] + TX - 1) / TX;
    pc.tiles_y = (p.g.n[1] + TY - 1) / TY;
    // one instantiation per staging and limiter (the limiter is a compile-time constant in the kernel)
    auto pick = [&](auto tma) {
        constexpr bool T = decltype(tma)::value;
        return p.g.limiter == LIM_MC ? corrector_kernel<TX, TY, T, LIM_MC>
               : p.g.limiter == LIM_NONE ? corrector_kernel<TX, TY, T, LIM_NONE>
                                         : corrector_kernel<TX, TY, T, LIM_MINMOD>;
    };
    auto k = p.staging == 1 ? pick(std::true_type{}) : pick(std::false_type{});
    const size_t smem = GeoCorr<TX, TY>::bytes() + 128;  // + alignment slack for TMA destinations
    static SmemLimitOnce smem_once;
    cudaError_t e = smem_once.set(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(pc.tiles_x * pc.tiles_y), (unsigned)((p.g.n[2] + zc - 1) / zc));
    k<<<grid, TX * TY, smem, s>>>(pc);
    return cudaGetLastError();
}

cudaError_t launch_twopass_split(const StepParams& p, cudaStream_t s)
{
    cudaError_t e = launch_twopass_predictor(p, s);
    return e != cudaSuccess ? e : launch_twopass_corrector(p, s);
}

// cuTensorMapEncodeTiled from the driver, found at run time (the library does not link libcuda)
static decltype(&cuTensorMapEncodeTiled) tensor_map_encoder()
{
    static decltype(&cuTensorMapEncodeTiled) fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        cudaGetLastError();
        return reinterpret_cast<decltype(&cuTensorMapEncodeTiled)>(p);
    }();
    return fn;
}

bool tma_available() { return tensor_map_encoder() != nullptr; }

__global__ void to_um32_kernel(float4* dst, const double* E, const double* G0, const double* G1, const double* G2,
                               long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = make_float4(d2f_trunc(E[i]), d2f_trunc(G0[i]), d2f_trunc(G1[i]), d2f_trunc(G2[i]));
}

cudaError_t launch_to_um32(float4* dst, const double* E, const double* G0, const double* G1, const double* G2,
                           long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long b = (n + 255) / 256;
    to_um32_kernel<<<(unsigned)(b < 152 * 16 ? b : 152 * 16), 256, 0, s>>>(dst, E, G0, G1, G2, n);
    return cudaGetLastError();
}

__global__ void to_gas4_kernel(float4* dst, const float* rho, const float* vx, const float* vy, const float* vz,
                               long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = make_float4(rho[i], vx ? vx[i] : 0.0f, vy ? vy[i] : 0.0f, vz ? vz[i] : 0.0f);
}

cudaError_t launch_to_gas4(float4* dst, const float* rho32, const float* vx, const float* vy, const float* vz,
                           long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long b = (n + 255) / 256;
    to_gas4_kernel<<<(unsigned)(b < 152 * 16 ? b : 152 * 16), 256, 0, s>>>(dst, rho32, vx, vy, vz, n);
    return cudaGetLastError();
}

bool encode_uhalf_map(CUtensorMap* map, float4* uhalf, const GridParams& g)
{
    auto enc = tensor_map_encoder();
    if (!enc || !uhalf || !g.pad[0] || !g.pad[1]) return false;
    constexpr int TX = 32, TY = 8;
    using G = GeoCorr<TX, TY>;
    // uhalf as floats: x = 4 (n0 + 4) floats per row, n1 + 4 rows, its stored planes; strides in bytes
    const cuuint64_t e0 = upad_extent(g, 0), e1 = upad_extent(g, 1), e2 = upad_extent(g, 2);
    const cuuint64_t dims[3] = {4ull * e0, e1, e2};
    const cuuint64_t strides[2] = {16ull * e0, 16ull * e0 * e1};
    const cuuint32_t box[3] = {4u * G::W2, (cuuint32_t)G::H2, 1u};  // the tile + 2-cell halo of one plane
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, uhalf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename K>
static int occupancy_of(K k, size_t smem, int threads)
{
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess || n < 1) return 1;
    return n;
}

cudaError_t launch_ensemble_predictor(const EnsembleParams& p, int n_ctas, cudaStream_t s)
{
    auto k = predictor_ens_kernel<32, 8>;
    const size_t smem = GeoPred<32, 8>::bytes();
    static SmemLimitOnce smem_once;
    cudaError_t e = smem_once.set(k, smem);
    if (e != cudaSuccess) return e;
    k<<<n_ctas, 256, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_ensemble_corrector(const EnsembleParams& p, int n_ctas, cudaStream_t s)
{
    // all grids of an ensemble share the limiter: one instantiation per limiter
    const int lim = p.n_grids > 0 ? p.limiter : LIM_MINMOD;
    auto k = lim == LIM_MC     ? corrector_ens_kernel<32, 8, LIM_MC>
             : lim == LIM_NONE ? corrector_ens_kernel<32, 8, LIM_NONE>
                               : corrector_ens_kernel<32, 8, LIM_MINMOD>;
    const size_t smem = GeoCorr<32, 8>::bytes();
    static SmemLimitOnce smem_once;
    cudaError_t e = smem_once.set(k, smem);
    if (e != cudaSuccess) return e;
    k<<<n_ctas, 256, smem, s>>>(p);
    return cudaGetLastError();
}

int ensemble_ctas_per_sm_predictor() { return occupancy_of(predictor_ens_kernel<32, 8>, GeoPred<32, 8>::bytes(), 256); }
int ensemble_ctas_per_sm_corrector()
{
    return occupancy_of(corrector_ens_kernel<32, 8, LIM_MINMOD>, GeoCorr<32, 8>::bytes(), 256);
}

int ensemble_ctas_per_sm_split() { return ens_occupancy<float, 32, 8, true>(); }

// Out-of-range index record of this module's kernels (debug builds; the release build has none and
// reports 0): copied to *out on stream s and, with reset, zeroed after the copy.
cudaError_t oob_read_split(OobRecord* out, int reset, cudaStream_t s)
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
bool bounds_checked_split()
{
#ifdef RHD_BOUNDS_CHECK
    return true;
#else
    return false;
#endif
}

}  // namespace rhd
