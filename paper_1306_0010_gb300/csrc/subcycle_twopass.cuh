// subcycle_twopass.cuh -- the split-precision subcycle for 3D grids as two kernels (included by
// subcycle.cuh after subcycle_pair.cuh).
//
//   predictor kernel: U^{m+1/2} of every cell of the grid with its ghost layers (two per face in
//     each direction that is not periodic on both faces; none in a periodic one) (the ghost cells
//     are the predictor applied to the ghost values of U^m, exactly as in the fused kernel and the
//     oracle), written as FP32 float4 (E, Gx, Gy, Gz);
//   corrector kernel: reconstruction, face states, HLL, divergence, sources, exchange and
//     realizability of the interior cells, reading U^{m+1/2} from the stored array (ghost positions,
//     or wrapped indices in periodic directions) and the FP64 state, updating the FP64 state.
// Each kernel marches column tiles through z.  Compared with the fused kernel the predictor is not
// recomputed on the corrector's halo, and each kernel needs far less shared memory and far fewer
// registers, so more warps are resident; the price is 32 bytes per cell of extra traffic (the FP32
// half-step state written once and read once).
#pragma once

// resident CTAs per SM the two kernels are compiled for (register budget 65536 / (256 x this))
#ifndef RHD_PRED_MIN_BLOCKS
#define RHD_PRED_MIN_BLOCKS 4
#endif
#ifndef RHD_CORR_MIN_BLOCKS
#define RHD_CORR_MIN_BLOCKS 3
#endif

namespace rhd {

// ------------------------------------------------------------------------------------------------
// TMA staging (tensor copies completed on an mbarrier), inline PTX
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// order this thread's earlier shared-memory accesses before later asynchronous-proxy accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// 3D tiled tensor copy global -> shared; (x, y, z) is the box origin in elements (x: floats, x*4 bytes
// a multiple of 16, every coordinate >= 0)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
// Wait until the barrier's phase with parity ph has completed; gives up after max_polls polls
// (each poll may suspend the thread for a bounded, implementation-defined time).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned ph, unsigned max_polls)
{
    const unsigned a = smem_addr(bar);
    for (unsigned it = 0; it < max_polls; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(ph)
            : "memory");
        if (done) return true;
    }
    return false;
}
constexpr unsigned kMaxPolls = 1u << 22;

// index of (x, y, z), each in [-pad, n + pad) of its direction, in the stored U^{m+1/2} array
__device__ __forceinline__ long long pad_index(const GridParams& g, int x, int y, int z)
{
    const long long px = upad_extent(g, 0), py = upad_extent(g, 1);
    return (long long)(x + g.pad[0]) + px * ((long long)(y + g.pad[1]) + py * (long long)(z + g.pad[2]));
}
// stored position, in direction d, of the U^{m+1/2} of coordinate p in [-2, n + 2) (further beyond the
// high face only for cells whose values are never used): p + 2 where ghost layers are stored, p wrapped
// into [0, n) where both faces are periodic
__device__ __forceinline__ int upad_pos(const GridParams& g, int d, int p)
{
    const int n = g.n[d];
    return g.pad[d] ? min(p, n + 1) + 2 : ((p % n) + n) % n;
}

// Work layout shared by both kernels: every thread owns one cell (tlx, tly) of the tile; the loops
// over cells, face-state records and faces are ordered so that the first passes are exactly one
// item per thread (its own cell), and the few items beyond the tile (halo cells, the faces of the
// tile's right column and top row) form one short last pass over the first threads.  No per-plane
// index arithmetic is needed and the passes over the own cells do not diverge.

// Gas of an interior cell at linear index li (split arrays; interior cells need no boundary rule).
__device__ __forceinline__ GasCell<float> gas_at(const GridParams& g, const GridArrays& a, long long li)
{
    GasCell<float> c;
    c.T = 0.0;
    c.rho = 0.0;
    li = chk(li, n_cells(g));
    const float r = __ldg(a.rho32 + li);
    c.rho32 = r;
    c.kP = a.kP32 ? __ldg(a.kP32 + li) : kappa_law_f(g.f_kappa_P, g.kpow, r);
    c.kF = a.kF32 ? __ldg(a.kF32 + li) : kappa_law_f(g.f_kappa_F, g.kpow, r);
#pragma unroll
    for (int d = 0; d < 3; ++d) c.v[d] = a.v32[d] ? __ldg(a.v32[d] + li) : 0.0f;
    c.j = a.j32 ? __ldg(a.j32 + li) : 0.0f;
    return c;
}

// One coordinate p of a cell in direction d mapped into [0, n) by the face's boundary rule, as one step
// of remap_cell: periodic wraps, reflect mirrors and flips the normal component (bit d of flip),
// outflow clamps; Dirichlet clamps too, or, when dir_ok and no earlier direction was Dirichlet,
// records the face (2 d + high) in dface.  The ghost layers whose values the predictor uses are at
// most three cells deep and active directions have n >= 3, so one step lands inside, as remap_cell's
// loop does; cells farther out (beyond the stored U^{m+1/2} in ragged tiles, values unused) are clamped
// into the grid so that every access stays in bounds.
__device__ __forceinline__ int ghost1(const GridParams& g, int d, int p, bool dir_ok, int& flip, int& dface)
{
    const int n = g.n[d];
    if ((unsigned)p < (unsigned)n) return p;
    const bool low = p < 0;
    const int bc = low ? g.bc_lo[d] : g.bc_hi[d];
    int r = low ? 0 : n - 1;
    if (bc == BC_DIRICHLET && dir_ok) {
        if (dface < 0) dface = 2 * d + (low ? 0 : 1);
    } else if (bc == BC_PERIODIC) {
        r = low ? p + n : p - n;
    } else if (bc == BC_REFLECT) {
        flip ^= 1 << d;
        r = low ? -p - 1 : 2 * n - 1 - p;
    }
    return min(max(r, 0), n - 1);
}

template <int TX, int TY>
struct GeoPred {
    static constexpr int NT = TX * TY;
    static constexpr int W1 = TX + 2, H1 = TY + 2;
    static constexpr int N1 = W1 * H1;
    static constexpr int NH = N1 - NT;  // halo cells of the tile + 1 region: rows -1 and TY, columns -1 and TX
    static_assert(NH <= NT && TX + TY <= NT, "one extra item per thread at most");
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    // float4 units: U^m of the tile + 1 region (two plane buffers), closure data, fluxes, and three
    // per-thread slots for the own cell's gas (rho, vx, vy, vz): plane p's gas is copied when plane p
    // is staged and read at the end of plane p + 1, after plane p + 2 has been issued
    static constexpr int UM = 0, CXo = UM + 2 * N1, CYo = CXo + N1, L3o = CYo + N1;
    static constexpr int FXo = L3o + (N1 + 1) / 2, FYo = FXo + NFX, GSo = FYo + NFY, END4 = GSo + 3 * NT;
    __host__ __device__ static constexpr size_t bytes() { return 16 * (size_t)END4; }
    __device__ static __forceinline__ int i1(int lx, int ly) { return (lx + 1) + W1 * (ly + 1); }
    // the h-th halo cell: rows ly = -1 and ly = TY with lx from -1 to TX, then columns lx = -1, TX
    __device__ static __forceinline__ void halo(int h, int& lx, int& ly)
    {
        if (h < 2 * W1) {
            ly = h < W1 ? -1 : TY;
            lx = (h < W1 ? h : h - W1) - 1;
        } else {
            const int hh = h - 2 * W1;
            ly = hh >> 1;
            lx = (hh & 1) ? TX : -1;
        }
    }
};

// Predictor over the column tile (x0, y0) of the stored U^{m+1/2} (coordinates in [-pad, n+pad))
// for planes [z0, z1).
template <int TX, int TY>
__device__ __forceinline__ void predictor_tile(const GridParams& g, const GridArrays& a, float4* uh, float chat,
                                               float dt, int x0, int y0, int z0, int z1, float4* sm, Counters& cnt)
{
    using G = GeoPred<TX, TY>;
    const int t = threadIdx.x;
    float4* Um0 = sm + G::UM;  // plane buffers Um0[buf * N1 + i]
    float4* CX = sm + G::CXo;
    float4* CY = sm + G::CYo;
    float2* L3 = reinterpret_cast<float2*>(sm + G::L3o);
    float4* Fx = sm + G::FXo;
    float4* Fy = sm + G::FYo;
    float4* gsl = sm + G::GSo + t;  // gsl[(p % 3) NT]: the own cell's (rho, vx, vy, vz) of plane p
    const float hdt = 0.5f * dt;
    const float idx = g.f_inv_dx[0], idy = g.f_inv_dx[1], idz = g.f_inv_dx[2];
    const int p1 = g.closure == 1, fixed = g.speeds == 1;
    const bool needT = g.exchange == EX_FROZEN_T;
    const long long nxy = (long long)g.n[0] * g.n[1];
    const int tlx = t % TX, tly = t / TX;
    const int gx = x0 + tlx, gy = y0 + tly;
    const bool own_in_pad = gx < g.n[0] + g.pad[0] && gy < g.n[1] + g.pad[1];
    const bool own_interior = gx >= 0 && gx < g.n[0] && gy >= 0 && gy < g.n[1];
    const bool has_h = t < G::NH;
    int hlx = 0, hly = 0;
    if (has_h) G::halo(t, hlx, hly);
    const int i_own = G::i1(tlx, tly), i_h = G::i1(hlx, hly);
    const int hx = x0 + hlx, hy = y0 + hly;
    // every cell of the tile + 1 region inside the grid in x and y: all loads of in-range planes are plain copies
    const bool xy_inside = x0 - 1 >= 0 && x0 + TX + 1 <= g.n[0] && y0 - 1 >= 0 && y0 + TY + 1 <= g.n[1];
    const int off_own = gx + g.n[0] * gy, off_h = hx + g.n[0] * hy;  // used only when xy_inside

    // Boundary rule of the x / y coordinates of the own and halo cells (fixed along the z march): the
    // source cell, the sign flips of the normal G components, and a Dirichlet face (state: dir_ok) or
    // clamping (gas: no Dirichlet values).
    int ox_fl = 0, ox_df = -1, hx_fl = 0, hx_df = -1, gx_fl = 0, gx_df = -1;
    int oxr = ghost1(g, 0, gx, true, ox_fl, ox_df);
    int oyr = ghost1(g, 1, gy, true, ox_fl, ox_df);
    const int hxr = ghost1(g, 0, hx, true, hx_fl, hx_df);
    const int hyr = ghost1(g, 1, hy, true, hx_fl, hx_df);
    const int gxr = ghost1(g, 0, gx, false, gx_fl, gx_df);
    const int gyr = ghost1(g, 1, gy, false, gx_fl, gx_df);
    (void)oxr;
    (void)oyr;
    // U^m of one cell into the plane buffer from the FP32 mirror (the FP64 state truncated toward zero):
    // in-grid cells directly, ghost cells from their source cell by the boundary rule (sign flips applied
    // once the copy has landed, by flip_ghosts) or, at a Dirichlet face, the face state truncated
    auto stage = [&](float4* d, int xr, int yr, int fl, int df, int off, int q, bool fast, long long zoff) {
        if (fast) {
            cp_async16(d, a.um32 + chk(zoff + off, n_cells(g)));
            return;
        }
        const int qr = ghost1(g, 2, q, true, fl, df);
        if (df >= 0) {
            const double* sd = (df & 1) ? g.dir_hi[df >> 1] : g.dir_lo[df >> 1];
            *d = make_float4(d2f_trunc(sd[0]), d2f_trunc(sd[1]), d2f_trunc(sd[2]), d2f_trunc(sd[3]));
        } else {
            cp_async16(d, a.um32 + lin(g, xr, yr, qr));
        }
    };
    // negate the G components of a staged ghost cell that the boundary rule mirrors
    auto flip_ghost = [&](float4* d, int fl, int df, int q) {
        ghost1(g, 2, q, true, fl, df);
        if (df < 0 && fl) {
            float4 v = *d;
            if (fl & 1) v.y = -v.y;
            if (fl & 2) v.z = -v.z;
            if (fl & 4) v.w = -v.w;
            *d = v;
        }
    };
    // zoff = q * nxy, carried by the caller
    auto issue_plane = [&](int q, long long zoff, int buf) {
        const bool fast = xy_inside && (unsigned)q < (unsigned)g.n[2];
        float4* Ub = Um0 + buf * G::N1;
        stage(Ub + i_own, oxr, oyr, ox_fl, ox_df, off_own, q, fast, zoff);
        if (has_h) stage(Ub + i_h, hxr, hyr, hx_fl, hx_df, off_h, q, fast, zoff);
        // the own cell's gas of plane q (the boundary rule's source cell for ghost cells), for its half
        // step one plane later
        if (own_in_pad && !needT) {
            int fl = gx_fl, df = -1;
            const int qr = ghost1(g, 2, q, false, fl, df);
            cp_async16(gsl + ((q + 3) % 3) * G::NT,
                       a.gas4 + chk((own_interior && (unsigned)q < (unsigned)g.n[2]) ? zoff + off_own : lin(g, gxr, gyr, qr),
                                    n_cells(g)));
        }
    };
    auto closure_xy = [&](int i, const float4& U, const ClosureScalars<float>& k) {
        float l1x, l3x, l1y, l3y;
        wave_speeds(k, U.y, chat, fixed, l1x, l3x);
        wave_speeds(k, U.z, chat, fixed, l1y, l3y);
        // explicitly rounded: own and halo cells (other tiles' own cells) must get the same bits
        const float bx = xmul(k.b, U.y), bz = xmul(k.b, U.z);
        const float Pxy = xmul(bx, U.z), Pxz = xmul(bx, U.w), Pyz = xmul(bz, U.w);
        CX[i] = make_float4(xfma(bx, U.y, k.a), Pxy, Pxz, l1x);
        CY[i] = make_float4(Pxy, xfma(bz, U.z, k.a), Pyz, l1y);
        L3[i] = make_float2(l3x, l3y);
    };
    const float4* Um = Um0;  // the current plane's buffer
    auto xface = [&](int iL, int iR) {
        iL = chk(iL, G::N1);
        iR = chk(iR, G::N1);
        const float4 UL = Um[iL], UR = Um[iR], CL = CX[iL], CR = CX[iR];
        const float4 FL = make_float4(UL.y, CL.x, CL.y, CL.z);  // fluxes per unit chat
        const float4 FR = make_float4(UR.y, CR.x, CR.y, CR.z);
        return hll4(UL, UR, FL, FR, CL.w, L3[iL].x, CR.w, L3[iR].x, chat);
    };
    auto yface = [&](int iL, int iR) {
        iL = chk(iL, G::N1);
        iR = chk(iR, G::N1);
        const float4 UL = Um[iL], UR = Um[iR], CL = CY[iL], CR = CY[iR];
        const float4 FL = make_float4(UL.z, CL.x, CL.y, CL.z);
        const float4 FR = make_float4(UR.z, CR.x, CR.y, CR.z);
        return hll4(UL, UR, FL, FR, CL.w, L3[iL].y, CR.w, L3[iR].y, chat);
    };

    float4 zU = make_float4(0.f, 0.f, 0.f, 0.f), zP = zU, dxy = zU, zfl = zU;
    float zl3 = 0.f;
    const int qbeg = z0 - 1, qend = z1 + 1;
    // running 64-bit offsets: the staged plane's, and the own cell's U^{m+1/2} at plane q - 1 in the
    // stored array
    long long zoff = (long long)qbeg * nxy;
    const long long pzs = (long long)upad_extent(g, 0) * upad_extent(g, 1);
    long long uoff = pad_index(g, gx, gy, qbeg - 1);  // negative before the first written plane
    issue_plane(qbeg, zoff, 0);
    zoff += nxy;
    cp_async_commit();
#pragma unroll 1
    for (int q = qbeg; q < qend; ++q, zoff += nxy, uoff += pzs) {
        const bool emit = q > qbeg + 1 && own_in_pad;
        const int buf = (q - qbeg) & 1;
        Um = Um0 + buf * G::N1;
        cp_async_wait_all();
        if (!(xy_inside && (unsigned)q < (unsigned)g.n[2])) {
            flip_ghost(Um0 + buf * G::N1 + i_own, ox_fl, ox_df, q);
            if (has_h) flip_ghost(Um0 + buf * G::N1 + i_h, hx_fl, hx_df, q);
        }
        __syncthreads();
        if (q + 1 < qend) issue_plane(q + 1, zoff, buf ^ 1);
        cp_async_commit();
        // closure of the own cell (x, y and its z-direction data) and of the halo cell
        float4 nU, nP;
        float nl3;
        {
            const float4 U = Um[i_own];
            const ClosureScalars<float> k = closure_scalars(U.x, U.y, U.z, U.w, chat, p1);
            closure_xy(i_own, U, k);
            float l1z, l3z;
            wave_speeds(k, U.w, chat, fixed, l1z, l3z);
            nU = U;
            const float bw = xmul(k.b, U.w);
            nP = make_float4(xmul(bw, U.y), xmul(bw, U.z), xfma(bw, U.w, k.a), l1z);
            nl3 = l3z;
        }
        if (has_h) {
            const float4 U = Um[i_h];
            closure_xy(i_h, U, closure_scalars(U.x, U.y, U.z, U.w, chat, p1));
        }
        __syncthreads();
        // x face left of the own cell, y face below it, then the tile's top row and right column
        Fx[chk(tly * (TX + 1) + tlx, G::NFX)] = xface(i_own - 1, i_own);
        Fy[chk(tly * TX + tlx, G::NFY)] = yface(i_own - G::W1, i_own);
        if (t < TX) {
            const int iL = G::i1(t, TY - 1);
            Fy[chk(TY * TX + t, G::NFY)] = yface(iL, iL + G::W1);
        } else if (t < TX + TY) {
            const int ly = t - TX, iL = G::i1(TX - 1, ly);
            Fx[chk(ly * (TX + 1) + TX, G::NFX)] = xface(iL, iL + 1);
        }
        __syncthreads();
        // own cell: x/y divergence of plane q, z face (q-1 | q), U^{m+1/2} of plane q - 1.  No barrier
        // follows: every shared array written in the next plane is written after that plane's first
        // barrier, which no thread passes before all threads have finished this block.
        {
            const int fl = tly * (TX + 1) + tlx, fb = tly * TX + tlx;
            const float4 ax = Fx[fl], bxf = Fx[fl + 1], ay = Fy[fb], by = Fy[fb + TX];
            const float4 nd = make_float4((bxf.x - ax.x) * idx + (by.x - ay.x) * idy,
                                          (bxf.y - ax.y) * idx + (by.y - ay.y) * idy,
                                          (bxf.z - ax.z) * idx + (by.z - ay.z) * idy,
                                          (bxf.w - ax.w) * idx + (by.w - ay.w) * idy);
            float4 zfh = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q > qbeg) {
                const float4 FL = make_float4(zU.w, zP.x, zP.y, zP.z);
                const float4 FR = make_float4(nU.w, nP.x, nP.y, nP.z);
                zfh = hll4(zU, nU, FL, FR, zP.w, zl3, nP.w, nl3, chat);
            }
            const int p = q - 1;
            if (emit) {
                // gas of the own cell of plane q - 1; zoff is (q + 1) nxy here, so that cell is at
                // off_own + zoff - 2 nxy in the interior arrays
                GasCell<float> gc;
                const bool opt = a.kP32 || a.kF32 || a.j32;  // optional per-cell opacity / emissivity arrays
                const bool inner = own_interior && (unsigned)(q - 1) < (unsigned)g.n[2];
                if (!needT && (!opt || inner)) {
                    // staged when plane q - 1 was issued (the boundary rule's source cell for ghost cells,
                    // whose mirrored velocity components are negated here)
                    const float4 gv = gsl[((q - 1 + 3) % 3) * G::NT];
                    int fl = gx_fl, df = -1;
                    ghost1(g, 2, q - 1, false, fl, df);
                    gc.T = 0.0;
                    gc.rho = 0.0;
                    gc.rho32 = gv.x;
                    gc.v[0] = (fl & 1) ? -gv.y : gv.y;
                    gc.v[1] = (fl & 2) ? -gv.z : gv.z;
                    gc.v[2] = (fl & 4) ? -gv.w : gv.w;
                    // read only with the optional arrays, which take this branch for interior cells alone
                    const long long li = (long long)off_own + zoff - 2 * nxy;
                    gc.kP = a.kP32 ? __ldg(a.kP32 + chk(li, n_cells(g))) : kappa_law_f(g.f_kappa_P, g.kpow, gv.x);
                    gc.kF = a.kF32 ? __ldg(a.kF32 + chk(li, n_cells(g))) : kappa_law_f(g.f_kappa_F, g.kpow, gv.x);
                    gc.j = a.j32 ? __ldg(a.j32 + chk(li, n_cells(g))) : 0.0f;
                } else {
                    gc = load_gas<float, true>(g, a, gx, gy, q - 1, needT, false);
                }
                const float U0a[4] = {zU.x, zU.y, zU.z, zU.w};
                const float div[4] = {dxy.x + (zfh.x - zfl.x) * idz, dxy.y + (zfh.y - zfl.y) * idz,
                                      dxy.z + (zfh.z - zfl.z) * idz, dxy.w + (zfh.w - zfl.w) * idz};
                float S[4];
                explicit_sources(g, gc, U0a, chat, S);
                float U[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) U[qq] = U0a[qq] - hdt * div[qq] + hdt * S[qq];
                theta_updates(g, gc, chat, hdt, U);
                const int fx_ = realize(U, g.f_E_floor);
                if (own_interior && p >= 0 && p < g.n[2]) cnt.fix += fx_;
                uh[chk(uoff, n_padded(g))] = f4(U);
            }
            zfl = zfh;
            zU = nU;
            zP = nP;
            zl3 = nl3;
            dxy = nd;
        }
    }
    cp_async_wait_all();
}

template <int TX, int TY>
struct GeoCorr {
    static constexpr int NT = TX * TY;
    static constexpr int W2 = TX + 4, H2 = TY + 4, N2 = W2 * H2;
    static constexpr int NR2 = (N2 + NT - 1) / NT;
    static constexpr int NSX = (TX + 2) * TY, NSY = TX * (TY + 2);
    static constexpr int NCX = (TX + 1) * TY, NCY = TX * (TY + 1);
    static constexpr int NHR = 2 * TX + 2 * TY;  // halo records: y records of rows -1, TY; x records of columns -1, TX
    static_assert(NHR <= NT && TX + TY <= NT, "one extra item per thread at most");
    // float4 units: two U^{m+1/2} plane buffers, face-state records, fluxes
    // records: 4 float4 each (minus state, plus state, closure coefficients, wave speeds; face_record_ab)
    static constexpr int UK = 0, SXo = UK + 2 * N2, SYo = SXo + 4 * NSX, CXo = SYo + 4 * NSY, CYo = CXo + NCX;
    static constexpr int END4 = CYo + NCY;
    // the own cell's FP64 state and T (5 doubles, SoA by field) and (rho, vx, vy, vz) (one float4), staged
    // per thread
    static constexpr int OD = 5, OG = 4;
    __host__ __device__ static constexpr size_t bytes() { return 16 * (size_t)END4 + 8 * (size_t)OD * NT + 4 * (size_t)OG * NT; }
    __device__ static __forceinline__ int i2(int lx, int ly) { return (lx + 2) + W2 * (ly + 2); }
    // record slots: x record of (lx, ly), lx in [-1, TX]; y record of (lx, ly), ly in [-1, TY]
    __device__ static __forceinline__ int sx(int lx, int ly) { return (lx + 1) + (TX + 2) * ly; }
    __device__ static __forceinline__ int sy(int lx, int ly) { return lx + TX * (ly + 1); }
};

// Corrector over the interior column tile (x0, y0) for planes [z0, z1).  TMA: the tile + 2-cell halo
// of each U^{m+1/2} plane arrives by one tensor copy (issued by thread 0, completed on mbar[buf]; map
// and mbar are then required, and sm must be 128-byte aligned); otherwise by per-thread cp.async.
template <int TX, int TY, bool TMA = false, int LIMK = -1>
__device__ __forceinline__ void corrector_tile(const GridParams& g, const GridArrays& a, const float4* uh,
                                               float chat, float dt, double chat_d, double dt_d, int x0, int y0,
                                               int z0, int z1, float4* sm,
                                               Counters& cnt, const CUtensorMap* map = nullptr,
                                               uint64_t* mbar = nullptr, unsigned wait_polls = kMaxPolls)
{
    using G = GeoCorr<TX, TY>;
    const int t = threadIdx.x;
    float4* Ubuf = sm + G::UK;
    float4* Sx = sm + G::SXo;
    float4* Sy = sm + G::SYo;
    float4* Cx = sm + G::CXo;
    float4* Cy = sm + G::CYo;
    double* oD = reinterpret_cast<double*>(sm + G::END4) + t;                       // oD[q NT]: E, Gx, Gy, Gz, T
    float4* oG = reinterpret_cast<float4*>(reinterpret_cast<double*>(sm + G::END4) + G::OD * G::NT) + t;  // gas
    const float idx = g.f_inv_dx[0], idy = g.f_inv_dx[1], idz = g.f_inv_dx[2];
    const SplitStiffConsts sk = split_stiff_consts(g, chat_d, dt_d);
    // LIMK >= 0: the limiter is a compile-time constant (only its code is generated); -1: g.limiter
    const int p1 = g.closure == 1, fixed = g.speeds == 1, lim = LIMK >= 0 ? LIMK : g.limiter;
    const bool needT = g.exchange == EX_FULL || g.exchange == EX_FROZEN_T;
    const int tlx = t % TX, tly = t / TX;
    const int gx = x0 + tlx, gy = y0 + tly;
    const bool own_col = gx < g.n[0] && gy < g.n[1];
    const long long pz = (long long)upad_extent(g, 0) * upad_extent(g, 1);
    const long long nxy = (long long)g.n[0] * g.n[1];

    // the R2 plane of U^{m+1/2}: rows of W2 float4 starting at (x0 - 2, y0 + ly), at their stored
    // positions (ghost layers, or wrapped where the direction is periodic; beyond the high edges of
    // ragged tiles clamped or wrapped, those values are never used)
    int c_gpos[G::NR2];
#pragma unroll
    for (int r = 0; r < G::NR2; ++r) {
        const int c = t + r * G::NT;
        const int lx = c % G::W2 - 2, ly = c / G::W2 - 2;
        c_gpos[r] = upad_pos(g, 0, x0 + lx) + upad_extent(g, 0) * upad_pos(g, 1, y0 + ly);
    }
    // shared-memory destinations of this thread's copies, for both buffers
    unsigned c_dsm[G::NR2];
#pragma unroll
    for (int r = 0; r < G::NR2; ++r) c_dsm[r] = (unsigned)__cvta_generic_to_shared(Ubuf + t + r * G::NT);
    const unsigned buf_bytes = 16u * G::N2;
    // base: the plane's first element in the stored U^{m+1/2}; k: the plane (TMA)
    auto issue_plane = [&](const float4* base, int buf, int k) {
        if constexpr (TMA) {
            if (t == 0) {
                fence_proxy_async();  // the buffer's earlier generic reads complete before the copy
                mbar_arrive_expect_tx(mbar + buf, 16u * G::N2);
                tma_load_3d(Ubuf + buf * G::N2, map, 4 * x0, y0, k + g.pad[2], mbar + buf);
            }
        } else {
#pragma unroll
            for (int r = 0; r < G::NR2; ++r) {
                const int c = t + r * G::NT;
                if (c < G::N2) {
                    const unsigned dsm = c_dsm[r] + (buf ? buf_bytes : 0u);
                    const float4* src = uh + chk((base - uh) + c_gpos[r], n_padded(g));
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dsm), "l"(src) : "memory");
                }
            }
        }
    };
    // the own cell in the plane buffer; its x and y neighbours (+-1, +-W2) are read, so the index must
    // lie in [W2, N2 - W2)
    const int ihc = G::W2 + chk(G::i2(tlx, tly) - G::W2, G::N2 - 2 * G::W2);
    const int sx_own = G::sx(tlx, tly), sy_own = G::sy(tlx, tly);
    // this thread's halo record, if any
    const bool has_hr = t < G::NHR, hr_is_y = t < 2 * TX;
    int hr_i = 0, hr_slot = 0;
    if (has_hr) {
        if (hr_is_y) {
            const int ly = t < TX ? -1 : TY, lx = t % TX;
            hr_i = G::W2 + chk(G::i2(lx, ly) - G::W2, G::N2 - 2 * G::W2);
            hr_slot = G::sy(lx, ly);
        } else {
            const int hh = t - 2 * TX, ly = hh >> 1, lx = (hh & 1) ? TX : -1;
            hr_i = G::W2 + chk(G::i2(lx, ly) - G::W2, G::N2 - 2 * G::W2);
            hr_slot = G::sx(lx, ly);
        }
    }
    // the own column of U^{m+1/2} (clamped for columns beyond ragged tile edges, whose values are unused)
    const long long colo = upad_pos(g, 0, gx) + (long long)upad_extent(g, 0) * upad_pos(g, 1, gy);
    auto col = [&](int k) { return uh[chk(colo + (long long)upad_pos(g, 2, k) * pz, n_padded(g))]; };
    auto store_rec = [](float4* S, int n, int slot, const float4 (&rec)[4]) {
        slot = chk(slot, n);
#pragma unroll
        for (int v = 0; v < 4; ++v) S[v * n + slot] = rec[v];
    };
    // HLL at the face between record slots iL (its plus state) and iR (its minus state)
    auto hll_x = [&](int iL, int iR) {
        iL = chk(iL, G::NSX);
        iR = chk(iR, G::NSX);
        const float4 UL = Sx[G::NSX + iL], UR = Sx[iR];
        const float4 cL = Sx[2 * G::NSX + iL], cR = Sx[2 * G::NSX + iR];
        const float4 LL = Sx[3 * G::NSX + iL], LR = Sx[3 * G::NSX + iR];
        return hll_pair(UL, UR, flux_ab<0>(UL, cL.z, cL.w), flux_ab<0>(UR, cR.x, cR.y), LL.z, LL.w, LR.x, LR.y, chat);
    };
    auto hll_y = [&](int iL, int iR) {
        iL = chk(iL, G::NSY);
        iR = chk(iR, G::NSY);
        const float4 UL = Sy[G::NSY + iL], UR = Sy[iR];
        const float4 cL = Sy[2 * G::NSY + iL], cR = Sy[2 * G::NSY + iR];
        const float4 LL = Sy[3 * G::NSY + iL], LR = Sy[3 * G::NSY + iR];
        return hll_pair(UL, UR, flux_ab<1>(UL, cL.z, cL.w), flux_ab<1>(UR, cR.x, cR.y), LL.z, LL.w, LR.x, LR.y, chat);
    };

    // lower z face of the first plane: face states of cells z0-1 and z0 from U^{m+1/2} at z0-2 .. z0+1
    float4 zpS, cfl;  // plus state of the previous cell in z, with its closure coefficients and speeds
    float zpa, zpb, zpl1, zpl3;
    float4 ukp1, ukp2;  // U^{m+1/2} of the own column at k+1, k+2
    {
        const float4 u_m2 = col(z0 - 2), u_m1 = col(z0 - 1), u_0 = col(z0), u_1 = col(z0 + 1);
        float4 ra[4], rb[4];
        face_record_ab<2>(u_m2, u_m1, u_0, chat, lim, p1, fixed, ra);
        const int fb = face_record_ab<2>(u_m1, u_0, u_1, chat, lim, p1, fixed, rb);
        cnt.face += (unsigned)(fb & (int)own_col);
        cfl = hll_pair(ra[1], rb[0], flux_ab<2>(ra[1], ra[2].z, ra[2].w), flux_ab<2>(rb[0], rb[2].x, rb[2].y), ra[3].z,
                       ra[3].w, rb[3].x, rb[3].y, chat);
        zpS = rb[1];
        zpa = rb[2].z;
        zpb = rb[2].w;
        zpl1 = rb[3].z;
        zpl3 = rb[3].w;
        ukp1 = u_1;
    }
    long long li = own_col ? (long long)gx + (long long)g.n[0] * gy + (long long)z0 * nxy : 0;
    // running pointers (64-bit offsets advanced once per plane): the next plane to stage, and the
    // own column of U^{m+1/2} two planes ahead
    const float4* next_plane = uh + (long long)(z0 + g.pad[2]) * pz;
    // the own column two planes ahead (k + 2) as a running offset: stored plane zs2 (k + 4 with ghost
    // layers, below n + 4; k + 2 wrapped into [0, n) where z is periodic)
    int zs2 = z0 + 2 + g.pad[2];
    if (zs2 >= upad_extent(g, 2)) zs2 -= g.n[2];
    long long col2 = colo + (long long)zs2 * pz;
    if constexpr (TMA) {
        if (t == 0) {
            mbar_init(mbar + 0, 1);
            mbar_init(mbar + 1, 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    issue_plane(next_plane, 0, z0);
    next_plane += pz;
    cp_async_commit();
    bool timed_out = false;
    int fail_buf = 0;
    unsigned fail_ph = 0;
#pragma unroll 1
    for (int k = z0; k < z1; ++k, li += nxy, next_plane += pz) {
        const int buf = (k - z0) & 1;
        ukp2 = uh[chk(col2, n_padded(g))];
        col2 += pz;
        if (++zs2 == upad_extent(g, 2)) {  // only where z is periodic
            zs2 = 0;
            col2 = colo;
        }
        if constexpr (TMA) {
            // completion of this plane's copy: buffer buf's ((k - z0) >> 1)-th use, phase parity = that & 1
            const unsigned ph = ((k - z0) >> 1) & 1;
            const bool ok = mbar_wait(mbar + buf, ph, wait_polls);
            if (__syncthreads_or(!ok)) {
                timed_out = true;
                fail_buf = buf;
                fail_ph = ph;
                break;
            }
        } else {
            cp_async_wait_all();
            __syncthreads();
        }
        // the own cell's data of this plane, one commit group, awaited before the own-cell block
        if (own_col) {
            const long long lc = chk(li, n_cells(g));
            cp_async8(oD + 0 * G::NT, a.E + lc);
            cp_async8(oD + 1 * G::NT, a.G[0] + lc);
            cp_async8(oD + 2 * G::NT, a.G[1] + lc);
            cp_async8(oD + 3 * G::NT, a.G[2] + lc);
            if (needT) cp_async8(oD + 4 * G::NT, a.T + lc);
            cp_async16(oG, a.gas4 + lc);
        }
        cp_async_commit();
        if (k + 1 < z1) issue_plane(next_plane, buf ^ 1, k + 1);
        cp_async_commit();
        const float4* Uk = Ubuf + buf * G::N2;
        // face-state records: the own cell along x and along y, then this thread's halo record
        {
            float4 rec[4];
            const int fb = face_record_ab<0>(Uk[ihc - 1], Uk[ihc], Uk[ihc + 1], chat, lim, p1, fixed, rec);
            cnt.face += (unsigned)(fb & (int)own_col);
            store_rec(Sx, G::NSX, sx_own, rec);
        }
        {
            float4 rec[4];
            const int fb = face_record_ab<1>(Uk[ihc - G::W2], Uk[ihc], Uk[ihc + G::W2], chat, lim, p1, fixed, rec);
            cnt.face += (unsigned)(fb & (int)own_col);
            store_rec(Sy, G::NSY, sy_own, rec);
        }
        if (has_hr) {
            float4 rec[4];
            if (hr_is_y) {
                face_record_ab<1>(Uk[hr_i - G::W2], Uk[hr_i], Uk[hr_i + G::W2], chat, lim, p1, fixed, rec);
                store_rec(Sy, G::NSY, hr_slot, rec);
            } else {
                face_record_ab<0>(Uk[hr_i - 1], Uk[hr_i], Uk[hr_i + 1], chat, lim, p1, fixed, rec);
                store_rec(Sx, G::NSX, hr_slot, rec);
            }
        }
        // the z face (k | k+1) of the own column
        float4 cfh;
        {
            float4 rec[4];
            const int fb = face_record_ab<2>(Uk[ihc], ukp1, ukp2, chat, lim, p1, fixed, rec);
            cnt.face += (unsigned)(fb & (int)(k + 1 < z1) & (int)own_col);
            cfh = hll_pair(zpS, rec[0], flux_ab<2>(zpS, zpa, zpb), flux_ab<2>(rec[0], rec[2].x, rec[2].y), zpl1, zpl3,
                           rec[3].x, rec[3].y, chat);
            zpS = rec[1];
            zpa = rec[2].z;
            zpb = rec[2].w;
            zpl1 = rec[3].z;
            zpl3 = rec[3].w;
        }
        __syncthreads();
        // fluxes: the x face left of the own cell, the y face below it, then the tile's top row and right column
        Cx[chk(tly * (TX + 1) + tlx, G::NCX)] = hll_x(sx_own - 1, sx_own);
        Cy[chk(tly * TX + tlx, G::NCY)] = hll_y(sy_own - TX, sy_own);
        if (t < TX) {
            Cy[chk(TY * TX + t, G::NCY)] = hll_y(G::sy(t, TY - 1), G::sy(t, TY));
        } else if (t < TX + TY) {
            const int ly = t - TX;
            Cx[chk(ly * (TX + 1) + TX, G::NCX)] = hll_x(G::sx(TX - 1, ly), G::sx(TX, ly));
        }
        __syncthreads();
        // own cell.  No barrier follows: every shared array written in the next plane is written after
        // that plane's first barrier, which no thread passes before all threads have finished this block.
        if constexpr (TMA) cp_async_wait_all();  // only the own-cell group is pending
        else cp_async_wait_1();                   // the own-cell group; the next plane's may still be pending
        if (own_col) {
            double U0[4], Tn = 0.0;
            U0[0] = oD[0 * G::NT];
            U0[1] = oD[1 * G::NT];
            U0[2] = oD[2 * G::NT];
            U0[3] = oD[3 * G::NT];
            if (needT) Tn = oD[4 * G::NT];
            GasCell<float> gc;
            gc.T = 0.0;
            gc.rho = 0.0;
            const float4 gv = *oG;
            const float rr = gv.x;
            gc.rho32 = rr;
            gc.v[0] = gv.y;
            gc.v[1] = gv.z;
            gc.v[2] = gv.w;
            const long long lo = chk(li, n_cells(g));
            gc.kP = a.kP32 ? __ldg(a.kP32 + lo) : kappa_law_f(g.f_kappa_P, g.kpow, rr);
            gc.kF = a.kF32 ? __ldg(a.kF32 + lo) : kappa_law_f(g.f_kappa_F, g.kpow, rr);
            gc.j = a.j32 ? __ldg(a.j32 + lo) : 0.0f;
            const int fl = tly * (TX + 1) + tlx, fb = tly * TX + tlx;
            const float4 ax = Cx[fl], bxf = Cx[fl + 1], ay = Cy[fb], by = Cy[fb + TX];
            const float div[4] = {(bxf.x - ax.x) * idx + (by.x - ay.x) * idy + (cfh.x - cfl.x) * idz,
                                  (bxf.y - ax.y) * idx + (by.y - ay.y) * idy + (cfh.y - cfl.y) * idz,
                                  (bxf.z - ax.z) * idx + (by.z - ay.z) * idy + (cfh.z - cfl.z) * idz,
                                  (bxf.w - ax.w) * idx + (by.w - ay.w) * idy + (cfh.w - cfl.w) * idz};
            const float4 Uhk4 = Uk[ihc];
            const float Uhk[4] = {Uhk4.x, Uhk4.y, Uhk4.z, Uhk4.w};
            const bool full = g.exchange == EX_FULL;
            float S[4];
            explicit_sources(g, gc, Uhk, chat, S);
            float d[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) d[qq] = -dt * div[qq] + dt * S[qq];
            double Un[4];
            split_stiff(g, a, sk, chat, dt, gc, U0, d, Tn, Un, cnt);
            // realizability: the FP32 mirror screens, the FP64 test runs only near the limit
            float4 m = make_float4(d2f_trunc(Un[0]), d2f_trunc(Un[1]), d2f_trunc(Un[2]), d2f_trunc(Un[3]));
            if (!(m.x > g.f_E_floor * 1.001f) || m.y * m.y + m.z * m.z + m.w * m.w > 0.9999f * m.x * m.x) {
                const int fx = realize(Un, g.E_floor);
                cnt.fix += fx;
                m = make_float4(d2f_trunc(Un[0]), d2f_trunc(Un[1]), d2f_trunc(Un[2]), d2f_trunc(Un[3]));
            }
            // non-finite, or beyond the FP32 range the split transport works in (the truncation maps both
            // to infinity): checked on the mirror's FP32 values
            const bool bad = !(isfinite(m.x) && isfinite(m.y) && isfinite(m.z) && isfinite(m.w)) ||
                             (full && !finite_d(Tn));
            cnt.nonfinite += bad;
            a.Eo[lo] = Un[0];
            a.Go[0][lo] = Un[1];
            a.Go[1][lo] = Un[2];
            a.Go[2][lo] = Un[3];
            // the FP32 mirror of U^{m+1} for the next subcycle's predictor
            a.um32[lo] = m;
            if (full) a.T[lo] = Tn;
        }
        cfl = cfh;
        ukp1 = ukp2;
    }
    cp_async_wait_all();
    if constexpr (TMA) {
        if (timed_out) {
            // a copy did not complete in time: count it, give the one copy in flight (the awaited one; the
            // next plane's copy is issued only after a successful wait) another wait with the full bound,
            // so that it lands before the CTA's shared memory is released, and leave the tile; the host
            // reports RHD_ERR_TIMEOUT
            if (t == 0) {
                cnt.timeout += 1;
                mbar_wait(mbar + fail_buf, fail_ph, kMaxPolls);
            }
            __syncthreads();
        }
    }
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX* TY, RHD_PRED_MIN_BLOCKS) predictor_kernel(const __grid_constant__ StepParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = blockIdx.x;
    const int x0 = (tile % P.tiles_x) * TX - P.g.pad[0], y0 = (tile / P.tiles_x) * TY - P.g.pad[1];
    const int z0 = (int)blockIdx.y * P.z_chunk - P.g.pad[2];
    const int z1 = min(z0 + P.z_chunk, P.g.n[2] + P.g.pad[2]);
    Counters cnt = {0, 0, 0, 0, 0, 0};
    predictor_tile<TX, TY>(P.g, P.a, P.uhalf, P.f_chat, P.f_dt, x0, y0, z0, z1, reinterpret_cast<float4*>(smem_raw), cnt);
    add_counter(&P.stats->n_fix, cnt.fix);
}

template <int TX, int TY, bool TMA, int LIMK>
__global__ void __launch_bounds__(TX* TY, RHD_CORR_MIN_BLOCKS) corrector_kernel(const __grid_constant__ StepParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    const int tile = blockIdx.x;
    const int x0 = (tile % P.tiles_x) * TX, y0 = (tile / P.tiles_x) * TY;
    const int z0 = (int)blockIdx.y * P.z_chunk;
    const int z1 = min(z0 + P.z_chunk, P.g.n[2]);
    Counters cnt = {0, 0, 0, 0, 0, 0};
    // TMA destinations need 128-byte alignment: the launch adds 128 bytes of slack
    float4* sm = reinterpret_cast<float4*>(smem_raw);
    if constexpr (TMA) sm = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    corrector_tile<TX, TY, TMA, LIMK>(P.g, P.a, P.uhalf, P.f_chat, P.f_dt, P.chat, P.dt, x0, y0, z0, z1, sm, cnt,
                                      &P.uh_map, mbar, P.wait_polls);
    add_counter(&P.stats->n_fix, cnt.fix);
    add_counter(&P.stats->n_face, cnt.face);
    add_counter(&P.stats->n_theta, cnt.theta);
    add_counter(&P.stats->n_newton_fb, cnt.newton_fb);
    add_counter(&P.stats->n_nonfinite, cnt.nonfinite);
    max_counter(&P.stats->newton_iter_max, cnt.iter_max);
    if (cnt.timeout) atomicAdd(&P.stats->n_timeout, cnt.timeout);
}

// ------------------------------------------------------------------------------------------------
// persistent ensemble kernels: CTAs pull (grid, tile, z chunk) items from a global counter; the item
// to grid map is a binary search over the grids' item prefix sums (predictor items cover each grid
// with its stored ghost layers, corrector items its interior)
// ------------------------------------------------------------------------------------------------

// Claim the next item; returns false when the queue is empty.  On true, eg holds the item's grid
// (copied to shared memory) and *local the item's index within that grid.
template <bool PRED>
__device__ __forceinline__ bool ens_next(const EnsembleParams& P, EnsembleGrid& eg, long long* item_s,
                                         long long* local)
{
    if (threadIdx.x == 0) *item_s = (long long)atomicAdd(P.counter, 1ull);
    __syncthreads();
    const long long item = *item_s;
    __syncthreads();
    if (item >= (PRED ? P.n_pitems : P.n_items)) return false;
    int lo = 0, hi = P.n_grids - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((PRED ? P.grids[mid].first_pitem : P.grids[mid].first_item) <= item) lo = mid;
        else hi = mid - 1;
    }
    {
        const int* src = reinterpret_cast<const int*>(P.grids + lo);
        int* dst = reinterpret_cast<int*>(&eg);
        for (int w = threadIdx.x; w < (int)(sizeof(EnsembleGrid) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    *local = item - (PRED ? eg.first_pitem : eg.first_item);
    return true;
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX* TY, RHD_PRED_MIN_BLOCKS) predictor_ens_kernel(const __grid_constant__ EnsembleParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long item_s;
    __shared__ __align__(16) EnsembleGrid eg;
    Counters cnt = {0, 0, 0, 0, 0, 0};
    long long local;
#pragma unroll 1
    while (ens_next<true>(P, eg, &item_s, &local)) {
        const long long nxy = (long long)eg.ptiles_x * eg.ptiles_y;
        const int txy = (int)(local % nxy), tz = (int)(local / nxy);
        const int x0 = (txy % eg.ptiles_x) * TX - eg.g.pad[0], y0 = (txy / eg.ptiles_x) * TY - eg.g.pad[1];
        const int z0 = tz * P.z_chunk - eg.g.pad[2], z1 = min(z0 + P.z_chunk, eg.g.n[2] + eg.g.pad[2]);
        predictor_tile<TX, TY>(eg.g, eg.a, eg.uhalf, P.f_chat, eg.f_dt, x0, y0, z0, z1,
                               reinterpret_cast<float4*>(smem_raw), cnt);
        __syncthreads();
    }
    add_counter(&P.stats->n_fix, cnt.fix);
}

template <int TX, int TY, int LIMK>
__global__ void __launch_bounds__(TX* TY, RHD_CORR_MIN_BLOCKS) corrector_ens_kernel(const __grid_constant__ EnsembleParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long item_s;
    __shared__ __align__(16) EnsembleGrid eg;
    Counters cnt = {0, 0, 0, 0, 0, 0};
    long long local;
#pragma unroll 1
    while (ens_next<false>(P, eg, &item_s, &local)) {
        const long long nxy = (long long)eg.tiles_x * eg.tiles_y;
        const int txy = (int)(local % nxy), tz = (int)(local / nxy);
        const int x0 = (txy % eg.tiles_x) * TX, y0 = (txy / eg.tiles_x) * TY;
        const int z0 = tz * P.z_chunk, z1 = min(z0 + P.z_chunk, eg.g.n[2]);
        corrector_tile<TX, TY, false, LIMK>(eg.g, eg.a, eg.uhalf, P.f_chat, eg.f_dt, P.chat, eg.dt, x0, y0, z0, z1,
                               reinterpret_cast<float4*>(smem_raw), cnt);
        __syncthreads();
    }
    add_counter(&P.stats->n_fix, cnt.fix);
    add_counter(&P.stats->n_face, cnt.face);
    add_counter(&P.stats->n_theta, cnt.theta);
    add_counter(&P.stats->n_newton_fb, cnt.newton_fb);
    add_counter(&P.stats->n_nonfinite, cnt.nonfinite);
    max_counter(&P.stats->newton_iter_max, cnt.iter_max);
}

}  // namespace rhd
