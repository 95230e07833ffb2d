// subcycle_twopass.cuh -- the split-precision subcycle for 3D grids as two kernels (included by
// subcycle.cuh after subcycle_pair.cuh).
//
//   predictor kernel: U^{m+1/2} of every cell of the grid padded by two ghost layers (the ghost cells
//     are the predictor applied to the ghost values of U^m, exactly as in the fused kernel and the
//     oracle), written as FP32 float4 (E, Gx, Gy, Gz);
//   corrector kernel: reconstruction, face states, HLL, divergence, sources, exchange and
//     realizability of the interior cells, reading U^{m+1/2} from the padded array (no boundary
//     remapping is needed there) and the FP64 state, updating the FP64 state.
// Each kernel marches column tiles through z.  Compared with the fused kernel the predictor is not
// recomputed on the corrector's halo, and each kernel needs far less shared memory and far fewer
// registers, so more warps are resident; the price is 32 bytes per cell of extra traffic (the FP32
// half-step state written once and read once).
#pragma once

namespace rhd {

// index of (x, y, z), each in [-2, n+2), in the padded U^{m+1/2} array
__device__ __forceinline__ long long pad_index(const GridParams& g, int x, int y, int z)
{
    const long long px = g.n[0] + 4, py = g.n[1] + 4;
    return (long long)(x + 2) + px * ((long long)(y + 2) + py * (long long)(z + 2));
}

template <int TX, int TY>
struct GeoPred {
    static constexpr int NT = TX * TY;
    static constexpr int W1 = TX + 2, H1 = TY + 2;
    static constexpr int N1 = W1 * H1;
    static constexpr int NR1 = (N1 + NT - 1) / NT;
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    // float4 units
    static constexpr int UM = 0, CXo = UM + N1, CYo = CXo + N1, L3o = CYo + N1;
    static constexpr int FXo = L3o + (N1 + 1) / 2, FYo = FXo + NFX, END4 = FYo + NFY;
    static constexpr int ST = 4 * N1;  // staged FP64 U^m, 4 per cell
    __host__ __device__ static constexpr size_t bytes() { return 16 * (size_t)END4 + 8 * (size_t)ST; }
    __device__ static __forceinline__ int i1(int lx, int ly) { return (lx + 1) + W1 * (ly + 1); }
};

// Predictor over the padded column tile (x0, y0) (coordinates in [-2, n+2)) for planes [z0, z1).
template <int TX, int TY>
__device__ __forceinline__ void predictor_tile(const GridParams& g, const GridArrays& a, float4* uh, double chat_d,
                                               double dt_d, int x0, int y0, int z0, int z1, float4* sm, Counters& cnt)
{
    using G = GeoPred<TX, TY>;
    const int t = threadIdx.x;
    float4* Um = sm + G::UM;
    float4* CX = sm + G::CXo;
    float4* CY = sm + G::CYo;
    float2* L3 = reinterpret_cast<float2*>(sm + G::L3o);
    float4* Fx = sm + G::FXo;
    float4* Fy = sm + G::FYo;
    double* stU = reinterpret_cast<double*>(sm + G::END4);
    const float chat = (float)chat_d, hdt = 0.5f * (float)dt_d;
    const float idx = (float)g.inv_dx[0], idy = (float)g.inv_dx[1], idz = (float)g.inv_dx[2];
    const int p1 = g.closure == 1, fixed = g.speeds == 1;
    const bool needT = g.exchange == EX_FROZEN_T;
    const long long nxy = (long long)g.n[0] * g.n[1];
    const int tlx = t % TX, tly = t / TX;
    const int gx = x0 + tlx, gy = y0 + tly;
    const bool own_in_pad = gx < g.n[0] + 2 && gy < g.n[1] + 2;
    const bool own_interior = gx >= 0 && gx < g.n[0] && gy >= 0 && gy < g.n[1];

    int c_i1[G::NR1], c_off[G::NR1];
    const bool xy_inside = x0 - 1 >= 0 && x0 + TX + 1 <= g.n[0] && y0 - 1 >= 0 && y0 + TY + 1 <= g.n[1];
#pragma unroll
    for (int r = 0; r < G::NR1; ++r) {
        const int c = t + r * G::NT;
        const int lx = c % G::W1 - 1, ly = c / G::W1 - 1;
        c_i1[r] = G::i1(lx, ly);
        c_off[r] = (x0 + lx) + g.n[0] * (y0 + ly);
    }
    auto issue_plane = [&](int q) {
        const bool fast = xy_inside && (unsigned)q < (unsigned)g.n[2];
        const long long zoff = (long long)q * nxy;
#pragma unroll
        for (int r = 0; r < G::NR1; ++r) {
            const int c = t + r * G::NT;
            if (c < G::N1) {
                double* d = stU + 4 * c;
                const int x = x0 + c % G::W1 - 1, y = y0 + c / G::W1 - 1;
                if (fast || inside(g, x, y, q)) {
                    const long long i = fast ? zoff + c_off[r] : lin(g, x, y, q);
                    cp_async8(d + 0, a.E + i);
                    cp_async8(d + 1, a.G[0] + i);
                    cp_async8(d + 2, a.G[1] + i);
                    cp_async8(d + 3, a.G[2] + i);
                } else {  // ghost cell: boundary rule (sign flips, Dirichlet values)
                    double U[4];
                    load_U(g, a, x, y, q, U);
                    d[0] = U[0];
                    d[1] = U[1];
                    d[2] = U[2];
                    d[3] = U[3];
                }
            }
        }
    };

    float4 zU = make_float4(0.f, 0.f, 0.f, 0.f), zP = zU, dxy = zU, zfl = zU;
    float zl3 = 0.f;
    const int qbeg = z0 - 1, qend = z1 + 1;
    issue_plane(qbeg);
    cp_async_commit();
#pragma unroll 1
    for (int q = qbeg; q < qend; ++q) {
        // gas of the own cell of plane q - 1, loaded here and used after the face phase
        const bool emit = q > qbeg + 1 && own_in_pad;
        GasCell<float> gc;
        if (emit) gc = load_gas<float, true>(g, a, gx, gy, q - 1, needT, false);
        cp_async_wait_all();
#pragma unroll
        for (int r = 0; r < G::NR1; ++r) {
            const int c = t + r * G::NT;
            if (c < G::N1) {
                const double* d = stU + 4 * c;
                Um[c_i1[r]] = make_float4(d2f_trunc(d[0]), d2f_trunc(d[1]), d2f_trunc(d[2]), d2f_trunc(d[3]));
            }
        }
        __syncthreads();
        if (q + 1 < qend) issue_plane(q + 1);
        cp_async_commit();
        // closure of the R1 cells; z data of the own cell
        float4 nU = zU, nP = zP;
        float nl3 = zl3;
#pragma unroll
        for (int r = 0; r < G::NR1; ++r) {
            const int c = t + r * G::NT;
            if (c < G::N1) {
                const int i = c_i1[r];
                const float4 U = Um[i];
                ClosureScalars<float> k = closure_scalars(U.x, U.y, U.z, U.w, chat, p1);
                const float bx = k.b * U.y;
                float l1x, l3x, l1y, l3y;
                wave_speeds(k, U.y, chat, fixed, l1x, l3x);
                wave_speeds(k, U.z, chat, fixed, l1y, l3y);
                const float Pxy = bx * U.z, Pxz = bx * U.w, Pyz = k.b * U.z * U.w;
                CX[i] = make_float4(k.a + bx * U.y, Pxy, Pxz, l1x);
                CY[i] = make_float4(Pxy, k.a + k.b * U.z * U.z, Pyz, l1y);
                L3[i] = make_float2(l3x, l3y);
            }
        }
        {
            // z data of the own cell (tlx, tly)
            const float4 U = Um[G::i1(tlx, tly)];
            ClosureScalars<float> k = closure_scalars(U.x, U.y, U.z, U.w, chat, p1);
            float l1z, l3z;
            wave_speeds(k, U.w, chat, fixed, l1z, l3z);
            nU = U;
            nP = make_float4(k.b * U.y * U.w, k.b * U.z * U.w, k.a + k.b * U.w * U.w, l1z);
            nl3 = l3z;
        }
        __syncthreads();
        // x and y faces of the tile rows / columns
        for (int f = t; f < G::NFX + G::NFY; f += G::NT) {
            if (f < G::NFX) {
                const int ly = f / (TX + 1), lx = f % (TX + 1);
                const int iL = G::i1(lx - 1, ly), iR = iL + 1;
                const float4 UL = Um[iL], UR = Um[iR], CL = CX[iL], CR = CX[iR];
                const float4 FL = make_float4(chat * UL.y, chat * CL.x, chat * CL.y, chat * CL.z);
                const float4 FR = make_float4(chat * UR.y, chat * CR.x, chat * CR.y, chat * CR.z);
                Fx[f] = hll_pair(UL, UR, FL, FR, CL.w, L3[iL].x, CR.w, L3[iR].x);
            } else {
                const int fc = f - G::NFX;
                const int ly = fc / TX, lx = fc % TX;
                const int iL = G::i1(lx, ly - 1), iR = iL + G::W1;
                const float4 UL = Um[iL], UR = Um[iR], CL = CY[iL], CR = CY[iR];
                const float4 FL = make_float4(chat * UL.z, chat * CL.x, chat * CL.y, chat * CL.z);
                const float4 FR = make_float4(chat * UR.z, chat * CR.x, chat * CR.y, chat * CR.z);
                Fy[fc] = hll_pair(UL, UR, FL, FR, CL.w, L3[iL].y, CR.w, L3[iR].y);
            }
        }
        __syncthreads();
        // own cell: x/y divergence of plane q, z face (q-1 | q), U^{m+1/2} of plane q - 1
        {
            const int fl = tly * (TX + 1) + tlx, fb = tly * TX + tlx;
            const float4 ax = Fx[fl], bxf = Fx[fl + 1], ay = Fy[fb], by = Fy[fb + TX];
            const float4 nd = make_float4((bxf.x - ax.x) * idx + (by.x - ay.x) * idy,
                                          (bxf.y - ax.y) * idx + (by.y - ay.y) * idy,
                                          (bxf.z - ax.z) * idx + (by.z - ay.z) * idy,
                                          (bxf.w - ax.w) * idx + (by.w - ay.w) * idy);
            float4 zfh = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q > qbeg) {
                const float4 FL = make_float4(chat * zU.w, chat * zP.x, chat * zP.y, chat * zP.z);
                const float4 FR = make_float4(chat * nU.w, chat * nP.x, chat * nP.y, chat * nP.z);
                zfh = hll_pair(zU, nU, FL, FR, zP.w, zl3, nP.w, nl3);
            }
            const int p = q - 1;
            if (emit) {
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
                uh[pad_index(g, gx, gy, p)] = f4(U);
            }
            zfl = zfh;
            zU = nU;
            zP = nP;
            zl3 = nl3;
            dxy = nd;
        }
        __syncthreads();
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
    // float4 units: two U^{m+1/2} plane buffers, face-state records, fluxes
    static constexpr int UK = 0, SXo = UK + 2 * N2, SYo = SXo + 5 * NSX, CXo = SYo + 5 * NSY, CYo = CXo + NCX;
    static constexpr int END4 = CYo + NCY;
    __host__ __device__ static constexpr size_t bytes() { return 16 * (size_t)END4; }
    __device__ static __forceinline__ int i2(int lx, int ly) { return (lx + 2) + W2 * (ly + 2); }
};

// Corrector over the interior column tile (x0, y0) for planes [z0, z1).
template <int TX, int TY>
__device__ __forceinline__ void corrector_tile(const GridParams& g, const GridArrays& a, const float4* uh,
                                               double chat_d, double dt_d, int x0, int y0, int z0, int z1, float4* sm,
                                               Counters& cnt)
{
    using G = GeoCorr<TX, TY>;
    const int t = threadIdx.x;
    float4* Ubuf = sm + G::UK;
    float4* Sx = sm + G::SXo;
    float4* Sy = sm + G::SYo;
    float4* Cx = sm + G::CXo;
    float4* Cy = sm + G::CYo;
    const float chat = (float)chat_d, dt = (float)dt_d;
    const float idx = (float)g.inv_dx[0], idy = (float)g.inv_dx[1], idz = (float)g.inv_dx[2];
    const int p1 = g.closure == 1, fixed = g.speeds == 1, lim = g.limiter;
    const bool needT = g.exchange == EX_FULL || g.exchange == EX_FROZEN_T;
    const int tlx = t % TX, tly = t / TX;
    const int gx = x0 + tlx, gy = y0 + tly;
    const bool own_col = gx < g.n[0] && gy < g.n[1];
    const long long pz = (long long)(g.n[0] + 4) * (g.n[1] + 4);

    // the R2 plane of U^{m+1/2}: rows of W2 float4 starting at (x0 - 2, y0 + ly); all inside the padded array
    // except beyond the high edges of ragged tiles, which are clamped (those values are never used)
    int c_gpos[G::NR2];
#pragma unroll
    for (int r = 0; r < G::NR2; ++r) {
        const int c = t + r * G::NT;
        const int lx = c % G::W2 - 2, ly = c / G::W2 - 2;
        const int xx = min(x0 + lx, g.n[0] + 1), yy = min(y0 + ly, g.n[1] + 1);
        c_gpos[r] = (xx + 2) + (g.n[0] + 4) * (yy + 2);
    }
    auto issue_plane = [&](int k, int buf) {
        const float4* base = uh + (long long)(k + 2) * pz;
#pragma unroll
        for (int r = 0; r < G::NR2; ++r) {
            const int c = t + r * G::NT;
            if (c < G::N2) {
                unsigned dsm = (unsigned)__cvta_generic_to_shared(Ubuf + buf * G::N2 + c);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dsm), "l"(base + c_gpos[r])
                             : "memory");
            }
        }
    };
    const int ihc = G::i2(tlx, tly);
    auto col = [&](int k) { return uh[(long long)(k + 2) * pz + (min(gx, g.n[0] + 1) + 2) + (long long)(g.n[0] + 4) * (min(gy, g.n[1] + 1) + 2)]; };

    // lower z face of the first plane: face states of cells z0-1 and z0 from U^{m+1/2} at z0-2 .. z0+1
    float4 zpS, zpF, cfl;
    float zpl1, zpl3;
    float4 ukp1, ukp2;  // U^{m+1/2} of the own column at k+1, k+2
    {
        const float4 u_m2 = col(z0 - 2), u_m1 = col(z0 - 1), u_0 = col(z0), u_1 = col(z0 + 1);
        float4 ra[5], rb[5];
        face_record<2>(u_m2, u_m1, u_0, chat, lim, p1, fixed, ra);
        const int fb = face_record<2>(u_m1, u_0, u_1, chat, lim, p1, fixed, rb);
        if (fb && own_col) cnt.face += 1;
        cfl = hll_pair(ra[2], rb[0], ra[3], rb[1], ra[4].z, ra[4].w, rb[4].x, rb[4].y);
        zpS = rb[2];
        zpF = rb[3];
        zpl1 = rb[4].z;
        zpl3 = rb[4].w;
        ukp1 = u_1;
    }
    issue_plane(z0, 0);
    cp_async_commit();
#pragma unroll 1
    for (int k = z0; k < z1; ++k) {
        const int buf = (k - z0) & 1;
        ukp2 = col(k + 2);
        // the own cell's FP64 state, temperature and gas, loaded here and used after the face phases
        double U0[4] = {0.0, 0.0, 0.0, 0.0}, Tn = 0.0;
        GasCell<float> gc;
        long long li = 0;
        if (own_col) {
            li = lin(g, gx, gy, k);
            U0[0] = __ldg(a.E + li);
            U0[1] = __ldg(a.G[0] + li);
            U0[2] = __ldg(a.G[1] + li);
            U0[3] = __ldg(a.G[2] + li);
            if (needT) Tn = a.T[li];
            gc = load_gas<float, true>(g, a, gx, gy, k, false, false);
        }
        cp_async_wait_all();
        __syncthreads();
        if (k + 1 < z1) issue_plane(k + 1, buf ^ 1);
        cp_async_commit();
        const float4* Uk = Ubuf + buf * G::N2;
        // face-state records along x and y, and the z face (k | k+1) of the own column
        for (int c = t; c < G::NSX + G::NSY; c += G::NT) {
            float4 rec[5];
            if (c < G::NSX) {
                const int ly = c / (TX + 2), lx = c % (TX + 2) - 1;
                const int i = G::i2(lx, ly);
                const int fb = face_record<0>(Uk[i - 1], Uk[i], Uk[i + 1], chat, lim, p1, fixed, rec);
                if (fb && lx >= 0 && lx < TX && x0 + lx < g.n[0] && y0 + ly < g.n[1]) cnt.face += 1;
#pragma unroll
                for (int v = 0; v < 5; ++v) Sx[v * G::NSX + c] = rec[v];
            } else {
                const int cy = c - G::NSX;
                const int ly = cy / TX - 1, lx = cy % TX;
                const int i = G::i2(lx, ly);
                const int fb = face_record<1>(Uk[i - G::W2], Uk[i], Uk[i + G::W2], chat, lim, p1, fixed, rec);
                if (fb && ly >= 0 && ly < TY && x0 + lx < g.n[0] && y0 + ly < g.n[1]) cnt.face += 1;
#pragma unroll
                for (int v = 0; v < 5; ++v) Sy[v * G::NSY + cy] = rec[v];
            }
        }
        float4 cfh;
        {
            float4 rec[5];
            const int fb = face_record<2>(Uk[ihc], ukp1, ukp2, chat, lim, p1, fixed, rec);
            if (fb && k + 1 < z1 && own_col) cnt.face += 1;
            cfh = hll_pair(zpS, rec[0], zpF, rec[1], zpl1, zpl3, rec[4].x, rec[4].y);
            zpS = rec[2];
            zpF = rec[3];
            zpl1 = rec[4].z;
            zpl3 = rec[4].w;
        }
        __syncthreads();
        for (int f = t; f < G::NCX + G::NCY; f += G::NT) {
            if (f < G::NCX) {
                const int ly = f / (TX + 1), lx = f % (TX + 1);
                const int iL = lx + (TX + 2) * ly, iR = iL + 1;
                const float4 LL = Sx[4 * G::NSX + iL], LR = Sx[4 * G::NSX + iR];
                Cx[f] = hll_pair(Sx[2 * G::NSX + iL], Sx[iR], Sx[3 * G::NSX + iL], Sx[G::NSX + iR], LL.z, LL.w,
                                 LR.x, LR.y);
            } else {
                const int fc = f - G::NCX;
                const int ly = fc / TX, lx = fc % TX;
                const int iL = lx + TX * ly, iR = iL + TX;
                const float4 LL = Sy[4 * G::NSY + iL], LR = Sy[4 * G::NSY + iR];
                Cy[fc] = hll_pair(Sy[2 * G::NSY + iL], Sy[iR], Sy[3 * G::NSY + iL], Sy[G::NSY + iR], LL.z, LL.w,
                                  LR.x, LR.y);
            }
        }
        __syncthreads();
        if (own_col) {
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
            float u0f[4], d[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                u0f[qq] = d2f_trunc(U0[qq]);
                d[qq] = -dt * div[qq] + dt * S[qq];
            }
            const float thF = g.f_theta_F, thE = g.f_theta_E;
            const float xF = chat * gc.kF * dt;
            const float wF = xF * rcp(1.0f + thF * xF);
#pragma unroll
            for (int qq = 1; qq < 4; ++qq) d[qq] -= (u0f[qq] + d[qq]) * wF;
            if (g.exchange == EX_ABSORB) {
                const float xP = chat * gc.kP * dt;
                d[0] -= (u0f[0] + d[0]) * (xP * rcp(1.0f + thE * xP));
            } else if (g.exchange == EX_FROZEN_T) {
                const float xP = chat * gc.kP * dt;
                const float Tf = d2f_trunc(Tn);
                const float aT4 = g.f_a_rad * (Tf * Tf) * (Tf * Tf);
                d[0] += xP * (aT4 - (u0f[0] + d[0])) * rcp(1.0f + thE * xP);
            }
            double Etr = U0[0] + f2d_exact(d[0]);
            if (full) {
                float Ef = u0f[0] + d[0];
                if (!(Ef > 2.0f * g.f_E_floor)) {
                    if (Etr < g.E_floor) Etr = g.E_floor;
                    Ef = d2f_trunc(Etr);
                }
                ExchangeOut o;
                float qv;
                const float del = exchange_delta_fp32(g, chat, dt, gc.rho32, gc.kP, Ef, d2f_trunc(Tn), o, qv);
                const float dE = (chat * g.f_inv_c) * del;
                Etr = Etr - f2d_exact(dE);
                d[0] = Ef - dE - u0f[0];
                Tn = Tn + f2d_exact(qv * del);
                cnt.theta += o.theta_fb;
                cnt.newton_fb += o.newton_fb;
                cnt.iter_max = max(cnt.iter_max, (unsigned)o.iters);
            }
            double Un[4] = {Etr, U0[1] + f2d_exact(d[1]), U0[2] + f2d_exact(d[2]), U0[3] + f2d_exact(d[3])};
            const float ef = u0f[0] + d[0];
            float g2f = 0.f;
#pragma unroll
            for (int qq = 1; qq < 4; ++qq) {
                const float gq = u0f[qq] + d[qq];
                g2f += gq * gq;
            }
            if (!(ef > g.f_E_floor * 1.001f) || g2f > 0.9999f * ef * ef) cnt.fix += realize(Un, g.E_floor);
            const bool bad = !(finite_d(Un[0]) && finite_d(Un[1]) && finite_d(Un[2]) && finite_d(Un[3]) &&
                               (!full || finite_d(Tn)));
            cnt.nonfinite += bad;
            a.Eo[li] = Un[0];
            a.Go[0][li] = Un[1];
            a.Go[1][li] = Un[2];
            a.Go[2][li] = Un[3];
            if (full) a.T[li] = Tn;
        }
        cfl = cfh;
        ukp1 = ukp2;
        __syncthreads();
    }
    cp_async_wait_all();
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX* TY, 4) predictor_kernel(const __grid_constant__ StepParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = blockIdx.x;
    const int x0 = (tile % P.tiles_x) * TX - 2, y0 = (tile / P.tiles_x) * TY - 2;
    const int z0 = (int)blockIdx.y * P.z_chunk - 2;
    const int z1 = min(z0 + P.z_chunk, P.g.n[2] + 2);
    Counters cnt = {0, 0, 0, 0, 0, 0};
    predictor_tile<TX, TY>(P.g, P.a, P.uhalf, P.chat, P.dt, x0, y0, z0, z1, reinterpret_cast<float4*>(smem_raw), cnt);
    add_counter(&P.stats->n_fix, cnt.fix);
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX* TY, 3) corrector_kernel(const __grid_constant__ StepParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = blockIdx.x;
    const int x0 = (tile % P.tiles_x) * TX, y0 = (tile / P.tiles_x) * TY;
    const int z0 = (int)blockIdx.y * P.z_chunk;
    const int z1 = min(z0 + P.z_chunk, P.g.n[2]);
    Counters cnt = {0, 0, 0, 0, 0, 0};
    corrector_tile<TX, TY>(P.g, P.a, P.uhalf, P.chat, P.dt, x0, y0, z0, z1, reinterpret_cast<float4*>(smem_raw), cnt);
    add_counter(&P.stats->n_fix, cnt.fix);
    add_counter(&P.stats->n_face, cnt.face);
    add_counter(&P.stats->n_theta, cnt.theta);
    add_counter(&P.stats->n_newton_fb, cnt.newton_fb);
    add_counter(&P.stats->n_nonfinite, cnt.nonfinite);
    max_counter(&P.stats->newton_iter_max, cnt.iter_max);
}

// ------------------------------------------------------------------------------------------------
// persistent ensemble kernels: CTAs pull (grid, tile, z chunk) items from a global counter; the item
// to grid map is a binary search over the grids' item prefix sums (predictor items cover each grid
// padded by two ghost layers, corrector items its interior)
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
__global__ void __launch_bounds__(TX* TY, 4) predictor_ens_kernel(const __grid_constant__ EnsembleParams P)
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
        const int x0 = (txy % eg.ptiles_x) * TX - 2, y0 = (txy / eg.ptiles_x) * TY - 2;
        const int z0 = tz * P.z_chunk - 2, z1 = min(z0 + P.z_chunk, eg.g.n[2] + 2);
        predictor_tile<TX, TY>(eg.g, eg.a, eg.uhalf, P.chat, eg.dt, x0, y0, z0, z1,
                               reinterpret_cast<float4*>(smem_raw), cnt);
        __syncthreads();
    }
    add_counter(&P.stats->n_fix, cnt.fix);
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX* TY, 3) corrector_ens_kernel(const __grid_constant__ EnsembleParams P)
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
        corrector_tile<TX, TY>(eg.g, eg.a, eg.uhalf, P.chat, eg.dt, x0, y0, z0, z1,
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
