// gas_index.h -- index arithmetic of the gas-step kernels (k_gas.cu): the ghost rule, the layouts of
// the extended grid and of the face-flux arrays.  Host-and-device code: the kernels compute every
// array index through these functions, and a host test enumerates them over whole grids to check that
// every index stays inside its array.
#pragma once

#include "gas_internal.h"

#ifdef __CUDACC__
#define GAS_HD __host__ __device__ __forceinline__
#else
#define GAS_HD inline
#endif

namespace rhd {

// Ghost rule along one axis (the rule of the radiation path, with the gas's Dirichlet reading):
// periodic wraps, outflow and Dirichlet take the nearest cell, reflect mirrors and flips the sign of
// the normal component.  Coordinates within 2n of the grid need at most two steps; the clamp keeps
// any other coordinate inside [0, n).
GAS_HD int gas_axis(int c, int n, int lo, int hi, int& s)
{
    for (int it = 0; it < 4 && (c < 0 || c >= n); ++it) {
        const bool low = c < 0;
        const int bc = low ? lo : hi;
        if (bc == 0) {            // periodic
            c = ((c % n) + n) % n;
        } else if (bc == 2) {     // reflect
            c = low ? -c - 1 : 2 * n - 1 - c;
            s = -s;
        } else {                  // outflow, Dirichlet
            c = low ? 0 : n - 1;
        }
    }
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// interior linear index of the cell at coordinates c (which may lie in the ghost layers) and the
// signs (+1 or -1) of its normal components s[d]
GAS_HD long long gas_remap(const GasParams& p, const int c[3], int s[3])
{
    int q[3];
    for (int d = 0; d < 3; ++d) {
        s[d] = 1;
        q[d] = gas_axis(c[d], p.n[d], p.bc_lo[d], p.bc_hi[d], s[d]);
    }
    return q[0] + (long long)p.n[0] * (q[1] + (long long)p.n[1] * q[2]);
}

GAS_HD void gas_unravel(long long i, const int e[3], int a[3])
{
    a[0] = (int)(i % e[0]);
    const long long t = i / e[0];
    a[1] = (int)(t % e[1]);
    a[2] = (int)(t / e[1]);
}

GAS_HD long long gas_ravel(const int a[3], const int e[3])
{
    return a[0] + (long long)e[0] * (a[1] + (long long)e[1] * a[2]);
}

// face-flux layouts of direction d: the predictor's faces bound the extended grid (m + e_d faces),
// the corrector's the interior (n + e_d); face a lies on the low side of cell a
GAS_HD void gas_pred_faces(const GasParams& p, int d, int e[3])
{
    for (int k = 0; k < 3; ++k) e[k] = p.m[k] + (k == d ? 1 : 0);
}

GAS_HD void gas_corr_faces(const GasParams& p, int d, int e[3])
{
    for (int k = 0; k < 3; ++k) e[k] = p.n[k] + (k == d ? 1 : 0);
}

GAS_HD long long gas_count(const int e[3]) { return (long long)e[0] * e[1] * e[2]; }

// elements of a face-flux array of direction d (the predictor's layout, the larger of the two)
inline long long gas_face_capacity(const GasParams& p, int d)
{
    int e[3];
    gas_pred_faces(p, d, e);
    return gas_count(e);
}

// the geometry fields of p (n, g, m, bc_lo, bc_hi) for a grid of n cells; a direction with n > 1 is active
inline void gas_set_geometry(GasParams& p, const int n[3], const int bc_lo[3], const int bc_hi[3])
{
    for (int d = 0; d < 3; ++d) {
        p.n[d] = n[d];
        p.g[d] = n[d] > 1 ? GAS_GHOST : 0;
        p.m[d] = n[d] + 2 * p.g[d];
        p.bc_lo[d] = bc_lo[d];
        p.bc_hi[d] = bc_hi[d];
    }
}

// ---- the indices each kernel thread touches (the kernels call these; the host test enumerates them)

// predictor flux, face f of direction d: the interior indices (and normal-component signs) of the cells
// on its low (L) and high (R) side
GAS_HD void gas_pred_flux_cells(const GasParams& p, int d, long long f, long long* iL, int sL[3], long long* iR,
                                int sR[3])
{
    int fe[3], A[3], cL[3], cR[3];
    gas_pred_faces(p, d, fe);
    gas_unravel(f, fe, A);
    for (int k = 0; k < 3; ++k) cR[k] = cL[k] = A[k] - p.g[k];
    cL[d] -= 1;
    *iL = gas_remap(p, cL, sL);
    *iR = gas_remap(p, cR, sR);
}

// predictor update, extended cell i: the interior cell k it is filled from (signs s), whether it is an
// interior cell, and its low / high faces in each active direction's predictor layout (-1: inactive)
GAS_HD void gas_pred_update_cells(const GasParams& p, long long i, long long* k, int s[3], bool* inside,
                                  long long lo[3], long long hi[3])
{
    int A[3], c[3];
    gas_unravel(i, p.m, A);
    *inside = true;
    for (int q = 0; q < 3; ++q) {
        c[q] = A[q] - p.g[q];
        *inside = *inside && c[q] >= 0 && c[q] < p.n[q];
    }
    *k = gas_remap(p, c, s);
    for (int d = 0; d < 3; ++d) {
        lo[d] = hi[d] = -1;
        if (p.n[d] <= 1) continue;
        int fe[3], B[3] = {A[0], A[1], A[2]};
        gas_pred_faces(p, d, fe);
        B[d] += 1;
        lo[d] = gas_ravel(A, fe);
        hi[d] = gas_ravel(B, fe);
    }
}

// corrector flux, face f of direction d: the extended-grid indices of the cells f - 2 e_d .. f + e_d
GAS_HD void gas_corr_flux_cells(const GasParams& p, int d, long long f, long long x[4])
{
    int fe[3], A[3];
    gas_corr_faces(p, d, fe);
    gas_unravel(f, fe, A);
    for (int j = 0; j < 4; ++j) {
        int X[3];
        for (int k = 0; k < 3; ++k) X[k] = A[k] + p.g[k];
        X[d] += j - 2;
        x[j] = gas_ravel(X, p.m);
    }
}

// corrector update, interior cell i: its extended-grid index and its low / high faces in each active
// direction's corrector layout (-1: inactive)
GAS_HD void gas_corr_update_cells(const GasParams& p, long long i, long long* x, long long lo[3], long long hi[3])
{
    int A[3], X[3];
    gas_unravel(i, p.n, A);
    for (int k = 0; k < 3; ++k) X[k] = A[k] + p.g[k];
    *x = gas_ravel(X, p.m);
    for (int d = 0; d < 3; ++d) {
        lo[d] = hi[d] = -1;
        if (p.n[d] <= 1) continue;
        int fe[3], B[3] = {A[0], A[1], A[2]};
        gas_corr_faces(p, d, fe);
        B[d] += 1;
        lo[d] = gas_ravel(A, fe);
        hi[d] = gas_ravel(B, fe);
    }
}

}  // namespace rhd
