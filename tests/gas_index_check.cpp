// Host enumeration of every array index the gas-step kernels compute (through the functions of
// gas_index.h that the kernels call), for a set of grid shapes and boundary conditions: each index must
// lie inside its array.  Also prints the ghost rule along one axis for comparison with the oracle.
//
// Usage: gas_index_check            -> "ok <cases>" or the first violation, exit status 0 / 1
//        gas_index_check axis n lo hi g -> "c index sign" lines for c = -g .. n+g-1
#include <cstdio>
#include <cstdlib>
#include <string_view>

#include "gas_index.h"

using namespace rhd;

static int fail_count = 0;

static void check(bool ok, const char* what, long long v, long long extent, const int n[3])
{
    if (ok) return;
    if (fail_count++ < 5)
        std::printf("violation: %s = %lld outside [0, %lld) for n = (%d, %d, %d)\n", what, v, extent, n[0], n[1], n[2]);
}

static void check_grid(const int n[3], const int lo[3], const int hi[3])
{
    GasParams p{};
    gas_set_geometry(p, n, lo, hi);
    const long long ncell = gas_count(p.n), next = gas_count(p.m);
    long long cap[3];
    for (int d = 0; d < 3; ++d) cap[d] = gas_face_capacity(p, d);
    for (int d = 0; d < 3; ++d) {
        if (p.n[d] <= 1) continue;
        int fe[3];
        gas_pred_faces(p, d, fe);
        for (long long f = 0; f < gas_count(fe); ++f) {
            check(f < cap[d], "predictor face", f, cap[d], n);
            long long iL, iR;
            int sL[3], sR[3];
            gas_pred_flux_cells(p, d, f, &iL, sL, &iR, sR);
            check(iL >= 0 && iL < ncell, "predictor flux iL", iL, ncell, n);
            check(iR >= 0 && iR < ncell, "predictor flux iR", iR, ncell, n);
        }
        gas_corr_faces(p, d, fe);
        for (long long f = 0; f < gas_count(fe); ++f) {
            check(f < cap[d], "corrector face", f, cap[d], n);
            long long x[4];
            gas_corr_flux_cells(p, d, f, x);
            for (int j = 0; j < 4; ++j) check(x[j] >= 0 && x[j] < next, "corrector flux cell", x[j], next, n);
        }
    }
    for (long long i = 0; i < next; ++i) {
        long long k, l[3], h[3];
        int s[3];
        bool inside;
        gas_pred_update_cells(p, i, &k, s, &inside, l, h);
        check(k >= 0 && k < ncell, "predictor update cell", k, ncell, n);
        for (int d = 0; d < 3; ++d) {
            if (p.n[d] <= 1) continue;
            int fe[3];
            gas_pred_faces(p, d, fe);
            check(l[d] >= 0 && l[d] < gas_count(fe), "predictor update low face", l[d], gas_count(fe), n);
            check(h[d] >= 0 && h[d] < gas_count(fe), "predictor update high face", h[d], gas_count(fe), n);
        }
    }
    for (long long i = 0; i < ncell; ++i) {
        long long x, l[3], h[3];
        gas_corr_update_cells(p, i, &x, l, h);
        check(x >= 0 && x < next, "corrector update cell", x, next, n);
        for (int d = 0; d < 3; ++d) {
            if (p.n[d] <= 1) continue;
            int fe[3];
            gas_corr_faces(p, d, fe);
            check(l[d] >= 0 && l[d] < gas_count(fe), "corrector update low face", l[d], gas_count(fe), n);
            check(h[d] >= 0 && h[d] < gas_count(fe), "corrector update high face", h[d], gas_count(fe), n);
        }
    }
}

int main(int argc, char** argv)
{
    if (argc == 6 && std::string_view(argv[1]) == "axis") {
        const int n = std::atoi(argv[2]), lo = std::atoi(argv[3]), hi = std::atoi(argv[4]), g = std::atoi(argv[5]);
        for (int c = -g; c < n + g; ++c) {
            int s = 1;
            const int q = gas_axis(c, n, lo, hi, s);
            std::printf("%d %d %d\n", c, q, s);
        }
        return 0;
    }
    const int shapes[][3] = {{3, 1, 1}, {5, 1, 1}, {1, 4, 1}, {1, 1, 7}, {3, 3, 1}, {5, 3, 3}, {7, 4, 3},
                             {3, 5, 9}, {16, 3, 1}, {33, 9, 5}, {1, 6, 5}, {4, 1, 6}, {2, 2, 2}, {2, 3, 1}};
    int cases = 0;
    for (const auto& n : shapes)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const int lo[3] = {a, b, (a + b) % 4}, hi[3] = {b, (a + 1) % 4, a};
                check_grid(n, lo, hi);
                ++cases;
            }
    if (fail_count) {
        std::printf("%d violations\n", fail_count);
        return 1;
    }
    std::printf("ok %d\n", cases);
    return 0;
}
