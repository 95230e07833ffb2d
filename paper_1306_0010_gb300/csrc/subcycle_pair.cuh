// subcycle_pair.cuh -- FP32 closure, face-state and HLL helpers for the two-pass split kernels
// (included by subcycle.cuh).
//
// Same formulas and readings as closure_scalars / wave_speeds / face_states / hll in subcycle.cuh,
// laid out for instruction throughput on sm_103a: one float4 (E, Gx, Gy, Gz) per state, the two face
// values (minus, plus) of a cell run through the closure as one pair of FP32 lanes with the packed
// FP32x2 instructions (fadd2 / fmul2 / ffma2), and the HLL flux combines its four components as two
// such pairs.
#pragma once

namespace rhd {

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_s(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 p_rcp(float2 a) { return make_float2(rcp(a.x), rcp(a.y)); }
__device__ __forceinline__ float2 p_sqrt(float2 a) { return make_float2(sqrt_fast(a.x), sqrt_fast(a.y)); }
__device__ __forceinline__ float2 p_lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 p_hi(float4 v) { return make_float2(v.z, v.w); }

// Closure of two states at once (lane .x and lane .y) in direction D: flux chat (G_D, P_D.) and the
// wave speeds lambda_1, lambda_3 (same formulas as closure_scalars / wave_speeds / dir_flux).
template <int D>
__device__ __forceinline__ void closure_pair(float2 E, float2 gx, float2 gy, float2 gz, float chat, int p1, int fixed,
                                             float2 F[4], float2& l1, float2& l3)
{
    const float2 ch = p_s(chat);
    const float2 invE = p_rcp(E);
    const float2 g2 = p_fma(gz, gz, p_fma(gy, gy, p_mul(gx, gx)));
    float2 f2 = p_mul(g2, p_mul(invE, invE));
    f2.x = fminf(f2.x, 1.f);
    f2.y = fminf(f2.y, 1.f);
    const float2 s = p_sqrt(p_fma(p_s(-3.f), f2, p_s(4.f)));
    const float2 inv2ps = p_rcp(p_add(s, p_s(2.f)));
    const float2 sm1 = p_add(s, p_s(-1.f));
    float2 a, b;
    if (p1) {
        a = p_mul(E, p_s(1.f / 3.f));
        b = p_s(0.f);
    } else {
        a = p_mul(p_mul(sm1, E), p_s(1.f / 3.f));
        b = p_mul(p_mul(inv2ps, invE), p_s(3.f));
    }
    const float2 gd = D == 0 ? gx : (D == 1 ? gy : gz);
    const float2 bg = p_mul(b, gd);
    F[0] = p_mul(ch, gd);
    F[1] = p_mul(ch, D == 0 ? p_fma(bg, gx, a) : p_mul(bg, gx));
    F[2] = p_mul(ch, D == 1 ? p_fma(bg, gy, a) : p_mul(bg, gy));
    F[3] = p_mul(ch, D == 2 ? p_fma(bg, gz, a) : p_mul(bg, gz));
    if (fixed) {
        l3 = p_s(chat * 0.57735026918962576451f);
        l1 = p_s(-chat * 0.57735026918962576451f);
        return;
    }
    const float2 fd = p_mul(gd, invE);
    const float2 u = p_fma(p_s(-3.f), p_mul(p_mul(fd, fd), inv2ps), s);
    float2 rad = p_mul(p_mul(sm1, p_s(2.f / 3.f)), u);
    rad.x = fmaxf(rad.x, 0.f);
    rad.y = fmaxf(rad.y, 0.f);
    const float2 sr = p_sqrt(rad);
    const float2 cs = p_mul(ch, p_rcp(s));
    l1 = p_mul(p_sub(fd, sr), cs);
    l3 = p_mul(p_add(fd, sr), cs);
}

// Closure coefficients of two states (lanes .x, .y): P = a I + b G G^T (a, b of closure_scalars) and
// the wave speeds lambda_1, lambda_3 in direction D; the flux follows from (U, a, b) by flux_ab.
template <int D>
__device__ __forceinline__ void closure_ab_pair(float2 E, float2 gx, float2 gy, float2 gz, float chat, int p1,
                                                int fixed, float2& a, float2& b, float2& l1, float2& l3)
{
    const float2 ch = p_s(chat);
    const float2 invE = p_rcp(E);
    const float2 g2 = p_fma(gz, gz, p_fma(gy, gy, p_mul(gx, gx)));
    float2 f2 = p_mul(g2, p_mul(invE, invE));
    f2.x = fminf(f2.x, 1.f);
    f2.y = fminf(f2.y, 1.f);
    const float2 s = p_sqrt(p_fma(p_s(-3.f), f2, p_s(4.f)));
    const float2 inv2ps = p_rcp(p_add(s, p_s(2.f)));
    const float2 sm1 = p_add(s, p_s(-1.f));
    if (p1) {
        a = p_mul(E, p_s(1.f / 3.f));
        b = p_s(0.f);
    } else {
        a = p_mul(p_mul(sm1, E), p_s(1.f / 3.f));
        b = p_mul(p_mul(inv2ps, invE), p_s(3.f));
    }
    if (fixed) {
        l3 = p_s(chat * 0.57735026918962576451f);
        l1 = p_s(-chat * 0.57735026918962576451f);
        return;
    }
    const float2 gd = D == 0 ? gx : (D == 1 ? gy : gz);
    const float2 fd = p_mul(gd, invE);
    const float2 u = p_fma(p_s(-3.f), p_mul(p_mul(fd, fd), inv2ps), s);
    float2 rad = p_mul(p_mul(sm1, p_s(2.f / 3.f)), u);
    rad.x = fmaxf(rad.x, 0.f);
    rad.y = fmaxf(rad.y, 0.f);
    const float2 sr = p_sqrt(rad);
    const float2 cs = p_mul(ch, p_rcp(s));
    l1 = p_mul(p_sub(fd, sr), cs);
    l3 = p_mul(p_add(fd, sr), cs);
}

// Flux per unit chat, (G_D, P_D.), of state U in direction D from its closure coefficients; the HLL
// weights of hll_pair / hll4 carry the factor chat.
template <int D>
__device__ __forceinline__ float4 flux_ab(float4 U, float a, float b)
{
    const float gd = D == 0 ? U.y : (D == 1 ? U.z : U.w);
    const float bg = xmul(b, gd);
    return make_float4(gd, D == 0 ? xfma(bg, U.y, a) : xmul(bg, U.y), D == 1 ? xfma(bg, U.z, a) : xmul(bg, U.z),
                       D == 2 ? xfma(bg, U.w, a) : xmul(bg, U.w));
}

// minmod(a, b): the one of a, b nearer zero if they have the same sign, else 0, as three min / max:
// both positive -> min(a, b); both negative -> min(0, max(a, b)) = max(a, b); mixed signs -> max of
// a negative number and 0.
__device__ __forceinline__ float minmod_f(float a, float b) { return fmaxf(fminf(a, b), fminf(0.0f, fmaxf(a, b))); }

// Limited slope from the left and right differences (minmod, MC or none): the same values as
// `limited` in subcycle.cuh (MC = minmod(2 minmod(dl, dr), (dl + dr)/2)), as straight-line min / max
// code the compiler can interleave with the other direction's record; with lim a compile-time
// constant only the chosen limiter remains.
__device__ __forceinline__ float limited_f(float dl, float dr, int lim)
{
    const float avg = 0.5f * (dl + dr);
    const float mm = minmod_f(dl, dr);
    if (lim == LIM_NONE) return avg;
    if (lim == LIM_MC) return minmod_f(2.0f * mm, avg);
    return mm;
}

// E <= 0 or |G|^2 > (1 + tol) E^2, without short-circuit branches (same test as face_unrealizable)
__device__ __forceinline__ int unrealizable_f(float4 U)
{
    const float g2 = xfma(U.w, U.w, xfma(U.z, U.z, xmul(U.y, U.y)));
    return (int)(!(U.x > 0.0f)) | (int)(g2 > xmul(1.0f + Tol<float>::face, xmul(U.x, U.x)));
}

// Face-state record of one cell in direction D (see face_states): minus state, its flux, plus state,
// its flux, and (l1m, l3m, l1p, l3p).  Returns 1 if the slope was zeroed.
template <int D>
__device__ __forceinline__ int face_record(float4 um, float4 u0, float4 up, float chat, int lim, int p1, int fixed,
                                           float4 rec[5])
{
    float4 sl;
    sl.x = limited_f(u0.x - um.x, up.x - u0.x, lim);
    sl.y = limited_f(u0.y - um.y, up.y - u0.y, lim);
    sl.z = limited_f(u0.z - um.z, up.z - u0.z, lim);
    sl.w = limited_f(u0.w - um.w, up.w - u0.w, lim);
    float4 Sm = make_float4(u0.x - 0.5f * sl.x, u0.y - 0.5f * sl.y, u0.z - 0.5f * sl.z, u0.w - 0.5f * sl.w);
    float4 Sp = make_float4(u0.x + 0.5f * sl.x, u0.y + 0.5f * sl.y, u0.z + 0.5f * sl.z, u0.w + 0.5f * sl.w);
    const int fb = unrealizable_f(Sm) | unrealizable_f(Sp);
    Sm = fb ? u0 : Sm;
    Sp = fb ? u0 : Sp;
    float2 F[4], l1, l3;
    closure_pair<D>(make_float2(Sm.x, Sp.x), make_float2(Sm.y, Sp.y), make_float2(Sm.z, Sp.z),
                    make_float2(Sm.w, Sp.w), chat, p1, fixed, F, l1, l3);
    rec[0] = Sm;
    rec[1] = make_float4(F[0].x, F[1].x, F[2].x, F[3].x);
    rec[2] = Sp;
    rec[3] = make_float4(F[0].y, F[1].y, F[2].y, F[3].y);
    rec[4] = make_float4(l1.x, l3.x, l1.y, l3.y);
    return fb;
}

// Compact face-state record of one cell in direction D: minus state, plus state, their closure
// coefficients (a-, b-, a+, b+) and (l1-, l3-, l1+, l3+).  Returns 1 if the slope was zeroed.
template <int D>
__device__ __forceinline__ int face_record_ab(float4 um, float4 u0, float4 up, float chat, int lim, int p1, int fixed,
                                              float4 rec[4])
{
    float4 sl;
    sl.x = limited_f(u0.x - um.x, up.x - u0.x, lim);
    sl.y = limited_f(u0.y - um.y, up.y - u0.y, lim);
    sl.z = limited_f(u0.z - um.z, up.z - u0.z, lim);
    sl.w = limited_f(u0.w - um.w, up.w - u0.w, lim);
    float4 Sm = make_float4(u0.x - 0.5f * sl.x, u0.y - 0.5f * sl.y, u0.z - 0.5f * sl.z, u0.w - 0.5f * sl.w);
    float4 Sp = make_float4(u0.x + 0.5f * sl.x, u0.y + 0.5f * sl.y, u0.z + 0.5f * sl.z, u0.w + 0.5f * sl.w);
    const int fb = unrealizable_f(Sm) | unrealizable_f(Sp);
    Sm = fb ? u0 : Sm;
    Sp = fb ? u0 : Sp;
    float2 a, b, l1, l3;
    closure_ab_pair<D>(make_float2(Sm.x, Sp.x), make_float2(Sm.y, Sp.y), make_float2(Sm.z, Sp.z),
                       make_float2(Sm.w, Sp.w), chat, p1, fixed, a, b, l1, l3);
    rec[0] = Sm;
    rec[1] = Sp;
    rec[2] = make_float4(a.x, b.x, a.y, b.y);
    rec[3] = make_float4(l1.x, l3.x, l1.y, l3.y);
    return fb;
}

// HLL flux (Eq. hyperbolic:hllflux2) with the four components as two FP32 pairs; FL, FR are the
// states' fluxes per unit chat and the weights carry the factor chat.
__device__ __forceinline__ float4 hll_pair(float4 UL, float4 UR, float4 FL, float4 FR, float l1L, float l3L,
                                           float l1R, float l3R, float chat)
{
    const float SRp = fmaxf(fmaxf(l3L, l3R), 0.f), SLm = fminf(fminf(l1L, l1R), 0.f);
    const float den = SRp - SLm;
    if (den > 0.f) {
        const float2 a = p_s(SRp * chat), b = p_s(-SLm * chat), c = p_s(SRp * SLm), iv = p_s(rcp(den));
        const float2 lo =
            p_mul(p_fma(c, p_sub(p_lo(UR), p_lo(UL)), p_fma(b, p_lo(FR), p_mul(a, p_lo(FL)))), iv);
        const float2 hi =
            p_mul(p_fma(c, p_sub(p_hi(UR), p_hi(UL)), p_fma(b, p_hi(FR), p_mul(a, p_hi(FL)))), iv);
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    const float2 lo = p_mul(p_add(p_lo(FL), p_lo(FR)), p_s(0.5f * chat));
    const float2 hi = p_mul(p_add(p_hi(FL), p_hi(FR)), p_s(0.5f * chat));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// The same HLL flux with scalar FP32 operations (same operation order and fused multiply-adds as
// hll_pair, so the same bits): cheaper where the operands are not already register pairs.
__device__ __forceinline__ float4 hll4(float4 UL, float4 UR, float4 FL, float4 FR, float l1L, float l3L, float l1R,
                                       float l3R, float chat)
{
    const float SRp = fmaxf(fmaxf(l3L, l3R), 0.f), SLm = fminf(fminf(l1L, l1R), 0.f);
    const float den = SRp - SLm;
    if (den > 0.f) {
        const float a = xmul(SRp, chat), b = xmul(-SLm, chat), c = xmul(SRp, SLm), iv = rcp(den);
        return make_float4(xmul(xfma(c, xadd(UR.x, -UL.x), xfma(b, FR.x, xmul(a, FL.x))), iv),
                           xmul(xfma(c, xadd(UR.y, -UL.y), xfma(b, FR.y, xmul(a, FL.y))), iv),
                           xmul(xfma(c, xadd(UR.z, -UL.z), xfma(b, FR.z, xmul(a, FL.z))), iv),
                           xmul(xfma(c, xadd(UR.w, -UL.w), xfma(b, FR.w, xmul(a, FL.w))), iv));
    }
    const float h = 0.5f * chat;
    return make_float4((FL.x + FR.x) * h, (FL.y + FR.y) * h, (FL.z + FR.z) * h, (FL.w + FR.w) * h);
}

__device__ __forceinline__ float4 f4(const float U[4]) { return make_float4(U[0], U[1], U[2], U[3]); }

}  // namespace rhd
