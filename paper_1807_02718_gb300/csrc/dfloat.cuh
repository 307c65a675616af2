// Double-float ("df") arithmetic on the FP32 pipe, and the Hankel-form
// Bessel functions of orders 0 and 1 at x >= 8 evaluated with it.
//
// A df value is hi + lo with |lo| <= ulp(hi) / 2, ~2^-48 relative.  Products
// use the exact FMA residual (two-product), sums Knuth's two-sum; each
// operation is accurate to a few 2^-46 relative.  FP32 issues 64 times as
// many operations per clock as FP64 on this GPU, so a df operation (5-15
// FP32 instructions) costs a fraction of one FP64 instruction's issue slot.
//
// Hankel form (x >= 8, A&S 9.2.5-9.2.6, 9.2.9-9.2.10):
//   H_nu(x) = sqrt(2/(pi x)) (P_nu + i Q_nu) e^{i (x - (2 nu + 1) pi/4)},
//   P0 = 1 - 9u/8192 + u^2 G0,   Q0 = (8/x)(-1/64 + 75u/524288 + u^2 G1),
//   P1 = 1 + 15u/8192 + u^2 G2,  Q1 = (8/x)(3/64 - 105u/524288 + u^2 G3),
// u = (8/x)^2.  The leading coefficients are exact binary32 numbers; each
// remainder u^2 G_k (|.| <= 1e-4) is a polynomial whose constant term is a
// df pair and whose other terms (|.| <= 1e-6) are binary32 (bessel_cheb.h),
// so the df results carry ~1e-14 absolute error.
#pragma once

#include "bessel_cheb.h"

namespace fh {

struct dfv {
    float hi, lo;
};

__device__ __forceinline__ dfv df_make(float hi, float lo) { return {hi, lo}; }

__device__ __forceinline__ dfv df_from(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_to(dfv a) { return (double)a.hi + (double)a.lo; }

// A complex FP64 value as double-float pairs (re hi, re lo, im hi, im lo).
__device__ __forceinline__ float4 df_pack(double re, double im) {
    const dfv r = df_from(re), i = df_from(im);
    return make_float4(r.hi, r.lo, i.hi, i.lo);
}

__device__ __forceinline__ dfv df_quick(float s, float e) {   // |s| >= |e|
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ dfv df_add(dfv a, dfv b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    return df_quick(s, e);
}

__device__ __forceinline__ dfv df_add_f(dfv a, float b) {
    const float s = a.hi + b;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b - bb)) + a.lo;
    return df_quick(s, e);
}

__device__ __forceinline__ dfv df_neg(dfv a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfv df_mul(dfv a, dfv b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}

__device__ __forceinline__ dfv df_mul_f(dfv a, float b) {
    const float p = a.hi * b;
    const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
    return df_quick(p, e);
}

// a * b + c
__device__ __forceinline__ dfv df_fma(dfv a, dfv b, dfv c) { return df_add(df_mul(a, b), c); }

// a * b + c with one renormalisation: the exact product of the hi parts (FMA
// residual) and the cross terms, the sum of the two leading parts by two-sum,
// every small part added into one error term.
__device__ __forceinline__ dfv df_mad(dfv a, dfv b, dfv c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = p + c.hi;
    const float bb = s - p;
    return df_quick(s, ((p - (s - bb)) + (c.hi - bb)) + (e + c.lo));
}

// a * b + c * d with one renormalisation (two exact products, one two-sum).
__device__ __forceinline__ dfv df_dot2(dfv a, dfv b, dfv c, dfv d) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float q = c.hi * d.hi;
    float f = fmaf(c.hi, d.hi, -q);
    f = fmaf(c.hi, d.lo, f);
    f = fmaf(c.lo, d.hi, f);
    const float s = p + q;
    const float bb = s - p;
    return df_quick(s, ((p - (s - bb)) + (q - bb)) + (e + f));
}

// acc += a * b (or -= when neg): exact FP32 product hi*hi with its FMA
// residual and the cross terms; the running sum (sh, sl) is a two-sum pair
// that the caller renormalises (df_quick) every few terms.
__device__ __forceinline__ void df_acc(float &sh, float &sl, dfv a, dfv b, bool neg) {
    float p = a.hi * b.hi;
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    if (neg) { p = -p; pe = -pe; }
    const float t = sh + p;
    const float z = t - sh;
    sl += ((sh - (t - z)) + (p - z)) + pe;
    sh = t;
}

__device__ __forceinline__ dfv df_sqrt(dfv a) {
    const float s = sqrtf(a.hi);
    const float e = (fmaf(-s, s, a.hi) + a.lo) * (0.5f / s);
    return df_quick(s, e);
}

__device__ __forceinline__ dfv df_rcp(dfv a) {
    const float r = 1.0f / a.hi;
    const float t = fmaf(-a.hi, r, 1.0f) - a.lo * r;   // 1 - a r
    return df_quick(r, r * t);
}

// sin and cos of a df argument |y| <= pi/4 (Taylor series to degree 17 / 16,
// truncation < 2^-53).  Horner in y^2; the coefficients of y^12 and beyond
// (<= 1/12! = 2.1e-9, times y^12 <= 0.055) need only binary32, the rest are
// df multiply-adds.
__device__ __forceinline__ void df_sincos_small(dfv y, dfv &sn, dfv &cs) {
    const dfv y2 = df_mul(y, y);
    float ts = kSinDF[16], tc = kCosDF[16];
#pragma unroll
    for (int k = 7; k >= 6; --k) {
        ts = fmaf(ts, y2.hi, kSinDF[2 * k]);
        tc = fmaf(tc, y2.hi, kCosDF[2 * k]);
    }
    dfv ps = df_make(ts, 0.f), pc = df_make(tc, 0.f);
#pragma unroll
    for (int k = 5; k >= 0; --k) {
        ps = df_mad(ps, y2, df_make(kSinDF[2 * k], kSinDF[2 * k + 1]));
        pc = df_mad(pc, y2, df_make(kCosDF[2 * k], kCosDF[2 * k + 1]));
    }
    sn = df_mul(ps, y);
    cs = pc;
}

// e^{i y} for a double-float 0 <= y < 3.1 without FP64: the Taylor series at
// y / 2^h with y / 2^h <= 0.78 (h = 0, 1 or 2; halving is exact), then h
// double-angle steps cos 2a = 1 - 2 sin^2 a, sin 2a = 2 sin a cos a.  The
// frequency step e^{i dkappa r} of the wide-band fields reaches y ~ 1.6.
__device__ __forceinline__ void df_sincos_mid(dfv y, dfv &sn, dfv &cs) {
    const int h = (y.hi >= 0.78f) + (y.hi >= 1.56f);
    const float sc = h == 0 ? 1.f : h == 1 ? 0.5f : 0.25f;
    df_sincos_small(df_make(y.hi * sc, y.lo * sc), sn, cs);
    for (int k = 0; k < h; ++k) {
        const dfv s2 = df_mul(sn, sn);
        const dfv c2 = df_add_f(df_mul_f(s2, -2.f), 1.f);
        sn = df_mul_f(df_mul(sn, cs), 2.f);
        cs = c2;
    }
}

// e^{i x} for an FP64 argument 0 <= x < 2^20: quadrant reduction in FP64 (two
// FMAs with pi/2 split into two doubles), the rest in df.
__device__ __forceinline__ void df_expi(double x, dfv &c, dfv &s) {
    constexpr double kPio2Hi = 1.5707963267948966192;
    constexpr double kPio2Lo = 6.123233995736766036e-17;
    const double k = rint(x * 0.63661977236758134308);
    double y = fma(-k, kPio2Hi, x);
    y = fma(-k, kPio2Lo, y);
    dfv sn, cs;
    df_sincos_small(df_from(y), sn, cs);
    const int q = ((int)k) & 3;
    if (q == 0) { c = cs; s = sn; }
    else if (q == 1) { c = df_neg(sn); s = cs; }
    else if (q == 2) { c = df_neg(cs); s = df_neg(sn); }
    else { c = sn; s = df_neg(cs); }
}

// e^{i (x - pi/4)} for x = kappa r, kappa = k1 + k2 + k3 (three binary32
// pieces, exact for an FP64 kappa), r double-float, 0 <= k1 r.hi < kExpiKrMax.
// x - pi/4 - q pi/2 is formed without rounding x first (Cody-Waite with pi/2 =
// C1 + C2 + C3): k1 r.hi - q C1 exactly (FMA residual; q C1 exact and the
// difference exact by Sterbenz's lemma), the O(2^-24 x) terms k1 r.lo,
// k2 r.hi, q C2 exactly as double-float pairs, the O(2^-48 x) terms in
// binary32.  Then the Taylor series on |y| <= pi/4 and the quadrant q.
constexpr float kExpiKrMax = 6000.f;   // q < 2^12, so that q C1 is exact

__device__ __forceinline__ void df_expi_kr(float k1, float k2, float k3, dfv r, dfv &c, dfv &s) {
    const float p1 = k1 * r.hi;
    const float e1 = fmaf(k1, r.hi, -p1);
    const float qf = rintf((p1 - kPio4DF[0]) * 0.636619772f);
    const float y0 = fmaf(-qf, kPio2CW[0], p1);
    const float a = k1 * r.lo, ae = fmaf(k1, r.lo, -a);
    const float b = k2 * r.hi, be = fmaf(k2, r.hi, -b);
    const float m = qf * kPio2CW[1], me = fmaf(qf, kPio2CW[1], -m);
    dfv t = df_add(df_make(a, ae), df_make(b, be));
    t = df_add(t, df_make(-m, -me));
    t = df_add(t, df_make(-kPio4DF[0], -kPio4DF[1]));
    t = df_add_f(t, e1);
    const float tail = fmaf(k2, r.lo, fmaf(k3, r.hi, -qf * kPio2CW[2]));
    const dfv y = df_add_f(df_add(df_make(y0, 0.f), t), tail);
    dfv sn, cs;
    df_sincos_small(y, sn, cs);
    const int q = ((int)qf) & 3;
    if (q == 0) { c = cs; s = sn; }
    else if (q == 1) { c = df_neg(sn); s = cs; }
    else if (q == 2) { c = df_neg(cs); s = df_neg(sn); }
    else { c = sn; s = df_neg(cs); }
}

// Remainder polynomials staged in shared memory (threads of a warp may fall
// into different x intervals).
struct __align__(16) GShared {
    float c[kPQ_NI * 4 * kG_TERMS];   // read as float4 pairs (kG_TERMS = 8)
    float2 c0[kPQ_NI * 4];          // constant terms as (hi, lo)
    float uc[kPQ_NI], iuh[kPQ_NI];
};
static_assert(kG_TERMS == 8, "g_poly reads each remainder polynomial as two float4");

__device__ __forceinline__ void g_stage(GShared &tb) {
    for (int i = threadIdx.x; i < kPQ_NI * 4 * kG_TERMS; i += blockDim.x) tb.c[i] = kG[i];
    for (int i = threadIdx.x; i < kPQ_NI * 4; i += blockDim.x) tb.c0[i] = make_float2(kG0DF[2 * i], kG0DF[2 * i + 1]);
    for (int i = threadIdx.x; i < kPQ_NI; i += blockDim.x) {
        tb.uc[i] = kPQ_UCf[i];
        tb.iuh[i] = kPQ_IUHf[i];
    }
}

// The binary32 part of a remainder polynomial: G - c0 = t (c1 + c2 t + ...
// + c5 t^4), its coefficients (c0 unused) as two 16-byte loads of the eight
// table entries; c6 and c7 are zero on every interval (gen_bessel_cheb.py
// checks that at most six terms are needed).
__device__ __forceinline__ float g_poly(const float *c, float t) {
    const float4 lo = reinterpret_cast<const float4 *>(c)[0], hi = reinterpret_cast<const float4 *>(c)[1];
    float a = fmaf(hi.y, t, hi.x);
    a = fmaf(a, t, lo.w);
    a = fmaf(a, t, lo.z);
    a = fmaf(a, t, lo.y);
    return a * t;
}

// u k + u^2 G with G = c0 + at (c0 a df pair, at binary32, k an exact
// binary32 coefficient): the Hankel terms of P or Q after the constant one,
// summed with one renormalisation.
__device__ __forceinline__ dfv pq_rem(dfv u, float k, dfv u2, float2 c0, float at) {
    const dfv G = df_add_f(df_make(c0.x, c0.y), at);
    const float p = u.hi * k;
    const float e = fmaf(u.lo, k, fmaf(u.hi, k, -p));
    const float q = u2.hi * G.hi;
    float f = fmaf(u2.hi, G.hi, -q);
    f = fmaf(u2.hi, G.lo, f);
    f = fmaf(u2.lo, G.hi, f);
    const float sm = p + q;
    const float bb = sm - p;
    return df_quick(sm, ((p - (sm - bb)) + (q - bb)) + (e + f));
}

// Hankel-form J0, Y0 (and J1, Y1 when want1) at x = kappa r >= 8, scaled by
// the amplitude that the caller carries in the phase:
//   r8 = 8 / x (df), (c, s) = a e^{i (x - pi/4)} for any real a;
//   J0 = a' (P0 c - Q0 s), Y0 = a' (P0 s + Q0 c), and with e^{i (x - 3pi/4)}
//   = (s, -c): J1 = a' (P1 s + Q1 c), Y1 = a' (Q1 s - P1 c), where
//   a' = sqrt(2 / (pi x)) / a (a = sqrt(2 / (pi x)) gives J and Y themselves).
// P = 1 + dP: each value is the phase component plus one two-product dot
// product of the small corrections (|dP| <= 1.2e-3, |Q| <= 0.05).
template <bool want1>
__device__ __forceinline__ void df_hankel(const GShared &tb, float xf, dfv r8, dfv c, dfv s, dfv &J0,
                                          dfv &Y0, dfv &J1, dfv &Y1) {
    const dfv u = df_mul(r8, r8);
    const int k = (xf >= 10.f) + (xf >= 13.f) + (xf >= 18.f) + (xf >= 28.f) + (xf >= 60.f);
    const float t = (u.hi - tb.uc[k]) * tb.iuh[k];
    const dfv u2 = df_mul(u, u);
    const float *g = tb.c + k * 4 * kG_TERMS;
    const float4 g01 = reinterpret_cast<const float4 *>(tb.c0)[2 * k];
    // dP0 = P0 - 1, Q0 = r8 (-1/64 + 75 u / 524288 + u^2 G1)
    const dfv dP0 = pq_rem(u, -9.0f / 8192.0f, u2, make_float2(g01.x, g01.y), g_poly(g, t));
    const dfv Q0 = df_mul(r8, df_add_f(pq_rem(u, 75.0f / 524288.0f, u2, make_float2(g01.z, g01.w),
                                              g_poly(g + kG_TERMS, t)),
                                       -1.0f / 64.0f));
    J0 = df_add(c, df_dot2(dP0, c, df_neg(Q0), s));
    Y0 = df_add(s, df_dot2(dP0, s, Q0, c));
    if (want1) {
        const float4 g23 = reinterpret_cast<const float4 *>(tb.c0)[2 * k + 1];
        const dfv dP1 = pq_rem(u, 15.0f / 8192.0f, u2, make_float2(g23.x, g23.y), g_poly(g + 2 * kG_TERMS, t));
        const dfv Q1 = df_mul(r8, df_add_f(pq_rem(u, -105.0f / 524288.0f, u2, make_float2(g23.z, g23.w),
                                                  g_poly(g + 3 * kG_TERMS, t)),
                                           3.0f / 64.0f));
        J1 = df_add(s, df_dot2(dP1, s, Q1, c));
        Y1 = df_add(df_neg(c), df_dot2(Q1, s, df_neg(dP1), c));
    }
}

// ---- small arguments (x < 8) ----
// With t = x^2/32 - 1 (the A&S 9.1.10-9.1.11 ascending series with the
// logarithmic parts taken out, as in the FP64 routine):
//   J0 = A0(t),  Y0 = (2/pi) ln(x/2) J0 + A1(t),
//   J1 = x A2(t), Y1 = (2/pi) ln(x/2) J1 - 2/(pi x) + x A3(t),
// A_k Chebyshev series in t (bessel_cheb.h).  Clenshaw's recurrence runs in
// binary32 over the coefficients k >= kChebHead (all below 2^-24 of the
// largest, |c_k| <= 2e-10) and in double-float over the rest.
constexpr int kChebHead = 12;

template <int N>
__device__ __forceinline__ dfv df_clenshaw(const float *c, dfv t) {
    const float t2f = 2.f * t.hi;
    float f1 = 0.f, f2 = 0.f;
#pragma unroll
    for (int k = N - 1; k >= kChebHead; --k) {
        const float f0 = fmaf(t2f, f1, c[2 * k] - f2);
        f2 = f1;
        f1 = f0;
    }
    dfv b1 = df_make(f1, 0.f), b2 = df_make(f2, 0.f);
    const dfv t2 = df_make(2.f * t.hi, 2.f * t.lo);
#pragma unroll
    for (int k = kChebHead - 1; k >= 1; --k) {
        const dfv b0 = df_add(df_mul(t2, b1), df_add(df_make(c[2 * k], c[2 * k + 1]), df_neg(b2)));
        b2 = b1;
        b1 = b0;
    }
    return df_add(df_mul(t, b1), df_add(df_make(c[0], c[1]), df_neg(b2)));
}

// ln a for a double-float a > 0 (normal): a = m 2^e with m in [1/sqrt2, sqrt2),
// ln m = 2 s sum_k s^2k / (2k+1), s = (m - 1)/(m + 1), |s| <= 0.172; the
// series to k = 10 (truncation < 1e-17), terms k >= 5 (< 3e-9) in binary32.
__device__ __forceinline__ dfv df_log(dfv a) {
    int e;
    float m = frexpf(a.hi, &e);           // a.hi = m 2^e, m in [1/2, 1)
    if (m < 0.70710678f) {
        m *= 2.f;
        --e;
    }
    const dfv mm = df_make(m, ldexpf(a.lo, -e));   // exact power-of-two scaling
    const dfv s = df_mul(df_add_f(mm, -1.f), df_rcp(df_add_f(mm, 1.f)));
    const dfv s2 = df_mul(s, s);
    float pf = kAtanhDF[20];
#pragma unroll
    for (int k = 9; k >= 5; --k) pf = fmaf(pf, s2.hi, kAtanhDF[2 * k]);
    dfv p = df_make(pf, 0.f);
#pragma unroll
    for (int k = 4; k >= 0; --k) p = df_add(df_mul(p, s2), df_make(kAtanhDF[2 * k], kAtanhDF[2 * k + 1]));
    const dfv ln2 = df_make(kLogConstDF[0], kLogConstDF[1]);
    return df_add(df_mul_f(ln2, (float)e), df_mul(df_make(2.f * s.hi, 2.f * s.lo), p));
}

// J0, Y0 (and J1, Y1 when want1) at 0 < x < 8 from x and lnh = ln(x/2).
template <bool want1>
__device__ __forceinline__ void df_bessel_small(dfv x, dfv lnh, dfv &J0, dfv &Y0, dfv &J1, dfv &Y1) {
    const dfv x2 = df_mul(x, x);
    const dfv t = df_add_f(df_make(x2.hi * 0.03125f, x2.lo * 0.03125f), -1.f);
    const dfv L = df_mul(df_make(kLogConstDF[2], kLogConstDF[3]), lnh);   // (2/pi) ln(x/2)
    J0 = df_clenshaw<kA0_N>(kA0DF, t);
    Y0 = df_add(df_mul(L, J0), df_clenshaw<kA1_N>(kA1DF, t));
    if (want1) {
        J1 = df_mul(x, df_clenshaw<kA2_N>(kA2DF, t));
        const dfv tpx = df_mul(df_make(kLogConstDF[2], kLogConstDF[3]), df_rcp(x));   // 2/(pi x)
        Y1 = df_add(df_add(df_mul(L, J1), df_neg(tpx)), df_mul(x, df_clenshaw<kA3_N>(kA3DF, t)));
    }
}

// Out-of-line entry points for the rarely taken branches of the large kernels
// (their code stays out of the instruction stream of the common path).
static __device__ __noinline__ void df_expi_cold(double x, dfv &c, dfv &s) { df_expi(x, c, s); }

static __device__ __noinline__ void df_bessel_small0_cold(dfv x, dfv lnh, dfv &J0, dfv &Y0) {
    dfv J1, Y1;
    df_bessel_small<false>(x, lnh, J0, Y0, J1, Y1);
}

}  // namespace fh
