// Steps a6-a7 (steps T0-T6): band-limited recentred synthesis of u(x, t).
//
// The paper expands F(omega) = B_k^slow(omega) V(x, omega) on [-W, W) in a
// trigonometric series from its values at M = 2(J-1) equispaced nodes (Sec.
// 4.1 eq. fourier_approx, P = 2W) and integrates it exactly against
// e^{-i omega (t - s_k)} (eq. approx), giving per window
//   u_k(x, t) = Re[(1/2pi) sum_m c_m 2W sinc(W (t - s_k)/pi - m)],
// summed over k (step T5, eq. uk_def).  Exchanging the (linear) sums yields
// the same numbers as a contraction over the non-negative frequencies p:
//   u(x, t) = sum_p Re[V(x, w_p) G_p(t)],
//   G_p(t)  = (mu_p / 2pi) sum_k B_k^slow(w_p) D_p(t - s_k),
//   D_p(tau) = (2W/M) sum_{m=-h}^{h-1} e^{-2 pi i m p / M} sinc(W tau/pi - m),
// with h = M/2, mu_0 = mu_{J-1} = 1 and mu_p = 2 otherwise (the nodes -w_p
// carry conj F since the signal is real).  The weights G are independent of
// the targets (the O(1)-in-T part); the contraction over p is a real GEMM
// u = [Vr | Vi] [Gr ; -Gi] with inner dimension 2J.
//
// D_p for windows far from t (|y| >= 1.25 h, y = W tau/pi) uses the Chebyshev
// expansion of 1/(y - m) in x = m/h on [-1, 1]: with a = y/h,
// s = sign(a) sqrt(a^2 - 1) and rho = 1/(a + s) (|rho| <= 1/2 for |a| >= 1.25),
//   1/(a - x) = (2/s) [1/2 + sum_{r>=1} rho^r T_r(x)]
// (the generating function of the Chebyshev polynomials), so that
//   D_p = (2W/M) (sin(pi y)/pi) (2/(h s)) sum_r rho^r nu_{p,r},
//   nu_{p,r} = sum_m (-1)^m T_r(m/h) e^{-2 pi i m p / M}  (r = 0 halved),
// truncated once |rho|^r < 2^-48 (|nu_{p,r}| <= M) and summed by Horner's
// rule in double-float arithmetic, except the terms past R1 with
// |rho|^R1 <= 2^-25 / R, which Horner's rule takes in FP32 first (their
// relative error ~R 2^-24 enters scaled by |rho|^R1, the size of the
// truncation error).  Its ratio |rho| is below the Taylor ratio h/|y| (0.5
// against 0.8 at |y| = 1.25 h), hence fewer terms.  Near windows interpolate a
// table of the direct sums or sum the M terms directly.
#include "fh_internal.h"

namespace fh {
namespace {

// nu_{p,r} as a contraction: pw[m + h][r] = T_r(m/h) (three-term recurrence
// T_{r+1} = 2x T_r - T_{r-1}, stable on [-1, 1]; T_0 halved; one thread per
// m), then one CTA per p stages (-1)^k (cos, sin)(2 pi k p / M) of a chunk of
// k in shared memory and thread r accumulates the cosine (even r) or sine
// (odd r) sum over k = 1 .. h-1, m and -m paired.
__global__ void far_powers_kernel(int M, double *__restrict__ pw) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M) return;
    const int h = M / 2;
    const double xv = (double)(q - h) / (double)h;
    double t0 = 1.0, t1 = xv;
    pw[(long long)q * kFarTerms] = 0.5;
    for (int r = 1; r < kFarTerms; ++r) {
        pw[(long long)q * kFarTerms + r] = t1;
        const double t2 = 2.0 * xv * t1 - t0;
        t0 = t1;
        t1 = t2;
    }
}

constexpr int kFarChunk = 128;

__global__ void __launch_bounds__(128) far_table_kernel(int J, int M, const double *__restrict__ pw,
                                                       double2 *__restrict__ nu, float4 *__restrict__ nu_f,
                                                       float4 *__restrict__ ph) {
    const int p = blockIdx.x;
    const int r = threadIdx.x;
    const int h = M / 2;
    __shared__ double2 phs[kFarChunk];
    if (p == 0)
        for (int q = r; q < M; q += blockDim.x) {
            double sn, cs;
            sincospi(-2.0 * (double)q / (double)M, &sn, &cs);
            const float ch = (float)cs, sh = (float)sn;   // double-float (cos, sin)
            ph[q] = make_float4(ch, (float)(cs - (double)ch), sh, (float)(sn - (double)sh));
        }
    // Pairing m with -m (T_r(-x) = (-1)^r T_r(x), e^{-i th m} + (-1)^r e^{i th m} =
    // 2 cos(th m) for even r, -2i sin(th m) for odd r; th = 2 pi p / M):
    //   nu_{p,r} = T_r(0) + (-1)^(h+p+r) T_r(1)
    //            + 2 sum_{k=1}^{h-1} (-1)^k T_r(k/h) {cos(th k) | -i sin(th k)},
    // the m = -h term using e^{i th h} = (-1)^p (T_0 halved throughout).
    const bool odd_r = r & 1;
    double acc = 0.0;
    for (int k0 = 1; k0 < h; k0 += kFarChunk) {
        __syncthreads();
        for (int e = r; e < kFarChunk; e += blockDim.x) {
            const int k = k0 + e;
            double2 v = make_double2(0.0, 0.0);
            if (k < h) {
                const int q = (int)(((long long)k * p) % M);
                double sn, cs;
                sincospi(2.0 * (double)q / (double)M, &sn, &cs);
                const double sg = (k & 1) ? -1.0 : 1.0;
                v = make_double2(sg * cs, sg * sn);
            }
            phs[e] = v;
        }
        __syncthreads();
        if (r < kFarTerms) {
            const int ke = min(kFarChunk, h - k0);
            const double *col = pw + (long long)(k0 + h) * kFarTerms + r;
            for (int e = 0; e < ke; ++e) {
                const double w = col[(long long)e * kFarTerms];
                acc = fma(w, odd_r ? phs[e].y : phs[e].x, acc);
            }
        }
    }
    double sr = 0.0, si = 0.0;
    if (r < kFarTerms) {
        const double t0 = pw[(long long)h * kFarTerms + r];      // T_r(0) (T_0 halved)
        const double t1 = r == 0 ? 0.5 : 1.0;                    // T_r(1)
        const double edge = ((h + p + r) & 1) ? -t1 : t1;        // the m = -h term
        sr = t0 + edge + (odd_r ? 0.0 : 2.0 * acc);
        si = odd_r ? -2.0 * acc : 0.0;
    }
    if (r < kFarTerms) {
        if (nu) nu[(long long)r * J + p] = make_double2(sr, si);
        const float rh = (float)sr, ih = (float)si;   // double-float copy for the far Horner
        nu_f[(long long)r * J + p] = make_float4(rh, (float)(sr - (double)rh), ih, (float)(si - (double)ih));
    }
}

// Double-float (FP32 pair) arithmetic for the near-window sums: FP32 runs at
// 64x the FP64 rate on this GPU.  A value is hi + lo with |lo| <= ulp(hi)/2;
// products use the exact FMA residual (Dekker / Ogita-Rump-Oishi two-product),
// sums the two-sum of Knuth, giving ~2^-44 relative accuracy per operation.
struct dfl { float hi, lo; };

__device__ __forceinline__ dfl df_split(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

// acc += a * b (a, b double-float; acc double-float)
__device__ __forceinline__ void df_mac(float &sh, float &sl, dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    const float t = sh + p;
    const float z = t - sh;
    const float err = (sh - (t - z)) + (p - z);
    sl += err + pe;
    sh = t;
}

// a * b in double-float, renormalised
__device__ __forceinline__ dfl df_mulq(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return {h, e - (h - p)};
}

// a + b and 1 / a in double-float, renormalised
__device__ __forceinline__ dfl df_addq(dfl a, dfl b) {
    const float sum = a.hi + b.hi;
    const float bb = sum - a.hi;
    const float e = ((a.hi - (sum - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    const float h = sum + e;
    return {h, e - (h - sum)};
}

__device__ __forceinline__ dfl df_rcpq(dfl a) {
    const float r = 1.0f / a.hi;
    const float t = fmaf(-a.hi, r, 1.0f) - a.lo * r;
    const float h = r + r * t;
    return {h, r * t - (h - r)};
}

// a * r + v in double-float (r, v double-float; a updated)
__device__ __forceinline__ void df_horner(float &ah, float &al, dfl r, float vh, float vl) {
    const float p = ah * r.hi;
    float e = fmaf(ah, r.hi, -p);
    e = fmaf(ah, r.lo, e);
    e = fmaf(al, r.hi, e);
    const float s = p + vh;
    const float bb = s - p;
    float err = (p - (s - bb)) + (vh - bb);
    err += e + vl;
    ah = s + err;
    al = err - (ah - s);
}

__device__ __forceinline__ dfl df_negq(dfl a) { return {-a.hi, -a.lo}; }

// sqrt(a) in double-float (a > 0): s = sqrt(a.hi) in binary32, corrected by
// (a - s^2) / (2 s) with s^2 exact through the FMA residual.
__device__ __forceinline__ dfl df_sqrtq(dfl a) {
    const float s = sqrtf(a.hi);
    const float r = (fmaf(-s, s, a.hi) + a.lo) / (2.f * s);
    const float h = s + r;
    return {h, r - (h - s)};
}

// e^x in double-float for -88 < x <= 0: x = k ln2 + r with |r| <= ln2 / 2,
// ln2 = L1 + L2 where L1 holds 16 significant bits (k L1 exact for |k| < 2^8);
// e^r by its Taylor series at 0, the terms n = 8 .. 13 (below 6e-9 for
// |r| <= 0.347) in binary32 and the rest in double-float; then e^x = 2^k e^r.
constexpr double kLn2 = 0.69314718055994530942;
constexpr float kLn2A = 0.693145751953125f;
constexpr float kLn2B = (float)(kLn2 - 0.693145751953125);
constexpr float kLn2C = (float)(kLn2 - 0.693145751953125 - (double)kLn2B);
// 1/n! for n = 3 .. 7 as double-float pairs (1/0!, 1/1!, 1/2! are exact)
#define FH_INV_FACT(n, v) \
    constexpr float kIF##n##h = (float)(v); \
    constexpr float kIF##n##l = (float)((v) - (double)(float)(v));
FH_INV_FACT(3, 1.0 / 6.0)
FH_INV_FACT(4, 1.0 / 24.0)
FH_INV_FACT(5, 1.0 / 120.0)
FH_INV_FACT(6, 1.0 / 720.0)
FH_INV_FACT(7, 1.0 / 5040.0)
#undef FH_INV_FACT

__device__ __forceinline__ dfl df_expq(dfl x) {
    const float k = rintf(x.hi * 1.4426950408889634f);
    // r = x - k ln2: x.hi - k L1 is exact (Sterbenz), k L2 exact as a pair
    const float kb = k * kLn2B, kbe = fmaf(k, kLn2B, -kb);
    dfl r = df_addq({x.hi - k * kLn2A, x.lo}, {-kb, -fmaf(k, kLn2C, kbe)});
    float tail = 1.f / 6227020800.f;   // 1/13!
    tail = fmaf(tail, r.hi, 1.f / 479001600.f);
    tail = fmaf(tail, r.hi, 1.f / 39916800.f);
    tail = fmaf(tail, r.hi, 1.f / 3628800.f);
    tail = fmaf(tail, r.hi, 1.f / 362880.f);
    tail = fmaf(tail, r.hi, 1.f / 40320.f);
    dfl q = {tail, 0.f};
    q = df_addq(df_mulq(q, r), {kIF7h, kIF7l});
    q = df_addq(df_mulq(q, r), {kIF6h, kIF6l});
    q = df_addq(df_mulq(q, r), {kIF5h, kIF5l});
    q = df_addq(df_mulq(q, r), {kIF4h, kIF4l});
    q = df_addq(df_mulq(q, r), {kIF3h, kIF3l});
    q = df_addq(df_mulq(q, r), {0.5f, 0.f});
    q = df_addq(df_mulq(q, r), {1.f, 0.f});
    q = df_addq(df_mulq(q, r), {1.f, 0.f});
    const int ki = (int)k;
    return {ldexpf(q.hi, ki), ldexpf(q.lo, ki)};
}

// Direct near-window sum, unscaled, for the thread's p (all threads of the CTA
// call it; it begins and ends with a barrier):
//   (rh + rl) + i (ih + il) = sum_{m=-h}^{h-1} e^{-2 pi i m p / M} sinc(y - m)
//   = S(y) + (-1)^p S(y+h) + sum_{j=1}^{h-1} (cos_j (S(y-j) + S(y+j))
//     + i sin_j (S(y-j) - S(y+j))),
// S(v) = sinc(v), (cos_j, sin_j) the phase e^{-2 pi i j p / M} (its conjugate
// pairs -j with j).  The sinc row uses sin(pi (y - j)) = (-1)^j sin(pi y);
// sypi = sin(pi y) / pi.  ph4: M phases (shared), sc4: h + 1 float4 (shared).
__device__ void stage_sinc_row(double y, dfl sypi, int h, float4 *sc4) {
    for (int jj = threadIdx.x; jj < h + 1; jj += blockDim.x) {
        // jj = 0: S(y) and S(y + h) into slot 0; jj >= 1: S(y - jj) +- S(y + jj)
        const int ja = jj == 0 ? 0 : jj, jb = jj == 0 ? h : jj;
        dfl va, vb;
        {
            const double d = y - (double)ja;
            if (d == 0.0) va = {1.f, 0.f};
            else {
                va = df_mulq(sypi, df_rcpq(df_split(d)));
                if (ja & 1) va = {-va.hi, -va.lo};
            }
        }
        {
            const double d = y + (double)jb;
            if (d == 0.0) vb = {1.f, 0.f};
            else {
                vb = df_mulq(sypi, df_rcpq(df_split(d)));
                if (jb & 1) vb = {-vb.hi, -vb.lo};
            }
        }
        if (jj == 0) {
            sc4[0] = make_float4(va.hi, va.lo, vb.hi, vb.lo);   // S(y), S(y + h)
        } else if (jj < h) {
            const dfl sp = df_addq(va, vb), sm = df_addq(va, {-vb.hi, -vb.lo});
            sc4[jj] = make_float4(sp.hi, sp.lo, sm.hi, sm.lo);
        }
    }
}

__device__ void near_sum(double y, dfl sypi, int h, int M, int p, int J, const float4 *ph4,
                         float4 *sc4, float &rh, float &rl, float &ih, float &il) {
    __syncthreads();
    stage_sinc_row(y, sypi, h, sc4);
    __syncthreads();
    rh = rl = ih = il = 0.f;
    if (p < J) {
        const float4 s0 = sc4[0];
        const dfl r0 = df_addq({s0.x, s0.y}, (p & 1) ? dfl{-s0.z, -s0.w} : dfl{s0.z, s0.w});
        rh = r0.hi;
        rl = r0.lo;
        int q = p;
        for (int jj = 1; jj < h; ++jj) {
            const float4 e = ph4[q];     // one 16-byte gather: cos and sin
            const float4 v = sc4[jj];    // one 16-byte broadcast: both sinc sums
            df_mac(rh, rl, {e.x, e.y}, {v.x, v.y});
            df_mac(ih, il, {e.z, e.w}, {v.z, v.w});
            q += p;
            if (q >= M) q -= M;
            if ((jj & 31) == 31) {   // renormalise the accumulators
                float tr = rh + rl; rl = rl - (tr - rh); rh = tr;
                float ti = ih + il; il = il - (ti - ih); ih = ti;
            }
        }
    }
}

// The sampled near sums.  Odd rows (direct sums, sin(pi g / 2) = +-1): one
// CTA per kTabRows consecutive positive odd rows and kTabThreads columns p,
// so that each phase gathered from shared memory serves kTabRows rows; the
// negative odd rows follow from the positive ones by a conjugation and a
// real end-term correction.  Even rows:
// D_p(n) = e^{-2 pi i n p / M} for -h <= n < h, else 0 (sinc(n - m) vanishes
// off m = n), written by the CTAs past the odd ones (grid-stride, blockIdx.y
// 0 only).
constexpr int kTabRows = 4;
constexpr int kTabThreads = 128;

__global__ void __launch_bounds__(kTabThreads) sinc_table_kernel(int J, int M, int G, int odd_ctas,
                                                                 const float4 *__restrict__ ph_g,
                                                                 float4 *__restrict__ tab) {
    const int h = M / 2;
    if ((int)blockIdx.x >= odd_ctas) {
        if (blockIdx.y != 0) return;
        const int e_first = (G & 1) ? 1 - G : -G;           // first even row
        const long long n_even = (long long)((G - e_first) / 2 + 1) * J;
        const int nb = gridDim.x - odd_ctas;
        for (long long idx = (long long)(blockIdx.x - odd_ctas) * blockDim.x + threadIdx.x; idx < n_even;
             idx += (long long)nb * blockDim.x) {
            const int pp = (int)(idx % J);
            const int g = e_first + 2 * (int)(idx / J);
            const int n = g / 2;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (n >= -h && n < h) v = ph_g[(long long)(n + M) * pp % M];
            tab[(long long)(g + G) * J + pp] = v;
        }
        return;
    }
    extern __shared__ __align__(16) float4 sm4[];
    float4 *ph4 = sm4;        // M phases
    float4 *sc4 = sm4 + M;    // kTabRows rows of h sinc sums
    const int g0 = 1 + 2 * kTabRows * (int)blockIdx.x;   // positive odd rows; -g from g
    const int p = blockIdx.y * kTabThreads + threadIdx.x;
    for (int q = threadIdx.x; q < M; q += blockDim.x) ph4[q] = ph_g[q];
#pragma unroll 1
    for (int r = 0; r < kTabRows; ++r) {
        const int g = g0 + 2 * r;
        if (g <= G) {
            const double sy = (g & 3) == 1 ? 1.0 : -1.0;   // sin(pi g / 2)
            stage_sinc_row(0.5 * (double)g, df_split(sy / kPi), h, sc4 + r * h);
        } else {
            for (int jj = threadIdx.x; jj < h; jj += blockDim.x) sc4[r * h + jj] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();
    if (p >= J) return;
    float ac[kTabRows][4];
#pragma unroll
    for (int r = 0; r < kTabRows; ++r) {
        const float4 s0 = sc4[r * h];
        const dfl r0 = df_addq({s0.x, s0.y}, (p & 1) ? dfl{-s0.z, -s0.w} : dfl{s0.z, s0.w});
        ac[r][0] = r0.hi;
        ac[r][1] = r0.lo;
        ac[r][2] = ac[r][3] = 0.f;
    }
    int q = p;
    for (int jj = 1; jj < h; ++jj) {
        const float4 e = ph4[q];
#pragma unroll
        for (int r = 0; r < kTabRows; ++r) {
            const float4 v = sc4[r * h + jj];
            df_mac(ac[r][0], ac[r][1], {e.x, e.y}, {v.x, v.y});
            df_mac(ac[r][2], ac[r][3], {e.z, e.w}, {v.z, v.w});
        }
        q += p;
        if (q >= M) q -= M;
        if ((jj & 31) == 31) {   // renormalise the accumulators
#pragma unroll
            for (int r = 0; r < kTabRows; ++r) {
                float t0 = ac[r][0] + ac[r][1]; ac[r][1] = ac[r][1] - (t0 - ac[r][0]); ac[r][0] = t0;
                float t1 = ac[r][2] + ac[r][3]; ac[r][3] = ac[r][3] - (t1 - ac[r][2]); ac[r][2] = t1;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kTabRows; ++r) {
        const int g = g0 + 2 * r;
        if (g > G) break;
        const float tr = ac[r][0] + ac[r][1], ti = ac[r][2] + ac[r][3];
        const dfl re = {tr, ac[r][1] - (tr - ac[r][0])}, im = {ti, ac[r][3] - (ti - ac[r][2])};
        tab[(long long)(g + G) * J + p] = make_float4(re.hi, re.lo, im.hi, im.lo);
        // D_p(-y) = conj(D_p(y)) + (-1)^p (sinc(y - h) - sinc(y + h)): m and -m
        // swap, c_{-m} = conj(c_m), and the end terms m = -h, h differ; at
        // y = g/2, sinc(y -+ h) = (-1)^h sin(pi y) / (pi (y -+ h))
        const double y = 0.5 * (double)g, sy = (g & 3) == 1 ? 1.0 : -1.0;
        const double corr = ((h & 1) ? -sy : sy) * 2.0 * (double)h / (kPi * (y * y - (double)h * (double)h));
        const dfl c = df_split((p & 1) ? -corr : corr);
        const dfl rn = df_addq(re, c);
        tab[(long long)(G - g) * J + p] = make_float4(rn.hi, rn.lo, -im.hi, -im.lo);
    }
}

// Bytes of the per-window arrays of weights_kernel (y, sin(pi y) or the far
// prefactor, three double-float and three int arrays), rounded to 16.
__host__ __device__ inline size_t weights_smem_head(int K) {
    return ((size_t)K * (2 * sizeof(double) + 3 * sizeof(float2) + 3 * sizeof(int)) + 15) & ~(size_t)15;
}

constexpr float kBetaUHi = (float)(kSincBeta / kSincU);
constexpr float kBetaULo = (float)(kSincBeta / kSincU - (double)kBetaUHi);
constexpr float k2PiHi = (float)(2.0 * kPi);
constexpr float k2PiLo = (float)(2.0 * kPi - (double)k2PiHi);
constexpr float kInv2PiHi = (float)(0.5 / kPi);
constexpr float kInv2PiLo = (float)(0.5 / kPi - (double)kInv2PiHi);

// One CTA per time t, thread p.  The per-window quantities that do not depend
// on p (y, near or far, sin(pi y), the far ratio h/y and its truncation R)
// are formed once per CTA.  Near windows: with the sampled table, 42 samples
// around y weighted by sinc(2u) E(u) (weights formed once per window, FP64,
// then split); without it, the direct M-term sums (near_sum).  Far windows:
// Horner in double-float over the double-float copy of nu.
__global__ void __launch_bounds__(256) weights_kernel(
    int J, int M, double W, int K, const double *__restrict__ s, const double2 *__restrict__ B,
    const float4 *__restrict__ Bf, const float4 *__restrict__ nu_f, const float4 *__restrict__ ph_g,
    const float4 *__restrict__ tab, int G, const double *__restrict__ T, int n_T,
    double *__restrict__ Gr, double *__restrict__ Gm, float2 *__restrict__ Gs, int pitch_T) {
    extern __shared__ __align__(16) double smd[];
    __shared__ float2 swt[kSincPts];                          // interpolation weights, double-float
    double *wy = smd;                                        // K: y
    double *wf = wy + K;                                     // K: sin(pi y) (near) or the far prefactor
    float2 *wrho = reinterpret_cast<float2 *>(wf + K);       // K: rho (far) or 2W/M (near), double-float
    float2 *wfd = wrho + K;                                  // K: far prefactor or sin(2 pi y), double-float
    float2 *wu = wfd + K;                                    // K: u_c = y - g_c / 2 (near, table)
    int *wR = reinterpret_cast<int *>(wu + K);               // K: far terms R | R1 << 16, 0 = near
    int *wg = wR + K;                                        // K: first sample row g0 (near, table)
    int *wgc = wg + K;                                       // K: nearest sample row g_c (near, table)
    float4 *ph4 = reinterpret_cast<float4 *>(reinterpret_cast<char *>(smd) + weights_smem_head(K));
    float4 *sc4 = ph4 + M;   // h: [0] = (S(y), S(y+h)), [j] = (S(y-j) + S(y+j), S(y-j) - S(y+j))
    const int t = blockIdx.x;
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    const int h = M / 2;
    const double tt = T[t];
    const double scale = 2.0 * W / (double)M;
    if (!tab)   // phases for the direct near sums
        for (int q = threadIdx.x; q < M; q += blockDim.x) ph4[q] = ph_g[q];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double y = W * (tt - s[k]) * (1.0 / kPi);
        wy[k] = y;
        if (fabs(y) < 1.25 * (double)h) {
            wR[k] = 0;
            const dfl sd = df_split(scale);
            wrho[k] = make_float2(sd.hi, sd.lo);
            if (tab) {   // samples g0 .. g0 + 41 around y, sin(2 pi y)
                // offsets from the nearest sample g_c: u_c = y - g_c / 2 is exact in FP64
                // (|u_c| <= 1/4), so that sin(2 pi u) / u stays accurate as u -> 0
                const int gc = (int)rint(2.0 * y);
                const dfl uc = df_split(y - 0.5 * (double)gc);
                double sn, cs;
                sincospi(y, &sn, &cs);
                const dfl s2 = df_split(2.0 * sn * cs);
                wg[k] = (int)floor(2.0 * y) - (kSincPts / 2 - 1);
                wgc[k] = gc;
                wu[k] = make_float2(uc.hi, uc.lo);
                wfd[k] = make_float2(s2.hi, s2.lo);
            } else {
                wf[k] = sinpi(y);
            }
        } else {
            const double sy = sinpi(y);
            const double a = y / (double)h;
            const double sq = copysign(sqrt((a - 1.0) * (a + 1.0)), a);
            const double rho = 1.0 / (a + sq);
            // truncation from binary32 logarithms (a term count, not a value)
            const float lr = -logf(fabsf((float)rho));
            const int R = max(1, min((int)ceilf(48.f * 0.693147181f / lr), kFarTerms));
            const int R1 = max(1, min((int)ceilf((25.f * 0.693147181f + logf((float)R)) / lr), R));
            wR[k] = R | (R1 << 16);
            const dfl rr = df_split(rho);
            wrho[k] = make_float2(rr.hi, rr.lo);
            wf[k] = scale * sy * 2.0 / (kPi * (double)h * sq);
            const dfl fd = df_split(wf[k]);
            wfd[k] = make_float2(fd.hi, fd.lo);
        }
    }
    __syncthreads();
    // G accumulates in double-float: q += B_k(w_p) D_p(t - s_k)
    float qrh = 0.f, qrl = 0.f, qih = 0.f, qil = 0.f;
    for (int k = 0; k < K; ++k) {
        const int R = wR[k] & 0xffff, R1 = wR[k] >> 16;
        dfl dr = {0.f, 0.f}, di = {0.f, 0.f};
        if (R == 0 && tab) {          // near window, sampled (the same branch in the whole CTA)
            const int g0 = wg[k];
            __syncthreads();          // previous window's weights read
            if (threadIdx.x < kSincPts) {
                // sinc(2u) E(u) at u = y - g/2 = u_c + (g_c - g)/2 in double-float:
                // sin(2 pi u) = (-1)^g sin(2 pi y), E(u) = exp((beta/U) sqrt(U^2 - u^2) - beta)
                const int i = (int)threadIdx.x;
                const float2 uc2 = wu[k];
                const dfl u = df_addq({uc2.x, uc2.y}, {0.5f * (float)(wgc[k] - g0 - i), 0.f});
                dfl w = {1.f, 0.f};
                if (u.hi != 0.f || u.lo != 0.f) {
                    const dfl w2 = df_addq({(float)(kSincU * kSincU), 0.f}, df_negq(df_mulq(u, u)));
                    w = {0.f, 0.f};
                    if (w2.hi > 0.f) {
                        const dfl arg = df_addq(df_mulq(df_sqrtq(w2), {kBetaUHi, kBetaULo}),
                                                {(float)-kSincBeta, 0.f});
                        const float2 s22 = wfd[k];
                        const dfl s2 = ((g0 + i) & 1) ? dfl{-s22.x, -s22.y} : dfl{s22.x, s22.y};
                        w = df_mulq(df_mulq(s2, df_expq(arg)), df_rcpq(df_mulq(u, {k2PiHi, k2PiLo})));
                    }
                }
                swt[i] = make_float2(w.hi, w.lo);
            }
            __syncthreads();
            if (p < J) {
                const float4 *col = tab + (long long)(g0 + G) * J + p;
                float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll 6
                for (int i = 0; i < kSincPts; ++i) {
                    const float4 v = col[(long long)i * J];
                    const float2 w = swt[i];
                    df_mac(rh, rl, {w.x, w.y}, {v.x, v.y});
                    df_mac(ih, il, {w.x, w.y}, {v.z, v.w});
                }
                const float2 sd = wrho[k];   // 2W/M
                dr = df_mulq({rh, rl}, {sd.x, sd.y});
                di = df_mulq({ih, il}, {sd.x, sd.y});
            }
        } else if (R == 0) {          // near window, direct sums
            float rh, rl, ih, il;
            near_sum(wy[k], df_split(wf[k] * (1.0 / kPi)), h, M, p, J, ph4, sc4, rh, rl, ih, il);
            if (p < J) {
                const float2 sd = wrho[k];   // 2W/M
                dr = df_mulq({rh, rl}, {sd.x, sd.y});
                di = df_mulq({ih, il}, {sd.x, sd.y});
            }
        } else if (p < J) {
            const float2 r2 = wrho[k];
            const dfl rho = {r2.x, r2.y};
            float ah = 0.f, bh = 0.f;
            for (int r = R - 1; r >= R1; --r) {     // FP32 tail
                const float4 v = nu_f[(long long)r * J + p];
                ah = fmaf(ah, rho.hi, v.x);
                bh = fmaf(bh, rho.hi, v.z);
            }
            float al = 0.f, bl = 0.f;
            for (int r = R1 - 1; r >= 0; --r) {
                const float4 v = nu_f[(long long)r * J + p];
                df_horner(ah, al, rho, v.x, v.y);
                df_horner(bh, bl, rho, v.z, v.w);
            }
            const float2 f2 = wfd[k];
            const dfl f = {f2.x, f2.y};
            dr = df_mulq({ah, al}, f);
            di = df_mulq({bh, bl}, f);
        }
        if (p < J) {
            dfl br, bi;
            if (Bf) {
                const float4 b4 = Bf[(long long)k * J + p];
                br = {b4.x, b4.y};
                bi = {b4.z, b4.w};
            } else {
                const double2 b = B[(long long)k * J + p];
                br = df_split(b.x);
                bi = df_split(b.y);
            }
            // q += b * d (complex)
            df_mac(qrh, qrl, br, dr);
            df_mac(qrh, qrl, {-bi.hi, -bi.lo}, di);
            df_mac(qih, qil, br, di);
            df_mac(qih, qil, bi, dr);
        }
    }
    if (p < J) {   // G = (mu_p / 2 pi) q, mu_p / 2 pi = 1/(2 pi) or 1/pi, in double-float
        const bool edge = p == 0 || p == J - 1;
        const dfl c = edge ? dfl{kInv2PiHi, kInv2PiLo} : dfl{2.f * kInv2PiHi, 2.f * kInv2PiLo};
        const dfl a = df_mulq({qrh, qrl}, c), b = df_negq(df_mulq({qih, qil}, c));
        if (Gs) {
            Gs[(long long)p * pitch_T + t] = make_float2(a.hi, a.lo);
            Gs[(long long)(J + p) * pitch_T + t] = make_float2(b.hi, b.lo);
        } else {
            Gr[(long long)p * n_T + t] = (double)a.hi + (double)a.lo;
            Gm[(long long)p * n_T + t] = (double)b.hi + (double)b.lo;
        }
    }
}

// Split a complex FP64 table into double-float pairs (re hi, re lo, im hi, im lo).
__global__ void split_df_kernel(const double2 *__restrict__ B, float4 *__restrict__ Bf, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 b = B[i];
    const dfl r = df_split(b.x), m = df_split(b.y);
    Bf[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
}

constexpr int BM = 64, BN = 64, BK = 16;

// u[x][t] = sum_{kk < 2J} A[x][kk] Bm[kk][t], A = [Vr | Vi], Bm = [Gr ; Gm].
__global__ void __launch_bounds__(256) contract_kernel(int J, int n_x, int n_T,
                                                       const double2 *__restrict__ V,
                                                       const double *__restrict__ Gr,
                                                       const double *__restrict__ Gm,
                                                       double *__restrict__ u) {
    __shared__ double As[BK][BM];
    __shared__ double Bs[BK][BN + 2];
    const int x0 = blockIdx.y * BM, t0 = blockIdx.x * BN;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    const int K2 = 2 * J;
    for (int k0 = 0; k0 < K2; k0 += BK) {
        for (int e = tid; e < BK * BM; e += 256) {
            const int kk = e / BM, xx = e % BM;
            const int k = k0 + kk, x = x0 + xx;
            double v = 0.0;
            if (k < K2 && x < n_x) {
                const double2 vv = V[(long long)(k < J ? k : k - J) * n_x + x];
                v = (k < J) ? vv.x : vv.y;
            }
            As[kk][xx] = v;
        }
        for (int e = tid; e < BK * BN; e += 256) {
            const int kk = e / BN, tt = e % BN;
            const int k = k0 + kk, t = t0 + tt;
            double v = 0.0;
            if (k < K2 && t < n_T) v = (k < J) ? Gr[(long long)k * n_T + t] : Gm[(long long)(k - J) * n_T + t];
            Bs[kk][tt] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int x = x0 + ty * 4 + i;
        if (x >= n_x) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = t0 + tx * 4 + j;
            if (t < n_T) u[(long long)x * n_T + t] = acc[i][j];
        }
    }
}

// V[j][x] (complex FP64) as double-float rows of the contraction's left
// operand: row j holds the real parts, row J + j the imaginary parts (row
// pitch px, a multiple of 4).
__global__ void split_v_kernel(int J, int n_x, int px, const double2 *__restrict__ V,
                               float2 *__restrict__ Vs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (x >= px) return;
    float2 r = make_float2(0.f, 0.f), i = r;
    if (x < n_x) {
        const double2 v = V[(long long)j * n_x + x];
        const dfl a = df_split(v.x), b = df_split(v.y);
        r = make_float2(a.hi, a.lo);
        i = make_float2(b.hi, b.lo);
    }
    Vs[(long long)j * px + x] = r;
    Vs[(long long)(J + j) * px + x] = i;
}

// The contraction in double-float arithmetic (mixed-precision paths):
//   u[x][t] = sum_{kk < 2J} Vs[kk][x] Gs[kk][t],
// both operands double-float pairs (hi, lo) with rows along x and t.  Each
// product is formed exactly (FMA residual) plus the hi*lo cross terms and
// every output accumulates as a double-float pair (two-sum), ~2^-44 relative
// per step.  64 x 64 outputs per CTA, 4 x 4 per thread (t in two pairs 32
// apart, so that shared-memory reads of a warp are contiguous); the next
// 16-deep slice of both operands is loaded into registers while the current
// one is consumed from shared memory (two buffers, one barrier per slice).
// Operand elements past n_x, n_T or 2J are read as zero.
__global__ void __launch_bounds__(256) contract_df_kernel(int J, int n_x, int n_T, int px, int pt,
                                                          const float2 *__restrict__ Vs,
                                                          const float2 *__restrict__ Gs,
                                                          double *__restrict__ u) {
    __shared__ __align__(16) float2 As[2][BK][BM];
    __shared__ __align__(16) float2 Bs[2][BK][BN];
    const int x0 = blockIdx.y * BM, t0 = blockIdx.x * BN;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int K2 = 2 * J;
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;

    // slice loader: element e = tid + 256 h (h = 0, 1) is row e / 32, float2
    // pair e % 32 of the 16 x 64 slice
    float4 ra[2], rb[2];
    auto load = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = tid + 256 * h, kk = k0 + (e >> 5), c = 2 * (e & 31);
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (kk < K2) {
                const int x = x0 + c, t = t0 + c;
                if (x < n_x) {
                    a = __ldg(reinterpret_cast<const float4 *>(Vs + (long long)kk * px + x));
                    if (x + 1 >= n_x) a.z = a.w = 0.f;
                }
                if (t < n_T) {
                    b = __ldg(reinterpret_cast<const float4 *>(Gs + (long long)kk * pt + t));
                    if (t + 1 >= n_T) b.z = b.w = 0.f;
                }
            }
            ra[h] = a;
            rb[h] = b;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = tid + 256 * h, kk = e >> 5, c = 2 * (e & 31);
            *reinterpret_cast<float4 *>(&As[buf][kk][c]) = ra[h];
            *reinterpret_cast<float4 *>(&Bs[buf][kk][c]) = rb[h];
        }
    };
    load(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K2; k0 += BK) {
        const bool more = k0 + BK < K2;
        if (more) load(k0 + BK);
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[4], b[4];
            const float4 a01 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            const float4 a23 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4 + 2]);
            const float4 b01 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 2]);
            const float4 b23 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][32 + tx * 2]);
            a[0] = make_float2(a01.x, a01.y);
            a[1] = make_float2(a01.z, a01.w);
            a[2] = make_float2(a23.x, a23.y);
            a[3] = make_float2(a23.z, a23.w);
            b[0] = make_float2(b01.x, b01.y);
            b[1] = make_float2(b01.z, b01.w);
            b[2] = make_float2(b23.x, b23.y);
            b[3] = make_float2(b23.z, b23.w);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float pp = a[i].x * b[j].x;
                    float pe = fmaf(a[i].x, b[j].x, -pp);
                    pe = fmaf(a[i].x, b[j].y, pe);
                    pe = fmaf(a[i].y, b[j].x, pe);
                    const float t = sh[i][j] + pp;
                    const float z = t - sh[i][j];
                    sl[i][j] += ((sh[i][j] - (t - z)) + (pp - z)) + pe;
                    sh[i][j] = t;
                }
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int x = x0 + ty * 4 + i;
        if (x >= n_x) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = t0 + (j < 2 ? tx * 2 + j : 32 + tx * 2 + (j - 2));
            if (t < n_T) u[(long long)x * n_T + t] = (double)sh[i][j] + (double)sl[i][j];
        }
    }
}

}  // namespace

void launch_far_table(int J, int M, double *pw, double2 *nu, float4 *nu_f, float4 *phase_tab,
                      cudaStream_t st) {
    far_powers_kernel<<<(M + 127) / 128, 128, 0, st>>>(M, pw);
    far_table_kernel<<<J, 128, 0, st>>>(J, M, pw, nu, nu_f, phase_tab);
}

void launch_sinc_table(int J, int M, const float4 *phase_tab, float4 *tab, cudaStream_t st) {
    const int G = sinc_tab_half(J);
    if (!G) return;
    const size_t smem = (size_t)(M + kTabRows * (M / 2)) * sizeof(float4);
    static std::atomic<unsigned long long> attr{0};
    ensure_smem_attr((const void *)sinc_table_kernel, 200 * 1024, attr);
    const int odd_ctas = ((G + 1) / 2 + kTabRows - 1) / kTabRows;   // positive odd rows 1 .. G
    sinc_table_kernel<<<dim3(odd_ctas + 64, (J + kTabThreads - 1) / kTabThreads), kTabThreads, smem, st>>>(
        J, M, G, odd_ctas, phase_tab, tab);
}

size_t synth_weights_smem(int J, int K, bool table) {
    const int M = 2 * (J - 1);
    return weights_smem_head(K) + (table ? 0 : (size_t)(M + M / 2) * sizeof(float4));
}

void launch_synth_weights(int J, int M, double W, int K, const double *s, const double2 *B,
                          float4 *Bf, const float4 *nu_f, const float4 *phase_tab,
                          const float4 *sinc_tab, const double *T, int n_T, double *Gr, double *Gm,
                          float2 *Gs, cudaStream_t st) {
    if (n_T <= 0) return;
    const size_t smem = synth_weights_smem(J, K, sinc_tab != nullptr);
    static std::atomic<unsigned long long> attr{0};
    ensure_smem_attr((const void *)weights_kernel, (int)kWeightsMaxSmem, attr);
    if (Bf) {
        const long long n = (long long)K * J;
        split_df_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(B, Bf, n);
    }
    dim3 grid(n_T, (J + 255) / 256);
    weights_kernel<<<grid, 256, smem, st>>>(J, M, W, K, s, B, Bf, nu_f, phase_tab, sinc_tab,
                                            sinc_tab ? sinc_tab_half(J) : 0, T, n_T, Gr, Gm, Gs,
                                            synth_pitch(n_T));
}

void launch_synth_contract(int J, int n_x, int n_T, const double2 *V, const double *Gr,
                           const double *Gm, double *u, cudaStream_t st) {
    if (n_x <= 0 || n_T <= 0) return;
    dim3 grid((n_T + BN - 1) / BN, (n_x + BM - 1) / BM);
    contract_kernel<<<grid, 256, 0, st>>>(J, n_x, n_T, V, Gr, Gm, u);
}

void launch_synth_contract_df(int J, int n_x, int n_T, const double2 *V, float2 *Vs,
                              const float2 *Gs, double *u, cudaStream_t st) {
    if (n_x <= 0 || n_T <= 0) return;
    const int px = synth_pitch(n_x), pt = synth_pitch(n_T);
    split_v_kernel<<<dim3((px + 255) / 256, J), 256, 0, st>>>(J, n_x, px, V, Vs);
    dim3 grid((n_T + BN - 1) / BN, (n_x + BM - 1) / BM);
    contract_df_kernel<<<grid, 256, 0, st>>>(J, n_x, n_T, px, pt, Vs, Gs, u);
}

}  // namespace fh
