// The 2D synthesis with the low-frequency split (Sec. 4.2; Sec. 5 steps
// T1b-T2d) and the FFT-accelerated scaled convolution (Sec. 4.1.2).
//
// Split synthesis.  For each window k and target x the inverse transform of
// F_k(w) = B_k^slow(w) V(x, w) over [-W, W] is, by F(-w) = conj F(w),
//   u_k(x, t) = (1/pi) Re[ I_{w_c}^{W}[F_k](t - s_k) + I_0^{w_c}[F_k](t - s_k) ]
// (eq. fourier_sing_decomp).  The smooth piece uses the n = J - j_c
// equispaced samples of [w_c, W] (w_c = omega_{j_c}): their FC(Gram)
// continuation (d = 6, C = 31, fc_gram_table.h) has period P = (n + C) dw, its
// DFT gives the coefficients of eq. fourier_approx about delta = (w_c + W)/2,
// and the term-wise integral eq. approx gives the transform at any t.  The
// singular piece uses the Filon-Clenshaw-Curtis rule on the graded mesh
// mu_j = w_c (j/4)^9.1 (eq. gradedmesh), 8 Clenshaw-Curtis points on each of
// the subintervals [mu_{j-1}, mu_j], j = 2..4 (eq. gradedmeshIntRule): the
// degree-7 interpolant times e^{-iwt} integrated exactly through the
// Chebyshev moments rho_n(kappa) = int_{-1}^{1} T_n(x) e^{-i kappa x} dx
// (32-point Gauss-Legendre for |kappa| < 12, the forward three-term
// recurrence above, where it is stable).
//
// Everything is linear in the frequency samples, so, as in the periodic
// synthesis, the target dependence is one real contraction:
//   u(x, t) = Re sum_p V'_p(x) G'_p(t),
// V' the target fields at the n smooth and 24 singular frequencies and
//   G'_p(t) = (1/pi) sum_k B_k(w_p) D_p(t - s_k),
// D_p the transform weight of sample p: for the smooth samples
// D_p(t') = sum_m K_m(t') E[m][p] with E = (shifted DFT) o (FC extension) and
// K_m(t') = e^{-i delta t'} 2A sinc((2A/P)(alpha t' - m)), alpha = P / (2 pi);
// for the singular samples the FCC weights.
//
// Scaled convolution.  d_n = sum_m c_m b(beta n - gamma m) (eqs. conv_sum,
// conv_sum_2 with the index reading of eq. discConv) is approximated by eq.
// approx_conv_sum: C^{(gamma)}_p (gamma-fractional DFT of c zero-padded to
// L), B_p (DFT of b at the integers -L/2..L/2-1) and the inverse
// beta-fractional DFT of C B.  Each fractional DFT of length L is computed by
// the chirp factorisation 2mp = m^2 + p^2 - (p - m)^2 as one circular
// convolution of length Nf >= 2L (a power of two) by radix-2 FFTs.
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "fc_gram_table.h"
#include "fh_internal.h"

namespace fh {
namespace {

constexpr int kSM = 4, kSNq = 8;
constexpr double kSQ = 9.1;
constexpr int kNsing = (kSM - 1) * kSNq;
constexpr int kGl = 32;

__constant__ double c_cheb[kSNq][kSNq];   // interpolant coefficients a_n = sum_c c_cheb[n][c] f_c
__constant__ double c_glx[kGl], c_glw[kGl];
__constant__ double c_mu[kSM];

// acc += a * b (or -= when neg) with the low part compensated too: the
// running sum is (sh, sl, sc), the product's FMA residual and cross terms
// and the exact two-sum error of the high part enter sl by a second two-sum
// (the smooth weights' sums cancel strongly).
__device__ __forceinline__ void df_acc_c(float &sh, float &sl, float &sc, dfv a, dfv b, bool neg) {
    float p = a.hi * b.hi;
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    if (neg) { p = -p; pe = -pe; }
    const float t = sh + p;
    const float z = t - sh;
    const float x = ((sh - (t - z)) + (p - z)) + pe;
    const float u = sl + x;
    const float w = u - sl;
    sc += (sl - (u - w)) + (x - w);
    sl = u;
    sh = t;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 expi(double th) {
    double s, c;
    sincos(th, &s, &c);
    return make_double2(c, s);
}
// e^{i pi r} for a rational phase r = num / den, num reduced modulo 2 den in integers
__device__ __forceinline__ double2 expi_pi_ratio(long long num, long long den) {
    long long r = num % (2 * den);
    if (r < 0) r += 2 * den;
    double s, c;
    sincospi((double)r / (double)den, &s, &c);
    return make_double2(c, s);
}

// (a N / D) mod 2 for integers N, D > 0: N = q D + r exactly, a q as an
// exact two-term product, reduced modulo 2 before the small terms are added,
// so that the phase pi a N / D keeps its accuracy for large N.
__device__ __forceinline__ double mulmod2(double a, long long N, long long D) {
    long long q = N / D, r = N - q * D;
    if (r < 0) {
        r += D;
        --q;
    }
    const double hi = a * (double)q;
    const double lo = fma(a, (double)q, -hi);
    double v = fmod(hi, 2.0) + lo + a * (double)r / (double)D;
    v = fmod(v, 2.0);
    return v < 0.0 ? v + 2.0 : v;
}
__device__ __forceinline__ double2 expi_pi(double r) {   // e^{i pi r}
    double s, c;
    sincospi(r, &s, &c);
    return make_double2(c, s);
}

// Continuation rows: Xc[j * n + p] = d e_j / d f_p (right end blended to
// zero, plus the left end read backwards, blended and reversed).
__global__ void fc_rows_kernel(int n, double *__restrict__ Xc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (p >= n) return;
    double v = 0.0;
    if (p >= n - kFcD) {
        const int i = p - (n - kFcD);
        for (int k = 0; k < kFcD; ++k) v += kFcA[j][k] * kFcQ[i][k];
    }
    if (p < kFcD) {
        const int i = kFcD - 1 - p;
        for (int k = 0; k < kFcD; ++k) v += kFcA[kFcC - 1 - j][k] * kFcQ[i][k];
    }
    Xc[(long long)j * n + p] = v;
}

// E[mi * n + p] (mi = m + L/2): coefficient c'_m about the interval centre
// per unit sample p:  (1/L) e^{i pi m (n-1)/L} sum_l e^{-2 pi i m l / L} X[l][p].
__global__ void fc_dft_kernel(int n, int L, const double *__restrict__ Xc, float4 *__restrict__ E) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x, mi = blockIdx.y;
    if (p >= n) return;
    const long long m = mi - L / 2;
    double2 acc = expi_pi_ratio(-2 * m * p, L);
    for (int j = 0; j < kFcC; ++j) {
        const double w = Xc[(long long)j * n + p];
        const double2 e = expi_pi_ratio(-2 * m * (n + j), L);
        acc.x += w * e.x;
        acc.y += w * e.y;
    }
    const double2 sh = expi_pi_ratio(m * (n - 1), L);
    const double2 r = cmul(acc, sh);
    E[(long long)mi * n + p] = df_pack(r.x / L, r.y / L);   // double-float pairs for the weights
}

// Smooth-piece weights: one CTA per time; for every window the kernel row
// K_m(t - s_k) goes to shared memory, then each thread forms D_p = sum_m K_m
// E[m][p] for its samples and accumulates B_k(w_p) D_p.  Rows 0..n-1 of the
// weight planes: Gr = Re G / pi, Gm = -Im G / pi.  The kernel row (FP64) and
// E are held as double-float pairs and the L-term sums D_p run in
// double-float on the FP32 pipe (exact products, compensated two-sum
// accumulation); B_k D_p and the sum over windows stay FP64.  The pairs'
// ~2^-48 rounding, amplified like any input rounding by the FC(Gram)
// continuation, leaves ~1e-10 of u (measured 8.8e-11 on the small kite
// against 3.8e-11 with FP64 sums), 50x below the split rule's own error.
__global__ void __launch_bounds__(256) smooth_weights_kernel(
    int n, int L, double A, double P, double delta, int K, const double *__restrict__ s,
    const double2 *__restrict__ B, int J, int j_c, const float4 *__restrict__ E,
    const double *__restrict__ T, int n_T, double *__restrict__ Gr, double *__restrict__ Gm) {
    extern __shared__ float4 km[];   // L values (re hi, re lo, im hi, im lo)
    const int it = blockIdx.x;
    const double t = T[it];
    const double alpha = P / (2.0 * kPi), r = 2.0 * A / P;
    constexpr int kPer = 4;           // samples per thread and pass
    for (int p0 = 0; p0 < n; p0 += kPer * blockDim.x) {
        double2 acc[kPer];
        for (int q = 0; q < kPer; ++q) acc[q] = make_double2(0.0, 0.0);
        for (int k = 0; k < K; ++k) {
            const double tp = t - s[k];
            __syncthreads();
            const double2 ph = expi(-delta * tp);
            for (int mi = threadIdx.x; mi < L; mi += blockDim.x) {
                const double y = r * (alpha * tp - (double)(mi - L / 2));
                const double sv = y == 0.0 ? 1.0 : sinpi(y) / (kPi * y);
                km[mi] = df_pack(2.0 * A * sv * ph.x, 2.0 * A * sv * ph.y);
            }
            __syncthreads();
            for (int q = 0; q < kPer; ++q) {
                const int p = p0 + q * blockDim.x + threadIdx.x;
                if (p >= n) continue;
                float rh = 0.f, rl = 0.f, rc = 0.f, ih = 0.f, il = 0.f, ic = 0.f;
                for (int mi = 0; mi < L; ++mi) {
                    const float4 e = __ldg(&E[(long long)mi * n + p]);
                    const float4 kk = km[mi];
                    const dfv kr = df_make(kk.x, kk.y), ki = df_make(kk.z, kk.w);
                    const dfv er = df_make(e.x, e.y), ei = df_make(e.z, e.w);
                    df_acc_c(rh, rl, rc, kr, er, false);   // Re: kr er - ki ei
                    df_acc_c(rh, rl, rc, ki, ei, true);
                    df_acc_c(ih, il, ic, kr, ei, false);   // Im: kr ei + ki er
                    df_acc_c(ih, il, ic, ki, er, false);
                }
                const double2 d = make_double2((double)rh + (double)rl + (double)rc,
                                               (double)ih + (double)il + (double)ic);
                acc[q] = cadd(acc[q], cmul(B[(long long)k * J + j_c + p], d));
            }
        }
        for (int q = 0; q < kPer; ++q) {
            const int p = p0 + q * blockDim.x + threadIdx.x;
            if (p >= n) continue;
            Gr[(long long)p * n_T + it] = acc[q].x / kPi;
            Gm[(long long)p * n_T + it] = -acc[q].y / kPi;
        }
    }
}

// Chebyshev moments rho_n(kappa), n < 8.
__device__ void cheb_moments(double kap, double2 (&rho)[kSNq]) {
    if (fabs(kap) < 12.0) {
        for (int q = 0; q < kSNq; ++q) rho[q] = make_double2(0.0, 0.0);
        for (int g = 0; g < kGl; ++g) {
            const double x = c_glx[g];
            const double2 e = expi(-kap * x);
            double t0 = 1.0, t1 = x;
            for (int q = 0; q < kSNq; ++q) {
                const double tq = q == 0 ? 1.0 : (q == 1 ? x : 2.0 * x * t1 - t0);
                if (q >= 2) {
                    t0 = t1;
                    t1 = tq;
                }
                rho[q].x += c_glw[g] * tq * e.x;
                rho[q].y += c_glw[g] * tq * e.y;
            }
        }
        return;
    }
    double sn, cs;
    sincos(kap, &sn, &cs);
    rho[0] = make_double2(2.0 * sn / kap, 0.0);
    rho[1] = make_double2(0.0, -2.0 * (sn - kap * cs) / (kap * kap));
    const double x2 = 2.0 * ((kap * kap - 2.0) * sn + 2.0 * kap * cs) / (kap * kap * kap);
    rho[2] = make_double2(2.0 * x2 - rho[0].x, 0.0);
    const double2 em = make_double2(cs, -sn), ep = make_double2(cs, sn);
    for (int q = 2; q + 1 < kSNq; ++q) {
        const double sgn = ((q + 1) & 1) ? -1.0 : 1.0;   // (-1)^(q+1)
        const double2 sig = make_double2(em.x - sgn * ep.x, em.y - sgn * ep.y);
        const double f = 1.0 / (q + 1) - 1.0 / (q - 1);
        const double2 br = make_double2(2.0 * rho[q].x - f * sig.x, 2.0 * rho[q].y - f * sig.y);
        // (q+1)/(i kap) * br = -i (q+1)/kap * br
        const double a = (double)(q + 1) / kap;
        rho[q + 1] = make_double2(a * br.y + (double)(q + 1) / (q - 1) * rho[q - 1].x,
                                  -a * br.x + (double)(q + 1) / (q - 1) * rho[q - 1].y);
    }
}

// Singular-piece weights: one thread per (time, interval of the graded
// mesh); the interval's eight Clenshaw-Curtis points share its Chebyshev
// moments and phase, computed once per window.  Rows n .. n+23 of the weight
// planes (row n + 8 (jv - 1) + c for point c of interval jv).
__global__ void fcc_weights_kernel(int n, int K, const double *__restrict__ s, const double2 *__restrict__ Bs,
                                   const double *__restrict__ T, int n_T, double *__restrict__ Gr,
                                   double *__restrict__ Gm) {
    const int it = blockIdx.x * blockDim.x + threadIdx.x, jv = blockIdx.y + 1;
    if (it >= n_T) return;
    const double a = c_mu[jv - 1], b = c_mu[jv];        // interval [mu_{jv-1}, mu_jv] (0-based c_mu)
    const double h = 0.5 * (b - a), dl = 0.5 * (a + b);
    const int i0 = (jv - 1) * kSNq;
    double2 acc[kSNq];
    for (int c = 0; c < kSNq; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int k = 0; k < K; ++k) {
        const double tp = T[it] - s[k];
        double2 rho[kSNq];
        cheb_moments(h * tp, rho);
        const double2 ph = expi(-dl * tp);
#pragma unroll
        for (int c = 0; c < kSNq; ++c) {
            double2 w = make_double2(0.0, 0.0);
            for (int q = 0; q < kSNq; ++q) {
                w.x += c_cheb[q][c] * rho[q].x;
                w.y += c_cheb[q][c] * rho[q].y;
            }
            w = cmul(w, ph);
            acc[c] = cadd(acc[c], cmul(Bs[(long long)k * kNsing + i0 + c], make_double2(h * w.x, h * w.y)));
        }
    }
    for (int c = 0; c < kSNq; ++c) {
        Gr[(long long)(n + i0 + c) * n_T + it] = acc[c].x / kPi;
        Gm[(long long)(n + i0 + c) * n_T + it] = -acc[c].y / kPi;
    }
}

// V' = [V rows j_c .. J-1 ; Vs rows 0 .. 23]
__global__ void stack_fields_kernel(int n, int n_x, int j_c, const double2 *__restrict__ V,
                                    const double2 *__restrict__ Vs, double2 *__restrict__ Vp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
    if (x >= n_x) return;
    Vp[(long long)p * n_x + x] = p < n ? V[(long long)(j_c + p) * n_x + x] : Vs[(long long)(p - n) * n_x + x];
}

// ---- radix-2 FFT (Stockham, out of place), batched over rows of length Nf ----

__global__ void fft_stage_kernel(int Nf, int half_len, int batch, const double2 *__restrict__ in,
                                 double2 *__restrict__ out, double sign) {
    // stage with butterflies of span Ls = 2 * half_len: element index j in [0, Nf/2)
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int halfN = Nf / 2;
    if (g >= (long long)halfN * batch) return;
    const int b = (int)(g / halfN), j = (int)(g % halfN);
    const int k = j % half_len;                 // position within the group
    const int grp = j / half_len;
    const double2 *src = in + (long long)b * Nf;
    double2 *dst = out + (long long)b * Nf;
    const double2 x0 = src[j], x1 = src[j + halfN];
    double sw, cw;
    sincospi(sign * (double)k / (double)half_len, &sw, &cw);   // e^{sign i pi k / half_len}
    const double2 t = cmul(x1, make_double2(cw, sw));
    const int o = grp * 2 * half_len + k;
    dst[o] = make_double2(x0.x + t.x, x0.y + t.y);
    dst[o + half_len] = make_double2(x0.x - t.x, x0.y - t.y);
}

// Bluestein input: y[b][m'] = x[b][m'] e^{-i pi alpha m^2 / L} (m = m' - L/2),
// zero for m' >= L (rows of length Nf).
__global__ void chirp_in_kernel(int L, int Nf, int batch, double alpha, const double2 *__restrict__ x,
                                double2 *__restrict__ y) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)Nf * batch) return;
    const int b = (int)(g / Nf), i = (int)(g % Nf);
    double2 v = make_double2(0.0, 0.0);
    if (i < L) {
        const long long m = i - L / 2;
        v = cmul(x[(long long)b * L + i], expi_pi(-mulmod2(alpha, m * m, L)));
    }
    y[g] = v;
}

// Chirp filter z[k] = e^{i pi alpha k^2 / L} at k and Nf - k, |k| < L.
__global__ void chirp_filter_kernel(int L, int Nf, double alpha, double2 *__restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nf) return;
    long long k = -1;
    if (i < L) k = i;
    else if (i > Nf - L) k = Nf - i;
    z[i] = k >= 0 ? expi_pi(mulmod2(alpha, k * k, L)) : make_double2(0.0, 0.0);
}

// Y[b][i] *= Z[i] / Nf
__global__ void pointwise_kernel(int Nf, int batch, double2 *__restrict__ Y, const double2 *__restrict__ Z) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)Nf * batch) return;
    const double2 z = Z[g % Nf];
    const double2 r = cmul(Y[g], z);
    Y[g] = make_double2(r.x / Nf, r.y / Nf);
}

// X[b][p'] = e^{-i pi alpha p^2 / L} conv[b][p'] (p = p' - L/2), times the
// extra factor e^{2 pi i beta n0 p / L} * B[p'] when B is given (the middle of
// eq. approx_conv_sum) and the scale 1/L when scale_L is set.
__global__ void chirp_out_kernel(int L, int Nf, int batch, double alpha, const double2 *__restrict__ conv,
                                 double2 *__restrict__ X, const double2 *__restrict__ Bm, double beta,
                                 long long n0, int scale_L) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)L * batch) return;
    const int b = (int)(g / L), i = (int)(g % L);
    const long long p = i - L / 2;
    double2 v = cmul(conv[(long long)b * Nf + i], expi_pi(-mulmod2(alpha, p * p, L)));
    if (Bm) {
        v = cmul(v, Bm[i]);
        const long long np = n0 * p;                 // e^{2 pi i beta n0 p / L}
        const double ph = np >= 0 ? mulmod2(2.0 * beta, np, L) : -mulmod2(2.0 * beta, -np, L);
        v = cmul(v, expi_pi(ph));
    }
    if (scale_L) v = make_double2(v.x / L, v.y / L);
    X[g] = v;
}

// b at the integers -L/2 .. L/2 - 1 (one row)
__global__ void kernel_samples_kernel(int L, double A, double P, double2 *__restrict__ bq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const double y = (2.0 * A / P) * (double)(i - L / 2);
    bq[i] = make_double2(2.0 * A * (y == 0.0 ? 1.0 : sinpi(y) / (kPi * y)), 0.0);
}

// ---- host helpers ----

unsigned grid_of(long long n, int block) { return (unsigned)((n + block - 1) / block); }

// Batched FFT of rows of length Nf (a power of two) in place in buf, using
// tmp of the same size; sign -1 forward, +1 inverse (unscaled).
void fft_rows(double2 *buf, double2 *tmp, int Nf, int batch, double sign, cudaStream_t st) {
    double2 *in = buf, *out = tmp;
    for (int h = 1; h < Nf; h *= 2) {
        const long long work = (long long)(Nf / 2) * batch;
        fft_stage_kernel<<<grid_of(work, 256), 256, 0, st>>>(Nf, h, batch, in, out, sign);
        double2 *t = in;
        in = out;
        out = t;
    }
    if (in != buf) cudaMemcpyAsync(buf, in, (size_t)Nf * batch * sizeof(double2), cudaMemcpyDeviceToDevice, st);
}

// X = FRFT_alpha(x) for batch rows of length L (eq. approx_conv_sum's
// fractional transforms), with the optional middle factor of chirp_out_kernel.
void frft_rows(const double2 *x, double2 *X, int L, int batch, double alpha, double2 *y, double2 *tmp,
               double2 *z, double2 *ztmp, int Nf, const double2 *Bm, double beta, long long n0,
               int scale_L, cudaStream_t st) {
    chirp_in_kernel<<<grid_of((long long)Nf * batch, 256), 256, 0, st>>>(L, Nf, batch, alpha, x, y);
    fft_rows(y, tmp, Nf, batch, -1.0, st);
    chirp_filter_kernel<<<grid_of(Nf, 256), 256, 0, st>>>(L, Nf, alpha, z);
    fft_rows(z, ztmp, Nf, 1, -1.0, st);
    pointwise_kernel<<<grid_of((long long)Nf * batch, 256), 256, 0, st>>>(Nf, batch, y, z);
    fft_rows(y, tmp, Nf, batch, 1.0, st);
    chirp_out_kernel<<<grid_of((long long)L * batch, 256), 256, 0, st>>>(L, Nf, batch, alpha, y, X, Bm, beta, n0,
                                                                        scale_L);
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on P_n).
void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

struct Scratch {
    std::vector<void *> bufs;
    cudaStream_t st;
    template <class T> T *get(size_t count) {
        void *p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(count, 1) * sizeof(T), st) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return static_cast<T *>(p);
    }
    ~Scratch() {
        for (void *p : bufs) cudaFreeAsync(p, st);
    }
};

}  // namespace
}  // namespace fh

using namespace fh;

extern "C" fh_status fh_sing_frequencies(double omega_c, double *out) {
    if (!out || !(omega_c > 0.0) || !std::isfinite(omega_c)) return FH_EINVAL;
    for (int jv = 1; jv < kSM; ++jv) {
        const double a = omega_c * std::pow((double)jv / kSM, kSQ);
        const double b = omega_c * std::pow((double)(jv + 1) / kSM, kSQ);
        for (int c = 0; c < kSNq; ++c)
            out[(jv - 1) * kSNq + c] = 0.5 * (a + b) + 0.5 * (b - a) * std::cos(kPi * c / (kSNq - 1));
    }
    return FH_OK;
}

extern "C" fh_status fh_synthesize_sing(int J, double W, int j_c, int K, const double *d_s, const double *d_B,
                                        const double *d_Bs, const double *d_V, const double *d_Vs, int n_x,
                                        const double *d_T, int n_T, double *d_u, void *stream) {
    if (J < 2 || !(W > 0.0) || K < 1 || n_x < 0 || n_T < 0 || j_c < 1) return FH_EINVAL;
    const int n = J - j_c;
    if (n < 2 * kFcD || ((n + kFcC) & 1)) return FH_EINVAL;   // FC needs 2d samples; n + C even
    if (n_x == 0 || n_T == 0) return FH_OK;
    if (!d_s || !d_B || !d_Bs || !d_V || !d_Vs || !d_T || !d_u) return FH_EINVAL;
    if (cudaPeekAtLastError() != cudaSuccess) return FH_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double dw = W / (J - 1), wc = j_c * dw;
    const int L = n + kFcC, ns = n + kNsing;
    // constants of the rule on this stream
    double cheb[kSNq][kSNq], glx[kGl], glw[kGl], mu[kSM];
    for (int q = 0; q < kSNq; ++q)
        for (int c = 0; c < kSNq; ++c) {
            const double wt = (c == 0 || c == kSNq - 1) ? 0.5 : 1.0;
            double v = 2.0 / (kSNq - 1) * wt * std::cos(kPi * q * c / (kSNq - 1));
            if (q == 0 || q == kSNq - 1) v *= 0.5;
            cheb[q][c] = v;
        }
    gauss_legendre(kGl, glx, glw);
    for (int j = 0; j < kSM; ++j) mu[j] = wc * std::pow((double)(j + 1) / kSM, kSQ);
    if (cudaMemcpyToSymbolAsync(c_cheb, cheb, sizeof cheb, 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_glx, glx, sizeof glx, 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_glw, glw, sizeof glw, 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_mu, mu, sizeof mu, 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FH_ECUDA;
    fh_status status = FH_OK;
    {
        Scratch sc{{}, st};
        double *Xc = sc.get<double>((size_t)kFcC * n);
        float4 *E = sc.get<float4>((size_t)L * n);   // the FC operator as double-float pairs
        double2 *Vp = sc.get<double2>((size_t)ns * n_x);
        double *Gr = sc.get<double>((size_t)ns * n_T);
        double *Gm = sc.get<double>((size_t)ns * n_T);
        if (!Xc || !E || !Vp || !Gr || !Gm) {
            cudaGetLastError();
            return FH_ENOMEM;
        }
        fc_rows_kernel<<<dim3(grid_of(n, 128), kFcC), 128, 0, st>>>(n, Xc);
        fc_dft_kernel<<<dim3(grid_of(n, 128), L), 128, 0, st>>>(n, L, Xc, E);
        const double A = 0.5 * (W - wc), P = L * dw, delta = 0.5 * (wc + W);
        const size_t smem = (size_t)L * sizeof(float4);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(smooth_weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        smooth_weights_kernel<<<n_T, 256, smem, st>>>(n, L, A, P, delta, K, d_s,
                                                      reinterpret_cast<const double2 *>(d_B), J, j_c, E, d_T, n_T,
                                                      Gr, Gm);
        fcc_weights_kernel<<<dim3(grid_of(n_T, 64), kSM - 1), 64, 0, st>>>(   // 3 n_T / 64 CTAs
            n, K, d_s, reinterpret_cast<const double2 *>(d_Bs), d_T, n_T, Gr, Gm);
        stack_fields_kernel<<<dim3(grid_of(n_x, 128), ns), 128, 0, st>>>(
            n, n_x, j_c, reinterpret_cast<const double2 *>(d_V), reinterpret_cast<const double2 *>(d_Vs), Vp);
        launch_synth_contract(ns, n_x, n_T, Vp, Gr, Gm, d_u, st);
        if (cudaGetLastError() != cudaSuccess) status = FH_ECUDA;
    }
    return status;
}

extern "C" fh_status fh_scaled_convolution(const double *d_c, int M, int batch, double beta, double gamma,
                                           long long n0, int L, double A, double P, double *d_d, void *stream) {
    if (M < 2 || (M & 1) || batch < 1 || L < M || (L & 1) || !(A > 0.0) || !(P > 0.0) || !d_c || !d_d ||
        !std::isfinite(beta) || !std::isfinite(gamma) || L > (1 << 24))
        return FH_EINVAL;
    if (cudaPeekAtLastError() != cudaSuccess) return FH_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int Nf = 1;
    while (Nf < 2 * L) Nf *= 2;
    fh_status status = FH_OK;
    {
        Scratch sc{{}, st};
        double2 *x = sc.get<double2>((size_t)L * batch);       // c zero-padded to L
        double2 *Cg = sc.get<double2>((size_t)L * batch);
        double2 *y = sc.get<double2>((size_t)Nf * batch);
        double2 *tmp = sc.get<double2>((size_t)Nf * batch);
        double2 *z = sc.get<double2>((size_t)Nf);
        double2 *ztmp = sc.get<double2>((size_t)Nf);
        double2 *bq = sc.get<double2>((size_t)L);
        double2 *Bm = sc.get<double2>((size_t)L);
        if (!x || !Cg || !y || !tmp || !z || !ztmp || !bq || !Bm) {
            cudaGetLastError();
            return FH_ENOMEM;
        }
        cudaMemsetAsync(x, 0, (size_t)L * batch * sizeof(double2), st);
        cudaMemcpy2DAsync(x + (L / 2 - M / 2), (size_t)L * sizeof(double2), d_c, (size_t)M * sizeof(double2),
                          (size_t)M * sizeof(double2), batch, cudaMemcpyDeviceToDevice, st);
        // B_p: DFT of b at the integers (alpha = 1)
        kernel_samples_kernel<<<grid_of(L, 256), 256, 0, st>>>(L, A, P, bq);
        frft_rows(bq, Bm, L, 1, 1.0, y, tmp, z, ztmp, Nf, nullptr, 0.0, 0, 0, st);
        // C^{(gamma)}_p, times B_p e^{2 pi i beta n0 p / L}
        frft_rows(x, Cg, L, batch, gamma, y, tmp, z, ztmp, Nf, Bm, beta, n0, 0, st);
        // the inverse beta-fractional transform: d_{n0+n'} = (1/L) sum_p (...) e^{2 pi i beta n' p / L}
        frft_rows(Cg, reinterpret_cast<double2 *>(d_d), L, batch, -beta, y, tmp, z, ztmp, Nf, nullptr, 0.0, 0, 1,
                  st);
        if (cudaGetLastError() != cudaSuccess) status = FH_ECUDA;
    }
    return status;
}
