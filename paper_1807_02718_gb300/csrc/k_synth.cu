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
// D_p for windows far from t (|y| >= 1.25 h, y = W tau/pi) uses the convergent
// expansion 1/(y - m) = (1/y) sum_r (m/y)^r:
//   D_p = (2W/M) sin(pi y)/(pi y) sum_r (h/y)^r nu_{p,r},
//   nu_{p,r} = sum_m (-1)^m (m/h)^r e^{-2 pi i m p / M},
// truncated once (h/|y|)^r < 2^-54; near windows sum the M terms directly.
#include "fh_internal.h"

namespace fh {
namespace {

// One CTA per p: phases e^{-2 pi i m p / M} (-1)^m for a chunk of m are staged
// in shared memory; thread r accumulates sum_m phase_m (m/h)^r, the power by
// binary exponentiation.
__device__ __forceinline__ double ipow(double x, int r) {
    double y = 1.0;
    while (r) {
        if (r & 1) y *= x;
        x *= x;
        r >>= 1;
    }
    return y;
}

constexpr int kFarChunk = 256;

__global__ void __launch_bounds__(256) far_table_kernel(int J, int M, double2 *__restrict__ nu,
                                                       double2 *__restrict__ ph) {
    const int p = blockIdx.x;
    const int r = threadIdx.x;
    const int h = M / 2;
    __shared__ double2 phs[kFarChunk];
    if (p == 0)
        for (int q = r; q < M; q += blockDim.x) {
            double sn, cs;
            sincospi(-2.0 * (double)q / (double)M, &sn, &cs);
            ph[q] = make_double2(cs, sn);
        }
    double sr = 0.0, si = 0.0;
    for (int m0 = -h; m0 < h; m0 += kFarChunk) {
        __syncthreads();
        for (int e = r; e < kFarChunk; e += blockDim.x) {
            const int m = m0 + e;
            double2 v = make_double2(0.0, 0.0);
            if (m < h) {
                const long long mm = ((long long)(m % M) + M) % M;
                const int q = (int)((mm * p) % M);
                double sn, cs;
                sincospi(-2.0 * (double)q / (double)M, &sn, &cs);
                const double sg = (m & 1) ? -1.0 : 1.0;
                v = make_double2(sg * cs, sg * sn);
            }
            phs[e] = v;
        }
        __syncthreads();
        if (r < kFarTerms) {
            const int me = min(kFarChunk, h - m0);
            for (int e = 0; e < me; ++e) {
                const double pw = ipow((double)(m0 + e) / (double)h, r);
                sr = fma(pw, phs[e].x, sr);
                si = fma(pw, phs[e].y, si);
            }
        }
    }
    if (r < kFarTerms) nu[(long long)r * J + p] = make_double2(sr, si);
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

__global__ void __launch_bounds__(256) weights_kernel(
    int J, int M, double W, int K, const double *__restrict__ s, const double2 *__restrict__ B,
    const double2 *__restrict__ nu, const double2 *__restrict__ ph_g,
    const double *__restrict__ T, int n_T, double *__restrict__ Gr, double *__restrict__ Gm) {
    extern __shared__ float smf[];
    float2 *phc = reinterpret_cast<float2 *>(smf);          // M: cos (hi, lo)
    float2 *phs = phc + M;                                   // M: sin (hi, lo)
    float2 *sc = phs + M;                                    // M: sinc (hi, lo)
    const int t = blockIdx.x;
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    const int h = M / 2;
    for (int q = threadIdx.x; q < M; q += blockDim.x) {
        const double2 e = ph_g[q];
        const dfl c = df_split(e.x), sn = df_split(e.y);
        phc[q] = make_float2(c.hi, c.lo);
        phs[q] = make_float2(sn.hi, sn.lo);
    }
    const double tt = T[t];
    const double scale = 2.0 * W / (double)M;
    double qr = 0.0, qi = 0.0;
    for (int k = 0; k < K; ++k) {
        const double y = W * (tt - s[k]) / kPi;
        double dr = 0.0, di = 0.0;
        if (fabs(y) < 1.25 * (double)h) {
            __syncthreads();
            for (int m = threadIdx.x; m < M; m += blockDim.x) {
                const double d = y - (double)(m - h);
                const dfl v = df_split((d == 0.0) ? 1.0 : sinpi(d) / (kPi * d));
                sc[m] = make_float2(v.hi, v.lo);
            }
            __syncthreads();
            if (p < J) {
                float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
                int q = (int)((((long long)(-h) % M + M) % M) * p % M);
                for (int m = 0; m < M; ++m) {
                    const float2 v2 = sc[m];
                    const float2 c2 = phc[q], s2 = phs[q];
                    const dfl v = {v2.x, v2.y};
                    df_mac(rh, rl, {c2.x, c2.y}, v);
                    df_mac(ih, il, {s2.x, s2.y}, v);
                    q += p;
                    if (q >= M) q -= M;
                    if ((m & 31) == 31) {   // renormalise the accumulators
                        float tr = rh + rl; rl = rl - (tr - rh); rh = tr;
                        float ti = ih + il; il = il - (ti - ih); ih = ti;
                    }
                }
                dr = scale * ((double)rh + (double)rl);
                di = scale * ((double)ih + (double)il);
            }
        } else if (p < J) {
            const double rho = (double)h / y;
            const double lr = log(fabs(rho));
            int R = (int)ceil(-54.0 * 0.69314718055994531 / lr);
            R = max(1, min(R, kFarTerms));
            double ar = 0.0, ai = 0.0;
            for (int r = R - 1; r >= 0; --r) {
                const double2 v = nu[(long long)r * J + p];
                ar = ar * rho + v.x;
                ai = ai * rho + v.y;
            }
            const double f = scale * sinpi(y) / (kPi * y);
            dr = f * ar;
            di = f * ai;
        }
        if (p < J) {
            const double2 b = B[(long long)k * J + p];
            qr += b.x * dr - b.y * di;
            qi += b.x * di + b.y * dr;
        }
    }
    if (p < J) {
        const double mu = (p == 0 || p == J - 1) ? 1.0 : 2.0;
        const double c = mu / (2.0 * kPi);
        Gr[(long long)p * n_T + t] = c * qr;
        Gm[(long long)p * n_T + t] = -c * qi;
    }
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

}  // namespace

void launch_far_table(int J, int M, double2 *nu, double2 *phase_tab, cudaStream_t st) {
    far_table_kernel<<<J, 192, 0, st>>>(J, M, nu, phase_tab);
}

void launch_synth_weights(int J, int M, double W, int K, const double *s, const double2 *B,
                          const double2 *nu, const double2 *phase_tab, const double *T,
                          int n_T, double *Gr, double *Gm, cudaStream_t st) {
    if (n_T <= 0) return;
    const size_t smem = (size_t)M * 3 * sizeof(float2);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    dim3 grid(n_T, (J + 255) / 256);
    weights_kernel<<<grid, 256, smem, st>>>(J, M, W, K, s, B, nu, phase_tab, T, n_T, Gr, Gm);
}

void launch_synth_contract(int J, int n_x, int n_T, const double2 *V, const double *Gr,
                           const double *Gm, double *u, cudaStream_t st) {
    if (n_x <= 0 || n_T <= 0) return;
    dim3 grid((n_T + BN - 1) / BN, (n_x + BM - 1) / BM);
    contract_kernel<<<grid, 256, 0, st>>>(J, n_x, n_T, V, Gr, Gm, u);
}

}  // namespace fh
