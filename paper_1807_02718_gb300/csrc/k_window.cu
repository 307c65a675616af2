// Step a4 (steps F1-F2): windowed signal pieces and their recentred spectra
//
//   w(t)  = 1 - eta((t + H)/(H/2))  on [-H, -H/2],  1 on (-H/2, H/2),
//           eta((t - H/2)/(H/2))    on [H/2, H],    0 for |t| > H,
//   eta(u) = exp(2 e^{-1/u} / (u - 1))                    (Sec. 3.1, eq. window_func)
//   B_k^slow(omega) = int_{-H}^{H} w(tau) a(s_k + tau) e^{i omega tau} dtau
//                                                          (Sec. 3.2, eq. Bkslow_eqn)
// by the trapezoidal rule on tau_q = -H + q dt (the integrand vanishes at
// both ends).  Pass 1 forms the windowed samples wa[k][q]; pass 2 gives one
// CTA per frequency, which stages e^{i omega tau_q} for a chunk of q in
// shared memory and lets each warp reduce one window's dot product.
#include "fh_internal.h"

namespace fh {
namespace {

__device__ double eta_cut(double u) {
    if (u <= 0.0) return 1.0;
    if (u >= 1.0) return 0.0;
    return exp(2.0 * exp(-1.0 / u) / (u - 1.0));
}

__device__ double window_w(double t, double H) {
    if (fabs(t) > H) return 0.0;
    if (t <= -0.5 * H) return 1.0 - eta_cut((t + H) / (0.5 * H));
    if (t >= 0.5 * H) return eta_cut((t - 0.5 * H) / (0.5 * H));
    return 1.0;
}

__global__ void windowed_samples_kernel(const double *__restrict__ a, int n_samples,
                                        long long start0, long long step, int Q, double dt,
                                        double H, double *__restrict__ wa) {
    const int k = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > Q) return;
    const long long idx = start0 + (long long)k * step + q;
    const double v = (idx >= 0 && idx < n_samples) ? a[idx] : 0.0;
    wa[(long long)k * (Q + 1) + q] = v * window_w(-H + dt * q, H);
}

constexpr int kChunk = 1024;

__global__ void __launch_bounds__(256) spectra_kernel(const double *__restrict__ wa, int Q,
                                                      double dt, double H, int K, int J,
                                                      const double *__restrict__ omega,
                                                      double2 *__restrict__ B) {
    const int j = blockIdx.x;
    const double w = omega[j];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double2 ph[kChunk];
    for (int kg = 0; kg < K; kg += 8) {
        const int k = kg + warp;
        double sr = 0.0, si = 0.0;
        for (int q0 = 0; q0 <= Q; q0 += kChunk) {
            __syncthreads();
            for (int e = threadIdx.x; e < kChunk; e += 256) {
                const int q = q0 + e;
                double sn = 0.0, cs = 0.0;
                if (q <= Q) sincos(w * (-H + dt * q), &sn, &cs);
                ph[e] = make_double2(cs, sn);
            }
            __syncthreads();
            if (k < K) {
                const double *row = wa + (long long)k * (Q + 1);
                const int qe = min(kChunk, Q + 1 - q0);
                for (int e = lane; e < qe; e += 32) {
                    const double v = row[q0 + e];
                    sr += v * ph[e].x;
                    si += v * ph[e].y;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_down_sync(0xffffffffu, sr, o);
            si += __shfl_down_sync(0xffffffffu, si, o);
        }
        if (lane == 0 && k < K) B[(long long)k * J + j] = make_double2(dt * sr, dt * si);
    }
}

}  // namespace

void launch_window_spectra(const double *a, int n_samples, long long start0, long long step,
                           int Q, double dt, double H, int K, int J, const double *omega,
                           double *wa, double2 *B, cudaStream_t st) {
    if (K <= 0 || J <= 0) return;
    dim3 g1((Q + 1 + 255) / 256, K);
    windowed_samples_kernel<<<g1, 256, 0, st>>>(a, n_samples, start0, step, Q, dt, H, wa);
    spectra_kernel<<<J, 256, 0, st>>>(wa, Q, dt, H, K, J, omega, B);
}

}  // namespace fh
