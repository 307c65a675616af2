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
// shared memory once for all windows; each warp reduces the dot products of
// four windows in FP64.
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

// One CTA per frequency: for each chunk of 1024 samples the phases
// e^{i omega tau_q} are formed once, as the product of e^{i omega tau_{q0 + 32a}}
// (FP64 sincos, 32 per chunk) and e^{i omega dt b} (b < 32, once per CTA);
// warp w accumulates the FP64 dot products of windows kb + w, kb + w + 8, ...
// (four per warp, blocks of 32 windows), so that each phase serves every window.
__global__ void __launch_bounds__(256) spectra_kernel(const double *__restrict__ wa, int Q,
                                                      double dt, double H, int K, int J,
                                                      const double *__restrict__ omega,
                                                      double2 *__restrict__ B) {
    const int j = blockIdx.x;
    const double w = omega[j];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double2 ph[kChunk];
    __shared__ double2 e0[32], e1[kChunk / 32];
    if (threadIdx.x < 32) {
        double sn, cs;
        sincos(w * (dt * (double)threadIdx.x), &sn, &cs);
        e0[threadIdx.x] = make_double2(cs, sn);
    }
    for (int kb = 0; kb < K; kb += 32) {
        double sr[4] = {0.0, 0.0, 0.0, 0.0}, si[4] = {0.0, 0.0, 0.0, 0.0};
        for (int q0 = 0; q0 <= Q; q0 += kChunk) {
            __syncthreads();
            if (threadIdx.x < kChunk / 32) {
                double sn, cs;
                sincos(w * (-H + dt * (double)(q0 + 32 * (int)threadIdx.x)), &sn, &cs);
                e1[threadIdx.x] = make_double2(cs, sn);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < kChunk; e += 256) {
                const double2 a = e1[e >> 5], b = e0[e & 31];
                ph[e] = q0 + e <= Q ? make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x)
                                    : make_double2(0.0, 0.0);
            }
            __syncthreads();
            const int qe = min(kChunk, Q + 1 - q0);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int k = kb + warp + 8 * s;
                if (k >= K) continue;
                const double *row = wa + (long long)k * (Q + 1) + q0;
                for (int e = lane; e < qe; e += 32) {
                    const double v = row[e];
                    sr[s] += v * ph[e].x;
                    si[s] += v * ph[e].y;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            for (int o = 16; o > 0; o >>= 1) {
                sr[s] += __shfl_down_sync(0xffffffffu, sr[s], o);
                si[s] += __shfl_down_sync(0xffffffffu, si[s], o);
            }
            const int k = kb + warp + 8 * s;
            if (lane == 0 && k < K) B[(long long)k * J + j] = make_double2(dt * sr[s], dt * si[s]);
        }
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
