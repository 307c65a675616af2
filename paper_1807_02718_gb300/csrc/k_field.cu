// Step a5 (step F5): target fields from the resident densities
//
//   V(x, omega_j) = int_Gamma psi_p(r', omega_j) G_omega(x, r') dsigma(r')
//                 ~ (pi/n) sum_i (i/4) H0(kappa |x - z_i|) |z'_i| psi_i
// (Sec. 2.3 eq. freq_domain_repr, Sec. 3.2 eq. Ukslow_repr; trapezoidal rule
// on the Nystrom nodes).  omega = 0 has no solve; V(x, 0) := 1 there (the 2D
// low-frequency limit of the radiating field with data e^{i kappa p.r}).
//
// One CTA per (frequency, 128 targets); source nodes are staged through
// shared memory with the weights c_i = (pi/n) |z'_i| psi_i / 4 premultiplied.
#include "bessel.cuh"
#include "fh_internal.h"

namespace fh {
namespace {

constexpr int kTgt = 128;
constexpr int kSrc = 256;

__global__ void __launch_bounds__(kTgt) field_kernel(
    SolveTables t, const int *__restrict__ solve_j, const double2 *__restrict__ z,
    const double2 *__restrict__ dz, const double2 *__restrict__ psi,
    const double *__restrict__ x, int n_x, double2 *__restrict__ V) {
    const int s = blockIdx.y;
    const int N = t.N[s];
    const int vo = t.vec_off[s];
    const double kappa = t.kappa[s];
    const double w = 2.0 * kPi / (double)N * 0.25;   // (pi/n) / 4
    const int it = blockIdx.x * kTgt + threadIdx.x;
    double px = 0.0, py = 0.0;
    if (it < n_x) { px = x[2 * it]; py = x[2 * it + 1]; }
    __shared__ double2 zs[kSrc];
    __shared__ double2 cs[kSrc];
    double vr = 0.0, vi = 0.0;
    for (int i0 = 0; i0 < N; i0 += kSrc) {
        __syncthreads();
        for (int e = threadIdx.x; e < kSrc; e += kTgt) {
            const int i = i0 + e;
            if (i < N) {
                const double2 d = dz[vo + i];
                const double sp = sqrt(d.x * d.x + d.y * d.y) * w;
                const double2 p = psi[vo + i];
                zs[e] = z[vo + i];
                cs[e] = make_double2(p.x * sp, p.y * sp);
            } else {
                zs[e] = make_double2(0.0, 0.0);
                cs[e] = make_double2(0.0, 0.0);
            }
        }
        __syncthreads();
        if (it < n_x) {
            const int ne = min(kSrc, N - i0);
            for (int e = 0; e < ne; ++e) {
                const double d1 = px - zs[e].x, d2 = py - zs[e].y;
                const double arg = kappa * sqrt(d1 * d1 + d2 * d2);
                double J0, Y0;
                bessel_j0y0(arg, J0, Y0);
                // (i)(J0 + i Y0) c = (-Y0 + i J0) c
                const double2 c = cs[e];
                vr += -Y0 * c.x - J0 * c.y;
                vi += -Y0 * c.y + J0 * c.x;
            }
        }
    }
    if (it < n_x) V[(long long)solve_j[s] * n_x + it] = make_double2(vr, vi);
}

__global__ void field_zero_freq_kernel(int n_x, double2 *__restrict__ V) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_x) V[i] = make_double2(1.0, 0.0);
}

__global__ void bessel_eval_kernel(const double *__restrict__ x, int n, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double J0, Y0, J1, Y1;
    bessel_j0y0j1y1(x[i], J0, Y0, J1, Y1);
    double a, b;
    bessel_j0y0(x[i], a, b);
    out[6 * i + 0] = J0;
    out[6 * i + 1] = Y0;
    out[6 * i + 2] = J1;
    out[6 * i + 3] = Y1;
    out[6 * i + 4] = a;
    out[6 * i + 5] = b;
}

}  // namespace

void launch_bessel_eval(const double *x, int n, double *out, cudaStream_t st) {
    if (n > 0) bessel_eval_kernel<<<(n + 127) / 128, 128, 0, st>>>(x, n, out);
}

void launch_target_field(const SolveTables &t, int S, const int *solve_j, int maxN,
                         const double2 *z, const double2 *dz, const double2 *psi,
                         const double *x, int n_x, double2 *V, cudaStream_t st) {
    (void)maxN;
    if (n_x <= 0) return;
    field_zero_freq_kernel<<<(n_x + 255) / 256, 256, 0, st>>>(n_x, V);
    if (S <= 0) return;
    dim3 grid((n_x + kTgt - 1) / kTgt, S);
    field_kernel<<<grid, kTgt, 0, st>>>(t, solve_j, z, dz, psi, x, n_x, V);
}

}  // namespace fh
