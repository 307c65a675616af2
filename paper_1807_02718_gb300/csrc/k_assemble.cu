// Step a2: Nystrom assembly of the direct CFIE (Sec. 2.3, eq. CFIE_direct)
//
//   (1/2) psi + K* psi - i eta S psi = dB/dn - i eta B,  B = e^{i kappa p.r},
//
// with the logarithmic splitting of the S and K* kernels and Kress's weights
// R_d for ln(4 sin^2((t - tau)/2)) (the discretisation the paper cites as
// Colton & Kress Sec. 3.5).  With r = |z_l - z_i|, s = |z'|,
// N_il = z2'_i (z1_l - z1_i) - z1'_i (z2_l - z2_i):
//   M  = (i/4) H0(kappa r) s_l          M1 = -J0(kappa r) s_l / (4 pi)
//   L  = (i kappa/4) H1(kappa r)/r N_il s_l/s_i
//   L1 = -(kappa/4pi) J1(kappa r)/r N_il s_l/s_i
//   M2 = M - M1 ln(4 sin^2),  L2 = L - L1 ln(4 sin^2)
//   A  = I/2 + R o (L1 - i eta M1) + (pi/n)(L2 - i eta M2)
// Diagonal limits: M1 = -s/4pi, M2 = [i/4 - C/2pi - ln(kappa s/2)/2pi] s,
// L1 = 0, L2 = (z1'' z2' - z2'' z1') / (4 pi s^2).
//
// One CTA assembles one 32 x 32 tile of one frequency's matrix; tiles of all
// frequencies form one flat launch (prefix offsets tile_off).  Each warp
// writes 32 consecutive rows of a column: column-major stores of 512 B.
#include "bessel.cuh"
#include "fh_internal.h"

namespace fh {
namespace {

constexpr int kTile = 32;

__device__ __forceinline__ int find_solve(const long long *__restrict__ off, int S, long long b) {
    int lo = 0, hi = S;  // off[lo] <= b < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) assemble_kernel(
    SolveTables t, int S, const long long *__restrict__ tile_off,
    const double2 *__restrict__ z, const double2 *__restrict__ dz,
    const double2 *__restrict__ ddz, const double *__restrict__ kress,
    const double *__restrict__ logsin, double2 *__restrict__ A) {
    const long long b = blockIdx.x;
    const int s = find_solve(tile_off, S, b);
    const int N = t.N[s];
    const int nt = (N + kTile - 1) / kTile;
    const long long lt = b - tile_off[s];
    const int tr = (int)(lt % nt), tc = (int)(lt / nt);
    const int i = tr * kTile + (threadIdx.x & 31);
    if (i >= N) return;
    const int vo = t.vec_off[s];
    const int to = t.tab_off[t.tab[s]];
    const double kappa = t.kappa[s], eta = t.eta[s];
    const double pin = 2.0 * kPi / (double)N;   // pi / n
    const double2 zi = z[vo + i], dzi = dz[vo + i];
    const double si = sqrt(dzi.x * dzi.x + dzi.y * dzi.y);
    double2 *Acol = A + t.mat_off[s];
    const double inv4pi = 1.0 / (4.0 * kPi);

    for (int q = threadIdx.x >> 5; q < kTile; q += 8) {
        const int l = tc * kTile + q;
        if (l >= N) break;
        int d = i - l;
        if (d < 0) d += N;
        const double Rw = kress[to + d];
        const double2 dzl = dz[vo + l];
        const double sl = sqrt(dzl.x * dzl.x + dzl.y * dzl.y);
        double L1, L2r, L2i, M1, M2r, M2i;
        if (l == i) {
            const double2 dd = ddz[vo + i];
            M1 = -si * inv4pi;
            M2r = (-kEulerGamma / (2.0 * kPi) - log(kappa * si * 0.5) / (2.0 * kPi)) * si;
            M2i = 0.25 * si;
            L1 = 0.0;
            L2r = (dd.x * dzi.y - dd.y * dzi.x) * inv4pi / (si * si);
            L2i = 0.0;
        } else {
            const double2 zl = z[vo + l];
            const double d1 = zl.x - zi.x, d2 = zl.y - zi.y;
            const double r = sqrt(d1 * d1 + d2 * d2);
            const double x = kappa * r;
            double J0, Y0, J1, Y1;
            bessel_j0y0j1y1(x, J0, Y0, J1, Y1);
            const double Nil = dzi.y * d1 - dzi.x * d2;
            const double ls = logsin[to + d];
            const double g = Nil * sl / (si * r);
            // M = (i/4)(J0 + i Y0) s_l
            const double Mr = -0.25 * Y0 * sl, Mi = 0.25 * J0 * sl;
            M1 = -J0 * sl * inv4pi;
            M2r = Mr - M1 * ls;
            M2i = Mi;
            // L = (i kappa/4)(J1 + i Y1) g
            const double Lr = -0.25 * kappa * Y1 * g, Li = 0.25 * kappa * J1 * g;
            L1 = -kappa * inv4pi * J1 * g;
            L2r = Lr - L1 * ls;
            L2i = Li;
        }
        // R (L1 - i eta M1) + (pi/n)(L2 - i eta M2)
        double ar = Rw * L1 + pin * (L2r + eta * M2i);
        double ai = Rw * (-eta * M1) + pin * (L2i - eta * M2r);
        if (l == i) ar += 0.5;
        Acol[(long long)l * N + i] = make_double2(ar, ai);
    }
}

// g_i = dB/dn - i eta B = i (kappa p.nu_i - eta) e^{i kappa p.z_i}
__global__ void rhs_kernel(SolveTables t, const double2 *__restrict__ z,
                           const double2 *__restrict__ dz, double p0, double p1,
                           double2 *__restrict__ g) {
    const int s = blockIdx.y;
    const int N = t.N[s];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int o = t.vec_off[s] + i;
    const double kappa = t.kappa[s], eta = t.eta[s];
    const double2 zi = z[o], d = dz[o];
    const double sp = sqrt(d.x * d.x + d.y * d.y);
    const double pn = (p0 * d.y - p1 * d.x) / sp;
    const double a = kappa * pn - eta;
    double sn, cs;
    sincos(kappa * (p0 * zi.x + p1 * zi.y), &sn, &cs);
    g[o] = make_double2(-a * sn, a * cs);
}

}  // namespace

void launch_assemble(const SolveTables &t, int S, const long long *tile_off, long long n_tiles,
                     const double2 *z, const double2 *dz, const double2 *ddz,
                     const double *kress, const double *logsin, double2 *A, cudaStream_t st) {
    if (n_tiles <= 0) return;
    assemble_kernel<<<(unsigned)n_tiles, 256, 0, st>>>(t, S, tile_off, z, dz, ddz, kress,
                                                       logsin, A);
}

void launch_rhs(const SolveTables &t, int S, int maxN, const double2 *z, const double2 *dz,
                double p0, double p1, double2 *g, cudaStream_t st) {
    if (S <= 0) return;
    dim3 grid((maxN + 127) / 128, S);
    rhs_kernel<<<grid, 128, 0, st>>>(t, z, dz, p0, p1, g);
}

}  // namespace fh
