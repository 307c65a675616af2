// Step a1: Nystrom nodes and curve derivatives; Kress log-kernel weights.
//
// Nodes t_i = pi i / n, i < N = 2n (Sec. 2.3, Nystrom method of Colton &
// Kress Sec. 3.5 cited there).  Curves are the circle, the kite of Sec. 6.2
// and star shapes r(t)(cos t, sin t).
#include "fh_internal.h"

namespace fh {
namespace {

__device__ void curve_eval(const CurveParams &cp, double t, double2 &z, double2 &dz,
                           double2 &ddz) {
    double s1, c1;
    sincos(t, &s1, &c1);
    if (cp.kind == FH_CURVE_KITE) {
        double s2, c2;
        sincos(2.0 * t, &s2, &c2);
        z = make_double2(cp.cx + c1 + 0.65 * c2 - 0.65, cp.cy + 1.5 * s1);
        dz = make_double2(-s1 - 1.3 * s2, 1.5 * c1);
        ddz = make_double2(-c1 - 2.6 * c2, -1.5 * s1);
        return;
    }
    double r = cp.r0, dr = 0.0, ddr = 0.0;
    if (cp.kind == FH_CURVE_STAR) {
        for (int k = 1; k <= cp.n_harm; ++k) {
            double sk, ck;
            sincos(k * t + cp.phase[k - 1], &sk, &ck);
            const double a = cp.amp[k - 1];
            r += a * ck;
            dr += -k * a * sk;
            ddr += -(double)(k * k) * a * ck;
        }
    }
    z = make_double2(cp.cx + r * c1, cp.cy + r * s1);
    dz = make_double2(dr * c1 - r * s1, dr * s1 + r * c1);
    ddz = make_double2(ddr * c1 - 2.0 * dr * s1 - r * c1, ddr * s1 + 2.0 * dr * c1 - r * s1);
}

__device__ __forceinline__ float2 split2(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// Also writes double-float copies of z, z' (hi, lo of x then y) and |z'| for
// the mixed-precision kernels.
__global__ void geometry_kernel(const CurveParams *__restrict__ curves,
                                const int *__restrict__ prob, const int *__restrict__ Ns,
                                const int *__restrict__ vec_off, double2 *__restrict__ z,
                                double2 *__restrict__ dz, double2 *__restrict__ ddz,
                                float4 *__restrict__ zf, float4 *__restrict__ dzf,
                                float2 *__restrict__ sf) {
    const int s = blockIdx.y;
    const int N = Ns[s];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const CurveParams &cp = curves[prob[s]];
    const int n = N / 2;
    const double t = kPi * (double)i / (double)n;
    double2 a, b, c;
    curve_eval(cp, t, a, b, c);
    const int o = vec_off[s] + i;
    z[o] = a;
    dz[o] = b;
    ddz[o] = c;
    const float2 ax = split2(a.x), ay = split2(a.y), bx = split2(b.x), by = split2(b.y);
    zf[o] = make_float4(ax.x, ax.y, ay.x, ay.y);
    dzf[o] = make_float4(bx.x, bx.y, by.x, by.y);
    sf[o] = split2(sqrt(b.x * b.x + b.y * b.y));
}

// R_d = -(2 pi / n) sum_{m=1}^{n-1} cos(m pi d / n) / m - (pi / n^2) cos(pi d)
// and the log kernel ln(4 sin^2(pi d / N)) (d != 0), for d = 0..N-1.
// cos(pi q / n) for q < N and 1/m for m < n are staged in shared memory; the
// index m d mod N advances by d per term.
// Also writes W_d / pi = ((pi/n) ln(4 sin^2(pi d / N)) - R_d) / pi as double-float
// pairs (the combined weight of the mixed-precision assembly).
__global__ void kress_kernel(const int *__restrict__ tab_N, const int *__restrict__ tab_off,
                             double *__restrict__ kress, double *__restrict__ logsin,
                             float2 *__restrict__ wpf) {
    extern __shared__ double ksm[];
    const int tb = blockIdx.y;
    const int N = tab_N[tb];
    const int n = N / 2;
    if (blockIdx.x * blockDim.x >= N) return;
    double *ctab = ksm, *inv = ksm + N;
    for (int q = threadIdx.x; q < N; q += blockDim.x) ctab[q] = cospi((double)q / (double)n);
    for (int m = threadIdx.x; m < n; m += blockDim.x) inv[m] = m ? 1.0 / (double)m : 0.0;
    __syncthreads();
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= N) return;
    double acc = 0.0;
    int q = d;                                   // m d mod N for m = 1
    for (int m = 1; m < n; ++m) {
        acc = fma(ctab[q], inv[m], acc);         // cos(pi m d / n) / m
        q += d;
        if (q >= N) q -= N;
    }
    const double sgn = (d & 1) ? -1.0 : 1.0;
    const double Rd = -(2.0 * kPi / n) * acc - (kPi / ((double)n * n)) * sgn;
    kress[tab_off[tb] + d] = Rd;
    double ls = 0.0;
    if (d != 0) {
        const double sv = sinpi((double)d / (double)N);
        ls = log(4.0 * sv * sv);
    }
    logsin[tab_off[tb] + d] = ls;
    wpf[tab_off[tb] + d] = split2(fma(kPi / (double)n, ls, -Rd) * (1.0 / kPi));
}

}  // namespace

void launch_geometry(const CurveParams *curves, const int *prob, int S, int maxN, const int *N,
                     const int *vec_off, double2 *z, double2 *dz, double2 *ddz, float4 *zf,
                     float4 *dzf, float2 *sf, cudaStream_t st) {
    if (S <= 0) return;
    dim3 grid((maxN + 127) / 128, S);
    geometry_kernel<<<grid, 128, 0, st>>>(curves, prob, N, vec_off, z, dz, ddz, zf, dzf, sf);
}

void launch_kress_tables(int n_tab, int maxN, const int *tab_N, const int *tab_off,
                         double *kress, double *logsin, float2 *wpf, cudaStream_t st) {
    if (n_tab <= 0) return;
    dim3 grid((maxN + 127) / 128, n_tab);
    const size_t smem = (size_t)maxN * 3 / 2 * sizeof(double);
    static std::atomic<unsigned long long> attr{0};
    ensure_smem_attr((const void *)kress_kernel, 200 * 1024, attr);
    kress_kernel<<<grid, 128, smem, st>>>(tab_N, tab_off, kress, logsin, wpf);
}

}  // namespace fh
