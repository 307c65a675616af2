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
#include "dfloat.cuh"
#include "fh_internal.h"

namespace fh {
namespace {

constexpr int kTgt = 128;
constexpr int kChunk = kFieldChunk;   // largest number of source nodes per work item

// Work item w = (subgroup g, chunk of `chunk` <= kChunk nodes).  One CTA per (128 targets, item):
// for each target-node pair the distance r, 1/r, sqrt(2/(pi r)),
// e^{i(kappa_0 r - pi/4)} and the step e^{i dkappa r} are formed once; each
// frequency j of the subgroup then needs only the Horner P0/Q0 series
// (x = kappa_j r >= 8) or the small-argument series (x < 8).  The phase
// carries the exact kappa_j through a first-order correction
// e^{i (kappa_j - kappa_0 - j dkappa) r}.  Partial sums per item go to
// scratch; field_reduce_kernel adds them in a fixed order (the result does
// not depend on scheduling).
__global__ void __launch_bounds__(kTgt) field_partial_kernel(
    SolveTables t, Subgroups grp, const int2 *__restrict__ items, int item_begin, int chunk,
    const double2 *__restrict__ z, const double2 *__restrict__ dz,
    const double2 *__restrict__ psi, const double *__restrict__ x, int n_x,
    double2 *__restrict__ part) {
    const int w = blockIdx.y;
    const int2 item = items[item_begin + w];    // (subgroup, first node)
    const int g = item.x, i0 = item.y;
    const int2 sgv = grp.sg[g];
    const int s0 = sgv.x, cnt = sgv.y;
    const int N = t.N[s0];
    const int vo0 = t.vec_off[s0];
    const double wq = 2.0 * kPi / (double)N * 0.25;   // (pi/n) / 4
    const double dk = grp.dkappa[g];
    __shared__ double kap[kGroup], ikap[kGroup], isqk[kGroup], corr[kGroup];
    __shared__ double2 zs[kChunk];
    __shared__ double2 ps[kGroup][kChunk];   // (pi/n)|z'|/4 * psi_j at each node
    __shared__ PQShared pqt;
    pq_stage(pqt);
    if (threadIdx.x < kGroup) {
        const int j = threadIdx.x;
        const double k = (j < cnt) ? t.kappa[s0 + j] : 1.0;
        kap[j] = k;
        ikap[j] = 1.0 / k;
        isqk[j] = 1.0 / sqrt(k);
    }
    const int ne = min(chunk, N - i0);
    for (int e = threadIdx.x; e < kChunk; e += kTgt) {
        const int i = i0 + e;
        double2 zz = make_double2(0.0, 0.0);
        double sp = 0.0;
        if (e < ne) {
            const double2 d = dz[vo0 + i];
            sp = sqrt(d.x * d.x + d.y * d.y) * wq;
            zz = z[vo0 + i];
        }
        zs[e] = zz;
        for (int j = 0; j < kGroup; ++j) {
            double2 v = make_double2(0.0, 0.0);
            if (e < ne && j < cnt) {
                const double2 q = psi[t.vec_off[s0 + j] + i];
                v = make_double2(q.x * sp, q.y * sp);
            }
            ps[j][e] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < kGroup) corr[threadIdx.x] = kap[threadIdx.x] - (kap[0] + threadIdx.x * dk);
    __syncthreads();
    const int it = blockIdx.x * kTgt + threadIdx.x;
    if (it >= n_x) return;
    const double px = x[2 * it], py = x[2 * it + 1];
    double2 acc[kGroup];
#pragma unroll
    for (int j = 0; j < kGroup; ++j) acc[j] = make_double2(0.0, 0.0);
    for (int e = 0; e < ne; ++e) {
        const double d1 = px - zs[e].x, d2 = py - zs[e].y;
        const double r = sqrt(d1 * d1 + d2 * d2);
        const double ir = 1.0 / r;
        const double ar = sqrt(kTwoOverPi * ir);
        double sn, cs, ss, sc;
        sincos(kap[0] * r, &sn, &cs);
        sincos(dk * r, &ss, &sc);
        double c0 = (cs + sn) * kSqrtHalf, s0v = (sn - cs) * kSqrtHalf;   // e^{i(x0 - pi/4)}
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            if (j < cnt) {
                const double xj = kap[j] * r;
                double J0, Y0;
                if (xj >= 8.0) {
                    const double dl = corr[j] * r;
                    const double c = c0 - dl * s0v, sv = s0v + dl * c0;
                    double P0, Q0, P1, Q1;
                    pq_horner<false>(pqt, xj, 8.0 * ir * ikap[j], P0, Q0, P1, Q1);
                    const double A = ar * isqk[j];
                    J0 = A * (P0 * c - Q0 * sv);
                    Y0 = A * (P0 * sv + Q0 * c);
                } else {
                    bessel_small0(xj, J0, Y0);
                }
                const double2 q = ps[j][e];
                acc[j].x += -Y0 * q.x - J0 * q.y;
                acc[j].y += -Y0 * q.y + J0 * q.x;
                const double cn = c0 * sc - s0v * ss;
                s0v = s0v * sc + c0 * ss;
                c0 = cn;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kGroup; ++j)
        if (j < cnt) part[((long long)w * kGroup + j) * n_x + it] = acc[j];
}


// Mixed-precision variant of field_partial_kernel: the same sums with the
// distances, H0 (Hankel form for kappa r >= 8, the small-argument series with
// ln r formed once per target-node pair below it), the phases and the
// accumulation in double-float arithmetic (the phases e^{i kappa_0 r} and
// e^{i dkappa r} reduced in binary32 pieces, FP64 only for kappa_0 r >= 6000).
// The amplitude sqrt(2 / (pi r)) rides on the phase of each target-node pair
// and 1 / sqrt(kappa_j) on the staged densities, so that the Hankel form
// returns sqrt(kappa_j) H0 and needs no amplitude product per frequency.
template <int kG>   // largest subgroup size of the launch (<= kGroup)
__global__ void __launch_bounds__(kTgt, 5) field_partial_df_kernel(
    SolveTables t, Subgroups grp, const int2 *__restrict__ items, int item_begin, int chunk,
    const double2 *__restrict__ z, const double2 *__restrict__ dz,
    const double2 *__restrict__ psi, const double *__restrict__ x, int n_x,
    const float4 *__restrict__ zf, double2 *__restrict__ part) {
    const int w = blockIdx.y;
    const int2 item = items[item_begin + w];
    const int g = item.x, i0 = item.y;
    const int2 sgv = grp.sg[g];
    const int s0 = sgv.x, cnt = sgv.y;
    const int N = t.N[s0];
    const int vo0 = t.vec_off[s0];
    const double wq = 2.0 * kPi / (double)N * 0.25;   // (pi/n) / 4
    const double dk = grp.dkappa[g];
    const dfv dkd = df_from(dk);
    const float dkf = (float)dk;
    __shared__ double kap[kGroup];
    __shared__ float kapf[kGroup], corrf[kGroup];
    __shared__ dfv ikap8[kGroup], sqk[kGroup], kapd[kGroup], lnk2[kGroup];
    __shared__ double isqd[kGroup];
    __shared__ float k3s[3];   // kappa_0 as three binary32 pieces
    __shared__ float4 zs[kChunk];             // node coordinates, double-float
    __shared__ float4 ps[kGroup][kChunk];   // (pi/n)|z'|/4 psi_j / sqrt(kappa_j) as (re hi, re lo, im hi, im lo)
    // each thread's sums (re hi, re lo, im hi, im lo) per frequency, in its own
    // column: the frequency loop stays rolled (a small instruction footprint)
    __shared__ float accs[kG][4][kTgt];
    __shared__ GShared gt;
    g_stage(gt);
    if (threadIdx.x == 0) {
        const double k0 = t.kappa[s0];
        const float a = (float)k0, b = (float)(k0 - (double)a);
        k3s[0] = a;
        k3s[1] = b;
        k3s[2] = (float)(k0 - (double)a - (double)b);
    }
    if (threadIdx.x < kGroup) {
        const int j = threadIdx.x;
        const double k = (j < cnt) ? t.kappa[s0 + j] : 1.0;
        kap[j] = k;
        kapf[j] = (float)k;
        ikap8[j] = df_from(8.0 / k);
        sqk[j] = df_from(sqrt(k));
        isqd[j] = 1.0 / sqrt(k);
        kapd[j] = df_from(k);
        lnk2[j] = df_from(log(0.5 * k));   // ln(kappa/2): ln(x/2) = ln(kappa/2) + ln r
        corrf[j] = (float)(k - ((j < cnt ? t.kappa[s0] : 1.0) + j * dk));
    }
    __syncthreads();
    const int ne = min(chunk, N - i0);
    for (int e = threadIdx.x; e < kChunk; e += kTgt) {
        const int i = i0 + e;
        float4 zz = make_float4(0.f, 0.f, 0.f, 0.f);
        double sp = 0.0;
        if (e < ne) {
            const double2 d = dz[vo0 + i];
            sp = sqrt(d.x * d.x + d.y * d.y) * wq;
            zz = zf[vo0 + i];
        }
        zs[e] = zz;
        for (int j = 0; j < kG; ++j) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < ne && j < cnt) {
                const double2 q = psi[t.vec_off[s0 + j] + i];
                const double spj = sp * isqd[j];
                const dfv re = df_from(q.x * spj), im = df_from(q.y * spj);
                v = make_float4(re.hi, re.lo, im.hi, im.lo);
            }
            ps[j][e] = v;
        }
    }
    __syncthreads();
    const int it = blockIdx.x * kTgt + threadIdx.x;
    if (it >= n_x) return;
    const dfv npx = df_neg(df_from(x[2 * it])), npy = df_neg(df_from(x[2 * it + 1]));
    const dfv two_over_pi = df_make(0.6366197466850281f, 2.5682552973194106e-08f);   // 2/pi
#pragma unroll
    for (int j = 0; j < kG; ++j)
#pragma unroll
        for (int h = 0; h < 4; ++h) accs[j][h][threadIdx.x] = 0.f;
    for (int e = 0; e < ne; ++e) {
        const float4 z4 = zs[e];
        const dfv d1 = df_add(df_make(z4.x, z4.y), npx), d2 = df_add(df_make(z4.z, z4.w), npy);
        const dfv rd = df_sqrt(df_add(df_mul(d1, d1), df_mul(d2, d2)));
        const dfv ir = df_rcp(rd);
        const dfv amp0 = df_sqrt(df_mul(ir, two_over_pi));   // sqrt(2 / (pi r))
        dfv c, sv, sc, ss;
        if (kapf[0] * rd.hi < kExpiKrMax) df_expi_kr(k3s[0], k3s[1], k3s[2], rd, c, sv);
        else df_expi_cold(kap[0] * df_to(rd) - 0.78539816339744830962, c, sv);   // e^{i (kappa_0 r - pi/4)}
        if (dkf * rd.hi < 3.1f) df_sincos_mid(df_mul(dkd, rd), ss, sc);   // e^{i dkappa r}, no FP64 reduction
        else df_expi_cold(dk * df_to(rd), sc, ss);
        c = df_mul(c, amp0);
        sv = df_mul(sv, amp0);
        const dfv lnr = kapf[0] * rd.hi < 8.0f ? df_log(rd) : df_make(0.f, 0.f);   // shared by the group
        const bool renorm = (e & 15) == 15;
#pragma unroll 1
        for (int j = 0; j < kG; ++j) {
            if (j < cnt) {
                const float xf = kapf[j] * rd.hi;
                dfv J0, Y0;   // sqrt(kappa_j) J0, sqrt(kappa_j) Y0
                if (xf >= 8.0f) {
                    const float dl = corrf[j] * rd.hi;
                    const dfv cj = df_add_f(c, -dl * sv.hi), sj = df_add_f(sv, dl * c.hi);
                    dfv J1, Y1;
                    df_hankel<false>(gt, xf, df_mul(ir, ikap8[j]), cj, sj, J0, Y0, J1, Y1);
                } else {
                    df_bessel_small0_cold(df_mul(kapd[j], rd), df_add(lnr, lnk2[j]), J0, Y0);
                    J0 = df_mul(J0, sqk[j]);
                    Y0 = df_mul(Y0, sqk[j]);
                }
                const float4 q4 = ps[j][e];
                const dfv qr = df_make(q4.x, q4.y), qi = df_make(q4.z, q4.w);
                // acc += (-Y0 qr - J0 qi) + i (-Y0 qi + J0 qr)
                float *ac = &accs[j][0][threadIdx.x];
                float rh = ac[0], rl = ac[kTgt], ih = ac[2 * kTgt], il = ac[3 * kTgt];
                df_acc(rh, rl, Y0, qr, true);
                df_acc(rh, rl, J0, qi, true);
                df_acc(ih, il, Y0, qi, true);
                df_acc(ih, il, J0, qr, false);
                if (renorm) {   // every 16 nodes
                    const dfv vr = df_quick(rh, rl), vi = df_quick(ih, il);
                    rh = vr.hi;
                    rl = vr.lo;
                    ih = vi.hi;
                    il = vi.lo;
                }
                ac[0] = rh;
                ac[kTgt] = rl;
                ac[2 * kTgt] = ih;
                ac[3 * kTgt] = il;
                const dfv cn = df_dot2(c, sc, df_neg(sv), ss);
                sv = df_dot2(sv, sc, c, ss);
                c = cn;
            }
        }
    }
    for (int j = 0; j < cnt; ++j) {
        const float *ac = &accs[j][0][threadIdx.x];
        part[((long long)w * kGroup + j) * n_x + it] =
            make_double2((double)ac[0] + (double)ac[kTgt], (double)ac[2 * kTgt] + (double)ac[3 * kTgt]);
    }
}

// V[solve_j[s0 + j]][x] = sum over the subgroup's items, in item order.
__global__ void field_reduce_kernel(Subgroups grp, int g_begin, const int *__restrict__ item_first,
                                    int item_begin, const int *__restrict__ solve_j,
                                    const double2 *__restrict__ part, int n_x,
                                    double2 *__restrict__ V) {
    const int g = g_begin + blockIdx.y;
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n_x) return;
    const int2 sgv = grp.sg[g];
    const int w0 = item_first[g] - item_begin, w1 = item_first[g + 1] - item_begin;
    for (int j = 0; j < sgv.y; ++j) {
        double2 acc = make_double2(0.0, 0.0);
        for (int w = w0; w < w1; ++w) {
            const double2 v = part[((long long)w * kGroup + j) * n_x + it];
            acc.x += v.x;
            acc.y += v.y;
        }
        V[(long long)solve_j[sgv.x + j] * n_x + it] = acc;
    }
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

// J0, Y0, J1, Y1 through the double-float routines of the mixed-precision
// kernels (Hankel form for x >= 8, small-argument series with a double-float
// logarithm below), for testing them.
__global__ void bessel_eval_df_kernel(const double *__restrict__ x, int n, double *__restrict__ out) {
    __shared__ GShared gt;
    g_stage(gt);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xv = x[i];
    double J0, Y0, J1, Y1;
    if (xv >= 8.0) {
        dfv c, s, j0, y0, j1, y1;
        df_expi(xv - 0.78539816339744830962, c, s);
        const dfv amp = df_from(sqrt(kTwoOverPi / xv));   // carried by the phase
        df_hankel<true>(gt, (float)xv, df_from(8.0 / xv), df_mul(c, amp), df_mul(s, amp), j0, y0, j1, y1);
        J0 = df_to(j0);
        Y0 = df_to(y0);
        J1 = df_to(j1);
        Y1 = df_to(y1);
    } else {
        const dfv xd = df_from(xv);
        const dfv lnh = df_add(df_log(xd), df_make(kLogConstDF[4], kLogConstDF[5]));   // ln(x/2)
        dfv j0, y0, j1, y1;
        df_bessel_small<true>(xd, lnh, j0, y0, j1, y1);
        J0 = df_to(j0);
        Y0 = df_to(y0);
        J1 = df_to(j1);
        Y1 = df_to(y1);
    }
    out[4 * i + 0] = J0;
    out[4 * i + 1] = Y0;
    out[4 * i + 2] = J1;
    out[4 * i + 3] = Y1;
}

}  // namespace

void launch_bessel_eval(const double *x, int n, double *out, cudaStream_t st) {
    if (n > 0) bessel_eval_kernel<<<(n + 127) / 128, 128, 0, st>>>(x, n, out);
}

void launch_bessel_eval_df(const double *x, int n, double *out, cudaStream_t st) {
    if (n > 0) bessel_eval_df_kernel<<<(n + 127) / 128, 128, 0, st>>>(x, n, out);
}

void launch_target_field(const SolveTables &t, const Subgroups &g, int g_begin, int n_groups,
                         const int2 *items, int item_begin, int n_items, int chunk,
                         int group_max, const int *item_first, const int *solve_j,
                         const double2 *z, const double2 *dz, const double2 *psi, const double *x,
                         int n_x, const float4 *zf, double2 *part, double2 *V, bool double_float,
                         cudaStream_t st) {
    if (n_x <= 0) return;
    field_zero_freq_kernel<<<(n_x + 255) / 256, 256, 0, st>>>(n_x, V);
    if (n_groups <= 0 || n_items <= 0) return;
    dim3 grid((n_x + kTgt - 1) / kTgt, n_items);
    if (double_float && group_max <= 4)
        field_partial_df_kernel<4><<<grid, kTgt, 0, st>>>(t, g, items, item_begin, chunk, z, dz, psi, x,
                                                          n_x, zf, part);
    else if (double_float)
        field_partial_df_kernel<kGroup><<<grid, kTgt, 0, st>>>(t, g, items, item_begin, chunk, z, dz, psi,
                                                               x, n_x, zf, part);
    else
        field_partial_kernel<<<grid, kTgt, 0, st>>>(t, g, items, item_begin, chunk, z, dz, psi, x, n_x,
                                                    part);
    dim3 g2((n_x + 127) / 128, n_groups);
    field_reduce_kernel<<<g2, 128, 0, st>>>(g, g_begin, item_first, item_begin, solve_j, part, n_x, V);
}

}  // namespace fh
