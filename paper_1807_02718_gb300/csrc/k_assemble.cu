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
// One CTA assembles one 32 x 32 tile for up to kGroup frequencies; tiles of
// all frequencies (of all problems of a batch) form one flat launch (prefix
// offsets tile_off).  Each warp writes 32 consecutive rows of a column:
// column-major stores of 512 B (the double-float kernel also writes the
// transposed entries, 16 B per row, which meet in L2).
#include "bessel.cuh"
#include "dfloat.cuh"
#include "fh_internal.h"

namespace fh {
namespace {

constexpr int kTile = 32;
constexpr int kNearBand = 2;   // off-diagonals whose special functions stay FP64 (mixed paths)

__device__ __forceinline__ int find_solve(const long long *__restrict__ off, int S, long long b) {
    int lo = 0, hi = S;  // off[lo] <= b < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

// Grouped assembly: one CTA per 32 x 32 tile of a frequency subgroup (up to
// kGroup consecutive frequencies with the same N, hence the same nodes).  The
// geometry of each entry (r, N_il, Kress weight, log kernel, speeds) and the
// phase e^{i(kappa_0 r - pi/4)} with its step e^{i dkappa r} are computed once;
// each frequency then evaluates the P/Q series and writes its own matrix.
__global__ void __launch_bounds__(256) assemble_group_kernel(
    SolveTables t, Subgroups grp, int n_groups, const double2 *__restrict__ z,
    const double2 *__restrict__ dz, const double2 *__restrict__ ddz,
    const double *__restrict__ kress, const double *__restrict__ logsin,
    double2 *__restrict__ A, long long out_shift, long long tile_base) {
    const long long b = tile_base + blockIdx.x;
    const int g = find_solve(grp.tile_off, n_groups, b);
    const int2 sgv = grp.sg[g];
    const int s0 = sgv.x, cnt = sgv.y;
    const int N = t.N[s0];
    const int nt = (N + kTile - 1) / kTile;
    const long long lt = b - grp.tile_off[g];
    const int tr = (int)(lt % nt), tc = (int)(lt / nt);
    __shared__ double kap[kGroup], eta[kGroup], ikap[kGroup], isqk[kGroup], corr[kGroup];
    __shared__ long long moff[kGroup];
    __shared__ PQShared pqt;
    pq_stage(pqt);
    const double dk = grp.dkappa[g];
    if (threadIdx.x < kGroup) {
        const int j = threadIdx.x;
        const double k = (j < cnt) ? t.kappa[s0 + j] : 1.0;
        kap[j] = k;
        eta[j] = (j < cnt) ? t.eta[s0 + j] : 0.0;
        ikap[j] = 1.0 / k;
        isqk[j] = 1.0 / sqrt(k);
        moff[j] = ((j < cnt) ? t.mat_off[s0 + j] : 0) + out_shift;
    }
    __syncthreads();
    if (threadIdx.x < kGroup) corr[threadIdx.x] = kap[threadIdx.x] - (kap[0] + threadIdx.x * dk);
    __syncthreads();
    const int i = tr * kTile + (threadIdx.x & 31);
    if (i >= N) return;
    const int vo = t.vec_off[s0];
    const int to = t.tab_off[t.tab[s0]];
    const double pin = 2.0 * kPi / (double)N;   // pi / n
    const double2 zi = z[vo + i], dzi = dz[vo + i];
    const double si = sqrt(dzi.x * dzi.x + dzi.y * dzi.y);
    const double inv4pi = 1.0 / (4.0 * kPi);

    for (int q = threadIdx.x >> 5; q < kTile; q += 8) {
        const int l = tc * kTile + q;
        if (l >= N) break;
        int d = i - l;
        if (d < 0) d += N;
        const double Rw = kress[to + d];
        const double2 dzl = dz[vo + l];
        const double sl = sqrt(dzl.x * dzl.x + dzl.y * dzl.y);
        const long long e_off = (long long)l * N + i;
        if (l == i) {
            const double2 dd = ddz[vo + i];
            const double M1 = -si * inv4pi;
            const double L2r = (dd.x * dzi.y - dd.y * dzi.x) * inv4pi / (si * si);
            for (int j = 0; j < cnt; ++j) {
                const double M2r = (-kEulerGamma / (2.0 * kPi) - log(kap[j] * si * 0.5) / (2.0 * kPi)) * si;
                const double M2i = 0.25 * si;
                const double ar = 0.5 + pin * (L2r + eta[j] * M2i);
                const double ai = Rw * (-eta[j] * M1) + pin * (0.0 - eta[j] * M2r);
                A[moff[j] + e_off] = make_double2(ar, ai);
            }
            continue;
        }
        const double2 zl = z[vo + l];
        const double d1 = zl.x - zi.x, d2 = zl.y - zi.y;
        const double r = sqrt(d1 * d1 + d2 * d2);
        const double ir = 1.0 / r;
        const double Nil = dzi.y * d1 - dzi.x * d2;
        const double ls = logsin[to + d];
        const double gg = Nil * sl / (si * r);
        const double amp = sqrt(kTwoOverPi * ir);
        double sn, cs, ss, sc;
        sincos(kap[0] * r, &sn, &cs);
        sincos(dk * r, &ss, &sc);
        double c0 = (cs + sn) * kSqrtHalf, s0v = (sn - cs) * kSqrtHalf;   // e^{i(x0 - pi/4)}
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            if (j < cnt) {
                const double kappa = kap[j];
                const double x = kappa * r;
                double J0, Y0, J1, Y1;
                if (x >= 8.0) {
                    const double dl = corr[j] * r;
                    const double c = c0 - dl * s0v, sv = s0v + dl * c0;
                    double P0, Q0, P1, Q1;
                    pq_horner<true>(pqt, x, 8.0 * ir * ikap[j], P0, Q0, P1, Q1);
                    const double Am = amp * isqk[j];
                    J0 = Am * (P0 * c - Q0 * sv);
                    Y0 = Am * (P0 * sv + Q0 * c);
                    J1 = Am * (P1 * sv + Q1 * c);
                    Y1 = Am * (Q1 * sv - P1 * c);
                } else {
                    bessel_small(x, J0, Y0, J1, Y1);
                }
                const double Mr = -0.25 * Y0 * sl, Mi = 0.25 * J0 * sl;
                const double M1 = -J0 * sl * inv4pi;
                const double M2r = Mr - M1 * ls;
                const double Lr = -0.25 * kappa * Y1 * gg, Li = 0.25 * kappa * J1 * gg;
                const double L1 = -kappa * inv4pi * J1 * gg;
                const double L2r = Lr - L1 * ls;
                const double et = eta[j];
                const double ar = Rw * L1 + pin * (L2r + et * Mi);
                const double ai = Rw * (-et * M1) + pin * (Li - et * M2r);
                A[moff[j] + e_off] = make_double2(ar, ai);
                const double cn = c0 * sc - s0v * ss;
                s0v = s0v * sc + c0 * ss;
                c0 = cn;
            }
        }
    }
}

// Mixed-precision variant of assemble_group_kernel.  With
//   k4 = kappa N_il s_l / (4 s_i r),  e4 = eta s_l / 4,
//   W  = (pi/n) ln(4 sin^2((t_i - t_l)/2)) - R_{i-l},
// the off-diagonal entry is
//   Re A = k4 (W/pi J1 - (pi/n) Y1) + (pi/n) e4 J0,
//   Im A = (pi/n) k4 J1 + e4 ((pi/n) Y0 - W/pi J0),
// the same combination of M, M1, M2, L, L1, L2 as the FP64 kernel.  For
// entries off the band |i - l| <= kNearBand, the Bessel values (Hankel form
// for kappa r >= 8, the small-argument series with ln r formed once per node
// pair below it), the phases and this combination run in double-float
// arithmetic; the diagonal and the band (where ln r and the Kress log table
// nearly cancel), the Kress weights and the log table stay FP64.  Entries are
// stored as double-float pairs (re hi, re lo, im hi, im lo): the FP32 LU takes
// the hi parts and the refinement residual uses both.  Per node pair the
// amplitude sqrt(2 / (pi r)) rides on the phase and the geometry factors are
// combined once,
//   A1 = g4 W/pi, B1 = g4 pi/n, C1 = s4 pi/n, D1 = s4 W/pi
//   (g4 = N_il s_l / (4 s_i r), s4 = s_l / 4),
// so that with J' = sqrt(kappa_j) J (what the Hankel form returns)
//   Re A = sqrt(kappa) (A1 J1' - B1 Y1') + (eta / sqrt(kappa)) C1 J0',
//   Im A = sqrt(kappa) B1 J1' + (eta / sqrt(kappa)) (C1 Y0' - D1 J0').
// r, the Bessel values, the phases and the Kress log weight (even in i - l)
// are the same for A(i, l) and A(l, i): a CTA takes a tile (tr, tc) of the
// upper triangle (flat index tc (tc + 1) / 2 + tr within the subgroup) and
// writes both entries of every node pair (i < l on a diagonal tile), the
// second one with its own geometry factors (N_li, s_i, s_l swapped).  With
// A32 non-null the hi parts also go to the row-major FP32 copy that the
// tensor-core LU factors (A32(i, l) at i N + l, the same offsets as A).
__global__ void __launch_bounds__(256, 3) assemble_group_df_kernel(
    SolveTables t, Subgroups grp, int n_groups, const double2 *__restrict__ dz,
    const float4 *__restrict__ zf, const float4 *__restrict__ dzf, const float2 *__restrict__ sf,
    const float2 *__restrict__ wpf, float4 *__restrict__ A, float2 *__restrict__ A32, long long out_shift,
    long long tile_base) {
    const long long b = tile_base + blockIdx.x;
    const int g = find_solve(grp.tile_off, n_groups, b);
    const int2 sgv = grp.sg[g];
    const int s0 = sgv.x, cnt = sgv.y;
    const int N = t.N[s0];
    const long long lt = b - grp.tile_off[g];
    int tc = (int)((sqrtf(8.f * (float)lt + 1.f) - 1.f) * 0.5f);
    while (tc > 0 && (long long)tc * (tc + 1) / 2 > lt) --tc;
    while ((long long)(tc + 1) * (tc + 2) / 2 <= lt) ++tc;
    const int tr = (int)(lt - (long long)tc * (tc + 1) / 2);   // 0 <= tr <= tc < ceil(N / 32)
    __shared__ double kap[kGroup];
    __shared__ float kapf[kGroup], corrf[kGroup];
    __shared__ dfv kapd[kGroup], ikap8[kGroup], sqk[kGroup], eqk[kGroup], lnk2[kGroup];
    __shared__ long long moff[kGroup];
    __shared__ float k3s[3];   // kappa_0 as three binary32 pieces
    __shared__ GShared gt;
    g_stage(gt);
    const double dk = grp.dkappa[g];
    const dfv dkd = df_from(dk);
    const float dkf = (float)dk;
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
        const double e = (j < cnt) ? t.eta[s0 + j] : 0.0;
        kap[j] = k;
        kapf[j] = (float)k;
        kapd[j] = df_from(k);
        ikap8[j] = df_from(8.0 / k);
        sqk[j] = df_from(sqrt(k));
        eqk[j] = df_from(e / sqrt(k));
        lnk2[j] = df_from(log(0.5 * k));   // ln(kappa/2): ln(x/2) = ln(kappa/2) + ln r
        corrf[j] = (float)(k - ((j < cnt ? t.kappa[s0] : 1.0) + j * dk));
        moff[j] = ((j < cnt) ? t.mat_off[s0 + j] : 0) + out_shift;
    }
    __syncthreads();
    const int i = tr * kTile + (threadIdx.x & 31);
    if (i >= N) return;
    const int vo = t.vec_off[s0];
    const int to = t.tab_off[t.tab[s0]];
    const double pin = 2.0 * kPi / (double)N;   // pi / n
    const dfv pind = df_from(pin);
    const double2 dzi = dz[vo + i];
    const double si = sqrt(dzi.x * dzi.x + dzi.y * dzi.y);
    const dfv isi4 = df_from(0.25 / si);
    const dfv two_over_pi = df_make(0.6366197466850281f, 2.5682552973194106e-08f);
    const float4 zi4 = zf[vo + i], dzi4 = dzf[vo + i];
    const dfv nzix = df_make(-zi4.x, -zi4.y), nziy = df_make(-zi4.z, -zi4.w);
    const dfv dzix = df_make(dzi4.x, dzi4.y), dziy = df_make(dzi4.z, dzi4.w);
    const float2 si2 = sf[vo + i];
    const dfv si4 = df_mul_f(df_make(si2.x, si2.y), 0.25f);   // s_i / 4
    const dfv C2 = df_mul(si4, pind);

    for (int q = threadIdx.x >> 5; q < kTile; q += 8) {
        const int l = tc * kTile + q;
        if (l >= N) break;
        if (tr == tc && l <= i) continue;   // each pair once on a diagonal tile
        int d = i - l;
        if (d < 0) d += N;
        if (d <= kNearBand || d >= N - kNearBand) continue;   // assemble_band_kernel
        const long long e_il = (long long)l * N + i, e_li = (long long)i * N + l;
        // pair geometry in double-float from the double-float node tables
        const float4 zl4 = zf[vo + l], dzl4 = dzf[vo + l];
        const dfv d1 = df_add(df_make(zl4.x, zl4.y), nzix), d2 = df_add(df_make(zl4.z, zl4.w), nziy);
        const dfv rd = df_sqrt(df_add(df_mul(d1, d1), df_mul(d2, d2)));
        const dfv ir = df_rcp(rd);
        const dfv Nil = df_add(df_mul(dziy, d1), df_neg(df_mul(dzix, d2)));
        // N_li = z2'_l (z1_i - z1_l) - z1'_l (z2_i - z2_l)
        const dfv Nli = df_dot2(df_make(dzl4.x, dzl4.y), d2, df_make(-dzl4.z, -dzl4.w), d1);
        const float2 sl2 = sf[vo + l], wp2 = wpf[to + d], wq2 = wpf[to + N - d];
        const dfv sl = df_make(sl2.x, sl2.y), Wp = df_make(wp2.x, wp2.y);   // |z'_l|, W / pi at i - l
        const dfv Wq = df_make(wq2.x, wq2.y);                                // W / pi at l - i
        const dfv gg4 = df_mul(df_mul(Nil, sl), df_mul(ir, isi4));          // N_il s_l / (4 s_i r)
        const dfv gq4 = df_mul(df_mul(Nli, si4), df_mul(ir, df_rcp(sl)));   // N_li s_i / (4 s_l r)
        const dfv sl4 = df_mul_f(sl, 0.25f);
        const dfv A1 = df_mul(gg4, Wp), B1 = df_mul(gg4, pind), C1 = df_mul(sl4, pind), D1 = df_mul(sl4, Wp);
        const dfv A2 = df_mul(gq4, Wq), B2 = df_mul(gq4, pind), D2 = df_mul(si4, Wq);
        const dfv amp0 = df_sqrt(df_mul(ir, two_over_pi));
        dfv c, sv, sc, ss;
        if (kapf[0] * rd.hi < kExpiKrMax) df_expi_kr(k3s[0], k3s[1], k3s[2], rd, c, sv);
        else df_expi_cold(kap[0] * df_to(rd) - 0.78539816339744830962, c, sv);   // e^{i (kappa_0 r - pi/4)}
        if (dkf * rd.hi < 3.1f) df_sincos_mid(df_mul(dkd, rd), ss, sc);   // e^{i dkappa r}, no FP64 reduction
        else df_expi_cold(dk * df_to(rd), sc, ss);
        c = df_mul(c, amp0);
        sv = df_mul(sv, amp0);
        const dfv lnr = kapf[0] * rd.hi < 8.0f ? df_log(rd) : df_make(0.f, 0.f);   // shared by the group
#pragma unroll 1   // not unrolled: half the registers, twice the occupancy
        for (int j = 0; j < kGroup; ++j) {
            if (j < cnt) {
                const float xf = kapf[j] * rd.hi;
                dfv J0, Y0, J1, Y1;   // each times sqrt(kappa_j)
                if (xf >= 8.0f) {
                    const float dl = corrf[j] * rd.hi;
                    const dfv cj = df_add_f(c, -dl * sv.hi), sj = df_add_f(sv, dl * c.hi);
                    df_hankel<true>(gt, xf, df_mul(ir, ikap8[j]), cj, sj, J0, Y0, J1, Y1);
                } else {
                    df_bessel_small<true>(df_mul(kapd[j], rd), df_add(lnr, lnk2[j]), J0, Y0, J1, Y1);
                    const dfv q = sqk[j];
                    J0 = df_mul(J0, q);
                    Y0 = df_mul(Y0, q);
                    J1 = df_mul(J1, q);
                    Y1 = df_mul(Y1, q);
                }
                const dfv sq = sqk[j], eq = eqk[j];
                const long long mo = moff[j];
                {
                    const dfv ar = df_dot2(sq, df_dot2(A1, J1, df_neg(B1), Y1), eq, df_mul(C1, J0));
                    const dfv ai = df_dot2(sq, df_mul(B1, J1), eq, df_dot2(C1, Y0, df_neg(D1), J0));
                    A[mo + e_il] = make_float4(ar.hi, ar.lo, ai.hi, ai.lo);
                    if (A32) A32[mo + e_li] = make_float2(ar.hi, ai.hi);
                }
                {
                    const dfv br = df_dot2(sq, df_dot2(A2, J1, df_neg(B2), Y1), eq, df_mul(C2, J0));
                    const dfv bi = df_dot2(sq, df_mul(B2, J1), eq, df_dot2(C2, Y0, df_neg(D2), J0));
                    A[mo + e_li] = make_float4(br.hi, br.lo, bi.hi, bi.lo);
                    if (A32) A32[mo + e_il] = make_float2(br.hi, bi.hi);
                }
                const dfv cn = df_dot2(c, sc, df_neg(sv), ss);
                sv = df_dot2(sv, sc, c, ss);
                c = cn;
            }
        }
    }
}

// The diagonal and the band 0 < |i - l| <= kNearBand (cyclically) of the
// matrices of solves list[0 .. gridDim.y - 1] for the mixed paths, in
// FP64 with the FP64 kernel's formulas: there r is of the order of the node
// spacing and ln r nearly cancels against the Kress log table.  One thread
// per entry, so that no warp of assemble_group_df_kernel runs FP64 Bessel
// series for a few lanes.  A32 (may be null): the hi parts, row-major.
__global__ void __launch_bounds__(256) assemble_band_kernel(
    SolveTables t, const int *__restrict__ list, const double2 *__restrict__ z, const double2 *__restrict__ dz,
    const double2 *__restrict__ ddz, const double *__restrict__ kress,
    const double *__restrict__ logsin, float4 *__restrict__ A, float2 *__restrict__ A32, long long out_shift) {
    constexpr int kW = 2 * kNearBand + 1;
    const int s = list[blockIdx.y];
    const int N = t.N[s];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * kW) return;
    const int i = e / kW, o = e % kW - kNearBand;
    int l = i + o;
    if (l < 0) l += N;
    if (l >= N) l -= N;
    int d = i - l;
    if (d < 0) d += N;
    const int vo = t.vec_off[s], to = t.tab_off[t.tab[s]];
    const double kappa = t.kappa[s], et = t.eta[s];
    const double pin = 2.0 * kPi / (double)N;   // pi / n
    const double inv4pi = 1.0 / (4.0 * kPi);
    const double2 zi = z[vo + i], dzi = dz[vo + i];
    const double si = sqrt(dzi.x * dzi.x + dzi.y * dzi.y);
    const double Rw = kress[to + d];
    double ar, ai;
    if (l == i) {
        const double2 dd = ddz[vo + i];
        const double M1 = -si * inv4pi;
        const double L2r = (dd.x * dzi.y - dd.y * dzi.x) * inv4pi / (si * si);
        const double M2r = (-kEulerGamma / (2.0 * kPi) - log(kappa * si * 0.5) / (2.0 * kPi)) * si;
        const double M2i = 0.25 * si;
        ar = 0.5 + pin * (L2r + et * M2i);
        ai = Rw * (-et * M1) + pin * (0.0 - et * M2r);
    } else {
        const double ls = logsin[to + d];
        const double2 zl = z[vo + l], dzl = dz[vo + l];
        const double e1 = zl.x - zi.x, e2 = zl.y - zi.y;
        const double r = sqrt(e1 * e1 + e2 * e2);
        const double sl = sqrt(dzl.x * dzl.x + dzl.y * dzl.y);
        const double gg = (dzi.y * e1 - dzi.x * e2) * sl / (si * r);
        double J0, Y0, J1, Y1;
        bessel_j0y0j1y1(kappa * r, J0, Y0, J1, Y1);
        const double Mr = -0.25 * Y0 * sl, Mi = 0.25 * J0 * sl;
        const double M1 = -J0 * sl * inv4pi;
        const double M2r = Mr - M1 * ls;
        const double Lr = -0.25 * kappa * Y1 * gg, Li = 0.25 * kappa * J1 * gg;
        const double L1 = -kappa * inv4pi * J1 * gg;
        const double L2r = Lr - L1 * ls;
        ar = Rw * L1 + pin * (L2r + et * Mi);
        ai = Rw * (-et * M1) + pin * (Li - et * M2r);
    }
    const float4 v = df_pack(ar, ai);
    A[t.mat_off[s] + out_shift + (long long)l * N + i] = v;
    if (A32) A32[t.mat_off[s] + out_shift + (long long)i * N + l] = make_float2(v.x, v.z);
}

// g_i = dB/dn - i eta B = i (kappa p.nu_i - eta) e^{i kappa p.z_i}
__global__ void rhs_kernel(SolveTables t, const double2 *__restrict__ z,
                           const double2 *__restrict__ dz, const int *__restrict__ prob,
                           const double2 *__restrict__ pdir, double2 *__restrict__ g) {
    const int s = blockIdx.y;
    const int N = t.N[s];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 pd = pdir[prob[s]];
    const double p0 = pd.x, p1 = pd.y;
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

void launch_assemble_groups(const SolveTables &t, const Subgroups &g, int n_groups,
                            long long tile_base, long long n_tiles, const int *band_list,
                            int band_count, int maxN,
                            const double2 *z, const double2 *dz,
                            const double2 *ddz, const double *kress, const double *logsin,
                            const float4 *zf, const float4 *dzf, const float2 *sf, const float2 *wpf,
                            double2 *A, float4 *Af, float2 *A32, long long out_shift, cudaStream_t st,
                            cudaStream_t band_st) {
    if (n_tiles <= 0 || n_groups <= 0) return;
    if (Af) {
        if (band_count > 0) {
            const dim3 grid((maxN * (2 * kNearBand + 1) + 255) / 256, band_count);
            assemble_band_kernel<<<grid, 256, 0, band_st>>>(t, band_list, z, dz, ddz, kress, logsin, Af,
                                                            A32, out_shift);
        }
        assemble_group_df_kernel<<<(unsigned)n_tiles, 256, 0, st>>>(t, g, n_groups, dz, zf, dzf, sf,
                                                                    wpf, Af, A32, out_shift, tile_base);
    } else
        assemble_group_kernel<<<(unsigned)n_tiles, 256, 0, st>>>(t, g, n_groups, z, dz, ddz, kress,
                                                                 logsin, A, out_shift, tile_base);
}

void launch_rhs(const SolveTables &t, int S, int maxN, const double2 *z, const double2 *dz,
                const int *prob, const double2 *pdir, double2 *g, cudaStream_t st) {
    if (S <= 0) return;
    dim3 grid((maxN + 127) / 128, S);
    rhs_kernel<<<grid, 128, 0, st>>>(t, z, dz, prob, pdir, g);
}

}  // namespace fh
