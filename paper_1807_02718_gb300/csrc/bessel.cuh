// J0, Y0, J1, Y1 in FP64 for x > 0, evaluated together (one sincos, one log).
//
//   x < 8:  J0 = A0(t), Y0 = (2/pi) ln(x/2) J0 + A1(t), J1 = x A2(t),
//           Y1 = (2/pi) ln(x/2) J1 - 2/(pi x) + x A3(t),   t = x^2/32 - 1
//           (A0..A3 are entire in x^2: the ascending series of A&S 9.1.10-9.1.11
//            with the logarithmic parts taken out);
//   x >= 8: H_nu(x) = sqrt(2/(pi x)) (P_nu + i Q_nu) e^{i (x - (2 nu + 1) pi/4)},
//           P0 = B0, Q0 = (8/x) B1, P1 = B2, Q1 = (8/x) B3 as functions of
//           u = (x0/x)^2 on [8, 20] and [20, inf)  (Hankel's form, A&S 9.2.5-9.2.6).
// Each A_k / B_k is a Chebyshev series (bessel_cheb.h, made by
// gen_bessel_cheb.py) summed by Clenshaw's recurrence.  Absolute error is
// ~2e-16 for O(1) values (see the GPU test against reference tables).
#pragma once

#include "bessel_cheb.h"

namespace fh {

template <int N>
__device__ __forceinline__ double clenshaw(const double *c, double t) {
    double b1 = 0.0, b2 = 0.0;
    const double t2 = 2.0 * t;
#pragma unroll
    for (int k = N - 1; k >= 1; --k) {
        const double b0 = fma(t2, b1, c[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(t, b1, c[0] - b2);
}

constexpr double kTwoOverPi = 0.63661977236758134308;
constexpr double kSqrtHalf = 0.70710678118654752440;

// Large-argument form: P0, Q0 (and P1, Q1 when want1) at x >= 8.
template <bool want1>
__device__ __forceinline__ void hankel_pq(double x, double &P0, double &Q0, double &P1,
                                          double &Q1) {
    const double r8 = 8.0 / x;
    if (x < 20.0) {
        const double u = r8 * r8;
        const double t = (u - kBLoU0) * (2.0 / (1.0 - kBLoU0)) - 1.0;
        P0 = clenshaw<kBLo0_N>(kBLo0, t);
        Q0 = r8 * clenshaw<kBLo1_N>(kBLo1, t);
        if (want1) {
            P1 = clenshaw<kBLo2_N>(kBLo2, t);
            Q1 = r8 * clenshaw<kBLo3_N>(kBLo3, t);
        }
    } else {
        const double r20 = 20.0 / x;
        const double t = 2.0 * r20 * r20 - 1.0;
        P0 = clenshaw<kBHi0_N>(kBHi0, t);
        Q0 = r8 * clenshaw<kBHi1_N>(kBHi1, t);
        if (want1) {
            P1 = clenshaw<kBHi2_N>(kBHi2, t);
            Q1 = r8 * clenshaw<kBHi3_N>(kBHi3, t);
        }
    }
}

// P0, Q0, P1, Q1 at x >= 8 given r8 = 8/x (shared by the grouped kernels).
template <bool want1>
__device__ __forceinline__ void hankel_pq_r8(double x, double r8, double &P0, double &Q0,
                                             double &P1, double &Q1) {
    if (x < 20.0) {
        const double t = (r8 * r8 - kBLoU0) * (2.0 / (1.0 - kBLoU0)) - 1.0;
        P0 = clenshaw<kBLo0_N>(kBLo0, t);
        Q0 = r8 * clenshaw<kBLo1_N>(kBLo1, t);
        if (want1) {
            P1 = clenshaw<kBLo2_N>(kBLo2, t);
            Q1 = r8 * clenshaw<kBLo3_N>(kBLo3, t);
        }
    } else {
        const double r20 = 2.5 * r8;
        const double t = 2.0 * r20 * r20 - 1.0;
        P0 = clenshaw<kBHi0_N>(kBHi0, t);
        Q0 = r8 * clenshaw<kBHi1_N>(kBHi1, t);
        if (want1) {
            P1 = clenshaw<kBHi2_N>(kBHi2, t);
            Q1 = r8 * clenshaw<kBHi3_N>(kBHi3, t);
        }
    }
}

// Horner form of P0, Q0 (and P1, Q1) for x >= 8 on the intervals of kPQ:
// the table is staged in shared memory by pq_stage() (threads of a warp may
// fall into different intervals).
struct PQShared {
    double c[kPQ_NI * 4 * kPQ_TERMS];
    double uc[kPQ_NI], iuh[kPQ_NI];
};

__device__ __forceinline__ void pq_stage(PQShared &tb) {
    for (int i = threadIdx.x; i < kPQ_NI * 4 * kPQ_TERMS; i += blockDim.x) tb.c[i] = kPQ[i];
    for (int i = threadIdx.x; i < kPQ_NI; i += blockDim.x) {
        tb.uc[i] = kPQ_UC[i];
        tb.iuh[i] = 1.0 / kPQ_UH[i];
    }
}

__device__ __forceinline__ double horner8(const double *c, double t) {
    double a = c[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) a = fma(a, t, c[k]);
    return a;
}

template <bool want1>
__device__ __forceinline__ void pq_horner(const PQShared &tb, double x, double r8, double &P0,
                                          double &Q0, double &P1, double &Q1) {
    const int k = (x >= 10.0) + (x >= 13.0) + (x >= 18.0) + (x >= 28.0) + (x >= 60.0);
    const double t = (r8 * r8 - tb.uc[k]) * tb.iuh[k];
    const double *c = tb.c + k * 4 * kPQ_TERMS;
    P0 = horner8(c, t);
    Q0 = r8 * horner8(c + kPQ_TERMS, t);
    if (want1) {
        P1 = horner8(c + 2 * kPQ_TERMS, t);
        Q1 = r8 * horner8(c + 3 * kPQ_TERMS, t);
    }
}

// Small-argument branch (x < 8) of the joint routine.
__device__ __forceinline__ void bessel_small(double x, double &J0, double &Y0, double &J1,
                                             double &Y1) {
    const double t = x * x * (1.0 / 32.0) - 1.0;
    J0 = clenshaw<kA0_N>(kA0, t);
    const double a1 = clenshaw<kA1_N>(kA1, t);
    const double a2 = clenshaw<kA2_N>(kA2, t);
    const double a3 = clenshaw<kA3_N>(kA3, t);
    const double L = kTwoOverPi * log(0.5 * x);
    Y0 = fma(L, J0, a1);
    J1 = x * a2;
    Y1 = fma(L, J1, fma(x, a3, -kTwoOverPi / x));
}

__device__ __forceinline__ void bessel_small0(double x, double &J0, double &Y0) {
    const double t = x * x * (1.0 / 32.0) - 1.0;
    J0 = clenshaw<kA0_N>(kA0, t);
    const double a1 = clenshaw<kA1_N>(kA1, t);
    Y0 = fma(kTwoOverPi * log(0.5 * x), J0, a1);
}

__device__ __forceinline__ void bessel_j0y0j1y1(double x, double &J0, double &Y0, double &J1,
                                                double &Y1) {
    if (x < 8.0) {
        const double t = x * x * (1.0 / 32.0) - 1.0;
        J0 = clenshaw<kA0_N>(kA0, t);
        const double a1 = clenshaw<kA1_N>(kA1, t);
        const double a2 = clenshaw<kA2_N>(kA2, t);
        const double a3 = clenshaw<kA3_N>(kA3, t);
        const double L = kTwoOverPi * log(0.5 * x);
        Y0 = fma(L, J0, a1);
        J1 = x * a2;
        Y1 = fma(L, J1, fma(x, a3, -kTwoOverPi / x));
    } else {
        double s, c;
        sincos(x, &s, &c);
        const double c0 = (c + s) * kSqrtHalf;   // cos(x - pi/4)
        const double s0 = (s - c) * kSqrtHalf;   // sin(x - pi/4)
        double P0, Q0, P1, Q1;
        hankel_pq<true>(x, P0, Q0, P1, Q1);
        const double A = sqrt(kTwoOverPi / x);
        J0 = A * (P0 * c0 - Q0 * s0);
        Y0 = A * (P0 * s0 + Q0 * c0);
        J1 = A * (P1 * s0 + Q1 * c0);   // chi_1 = chi_0 - pi/2
        Y1 = A * (Q1 * s0 - P1 * c0);
    }
}

__device__ __forceinline__ void bessel_j0y0(double x, double &J0, double &Y0) {
    if (x < 8.0) {
        const double t = x * x * (1.0 / 32.0) - 1.0;
        J0 = clenshaw<kA0_N>(kA0, t);
        const double a1 = clenshaw<kA1_N>(kA1, t);
        Y0 = fma(kTwoOverPi * log(0.5 * x), J0, a1);
    } else {
        double s, c;
        sincos(x, &s, &c);
        const double c0 = (c + s) * kSqrtHalf, s0 = (s - c) * kSqrtHalf;
        double P0, Q0, P1, Q1;
        hankel_pq<false>(x, P0, Q0, P1, Q1);
        const double A = sqrt(kTwoOverPi / x);
        J0 = A * (P0 * c0 - Q0 * s0);
        Y0 = A * (P0 * s0 + Q0 * c0);
    }
}

}  // namespace fh
