// Step a3: batched dense complex LU with partial pivoting and the solve
// A_s psi_s = g_s for every frequency (Sec. 5 step F3; the paper solves its 2D
// systems directly and notes LU for small problems in its appendix).
//
// FP64 path: one CTA per frequency, right-looking blocked LU (panel width
// NB) on the column-major matrix.  The right side is carried as column N so
// row swaps and eliminations reach it in flight; back substitution follows.
// The trailing update A22 -= L21 U12 is a complex rank-NB product staged in
// shared memory, 4 x 4 complex outputs per thread.
#include "fh_internal.h"

namespace fh {
namespace {

constexpr int NB = 16;   // panel width
constexpr int TT = 64;   // trailing tile edge

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cinv(double2 a) {
    const double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}

__global__ void __launch_bounds__(256) lu_solve_fp64_kernel(
    const int *__restrict__ order, const int *__restrict__ Ns,
    const long long *__restrict__ mat_off, const int *__restrict__ vec_off,
    double2 *__restrict__ A, double2 *__restrict__ B, int *__restrict__ info) {
    const int s = order[blockIdx.x];
    const int n = Ns[s];
    double2 *a = A + mat_off[s];
    double2 *y = B + vec_off[s];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;

    __shared__ double red_v[8];
    __shared__ int red_i[8];
    __shared__ int sh_piv, sh_bad;
    __shared__ double2 sh_val;
    __shared__ double2 Ls[TT][NB + 1];
    __shared__ double2 Us[NB][TT];

#define AT(i, j) a[(long long)(j) * n + (i)]

    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nb = min(NB, n - k0);
        // ---- panel factorisation, columns k0 .. k0+nb-1 ----
        for (int c = k0; c < k0 + nb; ++c) {
            double best = -1.0;
            int bi = n;
            for (int r = c + tid; r < n; r += 256) {
                const double2 v = AT(r, c);
                const double m = fabs(v.x) + fabs(v.y);
                if (m > best) { best = m; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                double bv = red_v[0];
                int bidx = red_i[0];
                for (int w = 1; w < 8; ++w)
                    if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bidx)) { bv = red_v[w]; bidx = red_i[w]; }
                int bad = !(bv > 0.0) || bidx >= n;
                double2 pv = make_double2(0.0, 0.0);
                if (!bad) {
                    pv = AT(bidx, c);
                    bad = !isfinite(pv.x) || !isfinite(pv.y);
                }
                if (bad) info[s] = c + 1;
                sh_bad = bad;
                sh_piv = bidx;
                if (!bad) sh_val = cinv(pv);
            }
            __syncthreads();
            if (sh_bad) return;
            const int p = sh_piv;
            if (p != c) {
                for (int j = tid; j < n; j += 256) {
                    const double2 t0 = AT(c, j);
                    AT(c, j) = AT(p, j);
                    AT(p, j) = t0;
                }
                if (tid == 0) { const double2 t0 = y[c]; y[c] = y[p]; y[p] = t0; }
            }
            __syncthreads();
            const double2 pinv = sh_val;
            for (int r = c + 1 + tid; r < n; r += 256) AT(r, c) = cmul(AT(r, c), pinv);
            __syncthreads();
            const int ncols = k0 + nb - c - 1;
            const int rows = n - c - 1;
            if (ncols > 0 && rows > 0) {
                for (int e = tid; e < rows * ncols; e += 256) {
                    const int r = c + 1 + e % rows;
                    const int j = c + 1 + e / rows;
                    const double2 l = AT(r, c), u = AT(c, j);
                    double2 v = AT(r, j);
                    v.x -= l.x * u.x - l.y * u.y;
                    v.y -= l.x * u.y + l.y * u.x;
                    AT(r, j) = v;
                }
            }
            __syncthreads();
        }
        // ---- U12 = L11^{-1} A12 (columns k0+nb .. n-1, column n = right side) ----
        for (int j = k0 + nb + tid; j <= n; j += 256) {
            double2 x[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) x[q] = (j < n) ? AT(k0 + q, j) : y[k0 + q];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                if (q < nb) {
#pragma unroll
                    for (int r = q + 1; r < NB; ++r) {
                        if (r < nb) {
                            const double2 l = AT(k0 + r, k0 + q);
                            x[r].x -= l.x * x[q].x - l.y * x[q].y;
                            x[r].y -= l.x * x[q].y + l.y * x[q].x;
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) {
                    if (j < n) AT(k0 + q, j) = x[q]; else y[k0 + q] = x[q];
                }
        }
        __syncthreads();
        // ---- trailing update A22 -= L21 U12 (column n = right side) ----
        const int r0 = k0 + nb;
        const int m = n - r0;
        if (m > 0) {
            const int ntr = (m + TT - 1) / TT, ntc = (m + 1 + TT - 1) / TT;
            const int tx = tid & 15, ty = tid >> 4;
            for (int tile = 0; tile < ntr * ntc; ++tile) {
                const int i0 = r0 + (tile % ntr) * TT, j0 = r0 + (tile / ntr) * TT;
                for (int e = tid; e < TT * NB; e += 256) {
                    const int rr = e % TT, q = e / TT;
                    double2 v = make_double2(0.0, 0.0);
                    if (i0 + rr < n && q < nb) v = AT(i0 + rr, k0 + q);
                    Ls[rr][q] = v;
                }
                for (int e = tid; e < TT * NB; e += 256) {
                    const int q = e % NB, cc = e / NB;
                    const int j = j0 + cc;
                    double2 v = make_double2(0.0, 0.0);
                    if (q < nb && j <= n) v = (j < n) ? AT(k0 + q, j) : y[k0 + q];
                    Us[q][cc] = v;
                }
                __syncthreads();
                double2 acc[4][4];
#pragma unroll
                for (int aa = 0; aa < 4; ++aa)
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        const int i = i0 + tx + 16 * aa, j = j0 + ty + 16 * bb;
                        double2 v = make_double2(0.0, 0.0);
                        if (i < n && j <= n) v = (j < n) ? AT(i, j) : y[i];
                        acc[aa][bb] = v;
                    }
#pragma unroll 4
                for (int q = 0; q < NB; ++q) {
                    double2 l[4], u[4];
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa) l[aa] = Ls[tx + 16 * aa][q];
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) u[bb] = Us[q][ty + 16 * bb];
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa)
#pragma unroll
                        for (int bb = 0; bb < 4; ++bb) {
                            acc[aa][bb].x -= l[aa].x * u[bb].x - l[aa].y * u[bb].y;
                            acc[aa][bb].y -= l[aa].x * u[bb].y + l[aa].y * u[bb].x;
                        }
                }
#pragma unroll
                for (int aa = 0; aa < 4; ++aa)
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        const int i = i0 + tx + 16 * aa, j = j0 + ty + 16 * bb;
                        if (i < n && j <= n) {
                            if (j < n) AT(i, j) = acc[aa][bb]; else y[i] = acc[aa][bb];
                        }
                    }
                __syncthreads();
            }
        }
    }
    // ---- back substitution U x = y ----
    for (int j = n - 1; j >= 0; --j) {
        if (tid == 0) {
            const double2 xj = cmul(y[j], cinv(AT(j, j)));
            y[j] = xj;
            sh_val = xj;
        }
        __syncthreads();
        const double2 xj = sh_val;
        for (int i = tid; i < j; i += 256) {
            const double2 u = AT(i, j);
            double2 v = y[i];
            v.x -= u.x * xj.x - u.y * xj.y;
            v.y -= u.x * xj.y + u.y * xj.x;
            y[i] = v;
        }
        __syncthreads();
    }
#undef AT
}

}  // namespace

void launch_lu_solve_fp64(const int *order, int S, const int *N, const long long *mat_off,
                          const int *vec_off, double2 *A, double2 *b, int *info, cudaStream_t st) {
    if (S <= 0) return;
    lu_solve_fp64_kernel<<<S, 256, 0, st>>>(order, N, mat_off, vec_off, A, b, info);
}

}  // namespace fh
