// Step a3, mixed precision: FP32 LU with partial pivoting, then iterative
// refinement with residuals r = g - A x against the double-float matrix
// (exact products, double-float sums: ~2^-46 relative per term).
//
// The CFIE matrices are well conditioned (second-kind equation), so each
// refinement sweep contracts the error by ~ cond * N * 2^-24; two or three
// sweeps bring the FP32 solution to the accuracy of the residual.  Refinement
// stops when the correction is below tol * ||x||_inf (max-norms); when the
// corrections contract steadily (ratio rho = ||d_k|| / ||d_(k-1)|| <= 1/2),
// the error left after adding d_k is about ||d_k|| rho / (1 - rho), and the
// sweep that would only confirm it is skipped once that estimate is below
// kEstTol * ||x||_inf; when the correction has stopped contracting (no better
// than half the previous one) below kStallTol * ||x||_inf, the level set by
// the residual's own rounding, it stops too.  It fails with FH_ENOCONV after
// max_iters sweeps.
//
// Kernels (largest systems first):
//   lu_factor_fp32_kernel  blocked right-looking LU (panel width 32) of the
//                          column-major complex64 copy, one CTA per system;
//   refine_*               x = 0, y = P g; per sweep: refine_solve_kernel
//                          (d = (LU)^-1 y in FP32, x += d; one CTA per
//                          system; 32-wide diagonal blocks solved by one warp,
//                          off-diagonal updates by the CTA), then
//                          refine_resid_kernel (y = P (g - A x), double-float
//                          products and sums, the difference from g in FP64;
//                          64 rows per CTA so that a sweep spreads over all
//                          SMs).  A system that has converged skips
//                          the remaining sweeps.  The factors may be
//                          column-major (SIMT LU) or row-major (tensor-core LU).
#include "fh_internal.h"

namespace fh {
namespace {

constexpr int NB = 32;   // panel width
constexpr int TT = 64;   // trailing tile edge

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(256) lu_factor_fp32_kernel(
    const int *__restrict__ order, const int *__restrict__ Ns,
    const long long *__restrict__ mat_off, const int *__restrict__ vec_off,
    float2 *__restrict__ A32, int *__restrict__ piv, int *__restrict__ info) {
    const int s = order[blockIdx.x];
    const int n = Ns[s];
    float2 *a = A32 + mat_off[s];
    int *pv = piv + vec_off[s];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    __shared__ float red_v[8];
    __shared__ int red_i[8];
    __shared__ int sh_piv, sh_bad;
    __shared__ float2 sh_val;
    __shared__ float2 Ls[TT][NB + 1];
    __shared__ float2 Us[NB][TT];
#define AT(i, j) a[(long long)(j) * n + (i)]
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nb = min(NB, n - k0);
        for (int c = k0; c < k0 + nb; ++c) {
            float best = -1.f;
            int bi = n;
            for (int r = c + tid; r < n; r += 256) {
                const float2 v = AT(r, c);
                const float m = fabsf(v.x) + fabsf(v.y);
                if (m > best) { best = m; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                float bv = red_v[0];
                int bidx = red_i[0];
                for (int w = 1; w < 8; ++w)
                    if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bidx)) { bv = red_v[w]; bidx = red_i[w]; }
                int bad = !(bv > 0.f) || bidx >= n;
                float2 p = make_float2(0.f, 0.f);
                if (!bad) {
                    p = AT(bidx, c);
                    bad = !isfinite(p.x) || !isfinite(p.y);
                }
                if (bad) info[s] = c + 1;
                sh_bad = bad;
                sh_piv = bidx;
                pv[c] = bidx;
                if (!bad) {
                    const float d = p.x * p.x + p.y * p.y;
                    sh_val = make_float2(p.x / d, -p.y / d);
                }
            }
            __syncthreads();
            if (sh_bad) return;
            const int p = sh_piv;
            if (p != c)
                for (int j = tid; j < n; j += 256) {
                    const float2 t0 = AT(c, j);
                    AT(c, j) = AT(p, j);
                    AT(p, j) = t0;
                }
            __syncthreads();
            const float2 pinv = sh_val;
            for (int r = c + 1 + tid; r < n; r += 256) AT(r, c) = cmulf(AT(r, c), pinv);
            __syncthreads();
            const int ncols = k0 + nb - c - 1, rows = n - c - 1;
            if (ncols > 0 && rows > 0)
                for (int e = tid; e < rows * ncols; e += 256) {
                    const int r = c + 1 + e % rows, j = c + 1 + e / rows;
                    const float2 l = AT(r, c), u = AT(c, j);
                    float2 v = AT(r, j);
                    v.x -= l.x * u.x - l.y * u.y;
                    v.y -= l.x * u.y + l.y * u.x;
                    AT(r, j) = v;
                }
            __syncthreads();
        }
        // U12 = L11^{-1} A12
        for (int j = k0 + nb + tid; j < n; j += 256) {
            float2 x[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) x[q] = AT(k0 + q, j);
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) {
#pragma unroll
                    for (int r = q + 1; r < NB; ++r)
                        if (r < nb) {
                            const float2 l = AT(k0 + r, k0 + q);
                            x[r].x -= l.x * x[q].x - l.y * x[q].y;
                            x[r].y -= l.x * x[q].y + l.y * x[q].x;
                        }
                }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nb) AT(k0 + q, j) = x[q];
        }
        __syncthreads();
        const int r0 = k0 + nb, m = n - r0;
        if (m > 0) {
            const int nt = (m + TT - 1) / TT;
            const int tx = tid & 15, ty = tid >> 4;
            for (int tile = 0; tile < nt * nt; ++tile) {
                const int i0 = r0 + (tile % nt) * TT, j0 = r0 + (tile / nt) * TT;
                for (int e = tid; e < TT * NB; e += 256) {
                    const int rr = e % TT, q = e / TT;
                    Ls[rr][q] = (i0 + rr < n && q < nb) ? AT(i0 + rr, k0 + q) : make_float2(0.f, 0.f);
                }
                for (int e = tid; e < TT * NB; e += 256) {
                    const int q = e % NB, cc = e / NB;
                    Us[q][cc] = (q < nb && j0 + cc < n) ? AT(k0 + q, j0 + cc) : make_float2(0.f, 0.f);
                }
                __syncthreads();
                float2 acc[4][4];
#pragma unroll
                for (int aa = 0; aa < 4; ++aa)
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        const int i = i0 + tx + 16 * aa, j = j0 + ty + 16 * bb;
                        acc[aa][bb] = (i < n && j < n) ? AT(i, j) : make_float2(0.f, 0.f);
                    }
#pragma unroll 8
                for (int q = 0; q < NB; ++q) {
                    float2 l[4], u[4];
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
                        if (i < n && j < n) AT(i, j) = acc[aa][bb];
                    }
                __syncthreads();
            }
        }
    }
#undef AT
    // Replace the swap sequence by the inverse row permutation: row i of the
    // original system becomes row iperm[i] of the factored one.
    extern __shared__ int perm[];
    for (int i = tid; i < n; i += 256) perm[i] = i;
    __syncthreads();
    if (tid == 0)
        for (int c = 0; c < n; ++c) {
            const int p = pv[c];
            if (p != c) { const int t0 = perm[c]; perm[c] = perm[p]; perm[p] = t0; }
        }
    __syncthreads();
    for (int k = tid; k < n; k += 256) pv[perm[k]] = k;
}

// y <- U^{-1} L^{-1} y in FP32 (y already in factored row order), y in shared
// memory.  L is unit lower.  Each 32-wide diagonal block is first loaded into
// registers (lane i holds row i of the block), so the warp's dependent chain
// runs on shuffles only; the rest of the CTA then applies the block to the
// remaining rows.
template <bool kRowMajor>
__device__ void lu_solve_shared(const float2 *__restrict__ a, int n, float2 *y) {
    const int tid = threadIdx.x, lane = tid & 31;
#define AT(i, j) (kRowMajor ? a[(long long)(i) * n + (j)] : a[(long long)(j) * n + (i)])
    for (int jb = 0; jb < n; jb += 32) {
        const int je = min(jb + 32, n);
        if (tid < 32) {
            const int i = jb + lane;
            float2 row[32];
#pragma unroll
            for (int q = 0; q < 32; ++q)
                row[q] = (i < je && jb + q < i) ? AT(i, jb + q) : make_float2(0.f, 0.f);
            float2 yi = (i < je) ? y[i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const float yjx = __shfl_sync(0xffffffffu, yi.x, q);
                const float yjy = __shfl_sync(0xffffffffu, yi.y, q);
                yi.x -= row[q].x * yjx - row[q].y * yjy;
                yi.y -= row[q].x * yjy + row[q].y * yjx;
            }
            if (i < je) y[i] = yi;
        }
        __syncthreads();
        for (int i = je + tid; i < n; i += blockDim.x) {
            float2 yi = y[i];
            for (int j = jb; j < je; ++j) {
                const float2 l = AT(i, j), yj = y[j];
                yi.x -= l.x * yj.x - l.y * yj.y;
                yi.y -= l.x * yj.y + l.y * yj.x;
            }
            y[i] = yi;
        }
        __syncthreads();
    }
    const int nblk = (n + 31) / 32;
    for (int b = nblk - 1; b >= 0; --b) {
        const int jb = b * 32, je = min(jb + 32, n);
        if (tid < 32) {
            const int i = jb + lane;
            float2 row[32];
#pragma unroll
            for (int q = 0; q < 32; ++q)
                row[q] = (i < je && jb + q >= i && jb + q < je) ? AT(i, jb + q) : make_float2(0.f, 0.f);
            float2 yi = (i < je) ? y[i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 31; q >= 0; --q) {
                if (jb + q == i && i < je) {
                    const float2 u = row[q];
                    const float d = u.x * u.x + u.y * u.y;
                    yi = make_float2((yi.x * u.x + yi.y * u.y) / d, (yi.y * u.x - yi.x * u.y) / d);
                }
                const float yjx = __shfl_sync(0xffffffffu, yi.x, q);
                const float yjy = __shfl_sync(0xffffffffu, yi.y, q);
                if (jb + q > i && jb + q < je) {
                    yi.x -= row[q].x * yjx - row[q].y * yjy;
                    yi.y -= row[q].x * yjy + row[q].y * yjx;
                }
            }
            if (i < je) y[i] = yi;
        }
        __syncthreads();
        for (int i = tid; i < jb; i += blockDim.x) {
            float2 yi = y[i];
            for (int j = jb; j < je; ++j) {
                const float2 u = AT(i, j), yj = y[j];
                yi.x -= u.x * yj.x - u.y * yj.y;
                yi.y -= u.x * yj.y + u.y * yj.x;
            }
            y[i] = yi;
        }
        __syncthreads();
    }
#undef AT
}

// Inverses of the 32 x 32 diagonal blocks of row-major factors, computed once
// per factorisation: one CTA (two warps) per block; warp 0 inverts the unit
// lower triangle, warp 1 the upper one, lane j solving for column j; the
// inverses are stored L^{-1} then U^{-1}, 2048 values per block, each as 16
// column pairs x 32 rows of float4 (entry (i, 2h + c) at 64 h + 2 i + c), so
// that the solve's diagonal warp reads a column pair of all 32 rows with one
// 512-byte load.  A partial last block is padded with the identity.
__global__ void __launch_bounds__(64) diag_inverse_kernel(const int2 *__restrict__ blocks,
                                                          const int *__restrict__ Ns,
                                                          const long long *__restrict__ mat_off,
                                                          const int *__restrict__ blk_off,
                                                          const float2 *__restrict__ LU32,
                                                          float2 *__restrict__ inv) {
    const int2 bk = blocks[blockIdx.x];
    const int s = bk.x, b = bk.y, n = Ns[s], jb = 32 * b, nbv = min(32, n - jb);
    const float2 *a = LU32 + mat_off[s];
    __shared__ float2 D[32][33];
    __shared__ float2 T[2][32][33];
    const int tid = threadIdx.x, w = tid >> 5, j = tid & 31;
    for (int e = tid; e < 1024; e += 64) {
        const int i = e >> 5, q = e & 31;
        D[i][q] = (i < nbv && q < nbv) ? a[(long long)(jb + i) * n + jb + q]
                                       : make_float2(i == q ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    float2 x[32];
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float2 v = make_float2(i == j ? 1.f : 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < i; ++k) {
                const float2 l = D[i][k];
                v.x -= l.x * x[k].x - l.y * x[k].y;
                v.y -= l.x * x[k].y + l.y * x[k].x;
            }
            x[i] = v;
        }
    } else {
#pragma unroll
        for (int i = 31; i >= 0; --i) {
            float2 v = make_float2(i == j ? 1.f : 0.f, 0.f);
#pragma unroll
            for (int k = i + 1; k < 32; ++k) {
                const float2 u = D[i][k];
                v.x -= u.x * x[k].x - u.y * x[k].y;
                v.y -= u.x * x[k].y + u.y * x[k].x;
            }
            const float2 d = D[i][i];
            const float rd = 1.f / (d.x * d.x + d.y * d.y);
            x[i] = make_float2((v.x * d.x + v.y * d.y) * rd, (v.y * d.x - v.x * d.y) * rd);
        }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) T[w][i][j] = x[i];
    __syncthreads();
    float2 *dst = inv + (long long)(blk_off[s] + b) * 2048;
    for (int e = tid; e < 2048; e += 64) {
        const int ww = e >> 10, h = (e >> 6) & 15, i = (e >> 1) & 31, c = e & 1;
        dst[e] = T[ww][i][2 * h + c];
    }
}

// Row-major factors (tensor-core LU), blockDim = 512: blocked substitution
// over 32-row blocks, forward (L) then backward (U).  The last warp forms each
// diagonal block's values as the product with its precomputed inverse (one
// warp, no dependent chain).  The other 15 warps own the 32-row chunks w, w +
// 15, ... and update every active row by its 32-column segment of the block:
// eight lanes per row, lane h holding columns 2h, 2h + 1, 16 + 2h, 17 + 2h
// (two 16-byte loads, so that one warp load covers four rows in four
// 128-byte lines), then the eight partial sums of a lane group's eight rows
// are reduced and scattered by shuffles so that lane h ends with row h's
// total.  The next block inverse and the segments of a warp's first chunk of
// the next step are loaded while the current step finishes.  N is even, so
// that every segment is 16-byte aligned.
__device__ void lu_solve_rowmajor(const float2 *__restrict__ a, int n, const float2 *__restrict__ inv,
                                  float2 *y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (int)(blockDim.x >> 5) - 1;   // row warps
    const bool dw = warp == nw;                  // the diagonal warp
    const int gq = lane >> 3, h = lane & 7;
    const int nblk = (n + 31) / 32, steps = 2 * nblk;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 r[16];   // next block inverse (diagonal warp) or the first chunk's segments
    auto block_of = [&](int k) { return k < nblk ? k : steps - 1 - k; };
    // chunks updated at step k: below the block (forward) or above it (backward)
    auto chunk_lo = [&](int k) { return k < nblk ? k + 1 : 0; };
    auto chunk_hi = [&](int k) { return k < nblk ? nblk : steps - 1 - k; };
    auto first_chunk = [&](int k) {   // the smallest c >= chunk_lo(k) with c = warp mod nw
        const int lo = chunk_lo(k);
        return lo + ((warp - lo % nw) + nw) % nw;
    };
    auto load_inv = [&](int k) {
        const float4 *blk = reinterpret_cast<const float4 *>(inv + (long long)block_of(k) * 2048 +
                                                             (k < nblk ? 0 : 1024));
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = blk[q * 32 + lane];
    };
    auto load_chunk = [&](int k, int c) {   // rows 32 c + 4 j + gq, j < 8
        const int jb = 32 * block_of(k), je = min(jb + 32, n);
        const bool v0 = jb + 2 * h < je, v1 = jb + 16 + 2 * h < je;   // je - jb is even
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = 32 * c + 4 * j + gq;
            const float4 *src = reinterpret_cast<const float4 *>(a + (long long)i * n + jb + 2 * h);
            r[2 * j] = (i < n && v0) ? src[0] : z4;
            r[2 * j + 1] = (i < n && v1) ? src[8] : z4;
        }
    };
    auto update_chunk = [&](int k, int c) {   // the chunk's segments in r
        const int jb = 32 * block_of(k), je = min(jb + 32, n);
        const bool v0 = jb + 2 * h < je, v1 = jb + 16 + 2 * h < je;
        const float2 z2 = make_float2(0.f, 0.f);
        const float2 ya = v0 ? y[jb + 2 * h] : z2, yb = v0 ? y[jb + 2 * h + 1] : z2;
        const float2 yc = v1 ? y[jb + 16 + 2 * h] : z2, yd = v1 ? y[jb + 17 + 2 * h] : z2;
        float sx[8], sy[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 l0 = r[2 * j], l1 = r[2 * j + 1];
            sx[j] = l0.x * ya.x - l0.y * ya.y + l0.z * yb.x - l0.w * yb.y + l1.x * yc.x - l1.y * yc.y +
                    l1.z * yd.x - l1.w * yd.y;
            sy[j] = l0.x * ya.y + l0.y * ya.x + l0.z * yb.y + l0.w * yb.x + l1.x * yc.y + l1.y * yc.x +
                    l1.z * yd.y + l1.w * yd.x;
        }
        // reduce over the eight lanes and scatter: lane h keeps row h's sum
        const bool b2 = (h >> 2) & 1, b1 = (h >> 1) & 1, b0 = h & 1;
        float ax[4], ay[4], bx[2], by[2];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            ax[t] = (b2 ? sx[t + 4] : sx[t]) + __shfl_xor_sync(0xffffffffu, b2 ? sx[t] : sx[t + 4], 4);
            ay[t] = (b2 ? sy[t + 4] : sy[t]) + __shfl_xor_sync(0xffffffffu, b2 ? sy[t] : sy[t + 4], 4);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            bx[t] = (b1 ? ax[t + 2] : ax[t]) + __shfl_xor_sync(0xffffffffu, b1 ? ax[t] : ax[t + 2], 2);
            by[t] = (b1 ? ay[t + 2] : ay[t]) + __shfl_xor_sync(0xffffffffu, b1 ? ay[t] : ay[t + 2], 2);
        }
        const float tx = (b0 ? bx[1] : bx[0]) + __shfl_xor_sync(0xffffffffu, b0 ? bx[0] : bx[1], 1);
        const float ty = (b0 ? by[1] : by[0]) + __shfl_xor_sync(0xffffffffu, b0 ? by[0] : by[1], 1);
        const int i = 32 * c + 4 * h + gq;
        if (i < n) {
            float2 yi = y[i];
            yi.x -= tx;
            yi.y -= ty;
            y[i] = yi;
        }
    };
    if (dw) load_inv(0);
    else if (first_chunk(0) < chunk_hi(0)) load_chunk(0, first_chunk(0));
    for (int k = 0; k < steps; ++k) {
        const int jb = 32 * block_of(k), je = min(jb + 32, n);
        if (dw) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (jb + 2 * q < je) {
                    const float2 y0 = y[jb + 2 * q], y1 = y[jb + 2 * q + 1];
                    acc.x += r[q].x * y0.x - r[q].y * y0.y + r[q].z * y1.x - r[q].w * y1.y;
                    acc.y += r[q].x * y0.y + r[q].y * y0.x + r[q].z * y1.y + r[q].w * y1.x;
                }
            if (k + 1 < steps) load_inv(k + 1);
            __syncwarp();
            if (jb + lane < je) y[jb + lane] = acc;
        }
        __syncthreads();
        if (!dw) {
            const int hi = chunk_hi(k);
            int c = first_chunk(k);
            if (c < hi) {
                update_chunk(k, c);
                for (c += nw; c < hi; c += nw) {
                    load_chunk(k, c);
                    update_chunk(k, c);
                }
            }
            if (k + 1 < steps && first_chunk(k + 1) < chunk_hi(k + 1)) load_chunk(k + 1, first_chunk(k + 1));
        }
        __syncthreads();
    }
}

__device__ double block_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    return r;
}

// Refinement state of one system.
struct RefineState {
    double gmax, dmax, xmax;
    double dprev;                 // correction of the sweep before (0 before sweep 2)
    unsigned long long rbits;     // max_i |r_i|_1 as the bits of a non-negative double
    int conv, pad;
};

// A correction that has stopped contracting is rounding noise of the residual;
// it is accepted as converged below this fraction of ||x||.
constexpr double kStallTol = 1e-10;
// Steady contraction: converged once the estimated remaining error is below
// this fraction of ||x|| (two orders below the correction tolerance, at the
// rounding level of the double-float residual).
constexpr double kEstTol = 1e-14;

__device__ __forceinline__ bool refine_done(const RefineState &r, double tol) {
    if (!(r.dmax > tol * r.xmax) || r.rbits == 0ull) return true;
    if (!(r.dprev > 0.0)) return false;
    if (r.dmax <= 0.5 * r.dprev) {
        const double rho = r.dmax / r.dprev;
        return r.dmax * rho <= kEstTol * (1.0 - rho) * r.xmax;
    }
    return r.dmax <= kStallTol * r.xmax;
}

// x = 0, y = P g (FP32), ||g||.
__global__ void __launch_bounds__(256) refine_setup_kernel(
    const int *__restrict__ order, const int *__restrict__ Ns, const int *__restrict__ vec_off,
    const int *__restrict__ piv,
    const double2 *__restrict__ G, double2 *__restrict__ X, float2 *__restrict__ Y32,
    RefineState *__restrict__ st, int *__restrict__ iters, const int *__restrict__ info) {
    __shared__ double red[32];
    const int s = order[blockIdx.x], n = Ns[s], vo = vec_off[s];
    double gmax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 gi = G[vo + i];
        X[vo + i] = make_double2(0.0, 0.0);
        Y32[vo + piv[vo + i]] = make_float2((float)gi.x, (float)gi.y);
        gmax = fmax(gmax, fabs(gi.x) + fabs(gi.y));
    }
    gmax = block_max(gmax, red);
    if (threadIdx.x == 0) {
        RefineState r;
        r.gmax = gmax;
        r.dmax = r.xmax = r.dprev = 0.0;
        r.rbits = 0ull;
        r.conv = info[s] != 0;
        r.pad = 0;
        st[s] = r;
        iters[s] = 0;
    }
}

// Sweep `it`: stop if sweep it-1 converged; else d = (LU)^{-1} y, x += d.
template <bool kRowMajor>
__global__ void __launch_bounds__(kRowMajor ? 512 : 256) refine_solve_kernel(
    const int *__restrict__ order, const int *__restrict__ Ns, const long long *__restrict__ mat_off,
    const int *__restrict__ vec_off, const float2 *__restrict__ LU32, const float2 *__restrict__ inv,
    const int *__restrict__ blk_off, double2 *__restrict__ X,
    const float2 *__restrict__ Y32, RefineState *__restrict__ st, int it, double tol,
    int *__restrict__ iters) {
    extern __shared__ float2 ys[];
    __shared__ double red[32];
    const int s = order[blockIdx.x];
    RefineState *rs = st + s;
    if (rs->conv) return;
    if (it > 1 && refine_done(*rs, tol)) {
        if (threadIdx.x == 0) rs->conv = 1;
        return;
    }
    const int n = Ns[s], vo = vec_off[s];
    for (int i = threadIdx.x; i < n; i += blockDim.x) ys[i] = Y32[vo + i];
    __syncthreads();
    if (kRowMajor) lu_solve_rowmajor(LU32 + mat_off[s], n, inv + (long long)blk_off[s] * 2048, ys);
    else lu_solve_shared<false>(LU32 + mat_off[s], n, ys);
    double dmax = 0.0, xmax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 d = ys[i];
        double2 xi = X[vo + i];
        xi.x += (double)d.x;
        xi.y += (double)d.y;
        X[vo + i] = xi;
        dmax = fmax(dmax, fabs((double)d.x) + fabs((double)d.y));
        xmax = fmax(xmax, fabs(xi.x) + fabs(xi.y));
    }
    dmax = block_max(dmax, red);
    xmax = block_max(xmax, red);
    if (threadIdx.x == 0) {
        rs->dprev = rs->dmax;
        rs->dmax = dmax;
        rs->xmax = xmax;
        rs->rbits = 0ull;
        iters[s] = it;
    }
}



// acc += a * b in double-float (exact product plus cross terms, two-sum)
__device__ __forceinline__ void dfmac(float &sh, float &sl, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float pe = fmaf(ah, bh, -p);
    pe = fmaf(ah, bl, pe);
    pe = fmaf(al, bh, pe);
    const float t = sh + p;
    const float z = t - sh;
    sl += ((sh - (t - z)) + (p - z)) + pe;
    sh = t;
}

// r = g - A x for 64 rows of one system (A column-major, double-float pairs);
// y = P r.  x is split into double-float pairs in shared memory; four column
// phases per row accumulate in double-float and are summed, then subtracted
// from g, in FP64 in a fixed order.
__global__ void __launch_bounds__(256) refine_resid_kernel(
    const int2 *__restrict__ chunks, const int *__restrict__ Ns, const long long *__restrict__ mat_off,
    const int *__restrict__ vec_off, const float4 *__restrict__ A, const int *__restrict__ piv,
    const double2 *__restrict__ G, const double2 *__restrict__ X, float2 *__restrict__ Y32,
    RefineState *__restrict__ st) {
    extern __shared__ float4 xs[];   // x_l as (re hi, re lo, im hi, im lo)
    __shared__ double2 part[4][kResidRows];
    __shared__ double red[32];
    const int2 ch = chunks[blockIdx.x];
    const int s = ch.x, r0 = ch.y;
    if (st[s].conv) return;
    const int n = Ns[s], vo = vec_off[s];
    const float4 *a = A + mat_off[s];
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        const double2 v = X[vo + l];
        const float rh = (float)v.x, ih = (float)v.y;
        xs[l] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
    }
    __syncthreads();
    const int ri = threadIdx.x & (kResidRows - 1), ph = threadIdx.x / kResidRows, i = r0 + ri;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    if (i < n)
        for (int l = ph; l < n; l += 4) {
            const float4 al = __ldcs(a + (long long)l * n + i);
            const float4 xl = xs[l];
            dfmac(rh, rl, al.x, al.y, xl.x, xl.y);      // re += ar xr - ai xi
            dfmac(rh, rl, -al.z, -al.w, xl.z, xl.w);
            dfmac(ih, il, al.x, al.y, xl.z, xl.w);      // im += ar xi + ai xr
            dfmac(ih, il, al.z, al.w, xl.x, xl.y);
        }
    part[ph][ri] = make_double2((double)rh + (double)rl, (double)ih + (double)il);
    __syncthreads();
    double m = 0.0;
    if (ph == 0 && i < n) {
        const double2 gi = G[vo + i];
        const double sr = ((part[0][ri].x + part[1][ri].x) + part[2][ri].x) + part[3][ri].x;
        const double si = ((part[0][ri].y + part[1][ri].y) + part[2][ri].y) + part[3][ri].y;
        const double r_re = gi.x - sr, r_im = gi.y - si;
        Y32[vo + piv[vo + i]] = make_float2((float)r_re, (float)r_im);
        m = fabs(r_re) + fabs(r_im);
    }
    m = block_max(m, red);
    if (threadIdx.x == 0 && m > 0.0)
        atomicMax(&st[s].rbits, (unsigned long long)__double_as_longlong(m));
}

// After the last sweep: convergence verdict and relative residual.
__global__ void refine_final_kernel(const int *__restrict__ order, int S, const RefineState *__restrict__ st,
                                    double tol, double *__restrict__ resid, int *__restrict__ info) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const int s = order[i];
    if (info[s] != 0) return;
    const RefineState r = st[s];
    const double rmax = __longlong_as_double((long long)r.rbits);
    if (!r.conv && !refine_done(r, tol)) info[s] = -1;
    resid[s] = r.gmax > 0.0 ? rmax / r.gmax : 0.0;
}

// FP32 copy: the hi parts of the double-float entries.
__global__ void convert_kernel(const float4 *__restrict__ A, float2 *__restrict__ B, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 v = A[i];
        B[i] = make_float2(v.x, v.z);
    }
}

}  // namespace

void launch_convert_fp32(const float4 *A, float2 *A32, long long n, cudaStream_t st) {
    if (n <= 0) return;
    convert_kernel<<<152 * 8, 256, 0, st>>>(A, A32, n);
}

void launch_lu_factor_fp32(const int *order, int S, const int *N, const long long *mat_off,
                           float2 *A32, int *piv, const int *vec_off, int *info, int maxN,
                           cudaStream_t st) {
    if (S <= 0) return;
    static std::atomic<unsigned long long> attr{0};
    ensure_smem_attr((const void *)lu_factor_fp32_kernel, 64 * 1024, attr);
    lu_factor_fp32_kernel<<<S, 256, maxN * sizeof(int), st>>>(order, N, mat_off, vec_off, A32, piv,
                                                              info);
}

size_t refine_state_bytes(int S) { return (size_t)S * sizeof(RefineState); }

void launch_lu_refine(bool row_major, const int *order, int S, const int *N,
                      const long long *mat_off, const int *vec_off, const int2 *chunks,
                      int n_chunks, const int2 *blocks, int n_blocks, const int *blk_off,
                      float2 *inv, const float4 *A, const float2 *LU32, const int *piv,
                      const double2 *g, double2 *x, float2 *y32, void *state, int max_iters,
                      double tol, int *iters, double *resid, int *info, int maxN, cudaStream_t st) {
    if (S <= 0) return;
    RefineState *rs = static_cast<RefineState *>(state);
    static std::atomic<unsigned long long> attr[3] = {{0}, {0}, {0}};
    ensure_smem_attr((const void *)refine_resid_kernel, 200 * 1024, attr[0]);
    ensure_smem_attr((const void *)refine_solve_kernel<true>, 200 * 1024, attr[1]);
    ensure_smem_attr((const void *)refine_solve_kernel<false>, 200 * 1024, attr[2]);
    if (row_major)
        diag_inverse_kernel<<<n_blocks, 64, 0, st>>>(blocks, N, mat_off, blk_off, LU32, inv);
    refine_setup_kernel<<<S, 256, 0, st>>>(order, N, vec_off, piv, g, x, y32, rs, iters, info);
    for (int it = 1; it <= max_iters; ++it) {
        if (row_major)
            refine_solve_kernel<true><<<S, 512, (size_t)maxN * sizeof(float2), st>>>(
                order, N, mat_off, vec_off, LU32, inv, blk_off, x, y32, rs, it, tol, iters);
        else
            refine_solve_kernel<false><<<S, 256, (size_t)maxN * sizeof(float2), st>>>(
                order, N, mat_off, vec_off, LU32, inv, blk_off, x, y32, rs, it, tol, iters);
        refine_resid_kernel<<<n_chunks, 256, (size_t)maxN * sizeof(float4), st>>>(
            chunks, N, mat_off, vec_off, A, piv, g, x, y32, rs);
    }
    refine_final_kernel<<<(S + 255) / 256, 256, 0, st>>>(order, S, rs, tol, resid, info);
}

}  // namespace fh
