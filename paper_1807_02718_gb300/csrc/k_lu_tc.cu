// Step a3 on the tensor cores: complex LU with partial pivoting whose trailing
// updates A22 -= L21 U12 run as tcgen05 MMAs (TF32 operands, FP32 accumulation
// in tensor memory); the refinement kernel of k_lu_mixed.cu then restores
// FP64 accuracy against the FP64 matrix.
//
// With L21 = Lr + i Li (m x nb) and U12 = Ur + i Ui (nb x m) the complex
// product is one real GEMM with K = 2 nb:
//   [Cr | Ci] -= [Lr | Li] [[Ur, Ui], [-Ui, Ur]].
// Each operand is split as x = hi + lo with hi = x rounded to TF32 and lo the
// FP32 remainder; hi*hi + hi*lo + lo*hi (three MMAs into one accumulator)
// carries ~FP32 accuracy ("3xTF32"), so refinement converges as fast as after
// an FP32 factorisation.
//
// One CTA (256 threads) per system, largest first.  Panel factorisation and
// the U12 solve are FP32 SIMT (as in lu_factor_fp32_kernel); per panel step
// the trailing matrix is covered by 128-row tiles x pairs of 128-column
// tiles, each pair accumulating in two 128 x 256 FP32 TMEM tiles (512
// columns).  Operands are staged by the threads into K-major shared-memory
// tiles (K chunks of 16 FP32); one thread issues the MMAs and commits them to
// an mbarrier; warps 0-3 and 4-7 apply the two accumulators to A22.
#include <algorithm>

#include "fh_internal.h"
#include "tc_gemm.cuh"

namespace fh {
namespace {

constexpr int NB = 32;                  // panel width (complex columns)
constexpr int KR = 2 * NB;              // real K of the trailing GEMM
constexpr int KC = 16;                  // FP32 K elements per shared stage
constexpr int KCB = KC * 4;             // bytes per row per stage
constexpr int TR = 128;                 // rows per tile (TMEM lanes)
constexpr int TCX = 128;                // complex columns per accumulator (256 TMEM columns)
constexpr long long kWaitLimit = 1LL << 22;

// shared-memory stage layout (bytes)
constexpr int kAT = TR * KCB;           // one A tile (hi or lo): 8 KiB
constexpr int kBT = 2 * TCX * KCB;      // one B tile (hi or lo), 256 rows: 16 KiB
constexpr int kStage = 2 * kAT + 4 * kBT;   // A hi/lo + two column tiles x B hi/lo: 80 KiB

__device__ __forceinline__ float tf32_hi(float v) {
    uint32_t u = __float_as_uint(v);
    u = (u + 0x1000u) & 0xFFFFE000u;     // round the 13 dropped mantissa bits to nearest
    return __uint_as_float(u);
}

__device__ __forceinline__ void put_split(uint8_t *hi, uint8_t *lo, uint32_t off, float v) {
    const float h = tf32_hi(v);
    *reinterpret_cast<float *>(hi + off) = h;
    *reinterpret_cast<float *>(lo + off) = v - h;
}

__global__ void __launch_bounds__(256, 1) lu_factor_tc_kernel(
    const int *__restrict__ order, const int *__restrict__ Ns,
    const long long *__restrict__ mat_off, const int *__restrict__ vec_off,
    float2 *__restrict__ A32, int *__restrict__ piv, int *__restrict__ info,
    int *__restrict__ err) {
    extern __shared__ uint8_t dsm[];
    uint8_t *stage = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    uint8_t *sAh = stage, *sAl = stage + kAT;
    uint8_t *sBh[2] = {stage + 2 * kAT, stage + 2 * kAT + 2 * kBT};
    uint8_t *sBl[2] = {stage + 2 * kAT + kBT, stage + 2 * kAT + 3 * kBT};
    int *perm = reinterpret_cast<int *>(stage + kStage);
    __shared__ float red_v[8];
    __shared__ int red_i[8];
    __shared__ int sh_piv, sh_bad;
    __shared__ float2 sh_val;
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;

    const int s = order[blockIdx.x];
    const int n = Ns[s];
    float2 *a = A32 + mat_off[s];
    int *pv = piv + vec_off[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = tslot;
    constexpr uint32_t idesc = tc::instr_desc(2u, TR, 2 * TCX);
    constexpr uint32_t sboA = (KCB / 16) * 128;
    uint32_t phase = 0;
    bool failed = false;

#define AT(i, j) a[(long long)(j) * n + (i)]
    for (int k0 = 0; k0 < n && !failed; k0 += NB) {
        const int nb = min(NB, n - k0);
        // ---- panel factorisation (FP32, SIMT) ----
        for (int c = k0; c < k0 + nb; ++c) {
            float best = -1.f;
            int bi = n;
            for (int r = c + tid; r < n; r += 256) {
                const float2 v = AT(r, c);
                const float mg = fabsf(v.x) + fabsf(v.y);
                if (mg > best) { best = mg; bi = r; }
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
            if (sh_bad) { failed = true; break; }
            const int p = sh_piv;
            if (p != c)
                for (int j = tid; j < n; j += 256) {
                    const float2 t0 = AT(c, j);
                    AT(c, j) = AT(p, j);
                    AT(p, j) = t0;
                }
            __syncthreads();
            const float2 pinv = sh_val;
            for (int r = c + 1 + tid; r < n; r += 256) {
                const float2 v = AT(r, c);
                AT(r, c) = make_float2(v.x * pinv.x - v.y * pinv.y, v.x * pinv.y + v.y * pinv.x);
            }
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
        if (failed) break;
        // ---- U12 = L11^{-1} A12 ----
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
        // ---- trailing update on the tensor cores ----
        const int r0 = k0 + nb;
        for (int rt = r0; rt < n && !failed; rt += TR) {
            for (int ct = r0; ct < n && !failed; ct += 2 * TCX) {
                for (int ch = 0; ch < KR / KC; ++ch) {
                    // real K index kk = ch*KC + e: panel column q = kk mod NB,
                    // real part for kk < NB, imaginary part otherwise
                    const bool imag = ch * KC >= NB;
                    const int q0 = ch * KC - (imag ? NB : 0);
                    if (tid < TR) {                       // A rows: [Lr | Li]
                        const int i = rt + tid;
                        for (int e = 0; e < KC; ++e) {
                            const int q = q0 + e;
                            float v = 0.f;
                            if (i < n && q < nb) {
                                const float2 l = AT(i, k0 + q);
                                v = imag ? l.y : l.x;
                            }
                            put_split(sAh, sAl, tc::kmajor_offset(tid, e * 4, KCB), v);
                        }
                    }
                    {                                     // B rows: one complex column per thread
                        const int t = tid >> 7, jl = tid & 127;
                        const int j = ct + t * TCX + jl;
                        for (int e = 0; e < KC; ++e) {
                            const int q = q0 + e;
                            float br = 0.f, bi = 0.f;     // rows for the Cr and Ci outputs
                            if (j < n && q < nb) {
                                const float2 u = AT(k0 + q, j);
                                br = imag ? -u.y : u.x;
                                bi = imag ? u.x : u.y;
                            }
                            put_split(sBh[t], sBl[t], tc::kmajor_offset(jl, e * 4, KCB), br);
                            put_split(sBh[t], sBl[t], tc::kmajor_offset(TCX + jl, e * 4, KCB), bi);
                        }
                    }
                    tc::fence_async_smem();
                    __syncthreads();
                    if (tid == 0) {
                        tc::tc_fence_after();
#pragma unroll
                        for (int ks = 0; ks < KC / 8; ++ks) {
                            const uint32_t off = ks * 256;
                            const uint64_t ah = tc::smem_desc(tc::smem_u32(sAh) + off, 128, sboA);
                            const uint64_t al = tc::smem_desc(tc::smem_u32(sAl) + off, 128, sboA);
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                const uint64_t bh = tc::smem_desc(tc::smem_u32(sBh[t]) + off, 128, sboA);
                                const uint64_t bl = tc::smem_desc(tc::smem_u32(sBl[t]) + off, 128, sboA);
                                const uint32_t d = taddr + (uint32_t)(t * 2 * TCX);
                                const uint32_t acc0 = (ch > 0 || ks > 0) ? 1u : 0u;
                                tc::mma<2>(d, ah, bh, idesc, acc0);
                                tc::mma<2>(d, ah, bl, idesc, 1u);
                                tc::mma<2>(d, al, bh, idesc, 1u);
                            }
                        }
                        tc::mma_commit(&bar);
                    }
                    const bool got = tc::mbar_wait(&bar, phase, kWaitLimit);
                    phase ^= 1;
                    tc::tc_fence_after();
                    if (!__syncthreads_and(got)) {
                        failed = true;
                        if (tid == 0) { atomicOr(err, 1); info[s] = -2; }
                        break;
                    }
                }
                if (failed) break;
                // epilogue: warps 0-3 apply accumulator 0, warps 4-7 accumulator 1
                {
                    const int t = warp >> 2, qd = warp & 3;
                    const int i = rt + qd * 32 + lane;
                    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
                    for (int c16 = 0; c16 < TCX; c16 += 16) {
                        float cr[16], ci[16];
                        tc::tmem_ld16(taddr + lane_base + (uint32_t)(t * 2 * TCX + c16), cr);
                        tc::tmem_ld16(taddr + lane_base + (uint32_t)(t * 2 * TCX + TCX + c16), ci);
                        if (i < n)
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                const int j = ct + t * TCX + c16 + e;
                                if (j < n) {
                                    float2 v = AT(i, j);
                                    v.x -= cr[e];
                                    v.y -= ci[e];
                                    AT(i, j) = v;
                                }
                            }
                    }
                }
                tc::tc_fence_before();
                __syncthreads();
            }
        }
    }
#undef AT
    if (failed) {
        // let any MMA still in flight complete before the tensor memory is freed
        tc::mbar_wait(&bar, phase ^ 1, kWaitLimit);
    } else {
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
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(taddr, 512);
}

}  // namespace

void launch_lu_factor_tc(const int *order, int S, const int *N, const long long *mat_off,
                         float2 *A32, int *piv, const int *vec_off, int *info, int *err, int maxN,
                         cudaStream_t st) {
    if (S <= 0) return;
    // >= 120 KiB keeps one CTA per SM, so a CTA never waits for the other's
    // 512 tensor-memory columns
    const size_t smem = std::max<size_t>(120 * 1024, 1024 + (size_t)kStage + (size_t)maxN * sizeof(int));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(lu_factor_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    lu_factor_tc_kernel<<<S, 256, smem, st>>>(order, N, mat_off, vec_off, A32, piv, info, err);
}

}  // namespace fh
