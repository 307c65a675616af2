// Step a3 on the tensor cores: batched complex LU with partial pivoting whose
// trailing updates A22 -= L21 U12 run as tcgen05 MMAs with FP32 accumulation in
// tensor memory; the refinement kernels of k_lu_mixed.cu then restore FP64
// accuracy against the FP64 matrix.
//
// Operands.  With L21 = Lr + i Li and U12 = Ur + i Ui the complex update is one
// real GEMM of inner dimension 2 nb.  K index 2q + {0, 1} holds (Lr, Li) of
// panel column q in A; B holds (Ur, -Ui) in the row that produces Re C and
// (Ui, Ur) in the row that produces Im C.  Interleaving those two B rows per
// complex column makes the accumulator columns come out in the order of the
// row-major complex matrix.  Each FP32 operand is split as hi + lo (hi rounded
// to TF32 or BF16, lo the remainder); hi*hi + hi*lo + lo*hi in one accumulator
// carries about 2^-21 (TF32) or 2^-16 (BF16) relative accuracy.
//
// Layout and parallelism.  The FP32 matrix is row-major.  A system of order n
// is factored by a cluster of cs >= ceil(n / 512) CTAs (1, 2, 4 or 8; more
// than the minimum spreads the trailing updates, lu_tc_cluster) of 512
// threads; thread t of CTA r owns panel row ("slot") 512 r + t, and a CTA
// whose slots are all past the active rows takes part with empty candidates.
// Per panel of
// nb = 32 columns:
//   1. the panel rows are loaded into registers (32 complex per thread) and
//      factored column by column: one arg-max per column over the cluster
//      (warp shuffles, then shared or distributed shared memory) that also
//      carries the winning row, after which every other row is eliminated in
//      registers.  Rows do not move; each thread tracks the position of its
//      row under the LAPACK swap sequence;
//   2. the panel is written to its final rows, and the rows that changed
//      position (at most 2 nb) are permuted in the columns outside the panel,
//      each CTA over its own column range, through shared memory;
//   3. U12 = L11^{-1} A12 by forward substitution, one column per thread, over
//      the same column ranges;
//   4. A22 -= L21 U12: 128-row tiles are dealt round-robin to the CTAs; per
//      row tile the A operand is staged once and 64-column B tiles are
//      double-buffered, so that staging and the epilogue of one tile overlap
//      the MMAs of the next (two 128-column TMEM accumulators).
// Cluster barriers separate the steps; a cluster of one uses __syncthreads.
#include <climits>
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "fh_internal.h"
#include "tc_gemm.cuh"

namespace cg = cooperative_groups;

namespace fh {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int NB = 32;                  // panel width (complex columns)
constexpr int TR = 128;                 // rows per tile (TMEM lanes)
constexpr int TCC = 32;                 // complex columns per tile (64 accumulator columns)
constexpr int kMaxCluster = 8;
constexpr int kMaxMoved = 2 * NB;
constexpr int kATile = TR * 2 * NB * 4;        // A operand (hi or lo) at 4 bytes per element: 32 KiB
constexpr int kBTile = 2 * TCC * 2 * NB * 4;   // B operand (hi or lo): 16 KiB
constexpr int kXPitch = 5;                     // float4 per row of an epilogue transpose buffer
constexpr int kXBytes = kWarps * 32 * kXPitch * 16;   // 40 KiB
constexpr int kDynSmem = 1024 + 2 * kATile + 4 * kBTile + kXBytes;
constexpr long long kWaitLimit = 1LL << 22;

template <int kKind> struct Op;
template <> struct Op<2> {              // TF32
    static constexpr int esize = 4;
    static constexpr int qpc = 2;       // complex panel columns per 16-byte chunk
};
template <> struct Op<1> {              // BF16
    static constexpr int esize = 2;
    static constexpr int qpc = 4;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float tf32_round(float v) {
    uint32_t u = __float_as_uint(v);
    u = (u + 0x1000u) & 0xFFFFE000u;     // round the 13 dropped mantissa bits to nearest
    return __uint_as_float(u);
}

// Split 2*qpc FP32 values into hi and lo 16-byte chunks of the operand type.
template <int kKind>
__device__ __forceinline__ void split_store(const float *v, uint8_t *hi, uint8_t *lo) {
    if constexpr (kKind == 2) {
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = tf32_round(v[e]);
            l[e] = v[e] - h[e];
        }
        *reinterpret_cast<float4 *>(hi) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(lo) = make_float4(l[0], l[1], l[2], l[3]);
    } else {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
            const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * e] - __low2float(hh),
                                                            v[2 * e + 1] - __high2float(hh));
            h[e] = *reinterpret_cast<const uint32_t *>(&hh);
            l[e] = *reinterpret_cast<const uint32_t *>(&ll);
        }
        *reinterpret_cast<uint4 *>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(lo) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Barrier over the system's CTAs.  with_global: also order global-memory
// writes before it for the other CTAs of the cluster.
__device__ __forceinline__ void sys_sync(int cs, bool with_global) {
    if (cs == 1) {
        __syncthreads();
    } else {
        if (with_global) __threadfence();
        cg::this_cluster().sync();
    }
}

// Pivot candidates are packed keys: hi = bits of |a|_1 (monotone for
// non-negative floats; NaN and Inf sort above every finite value), lo = ~row
// position (the smaller position wins a tie); an inactive row has key 0.
struct PanelShared {
    uint32_t kh[2][kWarps], kl[2][kWarps];      // per-warp best keys
    float2 wrow[2][kWarps][NB];                 // cluster of one: warp winners' rows
    uint32_t ckh[2][kMaxCluster], ckl[2][kMaxCluster];
    float2 crow[2][kMaxCluster][NB];            // cluster: CTA winners' rows
    float2 l11[NB][NB + 1];                     // unit lower L11 of the current panel
    int mv_dst[kMaxMoved], mv_src[kMaxMoved];
    int mv_cnt;
    uint64_t bar[2];
    uint32_t tslot;
    int wait_failed;                            // a completion wait of this CTA gave up
};

// Arg-max of packed keys over a warp; returns (hi, lo) of the best.
__device__ __forceinline__ void key_max(uint32_t h, uint32_t l, uint32_t &mh, uint32_t &ml) {
    mh = __reduce_max_sync(0xffffffffu, h);
    ml = __reduce_max_sync(0xffffffffu, h == mh ? l : 0u);
}

// A operand: rows i0 .. i0+127 of L21 (panel columns k0 .. k0+nb-1), K-major.
template <int kKind>
__device__ __forceinline__ void stage_a(const float2 *__restrict__ a, int n, int k0, int nb, int i0,
                                        uint8_t *sh, uint8_t *sl) {
    constexpr int qpc = Op<kKind>::qpc, kChunks = NB / qpc, kRowB = 2 * NB * Op<kKind>::esize;
    for (int e = threadIdx.x; e < TR * kChunks; e += kThreads) {
        const int r = e & (TR - 1), c = e / TR;
        const int i = i0 + r, q0 = c * qpc;
        float v[2 * qpc];
#pragma unroll
        for (int h = 0; h < qpc / 2; ++h) {
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n && q0 + 2 * h < nb)
                t = __ldcg(reinterpret_cast<const float4 *>(a + (long long)i * n + k0 + q0 + 2 * h));
            v[4 * h] = t.x;
            v[4 * h + 1] = t.y;
            v[4 * h + 2] = t.z;
            v[4 * h + 3] = t.w;
        }
        const uint32_t off = tc::kmajor_offset(r, c * 16, kRowB);
        split_store<kKind>(v, sh + off, sl + off);
    }
}

// B operand for complex columns j0 .. j0+TCC-1 of U12: row 2jj gives Re, row
// 2jj+1 gives Im of output column j0+jj.  load_b reads this thread's
// kBElems elements (qpc complex values each) into registers, store_b splits
// them into the K-major hi and lo tiles, so that the loads of the next tile
// can be in flight during the current tile's epilogue.
template <int kKind>
struct BRegs {
    static constexpr int qpc = Op<kKind>::qpc, kChunks = NB / qpc;
    static constexpr int kElems = 2 * TCC * kChunks / kThreads;
    float2 u[kElems][qpc];
};

template <int kKind>
__device__ __forceinline__ void load_b(const float2 *__restrict__ a, int n, int k0, int nb, int j0,
                                       BRegs<kKind> &rb) {
    constexpr int qpc = Op<kKind>::qpc;
#pragma unroll
    for (int m = 0; m < BRegs<kKind>::kElems; ++m) {
        const int e = threadIdx.x + m * kThreads;
        const int b = e & (2 * TCC - 1), c = e / (2 * TCC);
        const int j = j0 + (b >> 1), q0 = c * qpc;
#pragma unroll
        for (int h = 0; h < qpc; ++h)
            rb.u[m][h] = (j < n && q0 + h < nb) ? __ldcg(a + (long long)(k0 + q0 + h) * n + j)
                                                : make_float2(0.f, 0.f);
    }
}

template <int kKind>
__device__ __forceinline__ void store_b(const BRegs<kKind> &rb, uint8_t *sh, uint8_t *sl) {
    constexpr int qpc = Op<kKind>::qpc, kRowB = 2 * NB * Op<kKind>::esize;
#pragma unroll
    for (int m = 0; m < BRegs<kKind>::kElems; ++m) {
        const int e = threadIdx.x + m * kThreads;
        const int b = e & (2 * TCC - 1), c = e / (2 * TCC);
        const bool im = b & 1;
        float v[2 * qpc];
#pragma unroll
        for (int h = 0; h < qpc; ++h) {
            const float2 u = rb.u[m][h];
            v[2 * h] = im ? u.y : u.x;
            v[2 * h + 1] = im ? u.x : -u.y;
        }
        const uint32_t off = tc::kmajor_offset(b, c * 16, kRowB);
        split_store<kKind>(v, sh + off, sl + off);
    }
}

// One 128 x 64 complex tile: hi*hi + hi*lo + lo*hi over the panel's K.
template <int kKind>
__device__ __forceinline__ void issue_mma(uint32_t tacc, uint32_t ah, uint32_t al, uint32_t bh,
                                          uint32_t bl, uint64_t *bar) {
    constexpr int kRowB = 2 * NB * Op<kKind>::esize;
    constexpr uint32_t sbo = (kRowB / 16) * 128;
    constexpr int ksteps = kRowB / 32;          // 32 bytes of K per MMA
    constexpr uint32_t idesc = tc::instr_desc(kKind == 2 ? 2u : 1u, TR, 2 * TCC);
#pragma unroll
    for (int ks = 0; ks < ksteps; ++ks) {
        const uint32_t o = (uint32_t)ks * 256u;
        const uint64_t dah = tc::smem_desc(ah + o, 128, sbo), dal = tc::smem_desc(al + o, 128, sbo);
        const uint64_t dbh = tc::smem_desc(bh + o, 128, sbo), dbl = tc::smem_desc(bl + o, 128, sbo);
        tc::mma<kKind>(tacc, dah, dbh, idesc, ks > 0 ? 1u : 0u);
        tc::mma<kKind>(tacc, dah, dbl, idesc, 1u);
        tc::mma<kKind>(tacc, dal, dbh, idesc, 1u);
    }
    tc::mma_commit(bar);
}

// C(i0.., j0..) -= accumulator.  Warp w owns TMEM lanes 32 (w % 4) .. and
// accumulator columns 16 (w / 4) .. (8 complex columns of each of its 32
// rows).  C is read eight rows at a time, four lanes covering the 64
// contiguous bytes of a row (epi_load, issued before the MMA wait); the
// accumulator is passed through the warp's shared-memory buffer into the same
// lane pattern (epi_store).
__device__ __forceinline__ void epi_load(const float2 *__restrict__ a, int n, int i0, int j0, float4 (&c)[4]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wq = warp & 3, wc = warp >> 2;
    const int j = j0 + 8 * wc + 2 * (lane & 3);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = i0 + 32 * wq + 8 * p + (lane >> 2);
        c[p] = (i < n && j < n) ? __ldcg(reinterpret_cast<const float4 *>(a + (long long)i * n + j))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ void epi_store(float2 *__restrict__ a, int n, int i0, int j0, uint32_t tacc,
                                          float4 *sX, const float4 (&c)[4]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wq = warp & 3, wc = warp >> 2;
    float d[16];
    tc::tmem_ld16(tacc + ((uint32_t)(32 * wq) << 16) + (uint32_t)(wc * 16), d);
    float4 *buf = sX + warp * 32 * kXPitch;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        buf[lane * kXPitch + k] = make_float4(d[4 * k], d[4 * k + 1], d[4 * k + 2], d[4 * k + 3]);
    __syncwarp();
    const int k = lane & 3, j = j0 + 8 * wc + 2 * k;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int rr = 8 * p + (lane >> 2), i = i0 + 32 * wq + rr;
        if (i < n && j < n) {
            const float4 dv = buf[rr * kXPitch + k];
            __stcg(reinterpret_cast<float4 *>(a + (long long)i * n + j),
                   make_float4(c[p].x - dv.x, c[p].y - dv.y, c[p].z - dv.z, c[p].w - dv.w));
        }
    }
    __syncwarp();
}

// Pointer into the shared memory of CTA r of this system's cluster.
template <typename T>
__device__ __forceinline__ T *at_rank(T *p, int cs, int r) {
    return cs == 1 ? p : cg::this_cluster().map_shared_rank(p, (unsigned)r);
}

// Blocks [cs * c, cs * c + cs) factor system order[c].  On return piv holds
// the inverse row permutation (original row i is row piv[i] of the factors).
template <int kKind, bool kMulti>
__global__ void __launch_bounds__(kThreads, 1) lu_factor_tc_kernel(
    const int *__restrict__ order, int cs_arg, const int *__restrict__ Ns,
    const long long *__restrict__ mat_off, const int *__restrict__ vec_off,
    float2 *__restrict__ A32, int *__restrict__ piv, int *__restrict__ info,
    int *__restrict__ err) {
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(16) PanelShared ps;
    uint8_t *stage = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    uint8_t *sAh = stage, *sAl = stage + kATile;
    uint8_t *sB = stage + 2 * kATile;                                   // 2 x (hi, lo)
    float4 *sX = reinterpret_cast<float4 *>(sB + 4 * kBTile);           // epilogue transposes
    float4 *gbuf = reinterpret_cast<float4 *>(sB);                      // row gather (B + X)
    constexpr int kGather = (4 * kBTile + kXBytes) / 16;                // float4 in gbuf

    const int cs = kMulti ? cs_arg : 1;
    const int rank = kMulti ? (int)cg::this_cluster().block_rank() : 0;
    const int s = order[blockIdx.x / cs];
    const int n = Ns[s];
    float2 *a = A32 + mat_off[s];
    int *pv = piv + vec_off[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int myslot = rank * kThreads + tid;

    if (warp == 0) tc::tmem_alloc(&ps.tslot, 4 * TCC);
    if (tid == 0) {
        tc::mbar_init(&ps.bar[0], 1);
        tc::mbar_init(&ps.bar[1], 1);
        ps.wait_failed = 0;
    }
    if (rank == 0)   // pv: factored position -> original row, while factoring
        for (int i = tid; i < n; i += kThreads) pv[i] = i;
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = ps.tslot;
    if (cs > 1) cg::this_cluster().sync();   // every CTA running before shared memory is addressed remotely

    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool failed = false, bad = false;
    int bsel = 0;

    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nb = min(NB, n - k0), m = n - k0;
        if (tid == 0) ps.mv_cnt = 0;
        const bool own = myslot < m;
        float2 v[NB];
        {
            const float4 *src = reinterpret_cast<const float4 *>(a + (long long)(k0 + (own ? myslot : 0)) * n + k0);
#pragma unroll
            for (int h = 0; h < NB / 2; ++h) {
                const float4 t = (own && 2 * h < nb) ? __ldcg(src + h) : make_float4(0.f, 0.f, 0.f, 0.f);
                v[2 * h] = make_float2(t.x, t.y);
                v[2 * h + 1] = make_float2(t.z, t.w);
            }
        }
        int mypos = myslot;
        bool active = own;

        // 1. panel factorisation in registers
#pragma unroll
        for (int cl = 0; cl < NB; ++cl) {
            if (cl >= nb || bad) continue;
            const int pb = cl & 1;
            const uint32_t khi = active ? __float_as_uint(fabsf(v[cl].x) + fabsf(v[cl].y)) : 0u;
            const uint32_t klo = active ? ~(uint32_t)mypos : 0u;
            uint32_t mh, ml;
            key_max(khi, klo, mh, ml);
            if (lane == 0) {
                ps.kh[pb][warp] = mh;
                ps.kl[pb][warp] = ml;
            }
            const float2 *row;
            if constexpr (!kMulti) {
                if (active && khi == mh && klo == ml) {   // this warp's best row
                    float4 *dst = reinterpret_cast<float4 *>(ps.wrow[pb][warp]);
#pragma unroll
                    for (int h = cl / 2; h < NB / 2; ++h)
                        dst[h] = make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
                }
                __syncthreads();
                const uint32_t h2 = lane < kWarps ? ps.kh[pb][lane] : 0u;
                const uint32_t l2 = lane < kWarps ? ps.kl[pb][lane] : 0u;
                key_max(h2, l2, mh, ml);
                const uint32_t hit = __ballot_sync(0xffffffffu, lane < kWarps && h2 == mh && l2 == ml);
                row = ps.wrow[pb][__ffs(hit) - 1];
            } else {
                __syncthreads();
                const uint32_t h2 = lane < kWarps ? ps.kh[pb][lane] : 0u;
                const uint32_t l2 = lane < kWarps ? ps.kl[pb][lane] : 0u;
                key_max(h2, l2, mh, ml);
                if (active && khi == mh && klo == ml)     // this CTA's best row, to every CTA
                    for (int r = 0; r < cs; ++r) {
                        *at_rank(&ps.ckh[pb][rank], cs, r) = mh;
                        *at_rank(&ps.ckl[pb][rank], cs, r) = ml;
                        float4 *dst = reinterpret_cast<float4 *>(at_rank(&ps.crow[pb][rank][0], cs, r));
#pragma unroll
                        for (int h = cl / 2; h < NB / 2; ++h)
                            dst[h] = make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
                    }
                if (mh == 0u && ml == 0u && tid == 0)    // no row of this CTA is left: empty candidate
                    for (int r = 0; r < cs; ++r) {
                        *at_rank(&ps.ckh[pb][rank], cs, r) = 0u;
                        *at_rank(&ps.ckl[pb][rank], cs, r) = 0u;
                    }
                sys_sync(cs, false);
                const uint32_t h3 = lane < cs ? ps.ckh[pb][lane] : 0u;
                const uint32_t l3 = lane < cs ? ps.ckl[pb][lane] : 0u;
                key_max(h3, l3, mh, ml);
                const uint32_t hit = __ballot_sync(0xffffffffu, lane < cs && h3 == mh && l3 == ml);
                row = ps.crow[pb][__ffs(hit) - 1];
            }
            // zero or non-finite pivot, or no row left: the same verdict in every CTA
            if (ml == 0u || mh == 0u || mh >= 0x7F800000u) {
                if (rank == 0 && tid == 0) info[s] = k0 + cl + 1;
                bad = true;
                continue;
            }
            const int wpos = (int)~ml;
            const float2 pvt = row[cl];
            const float rd = 1.f / (pvt.x * pvt.x + pvt.y * pvt.y);
            const float2 pinv = make_float2(pvt.x * rd, -pvt.y * rd);
            if (active && mypos == wpos) {
                mypos = cl;
                active = false;
            } else if (active && mypos == cl) {
                mypos = wpos;        // swapped with the pivot row's position
            }
            if (active) {
                const float2 l = cmul(v[cl], pinv);
                v[cl] = l;
#pragma unroll
                for (int q = cl + 1; q < NB; ++q) {
                    const float2 u = row[q];
                    v[q].x -= l.x * u.x - l.y * u.y;
                    v[q].y -= l.x * u.y + l.y * u.x;
                }
            }
        }
        if (bad) break;

        // 2. panel to its final rows; L11 and the moved rows to every CTA
        if (own) {
            float4 *dst = reinterpret_cast<float4 *>(a + (long long)(k0 + mypos) * n + k0);
#pragma unroll
            for (int h = 0; h < NB / 2; ++h)
                if (2 * h < nb) __stcg(dst + h, make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y));
            if (mypos < nb)
                for (int r = 0; r < cs; ++r) {
                    float2 *l = at_rank(&ps.l11[mypos][0], cs, r);
#pragma unroll
                    for (int q = 0; q < NB; ++q)
                        if (q < mypos) l[q] = v[q];
                }
            if (mypos != myslot)
                for (int r = 0; r < cs; ++r) {
                    const int idx = atomicAdd(at_rank(&ps.mv_cnt, cs, r), 1);
                    if (idx < kMaxMoved) {   // at most 2 nb rows change position
                        *at_rank(&ps.mv_dst[idx], cs, r) = mypos;
                        *at_rank(&ps.mv_src[idx], cs, r) = myslot;
                    }
                }
        }
        sys_sync(cs, true);

        // column range of this CTA outside the panel: c in [0, n - nb), column
        // c < k0 ? c : c + nb
        const int ncs = n - nb;
        const int W = (((ncs + cs - 1) / cs) + 1) & ~1;
        const int c_lo = min(ncs, rank * W), c_hi = min(ncs, c_lo + W);
        const int nmv = min(ps.mv_cnt, kMaxMoved);
        if (nmv > 0) {
            int t_perm = 0;
            if (rank == 0 && tid < nmv) t_perm = pv[k0 + ps.mv_src[tid]];
            const int CW2 = kGather / nmv;      // float4 (two columns) per moved row and chunk
            for (int cb = c_lo; cb < c_hi; cb += 2 * CW2) {
                const int cw2 = min(2 * CW2, c_hi - cb) / 2;
                const int tot = nmv * cw2;
                for (int e = tid; e < tot; e += kThreads) {
                    const int p = e / cw2, c = cb + 2 * (e - p * cw2);
                    const int j = c < k0 ? c : c + nb;
                    gbuf[e] = __ldcg(reinterpret_cast<const float4 *>(a + (long long)(k0 + ps.mv_src[p]) * n + j));
                }
                __syncthreads();
                for (int e = tid; e < tot; e += kThreads) {
                    const int p = e / cw2, c = cb + 2 * (e - p * cw2);
                    const int j = c < k0 ? c : c + nb;
                    __stcg(reinterpret_cast<float4 *>(a + (long long)(k0 + ps.mv_dst[p]) * n + j), gbuf[e]);
                }
                __syncthreads();
            }
            if (rank == 0) {
                __syncthreads();
                if (tid < nmv) pv[k0 + ps.mv_dst[tid]] = t_perm;
            }
        }

        // 3. U12 = L11^{-1} A12 over this CTA's columns right of the panel
        // (blocks of 8 rows; finished blocks are re-read from memory, which
        // keeps the register footprint at 8 complex values)
        for (int c = max(c_lo, k0) + tid; c < c_hi; c += kThreads) {
            float2 *col = a + (long long)k0 * n + c + nb;
#pragma unroll
            for (int B = 0; B < NB / 8; ++B) {
                if (8 * B >= nb) continue;
                float2 xb[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    xb[e] = 8 * B + e < nb ? __ldcg(col + (long long)(8 * B + e) * n) : make_float2(0.f, 0.f);
#pragma unroll
                for (int C = 0; C < B; ++C)
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float2 xq = col[(long long)(8 * C + q) * n];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const float2 l = ps.l11[8 * B + e][8 * C + q];
                            xb[e].x -= l.x * xq.x - l.y * xq.y;
                            xb[e].y -= l.x * xq.y + l.y * xq.x;
                        }
                    }
#pragma unroll
                for (int q = 0; q < 8; ++q)
#pragma unroll
                    for (int e = q + 1; e < 8; ++e) {
                        const float2 l = ps.l11[8 * B + e][8 * B + q];
                        xb[e].x -= l.x * xb[q].x - l.y * xb[q].y;
                        xb[e].y -= l.x * xb[q].y + l.y * xb[q].x;
                    }
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (8 * B + e < nb) col[(long long)(8 * B + e) * n] = xb[e];
            }
        }
        sys_sync(cs, true);

        // 4. A22 -= L21 U12 on the tensor cores
        const int r0 = k0 + nb, m2 = n - r0;
        if (m2 > 0) {
            const int nrt = (m2 + TR - 1) / TR, nct = (m2 + TCC - 1) / TCC;
            for (int rt = rank; rt < nrt; rt += cs) {
                const int i0 = r0 + rt * TR;
                BRegs<kKind> rb;
                load_b<kKind>(a, n, k0, nb, r0, rb);            // first column tile
                stage_a<kKind>(a, n, k0, nb, i0, sAh, sAl);
                int prev = -1, prev_j0 = 0;
                float4 cprev[4], ccur[4];
                for (int ct = 0; ct <= nct; ++ct) {
                    const int b = bsel;
                    const int j0 = r0 + ct * TCC;
                    if (ct < nct) {
                        uint8_t *bh = sB + 2 * b * kBTile, *bl = bh + kBTile;
                        store_b<kKind>(rb, bh, bl);
                        tc::fence_async_smem();
                        tc::tc_fence_before();
                        __syncthreads();
                        tc::tc_fence_after();
                        if (ps.wait_failed) failed = true;   // the same verdict in every thread
                        const bool issue = !failed;
                        if (tid == 0 && issue)
                            issue_mma<kKind>(taddr + (uint32_t)(b * 2 * TCC), tc::smem_u32(sAh), tc::smem_u32(sAl),
                                             tc::smem_u32(bh), tc::smem_u32(bl), &ps.bar[b]);
                        pending[b] = issue;
                        bsel ^= 1;
                        // in flight while this tile multiplies and the previous one is
                        // written back: the next tile's B and this tile's C
                        if (ct + 1 < nct) load_b<kKind>(a, n, k0, nb, j0 + TCC, rb);
                        epi_load(a, n, i0, j0, ccur);
                    }
                    if (prev >= 0) {   // epilogue of the previous tile while this one multiplies
                        // every thread waits for the completion itself (no barrier): its
                        // accumulator reads and the reuse of the tile's B buffer two tiles
                        // later follow its own wait; a give-up is shared through
                        // ps.wait_failed at the next barrier
                        bool got = true;
                        if (pending[prev]) {
                            got = tc::mbar_wait(&ps.bar[prev], phase[prev], kWaitLimit);
                            phase[prev] ^= 1u;
                            pending[prev] = false;
                        }
                        tc::tc_fence_after();
                        if (!got) {
                            failed = true;
                            ps.wait_failed = 1;
                        }
                        if (!failed) epi_store(a, n, i0, prev_j0, taddr + (uint32_t)(prev * 2 * TCC), sX, cprev);
                        tc::tc_fence_before();
                    }
#pragma unroll
                    for (int p = 0; p < 4; ++p) cprev[p] = ccur[p];
                    prev = b;
                    prev_j0 = j0;
                }
            }
        }
        sys_sync(cs, true);
    }

    __syncthreads();
    if (ps.wait_failed) failed = true;
    // after a failed wait, let any MMA still in flight finish before freeing
    for (int b = 0; b < 2; ++b)
        if (pending[b]) {
            tc::mbar_wait(&ps.bar[b], phase[b], kWaitLimit);
            pending[b] = false;
        }
    if (failed && tid == 0) {
        atomicOr(err, 1);
        info[s] = -2;
    }
    if (!bad && rank == 0) {   // position -> row  into  row -> position
        int *perm = reinterpret_cast<int *>(sAh);
        __syncthreads();
        for (int i = tid; i < n; i += kThreads) perm[i] = pv[i];
        __syncthreads();
        for (int i = tid; i < n; i += kThreads) pv[perm[i]] = i;
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(taddr, 4 * TCC);
    if (cs > 1) cg::this_cluster().sync();   // no CTA leaves while its shared memory may be addressed
}

// Row-major FP32 copy (the hi parts) of the column-major double-float
// matrices (32 x 32 tiles).
__global__ void __launch_bounds__(256) convert_rowmajor_kernel(const int *__restrict__ list,
                                                               const int *__restrict__ Ns,
                                                               const long long *__restrict__ mat_off,
                                                               const float4 *__restrict__ A,
                                                               float2 *__restrict__ A32) {
    __shared__ float2 t[32][33];
    const int s = list[blockIdx.x], n = Ns[s];
    const float4 *src = A + mat_off[s];
    float2 *dst = A32 + mat_off[s];
    const int nt = (n + 31) / 32;
    for (int tile = blockIdx.y; tile < nt * nt; tile += gridDim.y) {
        const int ti = tile % nt, tj = tile / nt;
        for (int k = threadIdx.y; k < 32; k += 8) {
            const int l = tj * 32 + k, i = ti * 32 + threadIdx.x;
            if (l < n && i < n) {
                const float4 v = src[(long long)l * n + i];   // (re hi, re lo, im hi, im lo)
                t[k][threadIdx.x] = make_float2(v.x, v.z);
            }
        }
        __syncthreads();
        for (int k = threadIdx.y; k < 32; k += 8) {
            const int i = ti * 32 + k, l = tj * 32 + threadIdx.x;
            if (i < n && l < n) dst[(long long)i * n + l] = t[threadIdx.x][k];
        }
        __syncthreads();
    }
}

template <int kKind>
cudaError_t launch_group(const int *order, int count, int cs, const int *N, const long long *mat_off,
                         float2 *A32, int *piv, const int *vec_off, int *info, int *err, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * cs));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kDynSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cs == 1)
        return cudaLaunchKernelEx(&cfg, lu_factor_tc_kernel<kKind, false>, order, cs, N, mat_off,
                                  vec_off, A32, piv, info, err);
    return cudaLaunchKernelEx(&cfg, lu_factor_tc_kernel<kKind, true>, order, cs, N, mat_off, vec_off,
                              A32, piv, info, err);
}

}  // namespace

// Every CTA owns kThreads = 512 panel rows, so at least ceil(n / 512) CTAs;
// smaller rows_per_cta spreads the trailing updates over more CTAs.
int lu_tc_cluster(int n, int rows_per_cta) {
    const int rows = rows_per_cta >= kThreads ? kThreads : rows_per_cta >= 256 ? 256 : 128;
    const int need = (n + rows - 1) / rows;
    int cs = 1;
    while (cs < need && cs < 8) cs *= 2;
    return cs;
}

int lu_tc_launches(const int *order_h, const int *N_h, int S, int rows_per_cta) {
    int count = 0;
    for (int i = 0; i < S; ++i)
        if (i == 0 || lu_tc_cluster(N_h[order_h[i]], rows_per_cta) !=
                          lu_tc_cluster(N_h[order_h[i - 1]], rows_per_cta))
            ++count;
    return count;
}

void launch_convert_rowmajor(const int *list, int count, const int *N, const long long *mat_off,
                             const float4 *A, float2 *A32, cudaStream_t st) {
    if (count <= 0) return;
    convert_rowmajor_kernel<<<dim3(count, 16), dim3(32, 8), 0, st>>>(list, N, mat_off, A, A32);
}

cudaError_t launch_lu_factor_tc(int kind, int rows_per_cta, const int *order, const int *order_h,
                                const int *N_h, int S,
                                const int *N, const long long *mat_off, float2 *A32, int *piv,
                                const int *vec_off, int *info, int *err, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    static std::atomic<unsigned long long> attr[4] = {{0}, {0}, {0}, {0}};
    {
        const void *fns[4] = {(const void *)lu_factor_tc_kernel<2, false>, (const void *)lu_factor_tc_kernel<2, true>,
                              (const void *)lu_factor_tc_kernel<1, false>, (const void *)lu_factor_tc_kernel<1, true>};
        for (int f = kind == 2 ? 0 : 2, e0 = f + 2; f < e0; ++f) {
            const cudaError_t e = ensure_smem_attr(fns[f], kDynSmem, attr[f]);
            if (e != cudaSuccess) return e;
        }
    }
    // order is sorted by decreasing N, so each cluster size is a contiguous run
    for (int first = 0; first < S;) {
        const int cs = lu_tc_cluster(N_h[order_h[first]], rows_per_cta);
        int last = first;
        while (last < S && lu_tc_cluster(N_h[order_h[last]], rows_per_cta) == cs) ++last;
        const cudaError_t e = kind == 2
            ? launch_group<2>(order + first, last - first, cs, N, mat_off, A32, piv, vec_off, info, err, st)
            : launch_group<1>(order + first, last - first, cs, N, mat_off, A32, piv, vec_off, info, err, st);
        if (e != cudaSuccess) return e;
        first = last;
    }
    return cudaSuccess;
}

}  // namespace fh
