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
//   4. A22 -= L21 U12: the items (128-row tile, 32-column tile) are split
//      evenly over the CTAs in row-tile order and processed by warp roles over a two-stage pipeline (TMEM accumulators
//      and output tiles) fed by a ring of two (TF32) or six (BF16) B tiles:
//      one thread (the producer) brings in the operand tiles with the TMA
//      engine -- the split L21 rows (bulk copy, once per row tile) and the
//      split U12 columns (bulk copy, per 32-column tile), both written in the
//      MMA's shared-memory layout by steps 2 and 3 -- one thread issues the
//      MMAs into the stage's accumulator, one group of four epilogue warps per
//      stage writes the negated accumulator into the stage's shared-memory
//      tile (128-byte swizzle), and one thread adds that tile into the
//      row-major matrix with a tiled tensor reduction (FP32 add at L2), so
//      that C is never loaded into the SM.  Stages are handed over through
//      mbarriers (bounded waits).
// Cluster barriers separate the steps; a cluster of one uses __syncthreads.
#include <climits>
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>
#include <type_traits>

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
constexpr int kMaxStages = 3;           // pipeline depth of the trailing update (C tiles, accumulators)
constexpr int kMaxBStages = 6;          // depth of the ring of B operand tiles
constexpr int kMaxCluster = 8;
constexpr int kMaxMoved = 2 * NB;
constexpr int kCBox = TR * 32 * 4;             // one 128 x 32-float box (tensor map box): 16 KiB
constexpr int kCBoxes = 2 * TCC / 32;          // boxes per C tile
constexpr int kCTile = kCBoxes * kCBox;
constexpr long long kWaitLimit = 1LL << 22;
constexpr int kEpiWarp0 = 4;                   // epilogue warps from 4: one group of four per stage
constexpr int kStoreTid = 64;                  // issues the tile stores (warp 2)
static_assert(TCC == 16 || TCC == 32, "a C tile is one or two tensor-map boxes");

// Bytes of one operand tile (hi or lo) of each kind: A is 128 L21 rows, B 64
// rows (32 complex columns x {Re, Im}) of the 2 NB-long K dimension.
template <int kKind> __host__ __device__ constexpr int a_tile_bytes() { return TR * 2 * NB * (kKind == 2 ? 4 : 2); }
template <int kKind> __host__ __device__ constexpr int b_tile_bytes() { return 2 * TCC * 2 * NB * (kKind == 2 ? 4 : 2); }

// Shared-memory staging of each kind: the split A operand of one row tile, a
// ring of split B operand tiles (one per column tile) and per pipeline stage
// the output tile.  With the half-size BF16 operands the tiles have room for
// two panels in K (kPair): the trailing matrix is then updated once per pair
// of panels, which halves its traffic.
template <int kKind> struct Layout {
    static constexpr int kAT = a_tile_bytes<kKind>(), kBT = b_tile_bytes<kKind>();
    static constexpr bool kPair = kKind == 1;
    static constexpr int kSlots = kPair ? 2 : 1;
    static constexpr int kASpace = 2 * kSlots * kAT, kBSlot = 2 * kSlots * kBT;   // A (hi, lo); one ring slot
    static constexpr int kStages = 2, kBStages = 2;
    static constexpr int kDyn = 1024 + kASpace + kBStages * kBSlot + kStages * TR * 2 * TCC * 4;
    static constexpr int kTmemCols = kStages * 2 * TCC <= 128 ? 128 : 256;   // accumulators (a power of two)
    static_assert(kStages <= kMaxStages && kBStages <= kMaxBStages && kStages * 2 * TCC <= kTmemCols,
                  "stages fit the barriers and TMEM");
};

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
struct __align__(16) Cand {                 // one CTA's pivot candidate: key, then its row
    uint32_t kh, kl, pad[2];
    float2 row[NB];
};
struct PanelShared {
    uint32_t kh[2][kWarps], kl[2][kWarps];      // per-warp best keys
    float2 wrow[2][kWarps][NB];                 // cluster of one: warp winners' rows
    Cand cand[2][kMaxCluster];                  // cluster: every CTA's candidate
    float2 l11[NB + 16][NB + 1];                // unit lower L11 of the current panel; rows NB.. stay zero
    int mv_dst[kMaxMoved], mv_src[kMaxMoved];
    int mv_cnt;
    uint64_t bar[2];
    uint32_t tslot;
    int wait_failed;                            // a completion wait of this CTA gave up
    int ffail[kMaxCluster];                     // diagonal-pivot fast path: verdict of every CTA
};

// Arg-max of packed keys over a warp; returns (hi, lo) of the best.
__device__ __forceinline__ void key_max(uint32_t h, uint32_t l, uint32_t &mh, uint32_t &ml) {
    mh = __reduce_max_sync(0xffffffffu, h);
    ml = __reduce_max_sync(0xffffffffu, h == mh ? l : 0u);
}

// Operand tiles hold kSlots panels side by side in K (one panel, or two for
// the combined update of a pair of panels); slot `slot` of a row holds the
// 2 NB K values of one panel.

// Step 2: row `r` (0..127) of L21 tile `tile` in the MMA operand layout
// (K-major core matrices, hi tile then lo tile), slot `slot`, from the 32
// complex panel values of that row.
template <int kKind, int kSlots>
__device__ __forceinline__ void put_a_row(uint8_t *tiles, int tile, int r, const float2 (&v)[NB], int slot) {
    constexpr int qpc = Op<kKind>::qpc, kPanB = 2 * NB * Op<kKind>::esize, kRowB = kSlots * kPanB;
    constexpr int kT = kSlots * a_tile_bytes<kKind>();
    uint8_t *hi = tiles + (size_t)tile * 2 * kT, *lo = hi + kT;
#pragma unroll
    for (int c = 0; c < NB / qpc; ++c) {
        float w[2 * qpc];
#pragma unroll
        for (int h = 0; h < qpc; ++h) {
            w[2 * h] = v[c * qpc + h].x;
            w[2 * h + 1] = v[c * qpc + h].y;
        }
        const uint32_t off = tc::kmajor_offset(r, slot * kPanB + c * 16, kRowB);
        split_store<kKind>(w, hi + off, lo + off);
    }
}

// Step 3, one group of four rows: the B-operand chunks of U12 rows
// [4 g, 4 g + 4) of column `jj` (local to the trailing block): row 2 (jj %
// 32) gives Re, row 2 (jj % 32) + 1 gives Im of output column jj, in B tile
// jj / 32, slot `slot`.
template <int kKind, int kSlots>
__device__ __forceinline__ void put_b_group(uint8_t *tiles, int jj, int g, const float2 *u, int slot) {
    constexpr int qpc = Op<kKind>::qpc, kPanB = 2 * NB * Op<kKind>::esize, kRowB = kSlots * kPanB;
    constexpr int kT = kSlots * b_tile_bytes<kKind>();
    uint8_t *hi = tiles + (size_t)(jj / TCC) * 2 * kT, *lo = hi + kT;
    const int b = 2 * (jj % TCC);
#pragma unroll
    for (int cc = 0; cc < 4 / qpc; ++cc) {
        const int c = g * (4 / qpc) + cc;
        float re[2 * qpc], im[2 * qpc];
#pragma unroll
        for (int h = 0; h < qpc; ++h) {
            const float2 x = u[cc * qpc + h];
            re[2 * h] = x.x;
            re[2 * h + 1] = -x.y;
            im[2 * h] = x.y;
            im[2 * h + 1] = x.x;
        }
        const uint32_t o0 = tc::kmajor_offset(b, slot * kPanB + c * 16, kRowB);
        const uint32_t o1 = tc::kmajor_offset(b + 1, slot * kPanB + c * 16, kRowB);
        split_store<kKind>(re, hi + o0, lo + o0);
        split_store<kKind>(im, hi + o1, lo + o1);
    }
}

// Where step 3 stages the B operand of column jj: columns jj < split into
// the one-panel tiles bt1 (column jj), the others into slot `slot` of the
// two-panel tiles bt2 (column jj - split).
struct BDest {
    uint8_t *bt1, *bt2;
    int split, slot;
};

// Step 3 for one column, rows in groups of four: x[0..3] are rows q0..q0+3,
// eliminated into x[4..kRows) (rows q0 + 4 ..), stored, then the column
// shifts down by four.  Two instances (kRows = 32 while q0 < 16, 16 after)
// keep the loop bodies short enough to stay in the instruction cache.
template <int kKind, int kRows>
__device__ __forceinline__ void trsm_groups(float2 (&x)[NB], int g0, int g1, const float2 (*l11)[NB + 1],
                                            float2 *col, long long n, int nb, const BDest &bd, int jj) {
#pragma unroll 1
    for (int g = g0; g < g1; ++g) {
        const int q0 = 4 * g;
        const float2 (*L)[NB + 1] = reinterpret_cast<const float2 (*)[NB + 1]>(&l11[q0][q0]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int e = i + 1; e < kRows; ++e) {   // rows past the panel read zero rows of l11
                const float2 l = L[e][i];
                x[e].x -= l.x * x[i].x - l.y * x[i].y;
                x[e].y -= l.x * x[i].y + l.y * x[i].x;
            }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (q0 + i < nb) __stcg(col + (long long)(q0 + i) * n, x[i]);
        if (nb == NB) {
            if (jj < bd.split) put_b_group<kKind, 1>(bd.bt1, jj, g, x, 0);
            else put_b_group<kKind, 2>(bd.bt2, jj - bd.split, g, x, bd.slot);
        }
#pragma unroll
        for (int e = 0; e + 4 < kRows; ++e) x[e] = x[e + 4];
    }
}

// One 128 x 32-complex tile: hi*hi + hi*lo + lo*hi over the K of kSlots panels.
template <int kKind, int kSlots>
__device__ __forceinline__ void issue_mma(uint32_t tacc, uint32_t ah, uint32_t al, uint32_t bh,
                                          uint32_t bl) {
    constexpr int kRowB = kSlots * 2 * NB * Op<kKind>::esize;
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
}

// Pipeline state of the trailing update, kept in shared memory: stage s of
// the B and C buffers and of the TMEM accumulators is used by items s, s+2, ...
struct Pipe {
    uint64_t a_full, a_empty;
    uint64_t b_full[kMaxBStages], b_empty[kMaxBStages], c_empty[kMaxStages];
    uint64_t acc_full[kMaxStages], acc_empty[kMaxStages], c_written[kMaxStages];
    // items (row tile, column tile) and row tiles processed over all panels;
    // the loads the producer armed on each full barrier, the MMA thread's commits
    long long n_item, n_rowt;
    int armed_a, armed_b[kMaxBStages], commits[kMaxStages], commits_b[kMaxBStages], commits_a;
};

// Pointer into the shared memory of CTA r of this system's cluster.
template <typename T>
__device__ __forceinline__ T *at_rank(T *p, int cs, int r) {
    return cs == 1 ? p : cg::this_cluster().map_shared_rank(p, (unsigned)r);
}

// Blocks [cs * c, cs * c + cs) factor system order[c].  On return piv holds
// the inverse row permutation (original row i is row piv[i] of the factors).
// tmaps[s]: tensor map of system s's row-major FP32 matrix (2n floats x n
// rows, 32 x 128 boxes, 128-byte swizzle); opnd + a_off[s] / b_off[s]: the
// system's staged L21 and U12 operand tiles (rewritten every panel).
template <int kKind, bool kMulti>
__global__ void __launch_bounds__(kThreads, 1) lu_factor_tc_kernel(
    const int *__restrict__ order, int cs_arg, const int *__restrict__ Ns,
    const long long *__restrict__ mat_off, const int *__restrict__ vec_off,
    float2 *__restrict__ A32, int *__restrict__ piv, int *__restrict__ info,
    int *__restrict__ err, const CUtensorMap *__restrict__ tmaps, uint8_t *__restrict__ opnd,
    const long long *__restrict__ a_off, const long long *__restrict__ b_off) {
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(16) PanelShared ps;
    __shared__ __align__(8) Pipe pp;
    using LT = Layout<kKind>;
    constexpr int kAT = LT::kAT, kBT = LT::kBT, kStages = LT::kStages, kBStages = LT::kBStages;
    constexpr int kTmemCols = LT::kTmemCols;
    uint8_t *stage = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = stage;                                                // hi, lo
    uint8_t *sB = stage + LT::kASpace;                                  // ring of B tiles (hi, lo)
    uint8_t *sC = sB + kBStages * LT::kBSlot;                           // stages x C tile (1 KiB aligned)
    float4 *gbuf = reinterpret_cast<float4 *>(sB);                      // row gather (B + C)
    constexpr int kGather = (kBStages * LT::kBSlot + kStages * kCTile) / 16;   // float4 in gbuf
    // second panel of a pair: L21 of the first panel in the rows of the
    // second's pivots (32 x 32), kept in the A space between the updates
    float2 (*lpq)[NB + 2] = reinterpret_cast<float2 (*)[NB + 2]>(sA);
    static_assert(NB * (NB + 2) * 8 <= LT::kASpace, "the pair's L block fits the A space");
    static_assert(NB * (NB + 2) * 8 <= LT::kASpace && (NB * (NB + 2)) % 2 == 0,
                  "the pivot-row table of the checked-pivot panel fits the A space as whole float4s");

    const int cs = kMulti ? cs_arg : 1;
    const int rank = kMulti ? (int)cg::this_cluster().block_rank() : 0;
    const int s = order[blockIdx.x / cs];
    const int n = Ns[s];
    float2 *a = A32 + mat_off[s];
    int *pv = piv + vec_off[s];
    const CUtensorMap *tmap = tmaps + s;
    uint8_t *atiles = opnd + a_off[s], *btiles = opnd + b_off[s];
    // two-panel B tiles after the one-panel ones (lu_tc_opnd_bytes)
    uint8_t *b2tiles = btiles + (size_t)((max(n - NB, 0) + TCC - 1) / TCC) * 2 * kBT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int myslot = rank * kThreads + tid;

    if (warp == 0) tc::tmem_alloc(&ps.tslot, kTmemCols);
    if (tid == 0) {
        tc::mbar_init(&pp.a_full, 1);
        tc::mbar_init(&pp.a_empty, 1);
        for (int b = 0; b < kBStages; ++b) {
            tc::mbar_init(&pp.b_full[b], 1);
            tc::mbar_init(&pp.b_empty[b], 1);
            pp.armed_b[b] = pp.commits_b[b] = 0;
        }
        for (int b = 0; b < kStages; ++b) {
            tc::mbar_init(&pp.c_empty[b], 1);
            tc::mbar_init(&pp.acc_full[b], 1);
            tc::mbar_init(&pp.acc_empty[b], 4);
            tc::mbar_init(&pp.c_written[b], 4);
        }
        ps.wait_failed = 0;
        pp.n_item = pp.n_rowt = 0;
        pp.armed_a = pp.commits_a = 0;
        for (int b = 0; b < kStages; ++b) pp.commits[b] = 0;
    }
    for (int i = tid; i < 16 * (NB + 1); i += kThreads) ps.l11[NB + i / (NB + 1)][i % (NB + 1)] = make_float2(0.f, 0.f);
    if (rank == 0)   // pv: factored position -> original row, while factoring
        for (int i = tid; i < n; i += kThreads) pv[i] = i;
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = ps.tslot;
    if (cs > 1) cg::this_cluster().sync();   // every CTA running before shared memory is addressed remotely

    bool failed = false, bad = false;
    // role of the panel: 0 alone, 1 first of a pair (its update reaches only
    // the second panel's columns), 2 second of a pair (one update of the
    // trailing matrix with both panels' K)
    int role = 0;

    for (int k0 = 0; k0 < n; k0 += NB) {
        role = role == 1 ? 2 : (LT::kPair && n - k0 > 2 * NB ? 1 : 0);
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

        // 1a. Checked fast path.  Partial pivoting keeps the diagonal row
        // whenever, at every column, no row below it has a larger key (the
        // same packed |re| + |im| keys and tie rule as below: the diagonal is
        // the smallest position, so it wins ties).  For the second-kind CFIE
        // systems that holds with a wide margin (the largest key below the
        // diagonal is ~1/4 of it), and then the per-column search and
        // exchange across the cluster decide nothing.  So: the warp owning
        // the panel's first rows (CTA 0, threads 0-31) eliminates the 32 x 32
        // diagonal block, checking the keys among its rows and writing each
        // pivot row and its reciprocal into u11 (the A staging space, idle
        // during the panel); u11 goes to every CTA; every other row is
        // eliminated against u11 with its own key checked; one verdict per
        // panel.  The arithmetic is that of the search path below.  If any
        // check fails (or a pivot is zero or not finite) the panel is
        // reloaded and factored by the search path.
        bool fast = false;
        {
            float2 (*u11)[NB + 2] = reinterpret_cast<float2 (*)[NB + 2]>(sA);   // [c][q]; pinv at [c][NB]
            uint32_t fail = 0u;
            const bool dwarp = rank == 0 && warp == 0;     // rows 0-31: the diagonal block
            const bool lrow = own && myslot >= nb;         // rows eliminated against u11
            auto diag_step = [&](auto rows_c, const int q0) {
                constexpr int kRows = decltype(rows_c)::value;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = q0 + i;
                    if (c < nb) {
                        if (lane == c) {
#pragma unroll
                            for (int e = i; e < kRows; ++e)
                                if (q0 + e < NB) u11[c][q0 + e] = v[e];
                        }
                        __syncwarp();
                        const float2 pvt = u11[c][c];
                        const uint32_t kd = __float_as_uint(fabsf(pvt.x) + fabsf(pvt.y));
                        const bool act = own && lane > c;
                        const uint32_t kr = act ? __float_as_uint(fabsf(v[i].x) + fabsf(v[i].y)) : 0u;
                        const uint32_t kmax = __reduce_max_sync(0xffffffffu, kr);
                        if (kmax > kd || kd == 0u || kd >= 0x7F800000u) fail = 1u;
                        const float rd = 1.f / (pvt.x * pvt.x + pvt.y * pvt.y);
                        const float2 pinv = make_float2(pvt.x * rd, -pvt.y * rd);
                        if (lane == 0) u11[c][NB] = pinv;
                        if (act) {
                            const float2 l = cmul(v[i], pinv);
                            v[i] = l;
#pragma unroll
                            for (int e = i + 1; e < kRows; ++e)
                                if (q0 + e < NB) {
                                    const float2 u = u11[c][q0 + e];
                                    v[e].x -= l.x * u.x - l.y * u.y;
                                    v[e].y -= l.x * u.y + l.y * u.x;
                                }
                        }
                        __syncwarp();
                    }
                }
                float2 t[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) t[e] = v[e];
#pragma unroll
                for (int e = 0; e + 4 < NB; ++e) v[e] = v[e + 4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[NB - 4 + e] = t[e];
            };
            auto row_step = [&](auto rows_c, const int q0) {
                constexpr int kRows = decltype(rows_c)::value;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = q0 + i;
                    if (c < nb && lrow) {
                        const float2 pvt = u11[c][c], pinv = u11[c][NB];
                        const uint32_t kd = __float_as_uint(fabsf(pvt.x) + fabsf(pvt.y));
                        if (__float_as_uint(fabsf(v[i].x) + fabsf(v[i].y)) > kd) fail = 1u;
                        const float2 l = cmul(v[i], pinv);
                        v[i] = l;
#pragma unroll
                        for (int e = i + 1; e < kRows; ++e)
                            if (q0 + e < NB) {
                                const float2 u = u11[c][q0 + e];
                                v[e].x -= l.x * u.x - l.y * u.y;
                                v[e].y -= l.x * u.y + l.y * u.x;
                            }
                    }
                }
                float2 t[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) t[e] = v[e];
#pragma unroll
                for (int e = 0; e + 4 < NB; ++e) v[e] = v[e + 4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[NB - 4 + e] = t[e];
            };
            if (dwarp) {
#pragma unroll 1
                for (int q0 = 0; q0 < NB / 2; q0 += 4) diag_step(std::integral_constant<int, NB>{}, q0);
#pragma unroll 1
                for (int q0 = NB / 2; q0 < NB; q0 += 4) diag_step(std::integral_constant<int, NB / 2>{}, q0);
                if constexpr (kMulti) {   // u11 (pivot rows and reciprocals) to the other CTAs
                    const float4 *src = reinterpret_cast<const float4 *>(&u11[0][0]);
                    constexpr int kU4 = NB * (NB + 2) / 2;
                    for (int r = 1; r < cs; ++r) {
                        float4 *dst = reinterpret_cast<float4 *>(at_rank(&u11[0][0], cs, r));
                        for (int e = lane; e < kU4; e += 32) dst[e] = src[e];
                    }
                }
            }
            sys_sync(cs, false);   // u11 in every CTA
            if (lrow) {
#pragma unroll 1
                for (int q0 = 0; q0 < NB / 2; q0 += 4) row_step(std::integral_constant<int, NB>{}, q0);
#pragma unroll 1
                for (int q0 = NB / 2; q0 < NB; q0 += 4) row_step(std::integral_constant<int, NB / 2>{}, q0);
            }
            const int any = __syncthreads_or((int)fail);
            if constexpr (kMulti) {
                if (tid == 0)
                    for (int r = 0; r < cs; ++r) *at_rank(&ps.ffail[rank], cs, r) = any;
                sys_sync(cs, false);
                int all = 0;
                for (int r = 0; r < cs; ++r) all |= ps.ffail[r];
                fast = all == 0;
            } else {
                fast = any == 0;
            }
            if (!fast) {   // the search path below, from the panel as loaded
                const float4 *src = reinterpret_cast<const float4 *>(a + (long long)(k0 + (own ? myslot : 0)) * n + k0);
#pragma unroll
                for (int h = 0; h < NB / 2; ++h) {
                    const float4 t = (own && 2 * h < nb) ? __ldcg(src + h) : make_float4(0.f, 0.f, 0.f, 0.f);
                    v[2 * h] = make_float2(t.x, t.y);
                    v[2 * h + 1] = make_float2(t.z, t.w);
                }
            }
        }

        // 1. panel factorisation in registers, four columns per step of a
        // short rolled loop: v rotates left by four after each step, so that
        // v[i] is column q0 + i of the step and v[e] column q0 + e (e < 32 - q0;
        // the finished columns wrap to the end and come back in place after
        // the eighth step).  Two loop bodies, all 32 entries while q0 < 16 and
        // the first 16 after, keep the code small enough for the instruction
        // cache; the entries past the panel are skipped by predicate.
        if (!fast) {
        if constexpr (kMulti) {
            auto panel_step = [&](auto rows_c, auto group_c, const int q0) {
                constexpr int kRows = decltype(rows_c)::value, kGroup = decltype(group_c)::value;
                {
    #pragma unroll
                    for (int i = 0; i < kGroup; ++i) {
                        const int cl = q0 + i;
                        if (cl >= nb || bad) continue;
                        const int pb = cl & 1;
                        const uint32_t khi = active ? __float_as_uint(fabsf(v[i].x) + fabsf(v[i].y)) : 0u;
                        const uint32_t klo = active ? ~(uint32_t)mypos : 0u;
                        uint32_t mh, ml;
                        key_max(khi, klo, mh, ml);
                        if (lane == 0) {
                            ps.kh[pb][warp] = mh;
                            ps.kl[pb][warp] = ml;
                        }
                        const float2 *row;
                        {
                            __syncthreads();
                            const uint32_t h2 = lane < kWarps ? ps.kh[pb][lane] : 0u;
                            const uint32_t l2 = lane < kWarps ? ps.kl[pb][lane] : 0u;
                            key_max(h2, l2, mh, ml);
                            // this CTA's candidate to every CTA: the winning thread (or, when no
                            // row of this CTA is left, warp 0 with an empty key) fills this
                            // CTA's slot, then its warp copies the slot to the other CTAs, one
                            // 16-byte chunk per lane and step (the key and the row from column cl)
                            const bool none = mh == 0u && ml == 0u;
                            const bool win = active && khi == mh && klo == ml;
                            if (none ? warp == 0 : __ballot_sync(0xffffffffu, win) != 0u) {
                                Cand &mine = ps.cand[pb][rank];
                                float4 *m4 = reinterpret_cast<float4 *>(&mine);
                                if (win) {
                                    m4[0] = make_float4(__uint_as_float(mh), __uint_as_float(ml), 0.f, 0.f);
    #pragma unroll
                                    for (int e = i & ~1; e < kRows; e += 2)
                                        if (q0 + e < NB)
                                            m4[1 + (q0 + e) / 2] = make_float4(v[e].x, v[e].y, v[e + 1].x, v[e + 1].y);
                                } else if (none && lane == 0) {
                                    m4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                                }
                                __syncwarp();
                                const int h0 = cl / 2, per = none ? 1 : 1 + NB / 2 - h0;
                                for (int t = lane; t < (cs - 1) * per; t += 32) {
                                    const int rr = t / per, j = t - rr * per;
                                    const int f = j == 0 ? 0 : h0 + j;
                                    float4 *dst = reinterpret_cast<float4 *>(at_rank(&mine, cs, rr < rank ? rr : rr + 1));
                                    dst[f] = m4[f];
                                }
                            }
                            sys_sync(cs, false);
                            const uint32_t h3 = lane < cs ? ps.cand[pb][lane].kh : 0u;
                            const uint32_t l3 = lane < cs ? ps.cand[pb][lane].kl : 0u;
                            key_max(h3, l3, mh, ml);
                            const uint32_t hit = __ballot_sync(0xffffffffu, lane < cs && h3 == mh && l3 == ml);
                            row = ps.cand[pb][__ffs(hit) - 1].row;
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
                            const float2 l = cmul(v[i], pinv);
                            v[i] = l;
    #pragma unroll
                            for (int e = i + 1; e < kRows; ++e)
                                if (q0 + e < NB) {
                                    const float2 u = row[q0 + e];
                                    v[e].x -= l.x * u.x - l.y * u.y;
                                    v[e].y -= l.x * u.y + l.y * u.x;
                                }
                        }
                    }
                    if constexpr (kGroup < NB) {
                        float2 t[kGroup];
    #pragma unroll
                        for (int e = 0; e < kGroup; ++e) t[e] = v[e];
    #pragma unroll
                        for (int e = 0; e + kGroup < NB; ++e) v[e] = v[e + kGroup];
    #pragma unroll
                        for (int e = 0; e < kGroup; ++e) v[NB - kGroup + e] = t[e];
                    }
                }
            };
#pragma unroll 1
            for (int q0 = 0; q0 < NB / 2; q0 += 4)
                panel_step(std::integral_constant<int, NB>{}, std::integral_constant<int, 4>{}, q0);
#pragma unroll 1
            for (int q0 = NB / 2; q0 < NB; q0 += 4)
                panel_step(std::integral_constant<int, NB / 2>{}, std::integral_constant<int, 4>{}, q0);
        } else {
            // a cluster of one: fully unrolled (the column work dominates here)
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
                // this CTA's candidate to every CTA: the winning thread (or, when no
                // row of this CTA is left, warp 0 with an empty key) fills this
                // CTA's slot, then its warp copies the slot to the other CTAs, one
                // 16-byte chunk per lane and step (the key and the row from column cl)
                const bool none = mh == 0u && ml == 0u;
                const bool win = active && khi == mh && klo == ml;
                if (none ? warp == 0 : __ballot_sync(0xffffffffu, win) != 0u) {
                    Cand &mine = ps.cand[pb][rank];
                    float4 *m4 = reinterpret_cast<float4 *>(&mine);
                    if (win) {
                        m4[0] = make_float4(__uint_as_float(mh), __uint_as_float(ml), 0.f, 0.f);
#pragma unroll
                        for (int h = cl / 2; h < NB / 2; ++h)
                            m4[1 + h] = make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
                    } else if (none && lane == 0) {
                        m4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    __syncwarp();
                    const int h0 = cl / 2, per = none ? 1 : 1 + NB / 2 - h0;
                    for (int i = lane; i < (cs - 1) * per; i += 32) {
                        const int rr = i / per, j = i - rr * per;
                        const int f = j == 0 ? 0 : h0 + j;
                        float4 *dst = reinterpret_cast<float4 *>(at_rank(&mine, cs, rr < rank ? rr : rr + 1));
                        dst[f] = m4[f];
                    }
                }
                sys_sync(cs, false);
                const uint32_t h3 = lane < cs ? ps.cand[pb][lane].kh : 0u;
                const uint32_t l3 = lane < cs ? ps.cand[pb][lane].kl : 0u;
                key_max(h3, l3, mh, ml);
                const uint32_t hit = __ballot_sync(0xffffffffu, lane < cs && h3 == mh && l3 == ml);
                row = ps.cand[pb][__ffs(hit) - 1].row;
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
        }
        }   // !fast
        if (bad) break;

        // 2. panel to its final rows (and the L21 rows to the staged A
        // operand); L11 and the moved rows to every CTA
        if (own) {
            float4 *dst = reinterpret_cast<float4 *>(a + (long long)(k0 + mypos) * n + k0);
#pragma unroll
            for (int h = 0; h < NB / 2; ++h)
                if (2 * h < nb) __stcg(dst + h, make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y));
            if (role != 2) {
                if (mypos >= nb && nb == NB)
                    put_a_row<kKind, 1>(atiles, (mypos - NB) / TR, (mypos - NB) % TR, v, 0);
            } else if (mypos >= NB) {
                put_a_row<kKind, 2>(atiles, (mypos - NB) / TR, (mypos - NB) % TR, v, 1);
            }
            if (mypos < nb)
                for (int r = 0; r < cs; ++r) {
                    float2 *l = at_rank(&ps.l11[mypos][0], cs, r);
#pragma unroll
                    for (int q = 0; q < NB; ++q)
                        if (q < mypos) l[q] = v[q];
                }
            if (role == 2) {
                // the row's L21 of the first panel (v is done with), from its
                // place before the swaps of this panel: into slot 0 of the
                // two-panel A tiles, or for a pivot row into row mypos of lpq
                // at every CTA
                const float4 *lp = reinterpret_cast<const float4 *>(a + (long long)(k0 + myslot) * n + (k0 - NB));
#pragma unroll
                for (int h = 0; h < NB / 2; ++h) {
                    const float4 t = __ldcg(lp + h);
                    v[2 * h] = make_float2(t.x, t.y);
                    v[2 * h + 1] = make_float2(t.z, t.w);
                }
                if (mypos >= NB) {
                    put_a_row<kKind, 2>(atiles, (mypos - NB) / TR, (mypos - NB) % TR, v, 0);
                } else {
                    for (int r = 0; r < cs; ++r) {
                        float4 *dst = reinterpret_cast<float4 *>(at_rank(&lpq[mypos][0], cs, r));
#pragma unroll
                        for (int h = 0; h < NB / 2; ++h)
                            dst[h] = make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
                    }
                }
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

        // column ranges of this CTA outside the panel: an even share of the
        // columns left of it, [lc_lo, lc_hi), and of those right of it, columns
        // nb + [rc_lo, rc_hi) (the swaps and U12 of one column stay in one CTA)
        const int ncs = n - nb, nr = ncs - k0;
        const int WL = (((k0 + cs - 1) / cs) + 1) & ~1, WR = (((nr + cs - 1) / cs) + 1) & ~1;
        const int lc_lo = min(k0, rank * WL), lc_hi = min(k0, lc_lo + WL);
        const int rc_lo = k0 + min(nr, rank * WR), rc_hi = k0 + min(nr, rank * WR + WR);
        const int nmv = min(ps.mv_cnt, kMaxMoved);
        if (nmv > 0) {
            int t_perm = 0;
            if (rank == 0 && tid < nmv) t_perm = pv[k0 + ps.mv_src[tid]];
            const int CW2 = kGather / nmv;      // float4 (two columns) per moved row and chunk
            for (int side = 0; side < 2; ++side) {
                const int c_lo = side == 0 ? lc_lo : rc_lo, c_hi = side == 0 ? lc_hi : rc_hi;
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
            }
            if (rank == 0) {
                __syncthreads();
                if (tid < nmv) pv[k0 + ps.mv_dst[tid]] = t_perm;
            }
        }

        // 3. U12 = L11^{-1} A12 over this CTA's columns right of the panel:
        // one column per thread, all nb values in registers (one round of
        // loads), forward substitution with L11 from shared memory, then the
        // column to the matrix and to the staged B operand
        // (second panel of a pair: first A12 -= L21(first panel) U12(first
        // panel) in these rows, the update the first panel left out)
        const BDest bd{btiles, b2tiles, role == 0 ? INT_MAX : role == 1 ? NB : 0, role == 2 ? 1 : 0};
        // (U12 of the first panel over this CTA's columns, rows k0 - NB ..,
        // into the gather space with coalesced loads: up[q][c - rc_lo])
        float2 *up = reinterpret_cast<float2 *>(gbuf);
        const int ncol = rc_hi - rc_lo;
        // (at most 512 columns: a CTA owns 512 rows, so cs >= n / 512)
        if (role == 2 && NB * ncol > 2 * kGather) failed = true;
        if (role == 2 && !failed) {
            for (int e = tid; e < NB * ncol; e += kThreads) {
                const int q = e / ncol, c = e - q * ncol;
                up[e] = __ldcg(a + (long long)(k0 - NB + q) * n + rc_lo + c + nb);
            }
            __syncthreads();
        }
        for (int c = rc_lo + tid; c < rc_hi; c += kThreads) {
            float2 *col = a + (long long)k0 * n + c + nb;
            float2 x[NB];
#pragma unroll
            for (int e = 0; e < NB; ++e)
                x[e] = e < nb ? __ldcg(col + (long long)e * n) : make_float2(0.f, 0.f);
            if (role == 2 && !failed) {
#pragma unroll 2
                for (int q = 0; q < NB; ++q) {
                    const float2 u = up[q * ncol + (c - rc_lo)];
#pragma unroll
                    for (int e = 0; e < NB; ++e) {
                        const float2 l = lpq[e][q];
                        x[e].x -= l.x * u.x - l.y * u.y;
                        x[e].y -= l.x * u.y + l.y * u.x;
                    }
                }
            }
            trsm_groups<kKind, NB>(x, 0, NB / 8, ps.l11, col, n, nb, bd, c - k0);
            trsm_groups<kKind, NB / 2>(x, NB / 8, NB / 4, ps.l11, col, n, nb, bd, c - k0);
        }
        // the swaps, U12 and the staged operands (generic stores to global
        // memory) are read by the TMA engine below, which also overwrites the
        // shared-memory gather buffer of the swaps
        tc::fence_async_all();
        sys_sync(cs, true);

        // 4. A22 -= L21 U12 on the tensor cores: rows and columns from r0,
        // nct column tiles; at / bt: the staged A and B tiles (kS panels in K)
        const int r0 = k0 + nb, m2 = n - r0;
        auto update = [&](auto slots_c, const int nct, const uint8_t *at, const uint8_t *bt) {
                constexpr int kS = decltype(slots_c)::value;   // panels in K
                const int nrt = (m2 + TR - 1) / TR;
                // this CTA's items: an even share of the (row tile, column tile)
                // sequence in row-tile order, i.e. up to two partial row tiles
                // ("segments") besides whole ones
                const long long n_items = (long long)nrt * nct;
                const int t_lo = (int)(n_items * rank / cs), t_hi = (int)(n_items * (rank + 1) / cs);
                const int n_seg = t_hi > t_lo ? (t_hi - 1) / nct - t_lo / nct + 1 : 0;
                if (tid == 0) {
                    // producer: A once per segment, B per item
                    long long it = pp.n_item, rtc = pp.n_rowt;
                    for (int t = t_lo; t < t_hi && !failed; ++t, ++it) {
                        const int rt = t / nct, ct = t - rt * nct;
                        if (t == t_lo || ct == 0) {
                            if (rtc > 0 && !tc::mbar_wait(&pp.a_empty, (uint32_t)((rtc - 1) & 1), kWaitLimit)) {
                                failed = true;
                                break;
                            }
                            tc::mbar_arrive_tx(&pp.a_full, 2 * kS * kAT);
                            tc::bulk_load(sA, at + (size_t)rt * 2 * kS * kAT, 2 * kS * kAT, &pp.a_full);
                            ++pp.armed_a;
                            ++rtc;
                        }
                        const int bs = (int)(it % kBStages);
                        const long long ub = it / kBStages;
                        if (ub > 0 && !tc::mbar_wait(&pp.b_empty[bs], (uint32_t)((ub - 1) & 1), kWaitLimit)) {
                            failed = true;
                            break;
                        }
                        tc::mbar_arrive_tx(&pp.b_full[bs], 2 * kS * kBT);
                        tc::bulk_load(sB + bs * LT::kBSlot, bt + (size_t)ct * 2 * kS * kBT, 2 * kS * kBT, &pp.b_full[bs]);
                        ++pp.armed_b[bs];
                    }
                    if (failed) ps.wait_failed = 1;
                } else if (tid == 32) {
                    // MMA issuer
                    long long it = pp.n_item, rtc = pp.n_rowt;
                    for (int t = t_lo; t < t_hi && !failed; ++t, ++it) {
                        const int ct = t % nct;
                        if ((t == t_lo || ct == 0) && !tc::mbar_wait(&pp.a_full, (uint32_t)((rtc++) & 1), kWaitLimit)) {
                            failed = true;
                            break;
                        }
                        const int st = (int)(it % kStages), bs = (int)(it % kBStages);
                        const long long u = it / kStages;
                        if (!tc::mbar_wait(&pp.b_full[bs], (uint32_t)((it / kBStages) & 1), kWaitLimit) ||
                            (u > 0 && !tc::mbar_wait(&pp.acc_empty[st], (uint32_t)((u - 1) & 1), kWaitLimit))) {
                            failed = true;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t bh = tc::smem_u32(sB + bs * LT::kBSlot);
                        issue_mma<kKind, kS>(taddr + (uint32_t)(st * 2 * TCC), tc::smem_u32(sA),
                                             tc::smem_u32(sA) + kS * kAT, bh, bh + kS * kBT);
                        tc::mma_commit(&pp.acc_full[st]);
                        tc::mma_commit(&pp.b_empty[bs]);
                        ++pp.commits[st];
                        ++pp.commits_b[bs];
                        if (t == t_hi - 1 || ct == nct - 1) {   // the segment's A tile is read
                            tc::mma_commit(&pp.a_empty);
                            ++pp.commits_a;
                        }
                    }
                    if (failed) ps.wait_failed = 1;
                } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4 * kStages) {
                    // epilogue, one group of four warps per stage (the groups work on
                    // consecutive items at once): the negated accumulator into the
                    // stage's shared-memory tile, once the reduction of the stage's
                    // previous item has read it; thread: row r, all 2 TCC columns
                    const int g = (warp - kEpiWarp0) >> 2, lg = warp & 3;   // group (= stage), TMEM lane group
                    const int r = 32 * lg + lane;                           // tile row
                    long long it = pp.n_item;
                    bool stop = false;
                    for (int t = t_lo; t < t_hi && !stop && !failed; ++t, ++it) {
                        {
                            if ((int)(it % kStages) != g) continue;
                            const uint32_t par = (uint32_t)((it / kStages) & 1);
                            bool got = tc::mbar_wait(&pp.acc_full[g], par, kWaitLimit);
                            if (it >= kStages) got = got && tc::mbar_wait(&pp.c_empty[g], par ^ 1u, kWaitLimit);
                            if (tc::bar_or(1 + g, 128, !got)) {   // the same verdict in the whole group
                                stop = true;
                                break;
                            }
                            tc::tc_fence_after();
                            const uint32_t tacc = taddr + (uint32_t)(g * 2 * TCC) + ((uint32_t)(32 * lg) << 16);
    #pragma unroll
                            for (int bx = 0; bx < kCBoxes; ++bx) {   // one 32-column box at a time
                                float d[32];
                                tc::tmem_ld16(tacc + 32 * bx, *reinterpret_cast<float(*)[16]>(d));
                                tc::tmem_ld16(tacc + 32 * bx + 16, *reinterpret_cast<float(*)[16]>(d + 16));
                                if (bx == kCBoxes - 1) {   // the accumulator is read
                                    tc::tc_fence_before();
                                    __syncwarp();
                                    if (lane == 0) tc::mbar_arrive(&pp.acc_empty[g]);
                                }
                                float4 *row = reinterpret_cast<float4 *>(sC + g * kCTile + bx * kCBox + r * 128);
    #pragma unroll
                                for (int c = 0; c < 8; ++c)   // 128-byte swizzle of the box
                                    row[c ^ (r & 7)] = make_float4(-d[4 * c], -d[4 * c + 1], -d[4 * c + 2], -d[4 * c + 3]);
                            }
                            tc::fence_async_smem();   // the tile reduction (async proxy) reads these writes
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(&pp.c_written[g]);
                        }
                    }
                    if (stop) {
                        failed = true;
                        if (lg == 0 && lane == 0) ps.wait_failed = 1;
                    }
                } else if (tid == kStoreTid) {
                    // tile reductions: each tile is added into the matrix (C +=
                    // -L21 U12, at L2) once its four epilogue warps have written
                    // it; its buffer is released when the reduction has read it
                    // (two reductions in flight: an item's buffer is released once
                    // the next item's reduction has been issued)
                    long long it = pp.n_item;
                    int prev = -1;   // stage of the previous item, its buffer not yet released
                    for (int t = t_lo; t < t_hi && !failed; ++t, ++it) {
                        const int rt = t / nct, ct = t - rt * nct, i0 = r0 + rt * TR;
                        {
                            const int st = (int)(it % kStages);
                            if (!tc::mbar_wait(&pp.c_written[st], (uint32_t)((it / kStages) & 1), kWaitLimit)) {
                                failed = true;
                                break;
                            }
                            const int x = 2 * (r0 + ct * TCC);
                            uint8_t *src = sC + st * kCTile;
    #pragma unroll
                            for (int bx = 0; bx < kCBoxes; ++bx)
                                tc::tma_reduce_add_2d(tmap, x + 32 * bx, i0, src + bx * kCBox);
                            tc::bulk_commit();
                            if (prev >= 0) {
                                tc::bulk_wait_read1();
                                tc::mbar_arrive(&pp.c_empty[prev]);
                            }
                            prev = st;
                        }
                    }
                    if (prev >= 0) {
                        tc::bulk_wait_read();
                        tc::mbar_arrive(&pp.c_empty[prev]);
                    }
                    if (failed) ps.wait_failed = 1;
                    // the reductions are in global memory before the next panel reads them
                    tc::bulk_wait_all();
                    tc::fence_async_global();
                }
                // drain: the producer's loads and the MMAs have landed (a no-op
                // unless a wait gave up) before the buffers are reused
                if (tid == 0) {
                    if (pp.armed_a) tc::mbar_wait(&pp.a_full, (uint32_t)((pp.armed_a - 1) & 1), kWaitLimit);
                    for (int b = 0; b < kBStages; ++b)
                        if (pp.armed_b[b]) tc::mbar_wait(&pp.b_full[b], (uint32_t)((pp.armed_b[b] - 1) & 1), kWaitLimit);
                } else if (tid == 32) {
                    for (int b = 0; b < kStages; ++b)
                        if (pp.commits[b]) tc::mbar_wait(&pp.acc_full[b], (uint32_t)((pp.commits[b] - 1) & 1), kWaitLimit);
                    for (int b = 0; b < kBStages; ++b)
                        if (pp.commits_b[b]) tc::mbar_wait(&pp.b_empty[b], (uint32_t)((pp.commits_b[b] - 1) & 1), kWaitLimit);
                    if (pp.commits_a) tc::mbar_wait(&pp.a_empty, (uint32_t)((pp.commits_a - 1) & 1), kWaitLimit);
                }
                tc::fence_async_smem();   // the staging buffers are reused by generic accesses next
                tc::tc_fence_before();
                __syncthreads();
                tc::tc_fence_after();
                if (ps.wait_failed) failed = true;
                if (tid == 0) {   // read again at the next panel's update, after its barriers
                    pp.n_item += t_hi - t_lo;
                    pp.n_rowt += n_seg;
                }
        };
        if (m2 > 0) {
            if (role == 2) update(std::integral_constant<int, 2>{}, (m2 + TCC - 1) / TCC, atiles, b2tiles);
            else update(std::integral_constant<int, 1>{}, role == 1 ? 1 : (m2 + TCC - 1) / TCC, atiles, btiles);
        }
        sys_sync(cs, true);
    }

    __syncthreads();
    if (ps.wait_failed) failed = true;
    if (failed && tid == 0) {
        atomicOr(err, 1);
        info[s] = -2;
    }
    if (!bad && rank == 0) {   // position -> row  into  row -> position
        int *perm = reinterpret_cast<int *>(sA);
        __syncthreads();
        for (int i = tid; i < n; i += kThreads) perm[i] = pv[i];
        __syncthreads();
        for (int i = tid; i < n; i += kThreads) pv[perm[i]] = i;
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(taddr, kTmemCols);
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
                         float2 *A32, int *piv, const int *vec_off, int *info, int *err,
                         const LuTcWork &w, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * cs));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = Layout<kKind>::kDyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const CUtensorMap *maps = static_cast<const CUtensorMap *>(w.maps);
    if (cs == 1)
        return cudaLaunchKernelEx(&cfg, lu_factor_tc_kernel<kKind, false>, order, cs, N, mat_off,
                                  vec_off, A32, piv, info, err, maps, w.opnd, w.a_off, w.b_off);
    return cudaLaunchKernelEx(&cfg, lu_factor_tc_kernel<kKind, true>, order, cs, N, mat_off, vec_off,
                              A32, piv, info, err, maps, w.opnd, w.a_off, w.b_off);
}

}  // namespace

// Every CTA owns kThreads = 512 panel rows, so at least ceil(n / 512) CTAs,
// and exactly that many (any cluster size up to 8: rows, items and U12
// columns are split by rank); smaller rows_per_cta spreads the trailing
// updates over more CTAs.
int lu_tc_cluster(int n, int rows_per_cta) {
    const int rows = rows_per_cta >= kThreads ? kThreads : rows_per_cta >= 256 ? 256 : 128;
    const int need = (n + rows - 1) / rows;
    return need < 1 ? 1 : need > kMaxCluster ? kMaxCluster : need;
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

size_t lu_tc_opnd_bytes(int kind, const int *N_h, int S, long long *a_off_h, long long *b_off_h) {
    const size_t at = kind == 2 ? a_tile_bytes<2>() : a_tile_bytes<1>();
    const size_t bt = kind == 2 ? b_tile_bytes<2>() : b_tile_bytes<1>();
    // per system: the A tiles (one-panel rows below the first panel, or for
    // BF16 the larger two-panel tiles below a pair), then the one-panel B
    // tiles and for BF16 the two-panel B tiles
    const bool pair = kind != 2;
    size_t off = 0;
    for (int s = 0; s < S; ++s) {
        const int m2 = std::max(N_h[s] - NB, 0), m3 = std::max(N_h[s] - 2 * NB, 0);
        if (a_off_h) a_off_h[s] = (long long)off;
        size_t a_sz = (size_t)((m2 + TR - 1) / TR) * 2 * at;
        if (pair) a_sz = std::max(a_sz, (size_t)((m3 + TR - 1) / TR) * 4 * at);
        off += a_sz;
        if (b_off_h) b_off_h[s] = (long long)off;
        off += (size_t)((m2 + TCC - 1) / TCC) * 2 * bt;
        if (pair) off += (size_t)((m3 + TCC - 1) / TCC) * 4 * bt;
    }
    return std::max(off, (size_t)16);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}
}  // namespace

size_t lu_tc_map_bytes(int S) { return (size_t)std::max(S, 1) * sizeof(CUtensorMap); }

cudaError_t lu_tc_encode_maps(const int *N_h, const long long *mat_off_h, int S, float2 *A32, void *maps_h) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap *m = static_cast<CUtensorMap *>(maps_h);
    for (int s = 0; s < S; ++s) {
        const cuuint64_t n = (cuuint64_t)N_h[s];
        const cuuint64_t dims[2] = {2 * n, n};                   // floats per row, rows
        const cuuint64_t strides[1] = {2 * n * sizeof(float)};   // bytes between rows
        const cuuint32_t box[2] = {32, (cuuint32_t)TR};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = enc(&m[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, A32 + mat_off_h[s], dims, strides,
                               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_lu_factor_tc(int kind, int rows_per_cta, const int *order, const int *order_h,
                                const int *N_h, int S,
                                const int *N, const long long *mat_off, float2 *A32, int *piv,
                                const int *vec_off, int *info, int *err, const LuTcWork &w,
                                cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    static std::atomic<unsigned long long> attr[4] = {{0}, {0}, {0}, {0}};
    {
        const void *fns[4] = {(const void *)lu_factor_tc_kernel<2, false>, (const void *)lu_factor_tc_kernel<2, true>,
                              (const void *)lu_factor_tc_kernel<1, false>, (const void *)lu_factor_tc_kernel<1, true>};
        for (int f = kind == 2 ? 0 : 2, e0 = f + 2; f < e0; ++f) {
            const cudaError_t e = ensure_smem_attr(fns[f], f < 2 ? Layout<2>::kDyn : Layout<1>::kDyn, attr[f]);
            if (e != cudaSuccess) return e;
        }
    }
    // order is sorted by decreasing N, so each cluster size is a contiguous run
    for (int first = 0; first < S;) {
        const int cs = lu_tc_cluster(N_h[order_h[first]], rows_per_cta);
        int last = first;
        while (last < S && lu_tc_cluster(N_h[order_h[last]], rows_per_cta) == cs) ++last;
        const cudaError_t e = kind == 2
            ? launch_group<2>(order + first, last - first, cs, N, mat_off, A32, piv, vec_off, info, err, w, st)
            : launch_group<1>(order + first, last - first, cs, N, mat_off, A32, piv, vec_off, info, err, w, st);
        if (e != cudaSuccess) return e;
        first = last;
    }
    return cudaSuccess;
}

}  // namespace fh
