// Step a7 on the tensor cores: u[x][t] = sum_{kk < 2J} A[x][kk] B[kk][t] with
// A = [Vr | Vi] and B = [Gr ; Gm] (Sec. 4.1 eq. approx in collapsed form),
// to FP64-class accuracy through exact BF16 products (an error-free slicing
// of the operands, the "Ozaki scheme").
//
// Each row x of A is scaled by a power of two sa_x >= max_kk |A[x][kk]| and
// cut into kSlices = 8 slices of kSliceBits = 6 bits, A[x][kk] / sa_x =
// sum_i a_i 2^-(6 (i + 1)) + O(2^-49), a_i integers with |a_i| <= 2^6;
// likewise each column t of B with sb_t.  Integers of 7 bits are exact in
// BF16, their products (<= 2^12) are exact in the FP32 accumulator, and a
// level d = i + j sums at most kSlices pairs over a K segment of kSegK = 512
// terms below 2^24 (8 x 512 x 2^12 = 2^24), so every level is an exact
// integer sum: TMEM holds one FP32 accumulator per level (kSlices x 64 = 512
// columns, all of it).  After each K segment the epilogue combines the
// levels, scaled by 2^-(kSliceBits (d + 2)), into double-float sums (one per
// output) and the next segment starts its levels afresh; at the end the sums
// are multiplied by sa_x sb_t.  The result differs from the exact product by
// the dropped slice pairs (i + j >= kSlices) and the remainders, ~K 2^-48
// sa_x sb_t at worst.
//
// Kernels: ozaki_scale_kernel (the power-of-two scale of each row of A and
// each column of B), ozaki_slice_kernel (slices in BF16, written directly in
// the MMA's shared-memory layout: per 128-row (A) or 64-row (B) tile and K
// chunk of 16, the eight slices' K-major core matrices in one contiguous
// block), contract_tc_kernel (one CTA per 128 x 64 output tile, warp
// specialised over a four-stage pipeline: one thread bulk-copies each chunk's
// A and B blocks (48 KB), one thread issues the kind::f16 MMAs of every slice
// pair into its level's accumulator, eight epilogue warps combine the levels
// after each segment; mbarriers with bounded waits hand the stages over).
#include <cuda_bf16.h>

#include "fh_internal.h"
#include "dfloat.cuh"
#include "tc_gemm.cuh"

namespace fh {
namespace {

constexpr int kSlices = 8;
constexpr int kSliceBits = 6;
constexpr int kTM = 128;                 // output rows (x) per CTA = TMEM lanes
constexpr int kTN = 64;                  // output columns (t) per CTA
constexpr int kKC = 16;                  // K elements per staged chunk: one MMA K step (32 bytes)
constexpr int kKBytes = kKC * 2;
constexpr int kKPad = 64;                // K padding of the slice arrays
constexpr int kThr = 256;
constexpr int kASlice = kTM * kKBytes;   // bytes of one A slice chunk (4 KiB)
constexpr int kBSlice = kTN * kKBytes;   // bytes of one B slice chunk (2 KiB)
constexpr int kABlock = kSlices * kASlice, kBBlock = kSlices * kBSlice;   // 32 + 16 KiB per chunk
constexpr int kStage = kABlock + kBBlock;                                 // 48 KiB
constexpr int kStages = 4;
constexpr int kSmem = 1024 + kStages * kStage;
constexpr int kSegK = 512;                  // K per exact segment
constexpr int kCtaThreads = 384;            // producer (warp 0), MMA (warp 1), epilogue (warps 4 .. 11)
constexpr long long kWaitLimit = 1LL << 22;

// Element (r, kk) of the operand whose rows are r: A rows are targets x (from
// V[kk][x] complex, real parts for kk < J, imaginary parts above), B rows are
// times t (from Gr[kk][t] for kk < J, Gm[kk - J][t] above).
struct Src {
    const double2 *V;        // A: V[j * ld + r]
    const double *G0, *G1;   // B: Gr, Gm [j * ld + r]
    int J, ld, rows;
    __device__ __forceinline__ double at(int r, int kk) const {
        if (r >= rows || kk >= 2 * J) return 0.0;
        const int j = kk < J ? kk : kk - J;
        if (V) {
            const double2 v = V[(long long)j * ld + r];
            return kk < J ? v.x : v.y;
        }
        return (kk < J ? G0 : G1)[(long long)j * ld + r];
    }
};

// e[r] with max_kk |src(r, kk)| < 2^e[r] (0 for a zero row).  A CTA takes 32
// rows: lane = row (consecutive rows are contiguous in both sources), the
// eight warps stride over kk, then a shared-memory maximum.
__global__ void __launch_bounds__(kThr) ozaki_scale_kernel(Src src, int K, int *__restrict__ e) {
    __shared__ double part[kThr / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * 32 + lane;
    double m = 0.0;
#pragma unroll 8
    for (int kk = warp; kk < K; kk += kThr / 32) m = fmax(m, fabs(src.at(r, kk)));
    part[warp][lane] = m;
    __syncthreads();
    if (warp == 0) {
        for (int w = 1; w < kThr / 32; ++w) m = fmax(m, part[w][lane]);
        int ex = 0;
        if (m > 0.0) frexp(m, &ex);   // m = f 2^ex, f in [1/2, 1)
        e[r] = ex;
    }
}

// Slices of a 64-row x 32-column block, in BF16, written into the tiled
// layout the contraction copies in bulk: for tile rows tr (128 for A, 64 for
// B) and K chunks of 16, block (r / tr) * nkc + kk / 16 holds the eight slices
// one after the other, each tr rows of 32 bytes as K-major core matrices
// (8 rows x 16 bytes; the two 16-byte halves of K 128 bytes apart, 8-row
// groups 256 bytes apart).
// In integer arithmetic on the FP64 bit pattern: V = round(src 2^(42 - e[r]))
// (|V| <= 2^48) = sum_s a_s 2^(42 - 6 s) with balanced digits, each the
// nearest multiple of the remainder (a_0 in [-64, 64], a_s in [-32, 32]), so
// that the dropped slice products carry no common sign: src / 2^e[r] =
// sum_s a_s 2^-(6 (s + 1)) to within 2^-49.
__global__ void __launch_bounds__(kThr) ozaki_slice_kernel(Src src, const int *__restrict__ e,
                                                           int kpad, int tr,
                                                           __nv_bfloat16 *__restrict__ out) {
    __shared__ __nv_bfloat16 t[kSlices][32][64 + 8];   // [slice][kk][r], padded rows
    const int r0 = blockIdx.y * 64, k0 = blockIdx.x * 32;
    for (int idx = threadIdx.x; idx < 64 * 32; idx += kThr) {
        const int rr = idx & 63, kk = idx >> 6;          // consecutive threads: consecutive rows
        const int r = r0 + rr;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(src.at(r, k0 + kk));
        const int bexp = (int)((bits >> 52) & 0x7FF);
        const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (bexp ? (1ull << 52) : 0ull);
        // |src| = mant 2^(E), E = bexp - 1075 (1 - 1075 for subnormals); V = mant 2^(E + 42 - e)
        const int sh = (bexp ? bexp : 1) - 1075 + kSlices * kSliceBits - e[r];   // <= -5
        long long V = 0;
        if (sh > -64) {
            const int rs = -sh;
            V = (long long)((mant + (1ull << (rs - 1))) >> rs);   // round half up on |V|
        }
        if (bits >> 63) V = -V;
#pragma unroll
        for (int s = 0; s < kSlices; ++s) {
            const int p = kSliceBits * (kSlices - 1 - s);   // 42, 36, ..., 0
            const long long a = p ? (V + (1ll << (p - 1))) >> p : V;   // nearest, ties up
            V -= a << p;                                    // |V| <= 2^(p - 1)
            t[s][kk][rr] = __float2bfloat16_rn((float)a);   // |a| <= 64: exact
        }
    }
    __syncthreads();
    // 16-byte pieces: 8 consecutive K of one row and slice
    const int nkc = kpad / kKC;
    uint8_t *ob = reinterpret_cast<uint8_t *>(out);
    for (int idx = threadIdx.x; idx < kSlices * 64 * 4; idx += kThr) {
        const int rr = idx & 63, k8 = (idx >> 6) & 3, s = idx >> 8;
        const int r = r0 + rr, kk = k0 + 8 * k8;
        __align__(16) __nv_bfloat16 w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = t[s][8 * k8 + q][rr];
        const size_t blk = ((size_t)(r / tr) * nkc + kk / kKC) * kSlices + s;
        const uint32_t off = tc::kmajor_offset(r % tr, (kk % kKC) * 2, kKBytes);
        *reinterpret_cast<uint4 *>(ob + blk * (size_t)tr * kKBytes + off) = *reinterpret_cast<const uint4 *>(w);
    }
}

__global__ void __launch_bounds__(kCtaThreads, 1) contract_tc_kernel(
    const uint8_t *__restrict__ As, const uint8_t *__restrict__ Bs, int kpad, const int *__restrict__ ea,
    const int *__restrict__ eb, int n_x, int n_T, double *__restrict__ u, int *__restrict__ err) {
    extern __shared__ uint8_t dsm[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[kStages], empty[kStages], lv_full, lv_empty;
    __shared__ uint32_t tslot;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.y * kTM, t0 = blockIdx.x * kTN;
    const int nkc = kpad / kKC, nseg = (kpad + kSegK - 1) / kSegK;
    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&lv_full, 1);
        tc::mbar_init(&lv_empty, 8);
        failed = 0;
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = tslot;
    const uint8_t *ablk = As + (size_t)blockIdx.y * nkc * kABlock;   // this tile's chunks, in K order
    const uint8_t *bblk = Bs + (size_t)blockIdx.x * nkc * kBBlock;
    if (tid == 0) {
        // producer: chunk k's A and B blocks into stage k % kStages
        for (int k = 0; k < nkc; ++k) {
            const int st = k % kStages;
            if (k >= kStages && !tc::mbar_wait(&empty[st], (uint32_t)(((k / kStages) - 1) & 1), kWaitLimit)) {
                failed = 1;
                break;
            }
            tc::mbar_arrive_tx(&full[st], kStage);
            tc::bulk_load(sm + st * kStage, ablk + (size_t)k * kABlock, kABlock, &full[st]);
            tc::bulk_load(sm + st * kStage + kABlock, bblk + (size_t)k * kBBlock, kBBlock, &full[st]);
        }
    } else if (tid == 32) {
        // MMA issuer.  The B slices of a stage are consecutive 64-row blocks of
        // one K-major operand, so A slice i against B slices j0 .. j0 + n - 1
        // (N = 64 n <= 256) writes the products a_i b_j to accumulator columns
        // 64 (i + j): the level of each pair.  Twelve MMAs cover the 36 pairs.
        constexpr uint32_t sbo = (kKBytes / 16) * 128;
        const uint64_t desc0 = tc::smem_desc(tc::smem_u32(sm), 128, sbo);
        for (int k = 0; k < nkc && !failed; ++k) {
            const int st = k % kStages, kin = k % (kSegK / kKC);
            if (!tc::mbar_wait(&full[st], (uint32_t)((k / kStages) & 1), kWaitLimit) ||
                (kin == 0 && k > 0 && !tc::mbar_wait(&lv_empty, (uint32_t)(((k / (kSegK / kKC)) - 1) & 1), kWaitLimit))) {
                failed = 1;
                break;
            }
            tc::tc_fence_after();
            const uint64_t ds = desc0 + (uint64_t)((st * kStage) >> 4);
#pragma unroll
            for (int i = 0; i < kSlices; ++i) {
                const uint64_t da = ds + (uint64_t)((i * kASlice) >> 4);
#pragma unroll
                for (int j0 = 0; j0 < kSlices - i; j0 += 4) {
                    const int n = (kSlices - i - j0) < 4 ? (kSlices - i - j0) : 4;   // slices of B
                    const uint64_t db = ds + (uint64_t)((kABlock + j0 * kBSlice) >> 4);
                    const uint32_t id = tc::instr_desc(1u, kTM, kTN * n);
                    tc::mma<1>(taddr + (uint32_t)((i + j0) * kTN), da, db, id, (kin == 0 && i == 0) ? 0u : 1u);
                }
            }
            tc::mma_commit(&empty[st]);
            if (kin == kSegK / kKC - 1 || k == nkc - 1) tc::mma_commit(&lv_full);   // a segment's levels
        }
    } else if (warp >= 4) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows), columns
        // 32 ((w - 4) / 4) .. of each level; double-float sums across segments
        const int q = warp & 3, ch = (warp - 4) >> 2;
        const int x = x0 + 32 * q + lane;
        float hi[2][16], lo[2][16];
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
            for (int c = 0; c < 16; ++c) hi[g][c] = lo[g][c] = 0.f;
        bool ok = true;
        for (int sg = 0; sg < nseg && ok; ++sg) {
            ok = tc::mbar_wait(&lv_full, (uint32_t)(sg & 1), kWaitLimit);
            if (tc::bar_or(1, 256, !ok)) {   // the same verdict in every epilogue thread
                ok = false;
                break;
            }
            tc::tc_fence_after();
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int c0 = 32 * ch + 16 * g;
                float h2[16], l2[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) h2[c] = l2[c] = 0.f;
#pragma unroll 1
                for (int d = kSlices - 1; d >= 0; --d) {   // smallest levels first
                    float v[16];
                    tc::tmem_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(d * kTN + c0), v);
                    const float sc = ldexpf(1.f, -kSliceBits * d);   // level d relative to level 0
#pragma unroll
                    for (int c = 0; c < 16; ++c) {          // (h2, l2) += v sc, two-sum
                        const float p = v[c] * sc;           // exact: integer times a power of two
                        const float t = h2[c] + p, bb = t - h2[c];
                        l2[c] += (h2[c] - (t - bb)) + (p - bb);
                        h2[c] = t;
                    }
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) {   // segment sum into the running sum
                    const dfv r = df_add(df_make(hi[g][c], lo[g][c]), df_make(h2[c], l2[c]));
                    hi[g][c] = r.hi;
                    lo[g][c] = r.lo;
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&lv_empty);   // the levels may be overwritten
        }
        if (!ok && lane == 0) failed = 1;
        if (ok && x < n_x) {
            const int ex = ea[x];
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int t = t0 + 32 * ch + 16 * g + c;
                    if (t < n_T)
                        u[(long long)x * n_T + t] =
                            ldexp((double)hi[g][c] + (double)lo[g][c], ex + eb[t] - 2 * kSliceBits);
                }
        }
    }
    // drain: loads and MMAs in flight have landed before the CTA ends (a
    // no-op unless a wait gave up)
    if (tid == 0) {
        for (int k = max(0, nkc - kStages); k < nkc; ++k)
            tc::mbar_wait(&full[k % kStages], (uint32_t)((k / kStages) & 1), kWaitLimit);
    } else if (tid == 32) {
        for (int k = max(0, nkc - kStages); k < nkc; ++k)
            tc::mbar_wait(&empty[k % kStages], (uint32_t)((k / kStages) & 1), kWaitLimit);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (failed && tid == 0) atomicOr(err, 1);
    if (warp == 0) tc::tmem_free(taddr, 512);
}

}  // namespace

int contract_tc_kpad(int J) { return (2 * J + kKPad - 1) / kKPad * kKPad; }
int contract_tc_rows(int n) { return (n + kTM - 1) / kTM * kTM; }
int contract_tc_cols(int n) { return (n + kTN - 1) / kTN * kTN; }
bool contract_tc_ok(int J) { return 2 * J <= kContractTcMaxK; }

size_t contract_tc_scratch_bytes(int J, int n_x, int n_T) {
    const size_t kp = (size_t)contract_tc_kpad(J);
    const size_t rx = (size_t)contract_tc_rows(n_x), rt = (size_t)contract_tc_cols(n_T);
    return (size_t)kSlices * (rx + rt) * kp * sizeof(__nv_bfloat16) + (rx + rt) * sizeof(int);
}

cudaError_t launch_contract_tc(int J, int n_x, int n_T, const double2 *V, const double *Gr,
                               const double *Gm, double *u, void *scratch, int *err, cudaStream_t st) {
    if (n_x <= 0 || n_T <= 0) return cudaSuccess;
    static std::atomic<unsigned long long> attr{0};
    {
        const cudaError_t e = ensure_smem_attr((const void *)contract_tc_kernel, kSmem, attr);
        if (e != cudaSuccess) return e;
    }
    const int kp = contract_tc_kpad(J), rx = contract_tc_rows(n_x), rt = contract_tc_cols(n_T);
    __nv_bfloat16 *As = static_cast<__nv_bfloat16 *>(scratch);
    __nv_bfloat16 *Bs = As + (size_t)kSlices * rx * kp;
    int *ea = reinterpret_cast<int *>(Bs + (size_t)kSlices * rt * kp);
    int *eb = ea + rx;
    const Src sa{V, nullptr, nullptr, J, n_x, n_x};
    const Src sbt{nullptr, Gr, Gm, J, n_T, n_T};
    ozaki_scale_kernel<<<rx / 32, kThr, 0, st>>>(sa, 2 * J, ea);
    ozaki_scale_kernel<<<rt / 32, kThr, 0, st>>>(sbt, 2 * J, eb);
    ozaki_slice_kernel<<<dim3(kp / 32, rx / 64), kThr, 0, st>>>(sa, ea, kp, kTM, As);
    ozaki_slice_kernel<<<dim3(kp / 32, rt / 64), kThr, 0, st>>>(sbt, eb, kp, kTN, Bs);
    contract_tc_kernel<<<dim3(rt / kTN, rx / kTM), kCtaThreads, kSmem, st>>>(
        reinterpret_cast<const uint8_t *>(As), reinterpret_cast<const uint8_t *>(Bs), kp, ea, eb, n_x, n_T, u, err);
    return cudaGetLastError();
}

}  // namespace fh
