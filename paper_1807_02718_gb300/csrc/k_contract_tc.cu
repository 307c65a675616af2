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
// level d = i + j sums at most kSlices pairs over K <= 512 terms below 2^24
// (8 x 512 x 2^12 = 2^24), so every level is an exact integer sum: TMEM holds
// one FP32 accumulator per level (kSlices x 64 = 512 columns, all of it).  The epilogue combines the levels, scaled by
// 2^-(kSliceBits (d + 2)), in double-float and multiplies by sa_x sb_t.  The
// result differs from the exact product by the dropped slice pairs (i + j >=
// kSlices) and the remainders, ~K 2^-48 sa_x sb_t at worst.
//
// Kernels: ozaki_scale_kernel (the power-of-two scale of each row of A and
// each column of B), ozaki_slice_kernel (slices, written K-major in BF16
// through a shared-memory transpose), contract_tc_kernel (one CTA per 128 x 64
// output tile; K in chunks of 64: all slices of the chunk staged in shared
// memory in the canonical no-swizzle K-major layout, one thread issues the
// kind::f16 MMAs of every pair into its level's accumulator, bounded mbarrier
// wait; then the double-float epilogue).
#include <cuda_bf16.h>

#include "fh_internal.h"
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
constexpr int kStage = kSlices * (kASlice + kBSlice);   // 42 KiB
constexpr int kStages = 4;                              // chunks k+1 .. k+3 in flight
constexpr int kSmem = 1024 + kStages * kStage;
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

// Slices of a 64-row x 32-column block: out[s][r][kk] (row pitch kpad, BF16).
// In integer arithmetic on the FP64 bit pattern: V = round(src 2^(42 - e[r]))
// (|V| <= 2^48) = sum_s a_s 2^(42 - 6 s) with balanced digits, each the
// nearest multiple of the remainder (a_0 in [-64, 64], a_s in [-32, 32]), so
// that the dropped slice products carry no common sign: src / 2^e[r] =
// sum_s a_s 2^-(6 (s + 1)) to within 2^-49.
__global__ void __launch_bounds__(kThr) ozaki_slice_kernel(Src src, const int *__restrict__ e,
                                                           int kpad, long long slice_stride,
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
    for (int idx = threadIdx.x; idx < kSlices * 64 * 32; idx += kThr) {
        const int kk = idx & 31, rr = (idx >> 5) & 63, s = idx >> 11;   // consecutive threads: consecutive kk
        out[s * slice_stride + (long long)(r0 + rr) * kpad + k0 + kk] = t[s][kk][rr];
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Every slice of K chunk k0 .. k0 + kKC - 1 into one stage: 16-byte rows of
// 8-row core matrices, copied asynchronously (in flight during the MMAs of
// the chunks before).  Thread t copies 16-byte chunk t % 2 of A row t / 2
// and, for t < 128, of B row t / 2, for every slice.  Always commits a
// group (empty past the last chunk), so that group counting stays uniform.
__device__ __forceinline__ void stage_chunk(const __nv_bfloat16 *__restrict__ a_row,
                                            const __nv_bfloat16 *__restrict__ b_row, long long a_stride,
                                            long long b_stride, bool has_b, int k0, bool live,
                                            uint32_t stage, uint32_t dA, uint32_t dB) {
    if (live) {
#pragma unroll
        for (int sl = 0; sl < kSlices; ++sl) {
            cp_async16(stage + sl * kASlice + dA, a_row + sl * a_stride + k0);
            if (has_b) cp_async16(stage + kSlices * kASlice + sl * kBSlice + dB, b_row + sl * b_stride + k0);
        }
    }
    cp_async_commit();
}

__global__ void __launch_bounds__(kThr, 1) contract_tc_kernel(
    const __nv_bfloat16 *__restrict__ As, const __nv_bfloat16 *__restrict__ Bs, long long a_stride,
    long long b_stride, int kpad, const int *__restrict__ ea, const int *__restrict__ eb, int n_x,
    int n_T, double *__restrict__ u, int *__restrict__ err) {
    extern __shared__ uint8_t dsm[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bar[kStages];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.y * kTM, t0 = blockIdx.x * kTN;
    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (tid == 0)
        for (int s = 0; s < kStages; ++s) tc::mbar_init(&bar[s], 1);
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = tslot;
    const uint32_t st0 = tc::smem_u32(sm);
    constexpr uint32_t sbo = (kKBytes / 16) * 128;
    const int nk = kpad / kKC;
    // this thread's copies: 16-byte chunk tid % 2 of A row tid / 2 (and of B row tid / 2)
    const int crow = tid >> 1, cch = tid & 1;
    const bool has_b = crow < kTN;
    const __nv_bfloat16 *a_row = As + (long long)(x0 + crow) * kpad + cch * 8;
    const __nv_bfloat16 *b_row = Bs + (long long)(t0 + (has_b ? crow : 0)) * kpad + cch * 8;
    const uint32_t dA = tc::kmajor_offset(crow, cch * 16, kKBytes), dB = dA;
    // MMA descriptors differ only in the start address field (address / 16)
    const uint64_t desc0 = tc::smem_desc(st0, 128, sbo);
    bool ok = true;
    uint32_t phase[kStages] = {};
    bool pending[kStages] = {};
    for (int k = 0; k < kStages - 1; ++k)
        stage_chunk(a_row, b_row, a_stride, b_stride, has_b, k * kKC, k < nk, st0 + k * kStage, dA, dB);
    for (int k = 0; k < nk; ++k) {
        const int s = k % kStages;
        cp_async_wait<kStages - 2>();   // chunk k has landed (k+1, k+2 may be in flight)
        tc::fence_async_smem();
        tc::tc_fence_before();
        ok = __syncthreads_and(ok) != 0;
        tc::tc_fence_after();
        if (!ok) break;
        if (tid == 0) {   // queued behind the previous chunks' MMAs
            // The B slices of a stage are consecutive 64-row blocks of one K-major
            // operand, so A slice i against B slices j0 .. j0 + n - 1 (N = 64 n <=
            // 256) writes the products a_i b_j to accumulator columns 64 (i + j):
            // the level of each pair.  Twelve MMAs cover the 36 pairs.
            const uint64_t ds = desc0 + (uint64_t)((s * kStage) >> 4);
#pragma unroll
            for (int i = 0; i < kSlices; ++i) {
                const uint64_t da = ds + (uint64_t)((i * kASlice) >> 4);
#pragma unroll
                for (int j0 = 0; j0 < kSlices - i; j0 += 4) {
                    const int n = (kSlices - i - j0) < 4 ? (kSlices - i - j0) : 4;   // slices of B
                    const uint64_t db = ds + (uint64_t)((kSlices * kASlice + j0 * kBSlice) >> 4);
                    const uint32_t id = tc::instr_desc(1u, kTM, kTN * n);
                    tc::mma<1>(taddr + (uint32_t)((i + j0) * kTN), da, db, id, (k == 0 && i == 0) ? 0u : 1u);
                }
            }
            tc::mma_commit(&bar[s]);
        }
        pending[s] = true;
        // refill the stage of chunk k - 1 with chunk k + kStages - 1 once that
        // chunk's MMAs (ahead of chunk k's in the tensor pipe) are done
        const int sp = (k + kStages - 1) % kStages;
        if (pending[sp]) {
            if (!tc::mbar_wait(&bar[sp], phase[sp], kWaitLimit)) ok = false;
            phase[sp] ^= 1u;
            pending[sp] = false;
        }
        const int kn = k + kStages - 1;
        stage_chunk(a_row, b_row, a_stride, b_stride, has_b, kn * kKC, ok && kn < nk, st0 + sp * kStage,
                    dA, dB);   // after a give-up the stage may still be read: nothing copied
    }
    cp_async_wait<0>();
    // the last chunk's MMAs (the MMAs of one thread complete in issue order)
    bool got = true;
    for (int s = 0; s < kStages; ++s)
        if (pending[s]) {
            const bool g = tc::mbar_wait(&bar[s], phase[s], kWaitLimit);
            phase[s] ^= 1u;
            got = got && g;
        }
    tc::tc_fence_after();
    ok = __syncthreads_and(ok && got) != 0;
    if (!ok) {
        if (tid == 0) atomicOr(err, 1);
    } else {
        // warp w: TMEM lanes 32 (w % 4) .. (rows), columns 32 (w / 4) .. of each level
        const int q = warp & 3, ch = warp >> 2;
        const int x = x0 + 32 * q + lane;
        const int ex = x < n_x ? ea[x] : 0;
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
            const int c0 = 32 * ch + 16 * g;
            float hi[16], lo[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) hi[k] = lo[k] = 0.f;
#pragma unroll 1
            for (int d = kSlices - 1; d >= 0; --d) {   // smallest levels first
                float v[16];
                tc::tmem_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(d * kTN + c0), v);
                const float sc = ldexpf(1.f, -kSliceBits * d);   // level d relative to level 0
#pragma unroll
                for (int k = 0; k < 16; ++k) {          // (hi, lo) += v sc, two-sum
                    const float p = v[k] * sc;           // exact: integer times a power of two
                    const float t = hi[k] + p, bb = t - hi[k];
                    lo[k] += (hi[k] - (t - bb)) + (p - bb);
                    hi[k] = t;
                }
            }
            if (x < n_x)
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int t = t0 + c0 + k;
                    if (t < n_T)
                        u[(long long)x * n_T + t] =
                            ldexp((double)hi[k] + (double)lo[k], ex + eb[t] - 2 * kSliceBits);
                }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
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
    ozaki_slice_kernel<<<dim3(kp / 32, rx / 64), kThr, 0, st>>>(sa, ea, kp, (long long)rx * kp, As);
    ozaki_slice_kernel<<<dim3(kp / 32, rt / 64), kThr, 0, st>>>(sbt, eb, kp, (long long)rt * kp, Bs);
    contract_tc_kernel<<<dim3(rt / kTN, rx / kTM), kThr, kSmem, st>>>(As, Bs, (long long)rx * kp,
                                                                    (long long)rt * kp, kp, ea, eb,
                                                                    n_x, n_T, u, err);
    return cudaGetLastError();
}

}  // namespace fh
