// Diagnostic tcgen05 GEMM: C = A B^T with A (M x K) and B (N x K) row-major
// FP32 in global memory, rounded to BF16 or used as TF32 by the tensor core,
// FP32 accumulation in TMEM.  Used to check the tensor-core building blocks
// (descriptors, TMEM, mbarrier protocol) against a host GEMM.
#include <cuda_bf16.h>

#include "fh.h"
#include "tc_gemm.cuh"

namespace {

constexpr int kBN = 256;            // output columns per CTA (TMEM columns)
constexpr int kKBytes = 128;        // bytes of K per row per stage (64 BF16 / 32 TF32)
constexpr long long kWaitLimit = 1LL << 20;

template <int kKind>
__global__ void __launch_bounds__(128) tc_gemm_test_kernel(const float *__restrict__ A,
                                                           const float *__restrict__ B,
                                                           float *__restrict__ C, int M, int N,
                                                           int K, int *__restrict__ err) {
    constexpr int esize = (kKind == 1) ? 2 : 4;
    constexpr int kc = kKBytes / esize;            // K elements per stage
    extern __shared__ uint8_t dsm[];
    // operand tiles at a 1 KiB-aligned offset inside the dynamic buffer
    uint8_t *sa = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    uint8_t *sb = sa + fh::tc::kM * kKBytes;
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * fh::tc::kM, n0 = blockIdx.x * kBN;
    if (warp == 0) fh::tc::tmem_alloc(&tslot, kBN);
    if (tid == 0) fh::tc::mbar_init(&bar, 1);
    fh::tc::fence_async_smem();
    fh::tc::tc_fence_before();
    __syncthreads();
    fh::tc::tc_fence_after();
    const uint32_t taddr = tslot;
    constexpr uint32_t idesc = fh::tc::instr_desc(kKind == 1 ? 1u : 2u, fh::tc::kM, kBN);
    constexpr uint32_t sbo = (kKBytes / 16) * 128;
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < K && ok; k0 += kc) {
        // stage A rows (one per thread) and B rows (two per thread)
        for (int r = tid; r < fh::tc::kM + kBN; r += 128) {
            const bool isA = r < fh::tc::kM;
            const int row = isA ? r : r - fh::tc::kM;
            const float *src = isA ? A + (long long)(m0 + row) * K + k0 : B + (long long)(n0 + row) * K + k0;
            uint8_t *dst = isA ? sa : sb;
            for (int k = 0; k < kc; ++k) {
                const float v = (k0 + k < K) ? src[k] : 0.f;
                const uint32_t off = fh::tc::kmajor_offset(row, k * esize, kKBytes);
                if (kKind == 1) *reinterpret_cast<__nv_bfloat16 *>(dst + off) = __float2bfloat16_rn(v);
                else *reinterpret_cast<float *>(dst + off) = v;
            }
        }
        fh::tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            fh::tc::tc_fence_after();
            const uint32_t a0 = fh::tc::smem_u32(sa), b0 = fh::tc::smem_u32(sb);
#pragma unroll
            for (int ki = 0; ki < kKBytes / 32; ++ki) {
                const uint64_t da = fh::tc::smem_desc(a0 + ki * 256, 128, sbo);
                const uint64_t db = fh::tc::smem_desc(b0 + ki * 256, 128, sbo);
                fh::tc::mma<kKind>(taddr, da, db, idesc, (k0 > 0 || ki > 0) ? 1u : 0u);
            }
            fh::tc::mma_commit(&bar);
        }
        const bool got = fh::tc::mbar_wait(&bar, phase, kWaitLimit);
        phase ^= 1;
        fh::tc::tc_fence_after();
        ok = __syncthreads_and(got) != 0;   // block-uniform before warp-collective loads
    }
    if (!ok) {
        if (tid == 0) atomicOr(err, 1);
        fh::tc::mbar_wait(&bar, phase ^ 1, kWaitLimit);   // let an in-flight MMA finish
    } else {
        const int row = warp * 32 + lane;
        for (int c = 0; c < kBN; c += 16) {
            float v[16];
            fh::tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (m0 + row < M)
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (n0 + c + i < N) C[(long long)(m0 + row) * N + n0 + c + i] = v[i];
        }
    }
    fh::tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) fh::tc::tmem_free(taddr, kBN);
}

}  // namespace

// kind: 1 = BF16 operands, 2 = TF32 operands.  M a multiple of 128, N of 256,
// K of 64; host arrays.  Returns FH_ETIMEOUT if an MMA completion wait ran out.
extern "C" fh_status fh_tc_gemm_test(int kind, int M, int N, int K, const float *A,
                                     const float *B, float *C) {
    if ((kind != 1 && kind != 2) || M <= 0 || N <= 0 || K <= 0 || M % 128 || N % kBN || K % 64 ||
        !A || !B || !C)
        return FH_EINVAL;
    float *dA = nullptr, *dB = nullptr, *dC = nullptr;
    int *derr = nullptr;
    fh_status st = FH_OK;
    if (cudaMalloc(&dA, sizeof(float) * M * K) != cudaSuccess ||
        cudaMalloc(&dB, sizeof(float) * N * K) != cudaSuccess ||
        cudaMalloc(&dC, sizeof(float) * M * N) != cudaSuccess || cudaMalloc(&derr, sizeof(int)) != cudaSuccess)
        st = FH_ENOMEM;
    if (st == FH_OK) {
        cudaMemcpy(dA, A, sizeof(float) * M * K, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, sizeof(float) * N * K, cudaMemcpyHostToDevice);
        cudaMemset(derr, 0, sizeof(int));
        dim3 grid(N / kBN, M / 128);
        // at most two CTAs per SM, so their 2 x 256 TMEM columns always fit
        const size_t smem = 100 * 1024;
        if (kind == 1) {
            cudaFuncSetAttribute(tc_gemm_test_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_gemm_test_kernel<1><<<grid, 128, smem>>>(dA, dB, dC, M, N, K, derr);
        } else {
            cudaFuncSetAttribute(tc_gemm_test_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_gemm_test_kernel<2><<<grid, 128, smem>>>(dA, dB, dC, M, N, K, derr);
        }
        int herr = 0;
        if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = FH_ECUDA;
        else if (herr)
            st = FH_ETIMEOUT;
        else if (cudaMemcpy(C, dC, sizeof(float) * M * N, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = FH_ECUDA;
    }
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(derr);
    cudaGetLastError();
    return st;
}
