// Arithmetic-peak probes, used to state the rooflines of the path's kernels
// on the device they run on:
//  * a long chain of independent FP64 (or FP32) FMAs per thread, enough warps
//    to fill every SM (the FP64 and double-float kernels);
//  * back-to-back tcgen05 MMAs (M = 128, N = 256, one K step) from operands
//    resident in shared memory, one CTA per SM (the TF32 / BF16 tensor-core
//    kernels): the tensor pipe's own rate, without operand traffic.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fh.h"
#include "tc_gemm.cuh"

namespace {

constexpr int kChains = 16;

template <class T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T *out, int iters, T seed) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T m = (T)0.999999, k = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)-1) out[blockIdx.x] = s;   // never true; keeps the chains live
}

template <class T>
fh_status probe(int device, int iters, double *tflops) {
    if (!tflops || iters < 1) return FH_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return FH_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * 4096) != cudaSuccess) return FH_ENOMEM;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // best of several occupancies (2..8 CTAs of 256 threads per SM)
    double best = 0.0;
    cudaError_t e = cudaSuccess;
    for (int per_sm = 2; per_sm <= 8 && e == cudaSuccess; per_sm *= 2) {
        const int blocks = sms * per_sm;
        fma_chain_kernel<T><<<blocks, 256>>>(out, 64, (T)1);   // warm-up
        cudaEventRecord(a);
        fma_chain_kernel<T><<<blocks, 256>>>(out, iters, (T)1);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && ms > 0.f)
            best = std::max(best, 2.0 * kChains * (double)iters * blocks * 256.0 / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess || best <= 0.0) return FH_ECUDA;
    *tflops = best;
    return FH_OK;
}

constexpr int kPeakN = 256;                 // accumulator columns per MMA
constexpr long long kPeakWait = 1LL << 26;  // bounded completion wait (far above the run)

// One elected thread issues `iters` MMAs of M = 128, N = 256 and one K step
// (32 bytes of K per row: 16 BF16 or 8 TF32 values) alternating between two
// TMEM accumulators; the operands are fixed tiles in shared memory.
template <int kKind>
__global__ void __launch_bounds__(128) mma_peak_kernel(int iters, int *err) {
    extern __shared__ uint8_t dsm[];
    uint8_t *sa = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
    uint8_t *sb = sa + fh::tc::kM * 32;
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    // small non-zero operand values (1 + k/64 in BF16 or TF32 bit patterns)
    for (int i = tid; i < (fh::tc::kM + kPeakN) * 8; i += 128) {
        const float v = 1.0f + (float)(i & 63) / 64.0f;
        uint32_t w = __float_as_uint(v);
        if (kKind == 1) w = (w >> 16) | (w & 0xFFFF0000u);   // two BF16 halves
        reinterpret_cast<uint32_t *>(sa)[i] = w;
    }
    if (warp == 0) fh::tc::tmem_alloc(&tslot, 2 * kPeakN);
    if (tid == 0) fh::tc::mbar_init(&bar, 1);
    fh::tc::fence_async_smem();
    fh::tc::tc_fence_before();
    __syncthreads();
    fh::tc::tc_fence_after();
    const uint32_t taddr = tslot;
    if (tid == 0) {
        constexpr uint32_t idesc = fh::tc::instr_desc(kKind == 1 ? 1u : 2u, fh::tc::kM, kPeakN);
        const uint64_t da = fh::tc::smem_desc(fh::tc::smem_u32(sa), 128, 256);
        const uint64_t db = fh::tc::smem_desc(fh::tc::smem_u32(sb), 128, 256);
        for (int i = 0; i < iters; ++i)
            fh::tc::mma<kKind>(taddr + (uint32_t)((i & 1) * kPeakN), da, db, idesc, i >= 2 ? 1u : 0u);
        fh::tc::mma_commit(&bar);
    }
    const bool got = fh::tc::mbar_wait(&bar, 0, kPeakWait);
    if (!got) atomicOr(err, 1);
    fh::tc::tc_fence_after();
    __syncthreads();
    if (warp == 0) fh::tc::tmem_free(taddr, 2 * kPeakN);
}

fh_status mma_probe(int device, int kind, int iters, double *tflops) {
    if (!tflops || iters < 2 || (kind != 1 && kind != 2)) return FH_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return FH_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return FH_ENOMEM;
    cudaMemset(err, 0, sizeof(int));
    // more shared memory than two CTAs can share, so that one CTA runs per SM
    // and its 512 TMEM columns are always free
    const int smem = 120 * 1024;
    const void *fn = kind == 1 ? (const void *)mma_peak_kernel<1> : (const void *)mma_peak_kernel<2>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double best = 0.0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a);
        if (kind == 1) mma_peak_kernel<1><<<sms, 128, smem>>>(rep == 0 ? 64 : iters, err);
        else mma_peak_kernel<2><<<sms, 128, smem>>>(rep == 0 ? 64 : iters, err);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double k_step = kind == 1 ? 16.0 : 8.0;
        if (rep > 0 && e == cudaSuccess && ms > 0.f)
            best = std::max(best, 2.0 * fh::tc::kM * kPeakN * k_step * (double)iters * sms / (ms * 1e-3) / 1e12);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(err);
    if (e != cudaSuccess) return FH_ECUDA;
    if (herr) return FH_ETIMEOUT;
    if (best <= 0.0) return FH_ECUDA;
    *tflops = best;
    return FH_OK;
}

}  // namespace

extern "C" fh_status fh_probe_mma_peak(int device, int kind, int iters, double *tflops) {
    return mma_probe(device, kind, iters, tflops);
}

extern "C" fh_status fh_probe_fma_peak(int device, int fp64, int iters, double *tflops) {
    return fp64 ? probe<double>(device, iters, tflops) : probe<float>(device, iters, tflops);
}
