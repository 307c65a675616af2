// Arithmetic-peak probes: a long chain of independent FP64 (or FP32) FMAs per
// thread, enough warps to fill every SM.  Used to state the ALU roofline of
// the FP64 kernels on the device they run on.
#include <cuda_runtime.h>

#include <algorithm>

#include "fh.h"

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

}  // namespace

extern "C" fh_status fh_probe_fma_peak(int device, int fp64, int iters, double *tflops) {
    return fp64 ? probe<double>(device, iters, tflops) : probe<float>(device, iters, tflops);
}
