// Diagnostics.
//
// FMA throughput of the device, measured: the denominator for the roofline of the deposit kernels,
// which are bound by FP32 (mixed) and FP64 (plain) arithmetic rather than by memory or tensor cores.
//
// Every thread runs kChains independent multiply-add chains a <- a * m + c (|m| < 1, so values stay
// bounded) in an unrolled loop; enough warps per SM cover the FMA latency, so the pipe, not the
// dependency, sets the rate.  One FMA counts as two flops.
#include <cuda_runtime.h>

#include "rd_internal.cuh"

namespace rd {

namespace {

constexpr int kChains = 8;
constexpr int kInner = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T m, T c, int iters, T* sink)
{
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kInner; ++u) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], m, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    // never true for these inputs; keeps every chain live without a store per thread
    if (s == (T)-1.0) sink[blockIdx.x] = s;
}

// TFLOP/s of one timed launch sized to run for about target_ms.
template <typename T>
cudaError_t measure(int sms, cudaStream_t s, T* sink, double target_ms, double* tflops)
{
    const int blocks = sms * kBlocksPerSm;
    const double flops_per_iter = 2.0 * kChains * kInner * (double)blocks * kThreads;
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return err;
    err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return err;
    }
    int iters = 64;
    float ms = 0.f;
    for (int round = 0; round < 4; ++round) {
        k_fma_peak<T><<<blocks, kThreads, 0, s>>>((T)0.999999, (T)1e-6, iters, sink);   // warm-up / sizing
        cudaEventRecord(e0, s);
        k_fma_peak<T><<<blocks, kThreads, 0, s>>>((T)0.999999, (T)1e-6, iters, sink);
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) break;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms >= 0.5 * target_ms) break;
        const double scale = target_ms / (ms > 1e-3f ? ms : 1e-3f);
        const double next = iters * (scale < 64.0 ? scale : 64.0);
        iters = next > 1e8 ? 100000000 : (int)next;
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) *tflops = flops_per_iter * iters / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

// One CTA waits, with the kernels' bounded wait, for phase 0 of an mbarrier that expects one arrival
// and gets none: the wait runs out after limit_ns and the CTA records RD_ERR_TIMEOUT the way the
// deposit and adjoint kernels do, then returns.  Nothing is left in flight.
__global__ void k_wait_probe(unsigned long long limit_ns, unsigned* errors)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded_ns(&bar, 0u, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(errors, ERRBIT_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_probe(unsigned long long limit_ns, unsigned* errors, cudaStream_t s)
{
    k_wait_probe<<<1, 32, 0, s>>>(limit_ns, errors);
    return cudaGetLastError();
}

cudaError_t measure_fma_peaks(cudaStream_t s, double* fp32_tflops, double* fp64_tflops)
{
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    void* sink = nullptr;
    err = cudaMalloc(&sink, sizeof(double) * sms * kBlocksPerSm);
    if (err != cudaSuccess) return err;
    if (fp32_tflops) err = measure<float>(sms, s, static_cast<float*>(sink), 20.0, fp32_tflops);
    if (err == cudaSuccess && fp64_tflops)
        err = measure<double>(sms, s, static_cast<double*>(sink), 20.0, fp64_tflops);
    cudaError_t e2 = cudaFree(sink);
    return err != cudaSuccess ? err : e2;
}

}  // namespace rd
