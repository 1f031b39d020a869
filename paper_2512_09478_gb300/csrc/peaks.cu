// Peak-rate microbenchmarks of the units the hot path uses: FP32 FMA (the
// leaf kernel's pair arithmetic), the FP32 reciprocal square root (one per
// pair), FP64 FMA (the FP64 mode) and the tcgen05 kind::f16 MMA in the shape
// the M2L kernel issues (M = 128, K = 16, 64-byte swizzled K-major operands,
// N = 160 and 256).  They give the roofline denominators that the measured
// copy bandwidth and cuBLAS GEMM rates do not cover.  Each kernel runs long
// independent chains on every SM; times come from CUDA events.
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace kifmm {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void k_peak_fma(int iters, T x, T y, T *sink) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] * x + y;
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)-1.2345) sink[0] = s;  // keeps the chains alive; never true
}

__global__ void k_peak_rsqrt(int iters, float *sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1.0f + 0.1f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = rsqrt_t<float>(a[c]);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.2345f) sink[0] = s;
}

// One CTA per SM: thread 0 issues `reps` x 2 MMAs (K = 16 each) into one TMEM
// accumulator from zero-filled operands, then waits (bounded) for them.
template <int N>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int reps, int *status) {
    __shared__ __align__(1024) unsigned char ops[kTcRows * 64 + N * 64];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int never;
    for (int i = threadIdx.x; i < (int)sizeof(ops) / 4; i += blockDim.x) ((uint32_t *)ops)[i] = 0u;
    if (threadIdx.x == 0) {
        never = 0;
        mbar_init(smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    fence_proxy_async();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    if (threadIdx.x == 0) {
        const uint32_t sA = smem_u32(ops), sB = sA + kTcRows * 64;
        const uint32_t id = idesc_f16(N);
        for (int r = 0; r < reps; ++r)
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
                mma_f16(tmem, sdesc_sw64(sA + 32 * kk), sdesc_sw64(sB + 32 * kk), id, (r | kk) ? 1u : 0u);
        mma_commit(smem_u32(&done));
        if (!mbar_wait(smem_u32(&done), 0, &never)) set_status(status, KIFMM_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
}

template <class F>
float best_ms(cudaStream_t s, int reps, F &&launch) {
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) best = std::min(best, time_launch(s, launch));
    return best;
}

}  // namespace
}  // namespace kifmm

using namespace kifmm;

extern "C" {

kifmm_status kifmm_measure_peaks(kifmm_peaks_t *out, kifmm_stream_t stream) {
    if (!out) return KIFMM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, clock_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KIFMM_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
    void *sink = nullptr;
    int *status = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess || cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
        cudaFree(sink);
        return KIFMM_ERR_CUDA;
    }
    cudaMemsetAsync(status, 0, sizeof(int), s);
    const int blocks = sms * 8, threads = 256;
    const int it32 = 1 << 14, it64 = 1 << 10, itr = 1 << 12;
    const double fma_ops = (double)blocks * threads * kChains;
    const float ms32 = best_ms(s, 3, [&] {
        k_peak_fma<float><<<blocks, threads, 0, s>>>(it32, 1.0000001f, 1e-7f, (float *)sink);
    });
    const float ms64 = best_ms(s, 3, [&] {
        k_peak_fma<double><<<blocks, threads, 0, s>>>(it64, 1.0000000001, 1e-12, (double *)sink);
    });
    const float msr = best_ms(s, 3, [&] { k_peak_rsqrt<<<blocks, threads, 0, s>>>(itr, (float *)sink); });
    const int reps = 1 << 14;
    const float ms160 = best_ms(s, 3, [&] { k_peak_mma<160><<<sms, 128, 0, s>>>(reps, status); });
    const float ms256 = best_ms(s, 3, [&] { k_peak_mma<256><<<sms, 128, 0, s>>>(reps, status); });
    int st = 0;
    cudaError_t e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(sink);
    cudaFree(status);
    if (e != cudaSuccess) return KIFMM_ERR_CUDA;
    if (st != 0) return (kifmm_status)st;
    out->fp32_fma_tflops = 2.0 * fma_ops * it32 / (ms32 * 1e-3) / 1e12;
    out->fp64_fma_tflops = 2.0 * fma_ops * it64 / (ms64 * 1e-3) / 1e12;
    out->rsqrt_per_s = fma_ops * itr / (msr * 1e-3);
    const double mma = (double)sms * reps * 2 * 2.0 * kTcRows * 16;
    out->f16_mma_n160_tflops = mma * 160 / (ms160 * 1e-3) / 1e12;
    out->f16_mma_n256_tflops = mma * 256 / (ms256 * 1e-3) / 1e12;
    out->sms = sms;
    out->clock_mhz = clock_khz / 1000.0;
    return KIFMM_OK;
}

}  // extern "C"
