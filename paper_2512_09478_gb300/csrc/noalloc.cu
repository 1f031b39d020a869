// Energy reduction that allocates nothing.
//
// Who needs it: callers that cannot allocate device memory at the point where
// they want the long-range energy.  A DEM step recorded into a CUDA graph
// cannot call cudaMalloc during capture; a host application that hands all
// device memory to its own pool may forbid allocations by libraries; a
// time-critical integration loop may not afford a trip through an allocator.
// kifmm_energy_noalloc computes U = 1/2 sum_i q_i pot_i with a deterministic
// two-stage reduction (fixed 4096-particle chunks, then one ordered sum of the
// chunk partials), the scheme kifmm_evaluate uses for its energy output, and
// equal to that output up to rounding; it keeps the partials in a fixed array
// that is part of the library's device image, not in plan workspace.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace kifmm {
namespace {

constexpr int64_t kNaChunk = 4096;       // particles per partial sum
constexpr int64_t kNaMaxChunks = 16384;  // 128 KiB of partials: at most 67,108,864 particles per call
constexpr int kNaMaxDevices = 64;

// Shared by every call on a device; holds the last call's partials.
static __device__ __align__(256) double g_na_partials[kNaMaxChunks];

std::mutex g_na_mutex;
double *g_na_ptr[kNaMaxDevices] = {nullptr};

template <typename T>
__global__ void k_na_partials(int64_t n, const T *__restrict__ q, const T *__restrict__ pot, double *partials) {
    __shared__ double red[256];
    const int64_t a = (int64_t)blockIdx.x * kNaChunk;
    const int64_t e = min(n, a + kNaChunk);
    double s = 0.0;
    for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) s += (double)q[i] * (double)pot[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// One block, fixed summation order: deterministic for a given n.
__global__ void k_na_final(int64_t nchunks, const double *__restrict__ partials, double *energy) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t c = threadIdx.x; c < nchunks; c += blockDim.x) s += partials[c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *energy = 0.5 * red[0];
}

// Device address of the partials for the current device (looked up once per
// device, with that device current).
cudaError_t na_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_na_partials);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace kifmm

extern "C" kifmm_status kifmm_energy_noalloc(int64_t n, int dtype, const void *q, const void *pot, double *energy,
                                             kifmm_stream_t stream) {
    using namespace kifmm;
    if (n < 0 || !energy || (n > 0 && (!q || !pot))) return KIFMM_ERR_ARG;
    if (dtype != KIFMM_DTYPE_F32 && dtype != KIFMM_DTYPE_F64) return KIFMM_ERR_ARG;
    const int64_t nchunks = (n + kNaChunk - 1) / kNaChunk;
    if (nchunks > kNaMaxChunks) return KIFMM_ERR_CAPACITY;
    double *scratch = nullptr;
    if (na_scratch(&scratch) != cudaSuccess) {
        (void)cudaGetLastError();
        return KIFMM_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (nchunks > 0) {
        if (dtype == KIFMM_DTYPE_F64)
            k_na_partials<double><<<(unsigned)nchunks, 256, 0, s>>>(n, (const double *)q, (const double *)pot, scratch);
        else
            k_na_partials<float><<<(unsigned)nchunks, 256, 0, s>>>(n, (const float *)q, (const float *)pot, scratch);
    }
    k_na_final<<<1, 256, 0, s>>>(nchunks, scratch, energy);
    if (cudaGetLastError() != cudaSuccess) return KIFMM_ERR_CUDA;
    return KIFMM_OK;
}
