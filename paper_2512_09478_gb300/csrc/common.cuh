// Device helpers shared by the KIFMM kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kifmm {

// Kernel launches issued by the library on this thread (profiling).
extern thread_local long long g_launches;

#define KIFMM_CUDA_TRY(expr)                       \
    do {                                           \
        cudaError_t e__ = (expr);                  \
        if (e__ != cudaSuccess) return e__;        \
    } while (0)

// Record the first device-detected error (kifmm_status numbering).
__device__ __forceinline__ void set_status(int *status, int code) {
    atomicCAS(status, 0, code);
}

// 1/(4 pi)
__host__ __device__ constexpr double kInv4Pi = 0.07957747154594767;

// Surface radii (multiples of the box half-width): upward equivalent 1.05,
// upward check 2.95, downward equivalent 2.95, downward check 1.05.
__host__ __device__ constexpr double kAlphaInner = 1.05;
__host__ __device__ constexpr double kAlphaOuter = 2.95;

// Two boxes (level, integer coordinates) are adjacent when their closed
// cubes intersect and neither contains the other.
__device__ __forceinline__ bool boxes_adjacent(int la, int ax, int ay, int az, int lb, int bx, int by,
                                               int bz) {
    const int L = la > lb ? la : lb;
    const int sa = L - la, sb = L - lb;
    const int a[3] = {ax, ay, az}, b[3] = {bx, by, bz};
    bool a_in_b = true, b_in_a = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int alo = a[d] << sa, ahi = (a[d] + 1) << sa;
        const int blo = b[d] << sb, bhi = (b[d] + 1) << sb;
        if (alo > bhi || blo > ahi) return false;
        a_in_b = a_in_b && (blo <= alo) && (ahi <= bhi);
        b_in_a = b_in_a && (alo <= blo) && (bhi <= ahi);
    }
    return !(a_in_b || b_in_a);
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double4;
};

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
// FP32: the hardware approximation (rsqrt.approx, relative error below
// 2^-22.9), flushing subnormal inputs; callers exclude r = 0 themselves.
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) {
    return rsqrt(x);
}

// Laplace kernel value and gradient (w.r.t. the target) for a displacement
// r = target - source, scaled by a source weight w; zero when r = 0.
template <typename T>
__device__ __forceinline__ void lap_accum(T rx, T ry, T rz, T w, T &pot, T &gx, T &gy, T &gz) {
    const T r2 = rx * rx + ry * ry + rz * rz;
    const T rinv = (r2 > T(0)) ? rsqrt_t<T>(r2) : T(0);
    const T wr = w * rinv;
    const T wr3 = wr * rinv * rinv;
    pot += wr;
    gx -= rx * wr3;
    gy -= ry * wr3;
    gz -= rz * wr3;
}

// The same without the r = 0 test, for sources that cannot coincide with
// the target.
template <typename T>
__device__ __forceinline__ void lap_accum_nz(T rx, T ry, T rz, T w, T &pot, T &gx, T &gy, T &gz) {
    const T r2 = rx * rx + ry * ry + rz * rz;
    const T rinv = rsqrt_t<T>(r2);
    const T wr = w * rinv;
    const T wr3 = wr * rinv * rinv;
    pot += wr;
    gx -= rx * wr3;
    gy -= ry * wr3;
    gz -= rz * wr3;
}

template <typename T>
__device__ __forceinline__ T lap_pot(T rx, T ry, T rz) {
    const T r2 = rx * rx + ry * ry + rz * rz;
    return (r2 > T(0)) ? rsqrt_t<T>(r2) : T(0);
}

}  // namespace kifmm
