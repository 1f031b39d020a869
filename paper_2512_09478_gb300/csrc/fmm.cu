// KIFMM evaluation passes (Sec. 2.2): upward pass (P2M, M2M), M2L over the
// V lists, P2L over the X lists, downward pass (L2L), leaf evaluation (L2P,
// M2P over the W lists) and the near field (P2P over the U lists).
//
// Units: positions are root-normalised (root cube side 1) and every box
// stores potentials of the kernel 1/r on its check surfaces:
//   u(b) on UC = c_b + 2.95 h_b S  (upward), d(b) on DC = c_b + 1.05 h_b S.
// The 1/(4 pi), the coefficient and the 1/side, 1/side^2 of physical units
// are applied once in the final scatter.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace kifmm {

cudaError_t m2l_tensor(Plan &P, cudaStream_t s);  // m2l_tc.cu

namespace {

constexpr int kLeafThreads = 128;
constexpr int kMaxNs = 6 * 9 * 9 + 2;  // n_s at the largest surface order, p = 10

template <typename T>
__device__ __forceinline__ T box_half(int level) {
    return (T)ldexp(1.0, -(level + 1));
}
template <typename T>
__device__ __forceinline__ T box_center(int c, int level) {
    return (T)(ldexp((double)(2 * c + 1), -(level + 1)));
}

// Offset of image s (13: the cell itself) in root units: the periodic cell is
// the root box, of side 1.
template <typename T>
__device__ __forceinline__ void image_offset(int s, T &x, T &y, T &z) {
    x = (T)(s / 9 - 1);
    y = (T)((s / 3) % 3 - 1);
    z = (T)(s % 3 - 1);
}


template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
    s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// P2M: u(b)_j = (1/h) sum_i q_i / |2.95 S_j - (x_i - c_b)/h|.  One block
// per leaf with a thread per check point (blockDim = n_s rounded up to a
// warp); particles staged through shared memory in chunks of blockDim.  The
// check surface lies outside the leaf, so no distance is zero.
template <typename T>
__global__ void k_p2m(const int32_t *__restrict__ leaves, const int32_t *__restrict__ lvl,
                      const int32_t *__restrict__ first, const int32_t *__restrict__ cnt,
                      const typename Vec4<T>::type *__restrict__ pts, const T *__restrict__ surf, int ns,
                      T *__restrict__ u, const T *__restrict__ wts = nullptr, int adj = 0,
                      const T *__restrict__ dip = nullptr) {
    // Adjoint with dip ([N][3] sorted, root units): each particle also carries
    // the dipole dL/dgrad, whose field at the surface point y is
    // g . (y - x) / |y - x|^3 (the transpose of the gradient evaluation).
    extern __shared__ __align__(16) unsigned char p2m_sm[];
    T *sx = (T *)p2m_sm, *sy = sx + blockDim.x, *sz = sy + blockDim.x, *sq = sz + blockDim.x;
    T *gx = sq + blockDim.x, *gy = gx + blockDim.x, *gz = gy + blockDim.x;
    const int b = leaves[blockIdx.x];
    const T h = box_half<T>(lvl[b]), hinv = T(1) / h;
    const int n = cnt[b], f = first[b];
    const T a = (T)kAlphaOuter;
    for (int j0 = 0; j0 < ns; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        T px = 0, py = 0, pz = 0;
        if (j < ns) {
            px = a * surf[3 * j];
            py = a * surf[3 * j + 1];
            pz = a * surf[3 * j + 2];
        }
        T acc = 0;
        for (int c0 = 0; c0 < n; c0 += blockDim.x) {
            __syncthreads();
            if (c0 + threadIdx.x < n) {
                const auto v = pts[f + c0 + threadIdx.x];
                sx[threadIdx.x] = v.x * hinv;
                sy[threadIdx.x] = v.y * hinv;
                sz[threadIdx.x] = v.z * hinv;
                sq[threadIdx.x] = wts ? wts[f + c0 + threadIdx.x] : v.w;
                if (dip) {  // in box units the dipole term carries 1/h
                    const size_t k = 3 * (size_t)(f + c0 + threadIdx.x);
                    gx[threadIdx.x] = dip[k] * hinv;
                    gy[threadIdx.x] = dip[k + 1] * hinv;
                    gz[threadIdx.x] = dip[k + 2] * hinv;
                }
            }
            __syncthreads();
            const int m = min((int)blockDim.x, n - c0);
            if (dip) {
                for (int i = 0; i < m; ++i) {
                    const T rx = px - sx[i], ry = py - sy[i], rz = pz - sz[i];
                    const T ri = rsqrt_t<T>(rx * rx + ry * ry + rz * rz);
                    acc += sq[i] * ri + (gx[i] * rx + gy[i] * ry + gz[i] * rz) * (ri * ri * ri);
                }
            } else {
#pragma unroll 4
                for (int i = 0; i < m; ++i) {
                    const T rx = px - sx[i], ry = py - sy[i], rz = pz - sz[i];
                    acc += sq[i] * rsqrt_t<T>(rx * rx + ry * ry + rz * rz);
                }
            }
        }
        // forward: u = sum q / |UC - x| (1/h from the unit surface); adjoint of
        // L2P: h * sum w / |DE - x| with the same unit geometry
        if (j < ns) u[(size_t)b * ns + j] = adj ? acc : acc * hinv;
    }
}


// P2M, FP32 forward form: kP2mLeaves leaves per block (a leaf's ~n_s x 30
// kernel evaluations are too little work for a block of their own) and the
// particle loop on packed f32x2 arithmetic, two particles per instruction
// (the chunk's odd tail padded with a null particle: weight 0, far away).
constexpr int kP2mLeaves = 4;
__global__ void k_p2m_f32(const int32_t *__restrict__ leaves, int64_t n_leaves, const int32_t *__restrict__ lvl,
                          const int32_t *__restrict__ first, const int32_t *__restrict__ cnt,
                          const float4 *__restrict__ pts, const float *__restrict__ surf, int ns,
                          float *__restrict__ u) {
    extern __shared__ __align__(16) unsigned char p2m_sm[];
    const int nt = blockDim.x;  // a multiple of 32
    float *sx = (float *)p2m_sm, *sy = sx + nt, *sz = sy + nt, *sq = sz + nt;
    const float a = (float)kAlphaOuter;
    const int64_t l0 = (int64_t)blockIdx.x * kP2mLeaves, l1 = min(n_leaves, l0 + kP2mLeaves);
    for (int64_t li = l0; li < l1; ++li) {
        const int b = leaves[li];
        const float hinv = 1.f / box_half<float>(lvl[b]);
        const int n = cnt[b], f = first[b];
        for (int j0 = 0; j0 < ns; j0 += nt) {
            const int j = j0 + threadIdx.x;
            float px = 0.f, py = 0.f, pz = 0.f;
            if (j < ns) {
                px = a * surf[3 * j];
                py = a * surf[3 * j + 1];
                pz = a * surf[3 * j + 2];
            }
            const float2 npx = make_float2(-px, -px), npy = make_float2(-py, -py), npz = make_float2(-pz, -pz);
            float2 acc = make_float2(0.f, 0.f);
            for (int c0 = 0; c0 < n; c0 += nt) {
                __syncthreads();
                const int m = min(nt, n - c0);
                if ((int)threadIdx.x < m) {
                    const float4 v = pts[f + c0 + threadIdx.x];
                    sx[threadIdx.x] = v.x * hinv;
                    sy[threadIdx.x] = v.y * hinv;
                    sz[threadIdx.x] = v.z * hinv;
                    sq[threadIdx.x] = v.w;
                } else if ((int)threadIdx.x == m) {  // m < nt: pad the odd tail
                    sx[m] = sy[m] = sz[m] = 1e4f;
                    sq[m] = 0.f;
                }
                __syncthreads();
#pragma unroll 4
                for (int i = 0; i < m; i += 2) {
                    const float2 rx = __fadd2_rn(*reinterpret_cast<const float2 *>(sx + i), npx);
                    const float2 ry = __fadd2_rn(*reinterpret_cast<const float2 *>(sy + i), npy);
                    const float2 rz = __fadd2_rn(*reinterpret_cast<const float2 *>(sz + i), npz);
                    float2 r2 = __fmul2_rn(rx, rx);
                    r2 = __ffma2_rn(ry, ry, r2);
                    r2 = __ffma2_rn(rz, rz, r2);
                    const float2 ri = make_float2(rsqrt_t<float>(r2.x), rsqrt_t<float>(r2.y));
                    acc = __ffma2_rn(*reinterpret_cast<const float2 *>(sq + i), ri, acc);
                }
            }
            if (j < ns) u[(size_t)b * ns + j] = (acc.x + acc.y) * hinv;
        }
    }
}

// P2L: d(b)_j += (1/h_b) sum_{a in X(b)} sum_i q_i / |1.05 S_j - (x_i - c_b)/h_b|
template <typename T>
__global__ void k_p2l(const int32_t *__restrict__ nx, const int32_t *__restrict__ xdense,
                      const int32_t *__restrict__ lvl, const int32_t *__restrict__ cx,
                      const int32_t *__restrict__ cy, const int32_t *__restrict__ cz,
                      const int32_t *__restrict__ first, const int32_t *__restrict__ cnt,
                      const typename Vec4<T>::type *__restrict__ pts, const T *__restrict__ surf, int ns,
                      T *__restrict__ d, const T *__restrict__ wts = nullptr, int adj = 0,
                      double *__restrict__ dbar = nullptr, const T *__restrict__ dip = nullptr,
                      const int8_t *__restrict__ x_sh = nullptr) {
    // With dbar (FP32-based modes) the mean of this box's contribution goes
    // to dbar and only the mean-free remainder to d.  With dip (adjoint of
    // M2P under a loss on the gradient) every particle also carries a dipole.
    __shared__ T sx[kLeafThreads], sy[kLeafThreads], sz[kLeafThreads], sq[kLeafThreads];
    __shared__ T gx[kLeafThreads], gy[kLeafThreads], gz[kLeafThreads];
    __shared__ T cv[kMaxNs];
    __shared__ double red[kLeafThreads / 32];
    const int b = blockIdx.x;
    if (nx[b] == 0) return;
    const int lb = lvl[b];
    const T hb = box_half<T>(lb), hinv = T(1) / hb;
    const T cbx = box_center<T>(cx[b], lb), cby = box_center<T>(cy[b], lb), cbz = box_center<T>(cz[b], lb);
    const T al = (T)kAlphaInner;
    for (int j0 = 0; j0 < ns; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        T px = 0, py = 0, pz = 0;
        if (j < ns) {
            px = al * surf[3 * j];
            py = al * surf[3 * j + 1];
            pz = al * surf[3 * j + 2];
        }
        T acc = 0;
        for (int e = 0; e < nx[b]; ++e) {
            const int a = xdense[(size_t)b * kMaxCoarse + e];
            const int la = lvl[a];
            T ox = box_center<T>(cx[a], la) - cbx, oy = box_center<T>(cy[a], la) - cby,
              oz = box_center<T>(cz[a], la) - cbz;
            if (x_sh) {  // the source leaf's image (periodic cell)
                T ix, iy, iz;
                image_offset<T>(x_sh[(size_t)b * kMaxCoarse + e], ix, iy, iz);
                ox += ix, oy += iy, oz += iz;
            }
            const int n = cnt[a], f = first[a];
            for (int c0 = 0; c0 < n; c0 += kLeafThreads) {
                __syncthreads();
                if (c0 + threadIdx.x < n) {
                    const auto v = pts[f + c0 + threadIdx.x];
                    sx[threadIdx.x] = (ox + v.x) * hinv;
                    sy[threadIdx.x] = (oy + v.y) * hinv;
                    sz[threadIdx.x] = (oz + v.z) * hinv;
                    sq[threadIdx.x] = wts ? wts[f + c0 + threadIdx.x] : v.w;
                    if (dip) {
                        const size_t k = 3 * (size_t)(f + c0 + threadIdx.x);
                        gx[threadIdx.x] = dip[k] * hinv;
                        gy[threadIdx.x] = dip[k + 1] * hinv;
                        gz[threadIdx.x] = dip[k + 2] * hinv;
                    }
                }
                __syncthreads();
                const int m = min(kLeafThreads, n - c0);
                if (dip) {
                    for (int i = 0; i < m; ++i) {
                        const T rx = px - sx[i], ry = py - sy[i], rz = pz - sz[i];
                        const T ri = rsqrt_t<T>(rx * rx + ry * ry + rz * rz);
                        acc += sq[i] * ri + (gx[i] * rx + gy[i] * ry + gz[i] * rz) * (ri * ri * ri);
                    }
                } else {
                    for (int i = 0; i < m; ++i) acc += sq[i] * lap_pot<T>(px - sx[i], py - sy[i], pz - sz[i]);
                }
            }
        }
        if (j < ns) {
            const T v = adj ? acc : acc * hinv;
            if (dbar) cv[j] = v; else d[(size_t)b * ns + j] += v;
        }
    }
    if (dbar) {
        __syncthreads();
        double sum = 0.0;
        for (int j = threadIdx.x; j < ns; j += blockDim.x) sum += (double)cv[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
        __syncthreads();
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        const double mean = tot / ns;
        for (int j = threadIdx.x; j < ns; j += blockDim.x) d[(size_t)b * ns + j] += (T)((double)cv[j] - mean);
        if (threadIdx.x == 0) dbar[b] += mean;
    }
}

// ---------------------------------------------------------------------------
// Gathered, class-tiled GEMM on SIMT cores:
//   out[t] (=|+=) sum_{s < nslots} Op_s  in[src(t, s)]
// for a list of targets.  A block owns 64 targets and all outputs (padded to
// 160); each thread keeps an 8 x 5 register tile (targets 8 ty .. 8 ty + 7,
// outputs tx + 32 c).  Operators are stored transposed ([k][j]); k advances in
// chunks of 8 through shared memory with the next chunk prefetched into
// registers.  Used for M2L (189 V slots), M2M (8 child octants), L2L (parent)
// and the two factors of the leaf pseudo-inverses.
// ---------------------------------------------------------------------------
constexpr int kGK = 16;

// Target ranges of up to 8 classes (blockIdx.y = class) in one launch.
struct ClassRanges {
    int64_t b[9];
};

// Operator blocks are [k][ld]: ld = n_s, or n_s + 1 when column n_s holds the
// mean row of a mean-free check-to-check block (FP32-based modes).
template <typename T>
struct GatherM2L {
    const int32_t *vdense;
    const int *slot_off;
    const T *ops;
    int ns, ld;
    __device__ int src(int t, int s, int) const { return vdense[(size_t)t * kVSlots + s]; }
    __device__ const T *op(int s, int cls) const { return ops + (size_t)slot_off[cls * kVSlots + s] * ns * ld; }
    __device__ double mean_base(int, const double *) const { return 0.0; }
};
template <typename T>
struct GatherChild {
    const int32_t *child8;
    const T *ops;
    int ns;
    __device__ int src(int t, int s, int) const { return child8[(size_t)t * 8 + s]; }
    __device__ const T *op(int s, int) const { return ops + (size_t)s * ns * ns; }
    __device__ double mean_base(int, const double *) const { return 0.0; }
};
// One operator per class (L2L: the octant of the child); the child inherits
// the parent's mean.
template <typename T>
struct GatherParent {
    const int32_t *parent;
    const T *ops;
    int ns, ld;
    __device__ int src(int t, int, int) const { return parent[t]; }
    __device__ const T *op(int, int cls) const { return ops + (size_t)cls * ns * ld; }
    __device__ double mean_base(int t, const double *dbar) const { return dbar[parent[t]]; }
};
template <typename T>
struct GatherSelf {
    const T *op0;
    __device__ int src(int t, int, int) const { return t; }
    __device__ const T *op(int, int) const { return op0; }
    __device__ double mean_base(int, const double *) const { return 0.0; }
};

// With dbar: output column n_s (operator column n_s, the mean row) goes to
// dbar[t] (FP64, plus the functor's mean_base) instead of out.
// Tile: NTY warps; thread (tx, ty) owns targets RT ty .. RT ty + RT-1 and
// outputs tx + 32 c (c < RC): TT = NTY RT targets by TJ = 32 RC outputs.
// SPLIT: blockIdx.z = slot * ncb + column block; the block writes that
// slot's partial product to part ([slot][target position][ld]) and
// k_ggemm_sum adds the slots in order (the same arithmetic as the unsplit
// form; used for the small-tile M2M levels, whose latency is otherwise
// 8 slots x n_s / 16 dependent steps per block).
// MULTI: more than one slot per block (FP32 then keeps per-slot partials and
// running sums); single-slot launches need half the accumulator registers
// and run two 256-thread blocks per SM.
template <typename T, class G, int NTY, int RT, int RC, bool SPLIT, bool MULTI>
__global__ void __launch_bounds__(32 * NTY, (sizeof(T) == 4 && NTY == 8 && !MULTI) ? 2 : 1) k_ggemm(G g, const int32_t *__restrict__ targets, ClassRanges cr,
                                                    int nslots, int ns, int ld, const T *__restrict__ in,
                                                    T *__restrict__ out, int accumulate, double *dbar, int ncb,
                                                    T *__restrict__ part) {
    constexpr int TT = NTY * RT, TJ = 32 * RC, NT = 32 * NTY;
    __shared__ __align__(16) T Us[kGK][TT];
    __shared__ __align__(16) T Ms[kGK][TJ];
    __shared__ int32_t tgt[TT];
    __shared__ int32_t src[TT];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int cls = blockIdx.y;
    const int j0 = (SPLIT ? (int)blockIdx.z % ncb : (int)blockIdx.z) * TJ;  // output columns [j0, j0 + TJ)
    const int s_lo = SPLIT ? (int)blockIdx.z / ncb : 0, s_hi = SPLIT ? s_lo + 1 : nslots;
    int64_t t_begin = 0, t_end = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c == cls) {
            t_begin = cr.b[c];
            t_end = cr.b[c + 1];
        }
    const int64_t t0 = t_begin + (int64_t)blockIdx.x * TT;
    if (t0 >= t_end) return;  // uniform for the block
    if (threadIdx.x < TT) tgt[threadIdx.x] = (t0 + threadIdx.x < t_end) ? targets[t0 + threadIdx.x] : -1;
    // FP32: each slot sums into a fresh partial that is then added to the
    // running total, so no rounding chain is longer than one slot's n_s terms.
    constexpr bool kTwoLevel = sizeof(T) == 4 && MULTI;
    T acc[RT][RC], run[RT][RC];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[a][c] = run[a][c] = T(0);
    const int nk = (ns + kGK - 1) / kGK;
    __syncthreads();
    for (int s = s_lo; s < s_hi; ++s) {
        if (threadIdx.x < TT) {
            const int32_t t = tgt[threadIdx.x];
            src[threadIdx.x] = (t >= 0) ? g.src(t, s, cls) : -1;
        }
        const T *M = g.op(s, cls);
        __syncthreads();
        constexpr int kRU = (TT * kGK + NT - 1) / NT, kRM = (kGK * TJ + NT - 1) / NT;
        T ru[kRU], rm[kRM];
        auto load = [&](int kc) {
            const int k0 = kc * kGK;
#pragma unroll
            for (int r = 0; r < kRU; ++r) {
                const int e = threadIdx.x + NT * r;
                const int t = e / kGK, k = e % kGK;
                ru[r] = T(0);
                if (t < TT) {
                    const int32_t sb = src[t];
                    if (sb >= 0 && k0 + k < ns) ru[r] = in[(size_t)sb * ns + k0 + k];
                }
            }
#pragma unroll
            for (int r = 0; r < kRM; ++r) {
                const int e = threadIdx.x + NT * r;
                const int k = e / TJ, j = e - k * TJ;
                rm[r] = (k < kGK && k0 + k < ns && j0 + j < ld) ? M[(size_t)(k0 + k) * ld + j0 + j] : T(0);
            }
        };
        load(0);
        for (int kc = 0; kc < nk; ++kc) {
#pragma unroll
            for (int r = 0; r < kRU; ++r) {
                const int e = threadIdx.x + NT * r;
                if (e < TT * kGK) Us[e % kGK][e / kGK] = ru[r];
            }
#pragma unroll
            for (int r = 0; r < kRM; ++r) {
                const int e = threadIdx.x + NT * r;
                const int k = e / TJ;
                if (k < kGK) Ms[k][e - k * TJ] = rm[r];
            }
            __syncthreads();
            if (kc + 1 < nk) load(kc + 1);
#pragma unroll
            for (int k = 0; k < kGK; ++k) {
                T uv[RT], mv[RC];
#pragma unroll
                for (int a = 0; a < RT; ++a) uv[a] = Us[k][RT * ty + a];
#pragma unroll
                for (int c = 0; c < RC; ++c) mv[c] = Ms[k][tx + 32 * c];
#pragma unroll
                for (int a = 0; a < RT; ++a)
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc[a][c] += uv[a] * mv[c];
            }
            __syncthreads();
        }
        if constexpr (kTwoLevel) {
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    run[a][c] += acc[a][c];
                    acc[a][c] = T(0);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < RT; ++a) {
        const int32_t t = tgt[RT * ty + a];
        if (t < 0) continue;
#pragma unroll
        for (int c = 0; c < RC; ++c) {
            const int j = j0 + tx + 32 * c;
            const T v = kTwoLevel ? run[a][c] : acc[a][c];
            if constexpr (SPLIT) {
                if (j < ld)
                    part[((size_t)s_lo * (size_t)(cr.b[gridDim.y] - cr.b[0]) + (size_t)(t0 + RT * ty + a - cr.b[0])) * ld +
                         j] = v;
            } else if (j < ns) {
                T *o = out + (size_t)t * ns + j;
                *o = accumulate ? *o + v : v;
            } else if (j == ns && dbar) {
                dbar[t] = (accumulate ? dbar[t] : 0.0) + (double)v + g.mean_base(t, dbar);
            }
        }
    }
}

// FP32 big tiles with vector shared-memory reads: 64 targets x 160 outputs
// per 320-thread block; thread (tn = t % 40, tm = t / 40) owns outputs
// 4 tn .. 4 tn + 3 and targets 8 tm .. 8 tm + 7, so each k step reads one
// float4 of the operator and two of the gathered inputs for 32 FMAs (the
// scalar tile above reads 13 values for 40).  The sums run over k in the same
// order, one fresh partial per slot, so the results equal the scalar form's
// bit for bit.  VEC: the input rows are 16-byte aligned (n_s a multiple of 4)
// and are read as float4.
constexpr int kV4Threads = 320;
// SPLIT: blockIdx.z = slot * ncb + column block, the slot's partial product
// to part ([slot][target position][ld]) as in the scalar tile's split form.
template <class G, bool MULTI, bool VEC, bool SPLIT = false>
__global__ void __launch_bounds__(kV4Threads, 2) k_ggemm_v4(G g, const int32_t *__restrict__ targets,
                                                            ClassRanges cr, int nslots, int ns, int ld,
                                                            const float *__restrict__ in, float *__restrict__ out,
                                                            int accumulate, double *dbar, int ncb = 1,
                                                            float *__restrict__ part = nullptr) {
    constexpr int TT = 64, TJ = 160;
    __shared__ __align__(16) float Us[kGK][TT];
    __shared__ __align__(16) float Ms[kGK][TJ];
    __shared__ int32_t tgt[TT];
    __shared__ int32_t src[TT];
    const int tid = threadIdx.x;
    const int tn = tid % 40, tm = tid / 40;
    const int cls = blockIdx.y;
    const int j0 = (SPLIT ? (int)blockIdx.z % ncb : (int)blockIdx.z) * TJ;
    const int s_lo = SPLIT ? (int)blockIdx.z / ncb : 0, s_hi = SPLIT ? s_lo + 1 : nslots;
    int64_t t_begin = 0, t_end = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c == cls) {
            t_begin = cr.b[c];
            t_end = cr.b[c + 1];
        }
    const int64_t t0 = t_begin + (int64_t)blockIdx.x * TT;
    if (t0 >= t_end) return;  // uniform for the block
    if (tid < TT) tgt[tid] = (t0 + tid < t_end) ? targets[t0 + tid] : -1;
    float acc[8][4], run[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = run[a][c] = 0.f;
    const int nk = (ns + kGK - 1) / kGK;
    __syncthreads();
    for (int s = s_lo; s < s_hi; ++s) {
        if (tid < TT) {
            const int32_t t = tgt[tid];
            src[tid] = (t >= 0) ? g.src(t, s, cls) : -1;
        }
        const float *M = g.op(s, cls);
        __syncthreads();
        // staged values: inputs as (target = e % 64, k quad = e / 64), four
        // k values each; operator rows as (k, j) with j fastest
        constexpr int kRM = kGK * TJ / kV4Threads;  // 8
        float4 ru = make_float4(0.f, 0.f, 0.f, 0.f);
        float rm[kRM];
        auto load = [&](int kc) {
            const int k0 = kc * kGK;
            if (tid < TT * (kGK / 4)) {
                const int t = tid % TT, k = 4 * (tid / TT);
                const int32_t sb = src[t];
                ru = make_float4(0.f, 0.f, 0.f, 0.f);
                if (sb >= 0) {
                    const float *row = in + (size_t)sb * ns + k0 + k;
                    if (VEC && k0 + k + 3 < ns) {
                        ru = *reinterpret_cast<const float4 *>(row);
                    } else {
                        if (k0 + k < ns) ru.x = row[0];
                        if (k0 + k + 1 < ns) ru.y = row[1];
                        if (k0 + k + 2 < ns) ru.z = row[2];
                        if (k0 + k + 3 < ns) ru.w = row[3];
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kRM; ++r) {
                const int e = tid + kV4Threads * r;
                const int k = e / TJ, j = e - k * TJ;
                rm[r] = (k0 + k < ns && j0 + j < ld) ? M[(size_t)(k0 + k) * ld + j0 + j] : 0.f;
            }
        };
        load(0);
        for (int kc = 0; kc < nk; ++kc) {
            if (tid < TT * (kGK / 4)) {
                const int t = tid % TT, k = 4 * (tid / TT);
                Us[k][t] = ru.x;
                Us[k + 1][t] = ru.y;
                Us[k + 2][t] = ru.z;
                Us[k + 3][t] = ru.w;
            }
#pragma unroll
            for (int r = 0; r < kRM; ++r) {
                const int e = tid + kV4Threads * r;
                Ms[e / TJ][e % TJ] = rm[r];
            }
            __syncthreads();
            if (kc + 1 < nk) load(kc + 1);
#pragma unroll
            for (int k = 0; k < kGK; ++k) {
                const float4 u0 = *reinterpret_cast<const float4 *>(&Us[k][8 * tm]);
                const float4 u1 = *reinterpret_cast<const float4 *>(&Us[k][8 * tm + 4]);
                const float4 m = *reinterpret_cast<const float4 *>(&Ms[k][4 * tn]);
                const float uv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] += uv[a] * mv[c];
            }
            __syncthreads();
        }
        if constexpr (MULTI) {
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    run[a][c] += acc[a][c];
                    acc[a][c] = 0.f;
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int32_t t = tgt[8 * tm + a];
        if (t < 0) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + 4 * tn + c;
            const float v = MULTI ? run[a][c] : acc[a][c];
            if constexpr (SPLIT) {
                if (j < ld)
                    part[((size_t)s_lo * (size_t)(cr.b[gridDim.y] - cr.b[0]) + (size_t)(t0 + 8 * tm + a - cr.b[0])) *
                             ld + j] = v;
            } else if (j < ns) {
                float *o = out + (size_t)t * ns + j;
                *o = accumulate ? *o + v : v;
            } else if (j == ns && dbar) {
                dbar[t] = (accumulate ? dbar[t] : 0.0) + (double)v + g.mean_base(t, dbar);
            }
        }
    }
}

// Slot-split form: out = the in-order sum of the slots' partial products.
template <typename T, class G>
__global__ void k_ggemm_sum(G g, const int32_t *__restrict__ targets, int64_t t_first, int64_t n_t, int nslots, int ns,
                            int ld, const T *__restrict__ part, T *__restrict__ out, int accumulate, double *dbar) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_t * ld) return;
    const int64_t i = idx / ld;
    const int j = (int)(idx - i * ld);
    T v = T(0);
    for (int s = 0; s < nslots; ++s) v += part[((size_t)s * n_t + i) * ld + j];
    const int32_t t = targets[t_first + i];
    if (j < ns) {
        T *o = out + (size_t)t * ns + j;
        *o = accumulate ? *o + v : v;
    } else if (j == ns && dbar) {
        dbar[t] = (accumulate ? dbar[t] : 0.0) + (double)v + g.mean_base(t, dbar);
    }
}

// ---------------------------------------------------------------------------
// Leaf evaluation, one warp per target leaf: far field (L2P from the leaf's
// downward density on DE = 2.95 h S; M2P from the upward densities on
// UE = 1.05 h S of the W-list boxes) and near field (P2P over the U list).
// All of it is one stream of (pseudo-)sources {position relative to the leaf
// centre, weight}: the segments (own surface, W surfaces, U leaves) are laid
// end to end, and the stream is staged through shared memory in chunks of
// 128.  The next chunk's loads are issued before the current chunk is
// summed, so their latency overlaps the arithmetic.
//
// Tiling <TPL, G>: the warp splits into G groups of 32/G lanes; lane m of a
// group owns targets tbase + m + (32/G) k (k < TPL) and the group takes every
// G-th source of each chunk.  Up to 64 sources per lane are summed plainly,
// then added to the totals with two-sum; the groups' totals are combined in
// FP64 with shuffles and the result overwrites res.  The tile is picked per
// leaf so that (32/G) TPL covers its targets with little waste.
//
// Only the leaf's own particles can sit at distance zero from a target (a
// particle's own position, or a coincident particle: equal positions have
// equal keys, hence the same leaf); that segment is summed with the r = 0
// test, every other one without it.  Distinct particles of different leaves
// whose separation rounds to zero in the compute type would give a
// non-finite sum: the kernel reports KIFMM_ERR_NONFINITE for them.
// ---------------------------------------------------------------------------
constexpr int kLW = 4;               // warps (target leaves) per block
constexpr int kLK = 4;               // sources per lane per chunk
constexpr int kLChunk = 32 * kLK;    // sources per staged chunk
constexpr int kLFlush = 64;          // sources per lane summed plainly before a compensated flush
constexpr int kLSeg = 32;            // segments per batch (one per lane)

template <typename T>
__device__ __forceinline__ T pow2(int e);
template <>
__device__ __forceinline__ float pow2<float>(int e) {
    return __int_as_float((127 + e) << 23);
}
template <>
__device__ __forceinline__ double pow2<double>(int e) {
    return __longlong_as_double((long long)(1023 + e) << 52);
}

// c_a - c_b along one axis for boxes (level, integer coordinate): both
// centres are odd multiples of 2^-(level+1), so the difference is an integer
// below 2^22 times 2^-(L+1) and exact in FP32.
template <typename T>
__device__ __forceinline__ T centre_diff(int ca, int la, int cb, int lb) {
    const int L = max(la, lb);
    const int na = (2 * ca + 1) << (L - la), nb = (2 * cb + 1) << (L - lb);
    return (T)(na - nb) * pow2<T>(-(L + 1));
}

template <typename T, int TPL>
struct LeafAcc {
    T tx[TPL], ty[TPL], tz[TPL];
    T part[TPL][4];             // plain partial sums since the last flush
    T acc[TPL][4], cmp[TPL][4]; // compensated totals (two-sum)
    int pend;                   // sources per lane in part (warp-uniform bound)
    // FP32: the pair loop runs on packed f32x2 arithmetic, two sources per
    // instruction: negated targets duplicated into both halves, and plain
    // partial sums per half (folded into part at each flush)
    float2 ntx[TPL], nty[TPL], ntz[TPL];
    float2 pk[TPL][4];
};

template <typename T, int TPL>
__device__ __forceinline__ void leaf_flush(LeafAcc<T, TPL> &L) {
#pragma unroll
    for (int k = 0; k < TPL; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if constexpr (sizeof(T) == 4) {
                L.part[k][c] = L.pk[k][c].x + L.pk[k][c].y;
                L.pk[k][c] = make_float2(0.f, 0.f);
            }
            T sum, err;
            two_sum<T>(L.acc[k][c], L.part[k][c], sum, err);
            L.acc[k][c] = sum;
            L.cmp[k][c] += err;
            L.part[k][c] = T(0);
        }
    L.pend = 0;
}

// One segment of the source stream: positions are r * raw + o (surfaces:
// unit-surface points; particles: r = 1, raw = position in the source leaf's
// frame), weights hw * raw weight.
template <typename T>
struct LeafSeg {
    T ox, oy, oz, r, hw;
    int base;   // first particle, or first weight of the surface
    int kind;   // 0 own surface, 1 W-list surface, 2 particles
};

template <typename T>
struct LeafSmem {
    typename Vec4<T>::type buf[2][kLChunk];
    LeafSeg<T> seg[kLSeg];
    int start[kLSeg];
};

struct LeafCtx {
    const int32_t *lvl, *cx, *cy, *cz, *first, *cnt;
    const uint32_t *u_ptr, *w_ptr;
    const int32_t *u_idx, *w_idx;
    int ns;
    const double *dbar;  // per-box mean of the downward check potential, or nullptr
    LeafTiling tile;     // tile id per remaining-target bucket
    int *status;         // device status word
    const int8_t *u_sh, *w_sh;  // image shifts of the U and W entries (periodic cell), or null
    // Forward evaluate of a free-space plan: the outputs in caller order with
    // the physical scales (coef / (4 pi side), / side^2 of the particle's
    // system), written by the pass itself next to its FP64 results; null
    // elsewhere (the results are scattered by k_finalize).
    const uint32_t *perm = nullptr;
    const int32_t *sys = nullptr;
    const double *out_scale = nullptr;
    void *pot = nullptr, *grad = nullptr;
    int out_f64 = 0;
};


// Source weights of the leaf stage.  Forward: own surface dn_dens * h_b,
// W surfaces up_dens * h_a, particles q.  Adjoint (same geometry): own
// surface u-bar, W surfaces d-bar, particles w.
template <typename T>
struct LeafW {
    const T *own;
    int own_h;
    const T *wl;
    int wl_h;
    const T *pw;  // sorted per-particle weights, or nullptr for the charges
};

// Sources j in [lo, hi) of a staged chunk with j = grp (mod G).
template <typename T, int TPL, int G, bool CHECK>
__device__ __forceinline__ void leaf_range(LeafAcc<T, TPL> &L, const typename Vec4<T>::type *buf, int lo, int hi,
                                           int grp) {
    // sources in flight per iteration: about four pair evaluations per lane
    constexpr int UNR = (sizeof(T) == 8 || TPL >= 3) ? 1 : (TPL == 2 ? 2 : 4);
#pragma unroll UNR
    for (int j = lo + ((grp - lo) & (G - 1)); j < hi; j += G) {
        const auto s = buf[j];
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            if constexpr (CHECK)
                lap_accum<T>(L.tx[k] - s.x, L.ty[k] - s.y, L.tz[k] - s.z, s.w, L.part[k][0], L.part[k][1],
                             L.part[k][2], L.part[k][3]);
            else
                lap_accum_nz<T>(L.tx[k] - s.x, L.ty[k] - s.y, L.tz[k] - s.z, s.w, L.part[k][0], L.part[k][1],
                                L.part[k][2], L.part[k][3]);
        }
    }
}

// FP32 chunks are staged as source pairs: pair p holds sources a and a + G
// with a = (p / G) 2G + p % G, as eight floats (x_a x_b y_a y_b z_a z_b w_a
// w_b), so group g (p % G = g) meets its own sources g, g + G, g + 2G, ...
// two at a time, each pair already in the register halves of the f32x2
// instructions.  Entries beyond the chunk's sources hold a null source
// (weight 0, far away), which adds exactly zero.
__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Pairs i in [ia, ie) of group grp (pair index grp + i G).
template <int TPL, int G, bool CHECK>
__device__ __forceinline__ void leaf_pairs(LeafAcc<float, TPL> &L, const float4 *__restrict__ pairs, int ia, int ie,
                                           int grp) {
    constexpr int UNR = TPL == 1 ? 4 : 1;  // eight pair evaluations in flight per lane (the FP32 chains are latency-bound)
#pragma unroll UNR
    for (int i = ia; i < ie; ++i) {
        const int p = grp + i * G;
        const float4 A = pairs[2 * p], B = pairs[2 * p + 1];
        const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
        const float2 sz = make_float2(B.x, B.y), sw = make_float2(B.z, B.w);
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            // r = source - target (the gradient sum below is then + r w / r^3)
            const float2 rx = __fadd2_rn(sx, L.ntx[k]);
            const float2 ry = __fadd2_rn(sy, L.nty[k]);
            const float2 rz = __fadd2_rn(sz, L.ntz[k]);
            float2 r2 = __fmul2_rn(rx, rx);
            r2 = __ffma2_rn(ry, ry, r2);
            r2 = __ffma2_rn(rz, rz, r2);
            float2 ri;
            if constexpr (CHECK) {
                ri.x = r2.x > 0.f ? rsqrt_t<float>(r2.x) : 0.f;
                ri.y = r2.y > 0.f ? rsqrt_t<float>(r2.y) : 0.f;
            } else {
                ri.x = rsqrt_t<float>(r2.x);
                ri.y = rsqrt_t<float>(r2.y);
            }
            const float2 wr = __fmul2_rn(sw, ri);
            const float2 wr3 = __fmul2_rn(wr, __fmul2_rn(ri, ri));
            L.pk[k][0] = __fadd2_rn(L.pk[k][0], wr);
            L.pk[k][1] = __ffma2_rn(rx, wr3, L.pk[k][1]);
            L.pk[k][2] = __ffma2_rn(ry, wr3, L.pk[k][2]);
            L.pk[k][3] = __ffma2_rn(rz, wr3, L.pk[k][3]);
        }
    }
}

// A staged FP32 chunk of m sources (pair layout); [olo, ohi) are the leaf's
// own particles: the pairs of group grp that touch them take the r = 0 test.
// Sub-blocks of kLFlush / 2 pairs keep every plain partial sum to at most
// kLFlush terms.
template <int TPL, int G>
__device__ __forceinline__ void leaf_chunk_pk(LeafAcc<float, TPL> &L, const float4 *pairs, int m, int olo, int ohi,
                                              int grp) {
    const int np = grp < m ? (m - grp + 2 * G - 1) / (2 * G) : 0;
    // pair i holds this group's sources 2 i G + grp and 2 i G + grp + G
    const int i_lo = max(0, floor_div(olo - grp - G + 2 * G - 1, 2 * G));
    const int i_hi = max(0, floor_div(ohi - grp + 2 * G - 1, 2 * G));
    for (int i0 = 0; i0 < np; i0 += kLFlush / 2) {
        const int i1 = min(np, i0 + kLFlush / 2);
        const int a = max(i0, min(i1, i_lo)), e = max(a, min(i1, i_hi));
        leaf_pairs<TPL, G, false>(L, pairs, i0, a, grp);
        if (a < e) leaf_pairs<TPL, G, true>(L, pairs, a, e, grp);
        leaf_pairs<TPL, G, false>(L, pairs, e, i1, grp);
        L.pend += 2 * (i1 - i0);
        if (L.pend >= kLFlush) leaf_flush<float, TPL>(L);
    }
}

// A staged chunk of m sources; [olo, ohi) are the leaf's own particles.
// Sub-blocks of kLFlush G sources keep every plain partial sum to at most
// kLFlush terms.
template <typename T, int TPL, int G>
__device__ __forceinline__ void leaf_chunk(LeafAcc<T, TPL> &L, const typename Vec4<T>::type *buf, int m, int olo,
                                           int ohi, int grp) {
    if constexpr (sizeof(T) == 4) {
        leaf_chunk_pk<TPL, G>(L, buf, m, olo, ohi, grp);
        return;
    }
    for (int s0 = 0; s0 < m; s0 += kLFlush * G) {
        const int s1 = min(m, s0 + kLFlush * G);
        const int a = max(s0, min(s1, olo)), e = max(a, min(s1, ohi));
        leaf_range<T, TPL, G, false>(L, buf, s0, a, grp);
        if (a < e) leaf_range<T, TPL, G, true>(L, buf, a, e, grp);
        leaf_range<T, TPL, G, false>(L, buf, e, s1, grp);
        L.pend += (s1 - s0 + G - 1) / G;
        if (L.pend >= kLFlush) leaf_flush<T, TPL>(L);
    }
}

// Loads of chunk c of a batch: lane l takes stream entries c kLChunk + l + 32 i.
template <typename T>
__device__ __forceinline__ void leaf_fetch(const LeafSmem<T> &S, int c, int total, int nb,
                                           const typename Vec4<T>::type *__restrict__ pts,
                                           const T *__restrict__ surf, const LeafW<T> &W,
                                           typename Vec4<T>::type (&raw)[kLK], int (&rs)[kLK]) {
    const int lane = threadIdx.x & 31;
    // the lane's entries increase with i: one binary search, then linear steps
    int s = 0;
#pragma unroll
    for (int i = 0; i < kLK; ++i) {
        const int j = c * kLChunk + lane + 32 * i;
        rs[i] = -1;
        if (j < total) {
            if (i == 0) {
#pragma unroll
                for (int step = kLSeg / 2; step > 0; step >>= 1)
                    if (s + step < nb && S.start[s + step] <= j) s += step;
            } else {
                while (s + 1 < nb && S.start[s + 1] <= j) ++s;
            }
            const int k = j - S.start[s];
            const int kind = S.seg[s].kind, base = S.seg[s].base;
            rs[i] = s;
            if (kind == 2) {
                raw[i] = pts[base + k];
                if (W.pw) raw[i].w = W.pw[base + k];
            } else {
                raw[i].x = surf[3 * k];
                raw[i].y = surf[3 * k + 1];
                raw[i].z = surf[3 * k + 2];
                raw[i].w = (kind == 0 ? W.own : W.wl)[base + k];
            }
        }
    }
}

// Place fetched entries (segment transform applied) in staging buffer slot;
// FP32 in the pair layout of leaf_chunk_pk, with null sources past the end.
template <typename T, int G>
__device__ __forceinline__ void leaf_store(LeafSmem<T> &S, int slot, const typename Vec4<T>::type (&raw)[kLK],
                                           const int (&rs)[kLK]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < kLK; ++i) {
        typename Vec4<T>::type v;
        if (rs[i] >= 0) {
            const LeafSeg<T> g = S.seg[rs[i]];
            v.x = g.r * raw[i].x + g.ox;
            v.y = g.r * raw[i].y + g.oy;
            v.z = g.r * raw[i].z + g.oz;
            v.w = raw[i].w * g.hw;
        } else {
            if constexpr (sizeof(T) == 8) continue;
            v.x = v.y = v.z = T(1e4);  // null source: weight 0 at a finite distance
            v.w = T(0);
        }
        const int j = lane + 32 * i;
        if constexpr (sizeof(T) == 4) {
            const int r = j % (2 * G), pair = (j / (2 * G)) * G + r % G, h = r / G;
            float *P = reinterpret_cast<float *>(&S.buf[slot][0]) + 8 * pair;
            P[h] = v.x;
            P[2 + h] = v.y;
            P[4 + h] = v.z;
            P[6 + h] = v.w;
        } else {
            S.buf[slot][j] = v;
        }
    }
}

template <typename T, int TPL, int G>
__device__ void leaf_pass(const LeafCtx &C, int b, int tbase, const typename Vec4<T>::type *__restrict__ pts,
                          const T *__restrict__ surf, const LeafW<T> &W, LeafSmem<T> &S,
                          double4 *__restrict__ res) {
    using V4 = typename Vec4<T>::type;
    constexpr int LG = 32 / G;  // lanes per group
    const int lane = threadIdx.x & 31, grp = lane / LG, mem = lane % LG;
    const int lb = C.lvl[b], bx = C.cx[b], by = C.cy[b], bz = C.cz[b];
    const int n = C.cnt[b], f = C.first[b], ns = C.ns;
    LeafAcc<T, TPL> L;
#pragma unroll
    for (int k = 0; k < TPL; ++k) {
        const int i = tbase + mem + LG * k;
        V4 v{};
        if (i < n) v = pts[f + i];
        L.tx[k] = v.x;
        L.ty[k] = v.y;
        L.tz[k] = v.z;
        if constexpr (sizeof(T) == 4) {
            L.ntx[k] = make_float2(-(float)v.x, -(float)v.x);
            L.nty[k] = make_float2(-(float)v.y, -(float)v.y);
            L.ntz[k] = make_float2(-(float)v.z, -(float)v.z);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            L.part[k][c] = L.acc[k][c] = L.cmp[k][c] = T(0);
            L.pk[k][c] = make_float2(0.f, 0.f);
        }
    }
    L.pend = 0;
    const uint32_t w0 = C.w_ptr[b], u0 = C.u_ptr[b];
    const int nw = (int)(C.w_ptr[b + 1] - w0), nu = (int)(C.u_ptr[b + 1] - u0);
    const int nseg = 1 + nw + nu;
    for (int sb = 0; sb < nseg; sb += kLSeg) {
        // lane e describes segment sb + e of (own surface, W list, U list)
        const int e = sb + lane;
        LeafSeg<T> d{T(0), T(0), T(0), T(1), T(1), 0, 2};
        int cnt = 0, own = 0;
        if (e == 0) {
            d.r = (T)kAlphaOuter * pow2<T>(-(lb + 1));
            d.hw = W.own_h ? pow2<T>(-(lb + 1)) : T(1);
            d.base = b * ns;
            d.kind = 0;
            cnt = ns;
        } else if (e <= nw) {
            const int a = C.w_idx[w0 + e - 1], la = C.lvl[a];
            d.ox = centre_diff<T>(C.cx[a], la, bx, lb);
            d.oy = centre_diff<T>(C.cy[a], la, by, lb);
            d.oz = centre_diff<T>(C.cz[a], la, bz, lb);
            if (C.w_sh) {
                T ix, iy, iz;
                image_offset<T>(C.w_sh[w0 + e - 1], ix, iy, iz);
                d.ox += ix, d.oy += iy, d.oz += iz;
            }
            d.r = (T)kAlphaInner * pow2<T>(-(la + 1));
            d.hw = W.wl_h ? pow2<T>(-(la + 1)) : T(1);
            d.base = a * ns;
            d.kind = 1;
            cnt = ns;
        } else if (e < nseg) {
            const int a = C.u_idx[u0 + e - 1 - nw], la = C.lvl[a];
            d.ox = centre_diff<T>(C.cx[a], la, bx, lb);
            d.oy = centre_diff<T>(C.cy[a], la, by, lb);
            d.oz = centre_diff<T>(C.cz[a], la, bz, lb);
            const int sa = C.u_sh ? (int)C.u_sh[u0 + e - 1 - nw] : 13;
            if (sa != 13) {
                T ix, iy, iz;
                image_offset<T>(sa, ix, iy, iz);
                d.ox += ix, d.oy += iy, d.oz += iz;
            }
            d.base = C.first[a];
            cnt = C.cnt[a];
            own = (a == b) && sa == 13;  // another image of the leaf is not its own particles
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned own_mask = __ballot_sync(0xffffffffu, own);
        int olo = 0, ohi = 0;
        if (own_mask) {
            const int o = __ffs(own_mask) - 1;
            ohi = __shfl_sync(0xffffffffu, incl, o);
            olo = ohi - __shfl_sync(0xffffffffu, cnt, o);
        }
        __syncwarp();  // the previous batch is done with seg, start and buf
        S.seg[lane] = d;
        S.start[lane] = (e < nseg) ? incl - cnt : total;
        __syncwarp();
        const int nb = min(kLSeg, nseg - sb);
        typename Vec4<T>::type raw[kLK];
        int rs[kLK];
        const int nchunks = (total + kLChunk - 1) / kLChunk;
        for (int c = 0; c < nchunks; ++c) {
            // double-buffered: the slot written here was last read two chunks ago
            leaf_fetch<T>(S, c, total, nb, pts, surf, W, raw, rs);
            leaf_store<T, G>(S, c & 1, raw, rs);
            __syncwarp();
            const int c0 = c * kLChunk;
            leaf_chunk<T, TPL, G>(L, S.buf[c & 1], min(kLChunk, total - c0), olo - c0, ohi - c0, grp);
        }
    }
    leaf_flush<T, TPL>(L);
#pragma unroll
    for (int k = 0; k < TPL; ++k) {
        double tot[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            tot[c] = (double)L.acc[k][c] + (double)L.cmp[k][c];
#pragma unroll
            for (int o = 16; o >= LG; o >>= 1) tot[c] += __shfl_xor_sync(0xffffffffu, tot[c], o);
        }
        if (C.dbar) tot[0] += C.dbar[b];  // the constant part of the local expansion
        const int i = tbase + mem + LG * k;
        if (grp == 0 && i < n) {
            res[f + i] = make_double4(tot[0], tot[1], tot[2], tot[3]);
            if (!isfinite(tot[0] + tot[1] + tot[2] + tot[3])) set_status(C.status, KIFMM_ERR_NONFINITE);
            if (C.pot || C.grad) {  // the finalisation, as k_finalize does it
                const uint32_t j = C.perm[f + i];
                const int sy = C.sys[b];
                const double c1 = C.out_scale[2 * sy], c2 = C.out_scale[2 * sy + 1];
                if (C.out_f64) {
                    if (C.pot) ((double *)C.pot)[j] = c1 * tot[0];
                    if (C.grad) {
                        double *g = (double *)C.grad + 3 * (size_t)j;
                        g[0] = c2 * tot[1];
                        g[1] = c2 * tot[2];
                        g[2] = c2 * tot[3];
                    }
                } else {
                    if (C.pot) ((float *)C.pot)[j] = (float)(c1 * tot[0]);
                    if (C.grad) {
                        float *g = (float *)C.grad + 3 * (size_t)j;
                        g[0] = (float)(c2 * tot[1]);
                        g[1] = (float)(c2 * tot[2]);
                        g[2] = (float)(c2 * tot[3]);
                    }
                }
            }
        }
    }
}
// Leaf work items: a leaf is covered greedily by passes (leaf, first
// target); the pass over r remaining targets uses the plan table's variant
// for r (bucket (r - 1) / 8) and covers (32 / G) TPL of them, so e.g. 40
// targets become a 32-target pass and an 8-target pass with four source
// groups, keeping every lane busy.  One kernel per variant, each with the
// registers its tile needs; k_leaf_partition lists the items of each
// variant (order within a list is immaterial: passes are independent).
__global__ void k_leaf_partition(int64_t n_leaves, const int32_t *__restrict__ leaves,
                                 const int32_t *__restrict__ cnt, LeafTiling tile, int64_t cap,
                                 int2 *__restrict__ lists, int32_t *__restrict__ counts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n_leaves;
    const int b = valid ? leaves[i] : -1;
    const int n = valid ? cnt[b] : 0;
    int t0 = 0;
    while (__any_sync(0xffffffffu, t0 < n)) {
        const int v = (t0 < n) ? leaf_variant(tile, n - t0) : -1;
#pragma unroll
        for (int u = 0; u < kLeafTiles; ++u) {
            const unsigned m = __ballot_sync(0xffffffffu, v == u);
            if (m == 0) continue;
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&counts[u], __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (v == u) lists[(int64_t)u * cap + base + __popc(m & ((1u << lane) - 1))] = make_int2(b, t0);
        }
        if (v >= 0) t0 += (32 / leaf_tile_groups(v)) * leaf_tile_tpl(v);
    }
}

// Each warp takes the next pass from a shared counter as it finishes one
// (passes differ in length by their source lists; a fixed stride left the
// last warps running alone).  Every pass writes only its own targets, so the
// order passes are taken in does not change any result.
template <typename T, int TPL, int G>
__global__ void __launch_bounds__(32 * kLW, sizeof(T) == 4 ? (TPL == 1 ? 5 : 4) : 2)
    k_leaf_all(LeafCtx C, const int2 *__restrict__ list, const int32_t *__restrict__ count, int32_t *next,
               const typename Vec4<T>::type *__restrict__ pts, const T *__restrict__ surf, LeafW<T> W,
               double4 *__restrict__ res) {
    __shared__ LeafSmem<T> bufs[kLW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nl = *count;
    while (true) {
        int li = 0;
        if (lane == 0) li = atomicAdd(next, 1);
        li = __shfl_sync(0xffffffffu, li, 0);
        if (li >= nl) break;
        const int2 it = list[li];
        leaf_pass<T, TPL, G>(C, it.x, it.y, pts, surf, W, bufs[warp], res);
    }
}

template <typename T, int TPL, int G>
void leaf_launch_variant(const Plan &P, const LeafCtx &C, int v, const typename Vec4<T>::type *pts, const T *surf,
                         const LeafW<T> &W, double4 *res, cudaStream_t caller) {
    // on the variant's own stream, after the partition; joined back below
    cudaStream_t s = P.leaf_streams[v];
    cudaStreamWaitEvent(s, P.leaf_fork, 0);
    constexpr int occ = sizeof(T) == 4 ? (TPL == 1 ? 5 : 4) : 2;
    const int64_t want = (P.n_leaves + kLW - 1) / kLW;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)P.num_sms * occ));
    ++g_launches, k_leaf_all<T, TPL, G><<<g, 32 * kLW, 0, s>>>(C, P.leaf_vlist + (int64_t)v * P.leaf_item_cap,
                                                                P.leaf_vcnt + v, P.leaf_vcnt + 8 + v, pts, surf,
                                                                W, res);
    cudaEventRecord(P.leaf_join[v], s);
    cudaStreamWaitEvent(caller, P.leaf_join[v], 0);
}

// All leaves: work items by variant, then one launch per variant the table
// uses, each on its own stream so that the short variants' tails (a pass of
// one warp over a leaf's whole source list) overlap the long one.
template <typename T>
void leaf_launch(const Plan &P, const LeafCtx &C, const typename Vec4<T>::type *pts, const T *surf,
                 const LeafW<T> &W, double4 *res, cudaStream_t s) {
    if (P.n_leaves == 0) return;
    cudaMemsetAsync(P.leaf_vcnt, 0, sizeof(int32_t) * 16, s);  // counts and next-pass counters
    ++g_launches, k_leaf_partition<<<(unsigned)((P.n_leaves + 255) / 256), 256, 0, s>>>(
                      P.n_leaves, P.leaves, P.cnt, C.tile, P.leaf_item_cap, P.leaf_vlist, P.leaf_vcnt);
    cudaEventRecord(P.leaf_fork, s);
    bool used[kLeafTiles] = {false};
    for (int i = 0; i < kLeafBuckets; ++i) used[C.tile.get(i)] = true;
    if (used[0]) leaf_launch_variant<T, 1, 4>(P, C, 0, pts, surf, W, res, s);
    if (used[1]) leaf_launch_variant<T, 2, 4>(P, C, 1, pts, surf, W, res, s);
    if (used[2]) leaf_launch_variant<T, 1, 2>(P, C, 2, pts, surf, W, res, s);
    if (used[3]) leaf_launch_variant<T, 2, 2>(P, C, 3, pts, surf, W, res, s);
    if (used[4]) leaf_launch_variant<T, 1, 1>(P, C, 4, pts, surf, W, res, s);
    if (used[5]) leaf_launch_variant<T, 2, 1>(P, C, 5, pts, surf, W, res, s);
}

// Scatter to caller order with 1/(4 pi), coef and physical units.
template <typename TO>
__global__ void k_finalize(int64_t n, const double4 *__restrict__ res, const uint32_t *__restrict__ perm,
                           const int64_t *__restrict__ off, int S, const double *__restrict__ out_scale,
                           TO *pot, TO *grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= (int64_t)j) lo = mid; else hi = mid - 1;
    }
    const double c1 = out_scale[2 * lo], c2 = out_scale[2 * lo + 1];  // coef / (4 pi side), / side^2
    const double4 r = res[i];
    if (pot) pot[j] = (TO)(c1 * r.x);
    if (grad) {
        grad[3 * j] = (TO)(c2 * r.y);
        grad[3 * j + 1] = (TO)(c2 * r.z);
        grad[3 * j + 2] = (TO)(c2 * r.w);
    }
}

// Energy partial sums over chunks that never straddle systems (sorted order).
template <typename T>
__global__ void k_energy_chunks(const int64_t *__restrict__ chunks, const double4 *__restrict__ res,
                                const typename Vec4<T>::type *__restrict__ pts, double *partial) {
    __shared__ double red[256];
    const int64_t a = chunks[2 * blockIdx.x], e = chunks[2 * blockIdx.x + 1];
    double s = 0.0;
    for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) s += (double)pts[i].w * res[i].x;
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_energy_sum(const int32_t *__restrict__ chunk_start, const double *__restrict__ partial,
                             const double *__restrict__ lo_side, double coef, int S, double *energy) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double e = 0.0;
    for (int c = chunk_start[s]; c < chunk_start[s + 1]; ++c) e += partial[c];
    energy[s] = 0.5 * coef * kInv4Pi / lo_side[s * 4 + 3] * e;
}

// Clump force and torque, FP64 accumulation, one thread per clump.
template <typename TO>
__global__ void k_clump(int64_t nc, const int64_t *__restrict__ off, const TO *__restrict__ xyz,
                        const TO *__restrict__ q, const TO *__restrict__ grad, const TO *__restrict__ ref,
                        TO *force, TO *torque) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double F[3] = {0, 0, 0}, Tq[3] = {0, 0, 0};
    const double rx = ref[3 * c], ry = ref[3 * c + 1], rz = ref[3 * c + 2];
    for (int64_t k = off[c]; k < off[c + 1]; ++k) {
        const double qk = q[k];
        const double f0 = -qk * (double)grad[3 * k], f1 = -qk * (double)grad[3 * k + 1],
                     f2 = -qk * (double)grad[3 * k + 2];
        const double dx = (double)xyz[3 * k] - rx, dy = (double)xyz[3 * k + 1] - ry,
                     dz = (double)xyz[3 * k + 2] - rz;
        F[0] += f0;
        F[1] += f1;
        F[2] += f2;
        Tq[0] += dy * f2 - dz * f1;
        Tq[1] += dz * f0 - dx * f2;
        Tq[2] += dx * f1 - dy * f0;
    }
    for (int d = 0; d < 3; ++d) {
        force[3 * c + d] = (TO)F[d];
        torque[3 * c + d] = (TO)Tq[d];
    }
}


inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// k_p2m launch shape: a thread per check point, four staged values per thread.
inline int p2m_threads(const Plan &P) { return (P.ns + 31) / 32 * 32; }
template <typename T>
inline size_t p2m_smem(const Plan &P) { return 7 * sizeof(T) * (size_t)p2m_threads(P); }

// Classes c < ncls own targets [starts[c], starts[c + 1]); one launch.
template <typename T, class G>
void ggemm_classes(Plan &P, const G &g, const int32_t *targets, const int64_t *starts, int ncls, int nslots,
                   const T *in, T *out, int accumulate, cudaStream_t s, int ld = 0, double *dbar = nullptr) {
    ClassRanges cr;
    int64_t most = 0, total = 0;
    for (int c = 0; c <= ncls; ++c) cr.b[c] = starts[c];
    for (int c = 0; c < ncls; ++c) {
        most = std::max<int64_t>(most, starts[c + 1] - starts[c]);
        total += starts[c + 1] - starts[c];
    }
    if (most <= 0) return;
    if (ld == 0) ld = P.ns;
    // 64 x 160 tiles while they fill the GPU twice over; else 16 x 32 tiles
    // (the coarse levels of M2M / L2L and small trees are latency-bound),
    // with up to 8 slots split over blocks for up to kSplitTargets targets.
    const int64_t big_blocks = grid_for(total, 64) * grid_for(ld, 160);
    if (big_blocks >= 2 * P.num_sms) {
        dim3 grid(grid_for(most, 64), ncls, grid_for(ld, 160));
        if constexpr (sizeof(T) == 4) {
            const bool vec = P.ns % 4 == 0;
            if (nslots > 1 && vec)
                ++g_launches, k_ggemm_v4<G, true, true><<<grid, kV4Threads, 0, s>>>(g, targets, cr, nslots, P.ns, ld,
                                                                                   in, out, accumulate, dbar);
            else if (nslots > 1)
                ++g_launches, k_ggemm_v4<G, true, false><<<grid, kV4Threads, 0, s>>>(g, targets, cr, nslots, P.ns,
                                                                                    ld, in, out, accumulate, dbar);
            else if (vec)
                ++g_launches, k_ggemm_v4<G, false, true><<<grid, kV4Threads, 0, s>>>(g, targets, cr, nslots, P.ns,
                                                                                    ld, in, out, accumulate, dbar);
            else
                ++g_launches, k_ggemm_v4<G, false, false><<<grid, kV4Threads, 0, s>>>(g, targets, cr, nslots, P.ns,
                                                                                     ld, in, out, accumulate, dbar);
            return;
        }
        if (nslots > 1)
            ++g_launches, k_ggemm<T, G, 8, 8, 5, false, true><<<grid, 256, 0, s>>>(g, targets, cr, nslots, P.ns, ld,
                                                                                  in, out, accumulate, dbar, 1, nullptr);
        else
            ++g_launches, k_ggemm<T, G, 8, 8, 5, false, false><<<grid, 256, 0, s>>>(g, targets, cr, nslots, P.ns, ld,
                                                                                   in, out, accumulate, dbar, 1, nullptr);
        return;
    }
    const bool splittable = nslots > 1 && nslots <= 8 && total <= kSplitTargets;
    if (splittable && big_blocks * nslots >= 2 * P.num_sms) {
        // big tiles, one slot per block (single-slot registers: two blocks per SM)
        T *part = (T *)P.gemm_part;
        const int ncb_big = (int)grid_for(ld, 160);
        dim3 grid(grid_for(most, 64), ncls, ncb_big * nslots);
        if constexpr (sizeof(T) == 4) {
            if (P.ns % 4 == 0)
                ++g_launches, k_ggemm_v4<G, false, true, true><<<grid, kV4Threads, 0, s>>>(
                                  g, targets, cr, nslots, P.ns, ld, in, out, accumulate, dbar, ncb_big, part);
            else
                ++g_launches, k_ggemm_v4<G, false, false, true><<<grid, kV4Threads, 0, s>>>(
                                  g, targets, cr, nslots, P.ns, ld, in, out, accumulate, dbar, ncb_big, part);
        } else {
            ++g_launches, k_ggemm<T, G, 8, 8, 5, true, false><<<grid, 256, 0, s>>>(g, targets, cr, nslots, P.ns, ld,
                                                                                    in, out, accumulate, dbar,
                                                                                    ncb_big, part);
        }
        ++g_launches, k_ggemm_sum<T, G><<<grid_for(total * ld, 256), 256, 0, s>>>(
                          g, targets, cr.b[0], total, nslots, P.ns, ld, part, out, accumulate, dbar);
        return;
    }
    const int ncb = (int)grid_for(ld, 32);
    int64_t small_blocks = 0;
    for (int c = 0; c < ncls; ++c) small_blocks += grid_for(starts[c + 1] - starts[c], 16);
    small_blocks *= ncb;
    if (splittable && small_blocks < 16 * P.num_sms) {
        T *part = (T *)P.gemm_part;
        dim3 grid(grid_for(most, 16), ncls, ncb * nslots);
        ++g_launches, k_ggemm<T, G, 4, 4, 1, true, false><<<grid, 128, 0, s>>>(g, targets, cr, nslots, P.ns, ld, in,
                                                                                out, accumulate, dbar, ncb, part);
        ++g_launches, k_ggemm_sum<T, G><<<grid_for(total * ld, 256), 256, 0, s>>>(
                          g, targets, cr.b[0], total, nslots, P.ns, ld, part, out, accumulate, dbar);
        return;
    }
    dim3 grid(grid_for(most, 16), ncls, ncb);
    ++g_launches, k_ggemm<T, G, 4, 4, 1, false, true><<<grid, 128, 0, s>>>(g, targets, cr, nslots, P.ns, ld, in,
                                                                            out, accumulate, dbar, ncb, nullptr);
}

template <typename T, class G>
void ggemm(Plan &P, const G &g, const int32_t *targets, int64_t a, int64_t e, int nslots, const T *in, T *out,
           int accumulate, cudaStream_t s) {
    const int64_t st[2] = {a, e};
    ggemm_classes<T, G>(P, g, targets, st, 1, nslots, in, out, accumulate, s);
}

// Periodic cell (Sec. 2.4): the images beyond the 26 nearest act on the
// root's downward check potential, d(root) += F u(root), with F the
// far-image composite; FP64 sums, one block.  With dbar (FP32-based modes)
// the mean goes to dbar and the mean-free rest to d.
template <typename T>
__global__ void k_far_root(int ns, const double *__restrict__ Ft, const double *__restrict__ u, T *__restrict__ d,
                           double *__restrict__ dbar) {
    __shared__ double v[kMaxNs];
    __shared__ double red[32];
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < ns; ++k) acc += Ft[(size_t)k * ns + j] * u[k];
        v[j] = acc;
    }
    __syncthreads();
    double mean = 0.0;
    if (dbar) {
        double sum = 0.0;
        for (int j = threadIdx.x; j < ns; j += blockDim.x) sum += v[j];
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
        __syncthreads();
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        mean = tot / ns;
        if (threadIdx.x == 0) dbar[0] += mean;
    }
    for (int j = threadIdx.x; j < ns; j += blockDim.x) d[j] += (T)(v[j] - mean);
}

// Periodic cell: the uniform potential term of the conducting-boundary
// lattice sum that the root's equivalent density does not carry, (2 pi / 3)
// (Q2 of the particles - Q2 of the density) for the unit cell (V = 1), Q2 the
// trace of the second moment about the cell centre.  The particles' Q2 is
// the sum of the per-leaf sums in leaf order, the density's is g . u(root).
// One block, fixed summation order.
__global__ void k_moment_term(int64_t nl, const double *__restrict__ leaf_q2, int ns, const double *__restrict__ g,
                              const double *__restrict__ u_root, double *pshift) {
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < nl; i += blockDim.x) a += leaf_q2[i];
    for (int j = threadIdx.x; j < ns; j += blockDim.x) b += g[j] * u_root[j];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double qa = 0.0, qb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) qa += red[0][w], qb += red[1][w];
        *pshift = (2.0 * 3.14159265358979323846 / 3.0) * (qa - qb);
    }
}

// FP32-based periodic plans: the root's upward check potential in FP64 from
// its children's (M2M composites in FP64, stored [k][j]); a root that is a
// leaf keeps its own.  One block.
__global__ void k_root_up64(int ns, const int32_t *__restrict__ child8, const int32_t *__restrict__ nchild,
                            const double *__restrict__ m2m64, const float *__restrict__ u, double *__restrict__ u64) {
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        double acc = 0.0;
        if (nchild[0] == 0) {
            acc = (double)u[j];
        } else {
            for (int c = 0; c < 8; ++c) {
                const int32_t ch = child8[c];
                if (ch < 0) continue;
                const double *M = m2m64 + (size_t)c * ns * ns;
                for (int k = 0; k < ns; ++k) acc += M[(size_t)k * ns + j] * (double)u[(size_t)ch * ns + k];
            }
        }
        u64[j] = acc;
    }
}

__global__ void k_add_shift(int64_t n, const double *__restrict__ pshift, double4 *__restrict__ res) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) res[i].x += *pshift;
}

template <typename T>
cudaError_t evaluate_t(Plan &P, void *pot, void *grad, double *energy, cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    const int ns = P.ns;
    const size_t nn = (size_t)ns * ns;
    const T *surf = P.f64 ? (const T *)P.surf64 : (const T *)P.surf32;
    T *u = (T *)P.u_chk, *d = (T *)P.d_chk, *tmp = (T *)P.tmp_chk;
    const V4 *pts = (const V4 *)P.pts;
    double4 *res = (double4 *)P.res;
    // upward pass
    stage_begin(P, KIFMM_STAGE_P2M, s);
    if constexpr (sizeof(T) == 4)
        ++g_launches, k_p2m_f32<<<(unsigned)((P.n_leaves + kP2mLeaves - 1) / kP2mLeaves), p2m_threads(P),
                                  4 * sizeof(float) * (size_t)p2m_threads(P), s>>>(P.leaves, P.n_leaves, P.lvl,
                                                                                   P.first, P.cnt, pts, surf, ns, u);
    else
        ++g_launches, k_p2m<T><<<(unsigned)P.n_leaves, p2m_threads(P), p2m_smem<T>(P), s>>>(
                          P.leaves, P.lvl, P.first, P.cnt, pts, surf, ns, u);
    stage_end(P, KIFMM_STAGE_P2M, s);
    stage_begin(P, KIFMM_STAGE_M2M, s);
    for (int l = P.max_level - 1; l >= 0; --l)
        ggemm<T>(P, GatherChild<T>{P.child8, (const T *)P.m2m_t, ns}, P.part_list[1],
                 P.part_start[1][1 + l], P.part_start[1][2 + l], 8, u, u, 0, s);
    stage_end(P, KIFMM_STAGE_M2M, s);
    KIFMM_CUDA_TRY(cudaGetLastError());
    // interactions
    stage_begin(P, KIFMM_STAGE_M2L, s);
    KIFMM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(T) * (size_t)P.nb * ns, s));
    const bool split_mean = !P.f64;  // FP32-based modes: d = dbar (FP64) + mean-free FP32 vector
    if (split_mean) KIFMM_CUDA_TRY(cudaMemsetAsync(P.dbar, 0, sizeof(double) * (size_t)P.nb, s));
    const bool tensor = (P.desc.precision == KIFMM_MIXED_FP16);
    if (tensor) {
        KIFMM_CUDA_TRY(m2l_tensor(P, s));
    } else {
        ggemm_classes<T>(P, GatherM2L<T>{P.vdense, P.slot_off, (const T *)P.m2l_t, ns, P.op_ld}, P.part_list[0],
                         P.part_start[0].data(), 8, kVSlots, u, d, 0, s, P.op_ld, split_mean ? P.dbar : nullptr);
    }
    stage_end(P, KIFMM_STAGE_M2L, s);
    if (P.n_x > 0) {
        stage_begin(P, KIFMM_STAGE_P2L, s);
        ++g_launches, k_p2l<T><<<(unsigned)P.nb, kLeafThreads, 0, s>>>(P.nx, P.xdense, P.lvl, P.cx, P.cy, P.cz,
                                                                        P.first, P.cnt, pts, surf, ns, d, nullptr,
                                                                        0, split_mean ? P.dbar : nullptr, nullptr,
                                                                        P.periodic ? P.x_sh : nullptr);
        stage_end(P, KIFMM_STAGE_P2L, s);
    }
    // the root's upward check potential in FP64 (periodic cell)
    const double *u_root = nullptr;
    if (P.periodic) {
        if constexpr (sizeof(T) == 8) {
            u_root = (const double *)u;
        } else {
            ++g_launches, k_root_up64<<<1, 256, 0, s>>>(ns, P.child8, P.nchild, P.m2m64, u, P.u_root64);
            u_root = P.u_root64;
        }
        // the far images, on the root (box 0) before the downward pass
        ++g_launches, k_far_root<T><<<1, 256, 0, s>>>(ns, P.far_t, u_root, d, split_mean ? P.dbar : nullptr);
    }
    // downward pass: per level, per octant class of the child
    stage_begin(P, KIFMM_STAGE_L2L, s);
    for (int l = 1; l <= P.max_level; ++l)
        ggemm_classes<T>(P, GatherParent<T>{P.parent, (const T *)P.l2l_t, ns, P.op_ld}, P.part_list[3],
                         P.part_start[3].data() + 8 * l, 8, 1, d, d, 1, s, P.op_ld, split_mean ? P.dbar : nullptr);
    stage_end(P, KIFMM_STAGE_L2L, s);
    KIFMM_CUDA_TRY(cudaGetLastError());
    // leaves: equivalent densities (two-step pseudo-inverse), then L2P + M2P + P2P
    stage_begin(P, KIFMM_STAGE_LEAF, s);
    if (P.n_w > 0) {
        ggemm<T>(P, GatherSelf<T>{(const T *)P.up_w_t}, P.part_list[2], 0, P.part_start[2][1], 1, u, tmp, 0, s);
        ggemm<T>(P, GatherSelf<T>{(const T *)P.up_v_t}, P.part_list[2], 0, P.part_start[2][1], 1, tmp,
                 (T *)P.up_dens, 0, s);
    }
    ggemm<T>(P, GatherSelf<T>{(const T *)P.dn_w_t}, P.leaves, 0, P.n_leaves, 1, d, tmp, 0, s);
    ggemm<T>(P, GatherSelf<T>{(const T *)P.dn_v_t}, P.leaves, 0, P.n_leaves, 1, tmp, (T *)P.dn_dens, 0, s);
    stage_end(P, KIFMM_STAGE_LEAF, s);
    stage_begin(P, KIFMM_STAGE_P2P, s);
    LeafCtx C{P.lvl, P.cx, P.cy, P.cz, P.first, P.cnt, P.u_ptr, P.w_ptr, P.u_idx, P.w_idx, ns,
              split_mean ? P.dbar : nullptr, P.leaf_tile, P.status, P.periodic ? P.u_sh : nullptr,
              P.periodic ? P.w_sh : nullptr};
    // free space: the leaf pass writes the outputs itself (a periodic cell
    // adds the uniform shift to the results afterwards, then k_finalize)
    const bool fused_out = !P.periodic && (pot || grad);
    if (fused_out) {
        C.perm = P.perm;
        C.sys = P.sys;
        C.out_scale = P.out_scale;
        C.pot = pot;
        C.grad = grad;
        C.out_f64 = P.io_f64 ? 1 : 0;
    }
    const LeafW<T> W{(const T *)P.dn_dens, 1, (const T *)P.up_dens, 1, nullptr};
    if (!P.tuned_leaf && tuning_wanted(P, s)) {
        // time every candidate table on this tree; keep the fastest
        float best = 1e30f;
        LeafTiling pick = P.leaf_tile;
        leaf_launch<T>(P, C, pts, surf, W, res, s);  // warm the caches first
        for (int c = 0; c < kLeafTilingCandidates; ++c) {
            LeafCtx Cc = C;
            Cc.tile = leaf_tiling_candidate(c);
            float ms = 1e30f;
            for (int rep = 0; rep < 2; ++rep)  // best of two
                ms = std::min(ms, time_launch(s, [&] { leaf_launch<T>(P, Cc, pts, surf, W, res, s); }));
            if (ms < best) {
                best = ms;
                pick = Cc.tile;
            }
        }
        P.leaf_tile = pick;
        C.tile = pick;
        P.tuned_leaf = true;
    }
    leaf_launch<T>(P, C, pts, surf, W, res, s);
    if (P.periodic) {
        ++g_launches, k_moment_term<<<1, 256, 0, s>>>(P.n_leaves, P.leaf_q2, ns, P.far_g, u_root, P.pshift);
        ++g_launches, k_add_shift<<<grid_for(P.n, 256), 256, 0, s>>>(P.n, P.pshift, res);
    }
    stage_end(P, KIFMM_STAGE_P2P, s);
    KIFMM_CUDA_TRY(cudaGetLastError());
    // outputs
    stage_begin(P, KIFMM_STAGE_OUT, s);
    if ((pot || grad) && !fused_out) {
        if (P.io_f64)
            ++g_launches, k_finalize<double><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, res, P.perm, P.sys_off_d, P.n_sys, P.out_scale, (double *)pot,
                              (double *)grad);
        else
            ++g_launches, k_finalize<float><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, res, P.perm, P.sys_off_d, P.n_sys, P.out_scale, (float *)pot,
                              (float *)grad);
    }
    if (energy) {
        ++g_launches, k_energy_chunks<T><<<(unsigned)P.n_energy_chunks, 256, 0, s>>>(P.energy_chunks, res, pts,
                                                                                   P.energy_partial);
        ++g_launches, k_energy_sum<<<grid_for(P.n_sys, 64), 64, 0, s>>>(P.energy_chunk_start, P.energy_partial,
                                                                         P.lo_side, P.coef, P.n_sys, energy);
    }
    stage_end(P, KIFMM_STAGE_OUT, s);
    P.fwd_valid = P.fwd_res_valid = true;
    return cudaGetLastError();
}

// Per-particle system (the last offset at or below the caller index j).
__device__ __forceinline__ int system_of(const int64_t *__restrict__ off, int S, uint32_t j) {
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= (int64_t)j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Adjoint weights in sorted order: ws = dL/dpot + (1/2) dL/dU_s q (the energy
// U_s = 1/2 sum q pot of the particle's system s, through its pot); with an
// energy loss the forward potential (root units) is kept for the explicit
// (1/2) dL/dU pot term of dq, since the transposed passes overwrite it.
template <typename TI, typename T>
__global__ void k_adj_weights(int64_t n, const uint32_t *__restrict__ perm, const int64_t *__restrict__ off, int S,
                              const typename Vec4<T>::type *__restrict__ pts, const TI *__restrict__ w,
                              const double *__restrict__ dLdU, const double4 *__restrict__ res, T *__restrict__ ws,
                              double *__restrict__ fwd_pot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    double v = w ? (double)w[j] : 0.0;
    if (dLdU) {
        v += 0.5 * dLdU[system_of(off, S, j)] * (double)pts[i].w;
        fwd_pot[i] = res[i].x;
    }
    ws[i] = (T)v;
}

// dq = c1 (psi + pd) (+ 1/2 dL/dU c1 pot), dx = w_tot grad + c2 (q grad(psi + pd) + hg),
// c1 = coef / (4 pi side), c2 = c1 / side; w_tot = dL/dpot + 1/2 dL/dU q.
template <typename TO, typename T>
__global__ void k_finalize_adj(int64_t n, const double4 *__restrict__ res, const uint32_t *__restrict__ perm,
                               const int64_t *__restrict__ off, int S, const double *__restrict__ out_scale,
                               const typename Vec4<T>::type *__restrict__ pts, const TO *__restrict__ w,
                               const double *__restrict__ dLdU, const double *__restrict__ fwd_pot,
                               const double4 *__restrict__ hg, const double4 *__restrict__ pd,
                               const TO *__restrict__ grad, TO *dq, TO *dx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    const int s = system_of(off, S, j);
    const double c1 = out_scale[2 * s], c2 = out_scale[2 * s + 1];  // coef / (4 pi side), / side^2
    double4 r = res[i];
    if (pd) {
        const double4 e = pd[i];
        r.x += e.x, r.y += e.y, r.z += e.z, r.w += e.w;
    }
    const double q = (double)pts[i].w;
    const double hu = dLdU ? 0.5 * dLdU[s] : 0.0;
    if (dq) dq[j] = (TO)(c1 * r.x + (dLdU ? hu * c1 * fwd_pot[i] : 0.0));
    if (dx) {
        const double wj = (w ? (double)w[j] : 0.0) + hu * q;
        double t[3] = {c2 * q * r.y, c2 * q * r.z, c2 * q * r.w};
        if (hg) {
            const double4 h = hg[i];
            t[0] += c2 * h.x, t[1] += c2 * h.y, t[2] += c2 * h.z;
        }
        if (grad)
            for (int d = 0; d < 3; ++d) t[d] += wj * (double)grad[3 * j + d];
        dx[3 * j] = (TO)t[0];
        dx[3 * j + 1] = (TO)t[1];
        dx[3 * j + 2] = (TO)t[2];
    }
}

// ---------------------------------------------------------------------------
// The Stokeslet (the tensor kernel Eq. 1 admits; Stokes flow, Sec. 2.4):
// G(r) = I / |r| + r r^T / |r|^3, the 1 / (8 pi) and coef applied at the
// output.  Sources carry forces, surfaces 3-vector densities (expansion
// vectors of 3 n_s values, point-major), targets receive velocities.  The
// same homogeneity as 1/r (degree -1), so the box-unit scalings carry over.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void stokes_acc(T rx, T ry, T rz, T fx, T fy, T fz, T &ux, T &uy, T &uz) {
    const T ri = rsqrt_t<T>(rx * rx + ry * ry + rz * rz);
    const T rf = (rx * fx + ry * fy + rz * fz) * (ri * ri * ri);
    ux += fx * ri + rx * rf;
    uy += fy * ri + ry * rf;
    uz += fz * ri + rz * rf;
}

// P2M: u(b)_{3j+a} = sum_i G_a.(UC_j - x_i) f_i, box units then 1/h; one
// block per leaf, a thread per check point, forces staged through shared memory.
template <typename T>
__global__ void k_p2m_stokes(const int32_t *__restrict__ leaves, const int32_t *__restrict__ lvl,
                             const int32_t *__restrict__ first, const int32_t *__restrict__ cnt,
                             const typename Vec4<T>::type *__restrict__ pts, const T *__restrict__ frc,
                             const T *__restrict__ surf, int npt, T *__restrict__ u) {
    __shared__ T sx[kLeafThreads], sy[kLeafThreads], sz[kLeafThreads], sfx[kLeafThreads], sfy[kLeafThreads],
        sfz[kLeafThreads];
    const int b = leaves[blockIdx.x];
    const T h = box_half<T>(lvl[b]), hinv = T(1) / h;
    const int n = cnt[b], f = first[b];
    const T a = (T)kAlphaOuter;
    for (int j0 = 0; j0 < npt; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        T px = 0, py = 0, pz = 0, ux = 0, uy = 0, uz = 0;
        if (j < npt) px = a * surf[3 * j], py = a * surf[3 * j + 1], pz = a * surf[3 * j + 2];
        for (int c0 = 0; c0 < n; c0 += kLeafThreads) {
            __syncthreads();
            for (int k = threadIdx.x; k < kLeafThreads && c0 + k < n; k += blockDim.x) {
                const auto v = pts[f + c0 + k];
                sx[k] = v.x * hinv, sy[k] = v.y * hinv, sz[k] = v.z * hinv;
                const size_t o = 3 * (size_t)(f + c0 + k);
                sfx[k] = frc[o], sfy[k] = frc[o + 1], sfz[k] = frc[o + 2];
            }
            __syncthreads();
            const int m = min(kLeafThreads, n - c0);
            for (int i = 0; i < m; ++i) stokes_acc<T>(px - sx[i], py - sy[i], pz - sz[i], sfx[i], sfy[i], sfz[i], ux, uy, uz);
        }
        if (j < npt) {
            T *o = u + (size_t)b * 3 * npt + 3 * j;
            o[0] = ux * hinv, o[1] = uy * hinv, o[2] = uz * hinv;
        }
    }
}

// P2L: d(b) += the forces of the leaves of X(b) on b's downward check surface.
template <typename T>
__global__ void k_p2l_stokes(const int32_t *__restrict__ nx, const int32_t *__restrict__ xdense,
                             const int32_t *__restrict__ lvl, const int32_t *__restrict__ cx,
                             const int32_t *__restrict__ cy, const int32_t *__restrict__ cz,
                             const int32_t *__restrict__ first, const int32_t *__restrict__ cnt,
                             const typename Vec4<T>::type *__restrict__ pts, const T *__restrict__ frc,
                             const T *__restrict__ surf, int npt, T *__restrict__ d) {
    __shared__ T sx[kLeafThreads], sy[kLeafThreads], sz[kLeafThreads], sfx[kLeafThreads], sfy[kLeafThreads],
        sfz[kLeafThreads];
    const int b = blockIdx.x;
    if (nx[b] == 0) return;
    const int lb = lvl[b];
    const T hb = box_half<T>(lb), hinv = T(1) / hb;
    const T al = (T)kAlphaInner;
    for (int j0 = 0; j0 < npt; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        T px = 0, py = 0, pz = 0, ux = 0, uy = 0, uz = 0;
        if (j < npt) px = al * surf[3 * j], py = al * surf[3 * j + 1], pz = al * surf[3 * j + 2];
        for (int e = 0; e < nx[b]; ++e) {
            const int a = xdense[(size_t)b * kMaxCoarse + e], la = lvl[a];
            const T ox = centre_diff<T>(cx[a], la, cx[b], lb), oy = centre_diff<T>(cy[a], la, cy[b], lb),
                    oz = centre_diff<T>(cz[a], la, cz[b], lb);
            const int n = cnt[a], f = first[a];
            for (int c0 = 0; c0 < n; c0 += kLeafThreads) {
                __syncthreads();
                for (int k = threadIdx.x; k < kLeafThreads && c0 + k < n; k += blockDim.x) {
                    const auto v = pts[f + c0 + k];
                    sx[k] = (ox + v.x) * hinv, sy[k] = (oy + v.y) * hinv, sz[k] = (oz + v.z) * hinv;
                    const size_t o = 3 * (size_t)(f + c0 + k);
                    sfx[k] = frc[o], sfy[k] = frc[o + 1], sfz[k] = frc[o + 2];
                }
                __syncthreads();
                const int m = min(kLeafThreads, n - c0);
                for (int i = 0; i < m; ++i)
                    stokes_acc<T>(px - sx[i], py - sy[i], pz - sz[i], sfx[i], sfy[i], sfz[i], ux, uy, uz);
            }
        }
        if (j < npt) {
            T *o = d + (size_t)b * 3 * npt + 3 * j;
            o[0] += ux * hinv, o[1] += uy * hinv, o[2] += uz * hinv;
        }
    }
}

// Leaves: L2P (own downward density on the 2.95 h_b surface), M2P (the W
// boxes' upward densities on their 1.05 h_a surfaces) and P2P (the U-list
// particles' forces, r = 0 skipped); root units, FP64 sums; one block per
// leaf, a thread per target.
template <typename T>
__global__ void __launch_bounds__(kLeafThreads) k_leaf_stokes(LeafCtx C, const int32_t *__restrict__ leaves,
                                                              const typename Vec4<T>::type *__restrict__ pts,
                                                              const T *__restrict__ frc, const T *__restrict__ surf,
                                                              int npt, const T *__restrict__ dn_dens,
                                                              const T *__restrict__ up_dens, double4 *__restrict__ res) {
    __shared__ T sx[kLeafThreads], sy[kLeafThreads], sz[kLeafThreads], sfx[kLeafThreads], sfy[kLeafThreads],
        sfz[kLeafThreads];
    const int b = leaves[blockIdx.x];
    const int lb = C.lvl[b], n = C.cnt[b], f = C.first[b];
    const T hb = box_half<T>(lb);
    const uint32_t w0 = C.w_ptr[b], u0 = C.u_ptr[b];
    const int nw = (int)(C.w_ptr[b + 1] - w0), nu = (int)(C.u_ptr[b + 1] - u0);
    for (int t0 = 0; t0 < n; t0 += kLeafThreads) {
        const int i = t0 + threadIdx.x;
        const bool valid = i < n;
        T x = 0, y = 0, z = 0;
        if (valid) {
            const auto v = pts[f + i];
            x = v.x, y = v.y, z = v.z;
        }
        double vx = 0, vy = 0, vz = 0;
        auto add = [&](T rx, T ry, T rz, T fx, T fy, T fz) {
            T ux = 0, uy = 0, uz = 0;
            stokes_acc<T>(rx, ry, rz, fx, fy, fz, ux, uy, uz);
            vx += (double)ux, vy += (double)uy, vz += (double)uz;
        };
        if (valid) {
            const T a = (T)kAlphaOuter * hb;
            for (int k = 0; k < npt; ++k) {
                const T *w = dn_dens + (size_t)b * 3 * npt + 3 * k;
                add(x - a * surf[3 * k], y - a * surf[3 * k + 1], z - a * surf[3 * k + 2], w[0] * hb, w[1] * hb,
                    w[2] * hb);
            }
            for (int e = 0; e < nw; ++e) {
                const int a_ = C.w_idx[w0 + e], la = C.lvl[a_];
                const T ha = box_half<T>(la), al = (T)kAlphaInner * ha;
                const T ox = centre_diff<T>(C.cx[a_], la, C.cx[b], lb), oy = centre_diff<T>(C.cy[a_], la, C.cy[b], lb),
                        oz = centre_diff<T>(C.cz[a_], la, C.cz[b], lb);
                for (int k = 0; k < npt; ++k) {
                    const T *w = up_dens + (size_t)a_ * 3 * npt + 3 * k;
                    add(x - (ox + al * surf[3 * k]), y - (oy + al * surf[3 * k + 1]), z - (oz + al * surf[3 * k + 2]),
                        w[0] * ha, w[1] * ha, w[2] * ha);
                }
            }
        }
        for (int e = 0; e < nu; ++e) {
            const int a_ = C.u_idx[u0 + e], la = C.lvl[a_];
            const T ox = centre_diff<T>(C.cx[a_], la, C.cx[b], lb), oy = centre_diff<T>(C.cy[a_], la, C.cy[b], lb),
                    oz = centre_diff<T>(C.cz[a_], la, C.cz[b], lb);
            const int na = C.cnt[a_], fa = C.first[a_];
            for (int c0 = 0; c0 < na; c0 += kLeafThreads) {
                __syncthreads();
                if (c0 + threadIdx.x < na) {
                    const int j = fa + c0 + threadIdx.x;
                    const auto v = pts[j];
                    sx[threadIdx.x] = ox + v.x, sy[threadIdx.x] = oy + v.y, sz[threadIdx.x] = oz + v.z;
                    sfx[threadIdx.x] = frc[3 * (size_t)j], sfy[threadIdx.x] = frc[3 * (size_t)j + 1],
                    sfz[threadIdx.x] = frc[3 * (size_t)j + 2];
                }
                __syncthreads();
                const int m = min(kLeafThreads, na - c0);
                if (valid)
                    for (int k = 0; k < m; ++k) {
                        const T rx = x - sx[k], ry = y - sy[k], rz = z - sz[k];
                        if (!(rx * rx + ry * ry + rz * rz > T(0))) continue;  // the particle itself, coincident points
                        add(rx, ry, rz, sfx[k], sfy[k], sfz[k]);
                    }
            }
        }
        if (valid) {
            res[f + i] = make_double4(vx, vy, vz, 0.0);
            if (!isfinite(vx + vy + vz)) set_status(C.status, KIFMM_ERR_NONFINITE);
        }
    }
}

// Velocities in the caller's order: coef / (8 pi side) times the root-unit sums.
template <typename TO>
__global__ void k_finalize_stokes(int64_t n, const double4 *__restrict__ res, const uint32_t *__restrict__ perm,
                                  const int64_t *__restrict__ off, int S, const double *__restrict__ out_scale,
                                  TO *__restrict__ vel) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= (int64_t)j) lo = mid; else hi = mid - 1;
    }
    const double c = 0.5 * out_scale[2 * lo];  // coef / (4 pi side) / 2
    const double4 r = res[i];
    vel[3 * (size_t)j] = (TO)(c * r.x);
    vel[3 * (size_t)j + 1] = (TO)(c * r.y);
    vel[3 * (size_t)j + 2] = (TO)(c * r.z);
}

template <typename T>
cudaError_t evaluate_stokes_t(Plan &P, void *vel, cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    const int ns = P.ns, npt = P.nsurf;
    const T *surf = P.f64 ? (const T *)P.surf64 : (const T *)P.surf32;
    T *u = (T *)P.u_chk, *d = (T *)P.d_chk, *tmp = (T *)P.tmp_chk;
    const V4 *pts = (const V4 *)P.pts;
    const T *frc = (const T *)P.frc;
    double4 *res = (double4 *)P.res;
    const unsigned thr = (unsigned)std::min(kLeafThreads, (npt + 31) / 32 * 32);
    stage_begin(P, KIFMM_STAGE_P2M, s);
    ++g_launches, k_p2m_stokes<T><<<(unsigned)P.n_leaves, thr, 0, s>>>(P.leaves, P.lvl, P.first, P.cnt, pts, frc,
                                                                       surf, npt, u);
    stage_end(P, KIFMM_STAGE_P2M, s);
    stage_begin(P, KIFMM_STAGE_M2M, s);
    for (int l = P.max_level - 1; l >= 0; --l)
        ggemm<T>(P, GatherChild<T>{P.child8, (const T *)P.m2m_t, ns}, P.part_list[1],
                 P.part_start[1][1 + l], P.part_start[1][2 + l], 8, u, u, 0, s);
    stage_end(P, KIFMM_STAGE_M2M, s);
    stage_begin(P, KIFMM_STAGE_M2L, s);
    KIFMM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(T) * (size_t)P.nb * ns, s));
    ggemm_classes<T>(P, GatherM2L<T>{P.vdense, P.slot_off, (const T *)P.m2l_t, ns, P.op_ld}, P.part_list[0],
                     P.part_start[0].data(), 8, kVSlots, u, d, 0, s, P.op_ld, nullptr);
    stage_end(P, KIFMM_STAGE_M2L, s);
    if (P.n_x > 0) {
        stage_begin(P, KIFMM_STAGE_P2L, s);
        ++g_launches, k_p2l_stokes<T><<<(unsigned)P.nb, thr, 0, s>>>(P.nx, P.xdense, P.lvl, P.cx, P.cy, P.cz,
                                                                       P.first, P.cnt, pts, frc, surf, npt, d);
        stage_end(P, KIFMM_STAGE_P2L, s);
    }
    stage_begin(P, KIFMM_STAGE_L2L, s);
    for (int l = 1; l <= P.max_level; ++l)
        ggemm_classes<T>(P, GatherParent<T>{P.parent, (const T *)P.l2l_t, ns, P.op_ld}, P.part_list[3],
                         P.part_start[3].data() + 8 * l, 8, 1, d, d, 1, s, P.op_ld, nullptr);
    stage_end(P, KIFMM_STAGE_L2L, s);
    KIFMM_CUDA_TRY(cudaGetLastError());
    stage_begin(P, KIFMM_STAGE_LEAF, s);
    if (P.n_w > 0) {
        ggemm<T>(P, GatherSelf<T>{(const T *)P.up_w_t}, P.part_list[2], 0, P.part_start[2][1], 1, u, tmp, 0, s);
        ggemm<T>(P, GatherSelf<T>{(const T *)P.up_v_t}, P.part_list[2], 0, P.part_start[2][1], 1, tmp,
                 (T *)P.up_dens, 0, s);
    }
    ggemm<T>(P, GatherSelf<T>{(const T *)P.dn_w_t}, P.leaves, 0, P.n_leaves, 1, d, tmp, 0, s);
    ggemm<T>(P, GatherSelf<T>{(const T *)P.dn_v_t}, P.leaves, 0, P.n_leaves, 1, tmp, (T *)P.dn_dens, 0, s);
    stage_end(P, KIFMM_STAGE_LEAF, s);
    stage_begin(P, KIFMM_STAGE_P2P, s);
    LeafCtx C{P.lvl, P.cx, P.cy, P.cz, P.first, P.cnt, P.u_ptr, P.w_ptr, P.u_idx, P.w_idx, ns, nullptr,
              P.leaf_tile, P.status, nullptr, nullptr};
    ++g_launches, k_leaf_stokes<T><<<(unsigned)P.n_leaves, kLeafThreads, 0, s>>>(
                      C, P.leaves, pts, frc, surf, npt, (const T *)P.dn_dens, (const T *)P.up_dens, res);
    stage_end(P, KIFMM_STAGE_P2P, s);
    stage_begin(P, KIFMM_STAGE_OUT, s);
    if (vel) {
        if (P.io_f64)
            ++g_launches, k_finalize_stokes<double><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, res, P.perm, P.sys_off_d, P.n_sys, P.out_scale, (double *)vel);
        else
            ++g_launches, k_finalize_stokes<float><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, res, P.perm, P.sys_off_d, P.n_sys, P.out_scale, (float *)vel);
    }
    stage_end(P, KIFMM_STAGE_OUT, s);
    P.fwd_valid = P.fwd_res_valid = true;
    return cudaGetLastError();
}


// Weights of a loss on the gradient, in sorted order and root units: the
// caller's dL/dgrad divided by the side of the particle's system (the
// gradient in caller units is the root-unit gradient over the side).
template <typename TI, typename T>
__global__ void k_gather_g(int64_t n, const uint32_t *__restrict__ perm, const int64_t *__restrict__ off, int S,
                           const double *__restrict__ lo_side, const TI *__restrict__ g, T *__restrict__ gs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= (int64_t)j) lo = mid; else hi = mid - 1;
    }
    const double side = lo_side[4 * lo + 3];
#pragma unroll
    for (int d = 0; d < 3; ++d) gs[3 * i + d] = (T)((double)g[3 * j + d] / side);
}

// The leaf-level terms of a loss on the gradient, one block per leaf b (its
// targets in chunks of the block), root units, FP64 sums:
//  hg[i]  = H_i g_i, the Hessian of the forward field at particle i applied
//           to its own dipole (the gradient's dependence on the particle's
//           position), from b's forward sources: its downward equivalent
//           density on the 2.95 h_b surface, the upward densities of its W
//           boxes on their 1.05 h_a surfaces, and the U-list particles;
//  pd[i]  = (psi, grad psi) at particle i of the dipoles g_j of the U-list
//           particles j != i (the near field of the transposed gradient).
// With H = grad grad (1/r), r = x_i - y:  H g = (3 (r.g) r - r^2 g) / r^5;
// a dipole g at y gives psi(x) = g . r / r^3, grad psi = g / r^3 - 3 (g.r) r / r^5.
template <typename T>
__global__ void __launch_bounds__(kLeafThreads) k_adj_leaf(LeafCtx C, const int32_t *__restrict__ leaves,
                                                           const typename Vec4<T>::type *__restrict__ pts,
                                                           const T *__restrict__ surf, const T *__restrict__ dn_dens,
                                                           const T *__restrict__ up_dens, const T *__restrict__ gs,
                                                           double4 *__restrict__ hg, double4 *__restrict__ pd) {
    __shared__ T sx[kLeafThreads], sy[kLeafThreads], sz[kLeafThreads], sq[kLeafThreads];
    __shared__ T sgx[kLeafThreads], sgy[kLeafThreads], sgz[kLeafThreads];
    const int b = leaves[blockIdx.x];
    const int lb = C.lvl[b], n = C.cnt[b], f = C.first[b], ns = C.ns;
    const T hb = box_half<T>(lb);
    const uint32_t w0 = C.w_ptr[b], u0 = C.u_ptr[b];
    const int nw = (int)(C.w_ptr[b + 1] - w0), nu = (int)(C.u_ptr[b + 1] - u0);
    for (int t0 = 0; t0 < n; t0 += kLeafThreads) {
        const int i = t0 + threadIdx.x;
        const bool valid = i < n;
        T x = 0, y = 0, z = 0, g0 = 0, g1 = 0, g2 = 0;
        if (valid) {
            const auto v = pts[f + i];
            x = v.x, y = v.y, z = v.z;
            g0 = gs[3 * (size_t)(f + i)], g1 = gs[3 * (size_t)(f + i) + 1], g2 = gs[3 * (size_t)(f + i) + 2];
        }
        double h0 = 0, h1 = 0, h2 = 0, p0 = 0, p1 = 0, p2 = 0, p3 = 0;
        // Hessian of one monopole w at offset (rx, ry, rz) = x_i - y, applied to g
        auto hess = [&](T rx, T ry, T rz, T w) {
            const T r2 = rx * rx + ry * ry + rz * rz;
            const T ri = rsqrt_t<T>(r2), ri2 = ri * ri, ri3 = ri * ri2;
            const T rg3 = T(3) * (rx * g0 + ry * g1 + rz * g2) * ri2;
            h0 += (double)(w * ri3 * (rg3 * rx - g0));
            h1 += (double)(w * ri3 * (rg3 * ry - g1));
            h2 += (double)(w * ri3 * (rg3 * rz - g2));
        };
        if (valid) {
            // own downward equivalent surface (weights dn_dens h_b)
            const T a = (T)kAlphaOuter * hb;
            for (int k = 0; k < ns; ++k)
                hess(x - a * surf[3 * k], y - a * surf[3 * k + 1], z - a * surf[3 * k + 2],
                     dn_dens[(size_t)b * ns + k] * hb);
            // W boxes' upward equivalent surfaces (weights up_dens h_a)
            for (int e = 0; e < nw; ++e) {
                const int a_ = C.w_idx[w0 + e], la = C.lvl[a_];
                const T ha = box_half<T>(la), al = (T)kAlphaInner * ha;
                const T ox = centre_diff<T>(C.cx[a_], la, C.cx[b], lb), oy = centre_diff<T>(C.cy[a_], la, C.cy[b], lb),
                        oz = centre_diff<T>(C.cz[a_], la, C.cz[b], lb);
                for (int k = 0; k < ns; ++k)
                    hess(x - (ox + al * surf[3 * k]), y - (oy + al * surf[3 * k + 1]), z - (oz + al * surf[3 * k + 2]),
                         up_dens[(size_t)a_ * ns + k] * ha);
            }
        }
        // U-list particles, staged through shared memory
        for (int e = 0; e < nu; ++e) {
            const int a_ = C.u_idx[u0 + e], la = C.lvl[a_];
            const T ox = centre_diff<T>(C.cx[a_], la, C.cx[b], lb), oy = centre_diff<T>(C.cy[a_], la, C.cy[b], lb),
                    oz = centre_diff<T>(C.cz[a_], la, C.cz[b], lb);
            const int na = C.cnt[a_], fa = C.first[a_];
            for (int c0 = 0; c0 < na; c0 += kLeafThreads) {
                __syncthreads();
                if (c0 + threadIdx.x < na) {
                    const int j = fa + c0 + threadIdx.x;
                    const auto v = pts[j];
                    sx[threadIdx.x] = ox + v.x;
                    sy[threadIdx.x] = oy + v.y;
                    sz[threadIdx.x] = oz + v.z;
                    sq[threadIdx.x] = v.w;
                    sgx[threadIdx.x] = gs[3 * (size_t)j];
                    sgy[threadIdx.x] = gs[3 * (size_t)j + 1];
                    sgz[threadIdx.x] = gs[3 * (size_t)j + 2];
                }
                __syncthreads();
                const int m = min(kLeafThreads, na - c0);
                if (valid) {
                    for (int k = 0; k < m; ++k) {
                        const T rx = x - sx[k], ry = y - sy[k], rz = z - sz[k];
                        const T r2 = rx * rx + ry * ry + rz * rz;
                        if (!(r2 > T(0))) continue;  // the particle itself and coincident points
                        hess(rx, ry, rz, sq[k]);
                        const T ri = rsqrt_t<T>(r2), ri2 = ri * ri, ri3 = ri * ri2;
                        const T gr = sgx[k] * rx + sgy[k] * ry + sgz[k] * rz;
                        const T gr3 = T(3) * gr * ri2;
                        p0 += (double)(gr * ri3);
                        p1 += (double)(ri3 * (sgx[k] - gr3 * rx));
                        p2 += (double)(ri3 * (sgy[k] - gr3 * ry));
                        p3 += (double)(ri3 * (sgz[k] - gr3 * rz));
                    }
                }
            }
        }
        if (valid) {
            hg[f + i] = make_double4(h0, h1, h2, 0.0);
            pd[f + i] = make_double4(p0, p1, p2, p3);
        }
    }
}

// Transposed passes with the tree frozen: psi = A^T w (Sec. 2.2 operators,
// transposed in reverse order), then the adjoint outputs.
template <typename T>
cudaError_t backward_t(Plan &P, const void *w_user, const void *g_user, const double *dLdU, const void *grad_user,
                       void *dq, void *dx, cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    const int ns = P.ns;
    const size_t nn = (size_t)ns * ns;
    const T *surf = P.f64 ? (const T *)P.surf64 : (const T *)P.surf32;
    T *ub = (T *)P.u_chk, *db = (T *)P.d_chk, *tmp = (T *)P.tmp_chk;
    // scratch of their own: the forward's equivalent densities stay intact
    // (the Hessian term reads them, and a second backward may follow)
    T *e1 = (T *)P.adj_e1, *e2 = (T *)P.adj_e2, *ws = (T *)P.w_sorted;
    T *gs = g_user ? (T *)P.g_sorted : nullptr;
    const T *adjp = (const T *)P.adj_pinv;
    const V4 *pts = (const V4 *)P.pts;
    double4 *res = (double4 *)P.res;
    double4 *hg = g_user ? (double4 *)P.adj_hg : nullptr, *pd = g_user ? (double4 *)P.adj_pd : nullptr;
    double *fwd_pot = dLdU ? P.adj_pot : nullptr;
    if (P.io_f64)
        ++g_launches, k_adj_weights<double, T><<<grid_for(P.n, 256), 256, 0, s>>>(
                          P.n, P.perm, P.sys_off_d, P.n_sys, pts, (const double *)w_user, dLdU, res, ws, fwd_pot);
    else
        ++g_launches, k_adj_weights<float, T><<<grid_for(P.n, 256), 256, 0, s>>>(
                          P.n, P.perm, P.sys_off_d, P.n_sys, pts, (const float *)w_user, dLdU, res, ws, fwd_pot);
    LeafCtx C{P.lvl, P.cx, P.cy, P.cz, P.first, P.cnt, P.u_ptr, P.w_ptr, P.u_idx, P.w_idx, ns, nullptr,
              P.leaf_tile, P.status, nullptr, nullptr};
    if (g_user) {
        if (P.io_f64)
            ++g_launches, k_gather_g<double, T><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, P.perm, P.sys_off_d, P.n_sys, P.lo_side, (const double *)g_user, gs);
        else
            ++g_launches, k_gather_g<float, T><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, P.perm, P.sys_off_d, P.n_sys, P.lo_side, (const float *)g_user, gs);
        // the forward field's Hessian term and the dipoles' near field (reads
        // the last evaluate's equivalent densities)
        ++g_launches, k_adj_leaf<T><<<(unsigned)P.n_leaves, kLeafThreads, 0, s>>>(
                          C, P.leaves, pts, surf, (const T *)P.dn_dens, (const T *)P.up_dens, gs, hg, pd);
    }
    // L2P^T: h * sum w / |DE - x| (+ the dipoles) at each leaf, then d-bar = W_dn^T V_dn^T (.)
    KIFMM_CUDA_TRY(cudaMemsetAsync(db, 0, sizeof(T) * (size_t)P.nb * ns, s));
    KIFMM_CUDA_TRY(cudaMemsetAsync(ub, 0, sizeof(T) * (size_t)P.nb * ns, s));
    ++g_launches, k_p2m<T><<<(unsigned)P.n_leaves, p2m_threads(P), p2m_smem<T>(P), s>>>(P.leaves, P.lvl, P.first, P.cnt, pts, surf,
                                                                        ns, e1, ws, 1, gs);
    ggemm<T>(P, GatherSelf<T>{adjp + 3 * nn}, P.leaves, 0, P.n_leaves, 1, e1, tmp, 0, s);
    ggemm<T>(P, GatherSelf<T>{adjp + 2 * nn}, P.leaves, 0, P.n_leaves, 1, tmp, db, 0, s);
    // M2P^T: W-list sources a receive h_a * sum w / |UE_a - x| (+ dipoles) from the leaves of X(a)
    if (P.n_x > 0) {
        KIFMM_CUDA_TRY(cudaMemsetAsync(e2, 0, sizeof(T) * (size_t)P.nb * ns, s));
        ++g_launches, k_p2l<T><<<(unsigned)P.nb, kLeafThreads, 0, s>>>(P.nx, P.xdense, P.lvl, P.cx, P.cy, P.cz,
                                                                        P.first, P.cnt, pts, surf, ns, e2, ws, 1,
                                                                        nullptr, gs);
        ggemm<T>(P, GatherSelf<T>{adjp + 1 * nn}, P.part_list[2], 0, P.part_start[2][1], 1, e2, tmp, 0, s);
        ggemm<T>(P, GatherSelf<T>{adjp}, P.part_list[2], 0, P.part_start[2][1], 1, tmp, ub, 0, s);
    }
    // L2L^T, bottom-up
    for (int l = P.max_level - 1; l >= 0; --l)
        ggemm<T>(P, GatherChild<T>{P.child8, (const T *)P.adj_l2l, ns}, P.part_list[1], P.part_start[1][1 + l],
                 P.part_start[1][2 + l], 8, db, db, 1, s);
    // M2L^T (V lists are symmetric; operator at the negated offset, transposed)
    ggemm_classes<T>(P, GatherM2L<T>{P.vdense, P.slot_off, (const T *)P.adj_m2l, ns, ns}, P.part_list[0],
                     P.part_start[0].data(), 8, kVSlots, db, ub, 1, s);
    // M2M^T, top-down
    for (int l = 1; l <= P.max_level; ++l)
        ggemm_classes<T>(P, GatherParent<T>{P.parent, (const T *)P.adj_m2m, ns, ns}, P.part_list[3],
                         P.part_start[3].data() + 8 * l, 8, 1, ub, ub, 1, s);
    // P2M^T (own UC surface, u-bar), P2L^T (W boxes' DC surfaces, d-bar), P2P^T (weights w)
    const LeafW<T> W{ub, 0, db, 0, ws};
    leaf_launch<T>(P, C, pts, surf, W, res, s);
    if (P.io_f64)
        ++g_launches, k_finalize_adj<double, T><<<grid_for(P.n, 256), 256, 0, s>>>(
                          P.n, res, P.perm, P.sys_off_d, P.n_sys, P.out_scale, pts, (const double *)w_user, dLdU,
                          fwd_pot, hg, pd, (const double *)grad_user, (double *)dq, (double *)dx);
    else
        ++g_launches, k_finalize_adj<float, T><<<grid_for(P.n, 256), 256, 0, s>>>(
                          P.n, res, P.perm, P.sys_off_d, P.n_sys, P.out_scale, pts, (const float *)w_user, dLdU,
                          fwd_pot, hg, pd, (const float *)grad_user, (float *)dq, (float *)dx);
    P.fwd_res_valid = false;  // res now holds the adjoint field
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_backward(Plan &P, const void *w, const void *g, const double *dLdU, const void *grad, void *dq,
                         void *dx, cudaStream_t s) {
    return P.f64 ? backward_t<double>(P, w, g, dLdU, grad, dq, dx, s)
                 : backward_t<float>(P, w, g, dLdU, grad, dq, dx, s);
}

cudaError_t run_evaluate(Plan &P, void *pot, void *grad, double *energy, cudaStream_t s) {
    if (P.stokes) return P.f64 ? evaluate_stokes_t<double>(P, pot, s) : evaluate_stokes_t<float>(P, pot, s);
    return P.f64 ? evaluate_t<double>(P, pot, grad, energy, s) : evaluate_t<float>(P, pot, grad, energy, s);
}

cudaError_t run_clump_reduce(Plan &P, int64_t n_clumps, const int64_t *offs, const void *xyz, const void *q,
                             const void *grad, const void *ref, void *force, void *torque, cudaStream_t s) {
    if (n_clumps == 0) return cudaSuccess;
    if (P.io_f64)
        ++g_launches, k_clump<double><<<grid_for(n_clumps, 128), 128, 0, s>>>(n_clumps, offs, (const double *)xyz, (const double *)q,
                                                               (const double *)grad, (const double *)ref,
                                                               (double *)force, (double *)torque);
    else
        ++g_launches, k_clump<float><<<grid_for(n_clumps, 128), 128, 0, s>>>(n_clumps, offs, (const float *)xyz, (const float *)q,
                                                              (const float *)grad, (const float *)ref,
                                                              (float *)force, (float *)torque);
    return cudaGetLastError();
}

}  // namespace kifmm
