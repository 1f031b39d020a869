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

template <typename T>
__device__ __forceinline__ T box_half(int level) {
    return (T)ldexp(1.0, -(level + 1));
}
template <typename T>
__device__ __forceinline__ T box_center(int c, int level) {
    return (T)(ldexp((double)(2 * c + 1), -(level + 1)));
}

template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
    s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// P2M: u(b)_j = (1/h) sum_i q_i / |2.95 S_j - (x_i - c_b)/h|
template <typename T>
__global__ void k_p2m(const int32_t *__restrict__ leaves, const int32_t *__restrict__ lvl,
                      const int32_t *__restrict__ first, const int32_t *__restrict__ cnt,
                      const typename Vec4<T>::type *__restrict__ pts, const T *__restrict__ surf, int ns,
                      T *__restrict__ u) {
    __shared__ T sx[kLeafThreads], sy[kLeafThreads], sz[kLeafThreads], sq[kLeafThreads];
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
        for (int c0 = 0; c0 < n; c0 += kLeafThreads) {
            __syncthreads();
            if (c0 + threadIdx.x < n) {
                const auto v = pts[f + c0 + threadIdx.x];
                sx[threadIdx.x] = v.x * hinv;
                sy[threadIdx.x] = v.y * hinv;
                sz[threadIdx.x] = v.z * hinv;
                sq[threadIdx.x] = v.w;
            }
            __syncthreads();
            const int m = min(kLeafThreads, n - c0);
            for (int i = 0; i < m; ++i) acc += sq[i] * lap_pot<T>(px - sx[i], py - sy[i], pz - sz[i]);
        }
        if (j < ns) u[(size_t)b * ns + j] = acc * hinv;
    }
}

// M2M for the non-leaf boxes of one level: u(b) = sum_c A_{oct(c)} u(c).
template <typename T>
__global__ void k_m2m(int64_t ls, const int32_t *__restrict__ child_first, const int32_t *__restrict__ nchild,
                      const int32_t *__restrict__ cx, const int32_t *__restrict__ cy, const int32_t *__restrict__ cz,
                      const T *__restrict__ m2m_t, int ns, T *__restrict__ u) {
    extern __shared__ unsigned char smem_raw[];
    T *uc = reinterpret_cast<T *>(smem_raw);
    const int64_t b = ls + blockIdx.x;
    if (nchild[b] == 0) return;
    T acc[4] = {0, 0, 0, 0};
    for (int c = child_first[b]; c < child_first[b] + nchild[b]; ++c) {
        const int o = 4 * (cx[c] & 1) + 2 * (cy[c] & 1) + (cz[c] & 1);
        __syncthreads();
        for (int k = threadIdx.x; k < ns; k += blockDim.x) uc[k] = u[(size_t)c * ns + k];
        __syncthreads();
        const T *A = m2m_t + (size_t)o * ns * ns;
        for (int r = 0; r < 4; ++r) {
            const int j = threadIdx.x + r * blockDim.x;
            if (j >= ns) continue;
            T s = 0;
            for (int k = 0; k < ns; ++k) s += A[(size_t)k * ns + j] * uc[k];
            acc[r] += s;
        }
    }
    for (int r = 0; r < 4; ++r) {
        const int j = threadIdx.x + r * blockDim.x;
        if (j < ns) u[(size_t)b * ns + j] = acc[r];
    }
}

// M2L on SIMT cores: a block owns 64 targets of one octant class and all
// check points (padded to 160); for each of the class's 189 slots it gathers
// the 64 source rows and multiplies by the slot's operator.
constexpr int kM2LT = 64;   // targets per block
constexpr int kM2LJ = 160;  // padded outputs
constexpr int kM2LK = 8;    // k chunk

template <typename T>
__global__ void __launch_bounds__(256) k_m2l_simt(const int32_t *__restrict__ targets, int64_t t_begin,
                                                  int64_t t_end, int cls, const int32_t *__restrict__ vdense,
                                                  const int *__restrict__ slot_off, const T *__restrict__ m2l_t,
                                                  int ns, const T *__restrict__ u, T *__restrict__ d) {
    __shared__ T Us[kM2LK][kM2LT];
    __shared__ T Ms[kM2LK][kM2LJ];
    __shared__ int32_t tgt[kM2LT];
    __shared__ int32_t src[kM2LT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t t0 = t_begin + (int64_t)blockIdx.x * kM2LT;
    if (threadIdx.x < kM2LT) tgt[threadIdx.x] = (t0 + threadIdx.x < t_end) ? targets[t0 + threadIdx.x] : -1;
    T acc[4][10];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 10; ++c) acc[a][c] = 0;
    __syncthreads();
    for (int s = 0; s < kVSlots; ++s) {
        if (threadIdx.x < kM2LT) {
            const int32_t t = tgt[threadIdx.x];
            src[threadIdx.x] = (t >= 0) ? vdense[(size_t)t * kVSlots + s] : -1;
        }
        const T *M = m2l_t + (size_t)slot_off[cls * kVSlots + s] * ns * ns;
        __syncthreads();
        for (int k0 = 0; k0 < ns; k0 += kM2LK) {
            // gather: 64 targets x 8 k values, k-contiguous per target
            for (int e = threadIdx.x; e < kM2LT * kM2LK; e += 256) {
                const int t = e / kM2LK, k = e % kM2LK;
                const int32_t sb = src[t];
                Us[k][t] = (sb >= 0 && k0 + k < ns) ? u[(size_t)sb * ns + k0 + k] : T(0);
            }
            for (int e = threadIdx.x; e < kM2LK * kM2LJ; e += 256) {
                const int k = e / kM2LJ, j = e % kM2LJ;
                Ms[k][j] = (k0 + k < ns && j < ns) ? M[(size_t)(k0 + k) * ns + j] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kM2LK; ++k) {
                T uv[4], mv[10];
#pragma unroll
                for (int a = 0; a < 4; ++a) uv[a] = Us[k][ty + 16 * a];
#pragma unroll
                for (int c = 0; c < 10; ++c) mv[c] = Ms[k][tx + 16 * c];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 10; ++c) acc[a][c] += uv[a] * mv[c];
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int32_t t = tgt[ty + 16 * a];
        if (t < 0) continue;
#pragma unroll
        for (int c = 0; c < 10; ++c) {
            const int j = tx + 16 * c;
            if (j < ns) d[(size_t)t * ns + j] = acc[a][c];
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
                      T *__restrict__ d) {
    __shared__ T sx[kLeafThreads], sy[kLeafThreads], sz[kLeafThreads], sq[kLeafThreads];
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
            const T ox = box_center<T>(cx[a], la) - cbx, oy = box_center<T>(cy[a], la) - cby,
                    oz = box_center<T>(cz[a], la) - cbz;
            const int n = cnt[a], f = first[a];
            for (int c0 = 0; c0 < n; c0 += kLeafThreads) {
                __syncthreads();
                if (c0 + threadIdx.x < n) {
                    const auto v = pts[f + c0 + threadIdx.x];
                    sx[threadIdx.x] = (ox + v.x) * hinv;
                    sy[threadIdx.x] = (oy + v.y) * hinv;
                    sz[threadIdx.x] = (oz + v.z) * hinv;
                    sq[threadIdx.x] = v.w;
                }
                __syncthreads();
                const int m = min(kLeafThreads, n - c0);
                for (int i = 0; i < m; ++i) acc += sq[i] * lap_pot<T>(px - sx[i], py - sy[i], pz - sz[i]);
            }
        }
        if (j < ns) d[(size_t)b * ns + j] += acc * hinv;
    }
}

// L2L for one level: d(b) += C_{oct(b)} d(parent(b)).
template <typename T>
__global__ void k_l2l(int64_t ls, const int32_t *__restrict__ parent, const int32_t *__restrict__ cx,
                      const int32_t *__restrict__ cy, const int32_t *__restrict__ cz,
                      const T *__restrict__ l2l_t, int ns, T *__restrict__ d) {
    extern __shared__ unsigned char smem_raw[];
    T *dp = reinterpret_cast<T *>(smem_raw);
    const int64_t b = ls + blockIdx.x;
    const int32_t p = parent[b];
    const int o = 4 * (cx[b] & 1) + 2 * (cy[b] & 1) + (cz[b] & 1);
    for (int k = threadIdx.x; k < ns; k += blockDim.x) dp[k] = d[(size_t)p * ns + k];
    __syncthreads();
    const T *C = l2l_t + (size_t)o * ns * ns;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        T s = 0;
        for (int k = 0; k < ns; ++k) s += C[(size_t)k * ns + j] * dp[k];
        d[(size_t)b * ns + j] += s;
    }
}

// dens = V (W chk): the two-step pseudo-inverse, normalised to a unit box.
template <typename T>
__device__ void pinv_apply(const T *__restrict__ w_t, const T *__restrict__ v_t, int ns, const T *chk, T *tmp,
                           T *dens) {
    for (int m = threadIdx.x; m < ns; m += blockDim.x) {
        T s = 0;
        for (int j = 0; j < ns; ++j) s += w_t[(size_t)j * ns + m] * chk[j];
        tmp[m] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        T s = 0;
        for (int m = 0; m < ns; ++m) s += v_t[(size_t)m * ns + k] * tmp[m];
        dens[k] = s;
    }
    __syncthreads();
}

template <typename T>
__global__ void k_up_dens(int64_t nb, const int32_t *__restrict__ flag, const T *__restrict__ w_t,
                          const T *__restrict__ v_t, int ns, const T *__restrict__ u, T *__restrict__ dens) {
    extern __shared__ unsigned char smem_raw[];
    T *chk = reinterpret_cast<T *>(smem_raw);
    T *tmp = chk + ns;
    T *out = tmp + ns;
    const int64_t b = blockIdx.x;
    if (!flag[b]) return;
    for (int k = threadIdx.x; k < ns; k += blockDim.x) chk[k] = u[(size_t)b * ns + k];
    __syncthreads();
    pinv_apply<T>(w_t, v_t, ns, chk, tmp, out);
    for (int k = threadIdx.x; k < ns; k += blockDim.x) dens[(size_t)b * ns + k] = out[k];
}

// Leaf far field: L2P from the downward density on DE = 2.95 h S and M2P
// from the upward densities (UE = 1.05 h S) of the W-list boxes.
template <typename T>
__global__ void k_leaf_far(const int32_t *__restrict__ leaves, const int32_t *__restrict__ lvl,
                           const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                           const int32_t *__restrict__ cz, const int32_t *__restrict__ first,
                           const int32_t *__restrict__ cnt, const typename Vec4<T>::type *__restrict__ pts,
                           const T *__restrict__ surf, int ns, const T *__restrict__ dn_w_t,
                           const T *__restrict__ dn_v_t, const T *__restrict__ d,
                           const uint32_t *__restrict__ w_ptr, const int32_t *__restrict__ w_idx,
                           const T *__restrict__ up_dens, double4 *__restrict__ res) {
    extern __shared__ unsigned char smem_raw[];
    T *chk = reinterpret_cast<T *>(smem_raw);
    T *tmp = chk + ns;
    T *dens = tmp + ns;
    const int b = leaves[blockIdx.x];
    const int lb = lvl[b];
    const T h = box_half<T>(lb), hinv = T(1) / h;
    for (int k = threadIdx.x; k < ns; k += blockDim.x) chk[k] = d[(size_t)b * ns + k];
    __syncthreads();
    pinv_apply<T>(dn_w_t, dn_v_t, ns, chk, tmp, dens);
    const int n = cnt[b], f = first[b];
    const T ao = (T)kAlphaOuter, ai = (T)kAlphaInner;
    // per-thread particles (up to 4 per thread for leaves above 128)
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        T pot = 0, gx = 0, gy = 0, gz = 0;
        T X = 0, Y = 0, Z = 0;
        typename Vec4<T>::type v{};
        if (i < n) {
            v = pts[f + i];
            X = v.x * hinv;
            Y = v.y * hinv;
            Z = v.z * hinv;
            for (int k = 0; k < ns; ++k)
                lap_accum<T>(X - ao * surf[3 * k], Y - ao * surf[3 * k + 1], Z - ao * surf[3 * k + 2], dens[k],
                             pot, gx, gy, gz);
            gx *= hinv;
            gy *= hinv;
            gz *= hinv;
        }
        // M2P
        for (uint32_t e = w_ptr[b]; e < w_ptr[b + 1]; ++e) {
            const int a = w_idx[e];
            const int la = lvl[a];
            const T ha = box_half<T>(la), hainv = T(1) / ha;
            __syncthreads();
            for (int k = threadIdx.x; k < ns; k += blockDim.x) tmp[k] = up_dens[(size_t)a * ns + k];
            __syncthreads();
            if (i < n) {
                const T ox = box_center<T>(cx[b], lb) - box_center<T>(cx[a], la);
                const T oy = box_center<T>(cy[b], lb) - box_center<T>(cy[a], la);
                const T oz = box_center<T>(cz[b], lb) - box_center<T>(cz[a], la);
                const T Xa = (ox + v.x) * hainv, Ya = (oy + v.y) * hainv, Za = (oz + v.z) * hainv;
                T p2 = 0, g2x = 0, g2y = 0, g2z = 0;
                for (int k = 0; k < ns; ++k)
                    lap_accum<T>(Xa - ai * surf[3 * k], Ya - ai * surf[3 * k + 1], Za - ai * surf[3 * k + 2], tmp[k],
                                 p2, g2x, g2y, g2z);
                pot += p2;
                gx += g2x * hainv;
                gy += g2y * hainv;
                gz += g2z * hainv;
            }
        }
        if (i < n) res[f + i] = make_double4((double)pot, (double)gx, (double)gy, (double)gz);
    }
}

// P2P over the U list; each source leaf's contribution is summed plainly and
// added to the running totals with a compensated (two-sum) update.
template <typename T>
__global__ void k_p2p(const int32_t *__restrict__ leaves, const int32_t *__restrict__ lvl,
                      const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                      const int32_t *__restrict__ cz, const int32_t *__restrict__ first,
                      const int32_t *__restrict__ cnt, const typename Vec4<T>::type *__restrict__ pts,
                      const uint32_t *__restrict__ u_ptr, const int32_t *__restrict__ u_idx,
                      double4 *__restrict__ res) {
    __shared__ T sx[kLeafThreads], sy[kLeafThreads], sz[kLeafThreads], sq[kLeafThreads];
    const int b = leaves[blockIdx.x];
    const int lb = lvl[b];
    const T cbx = box_center<T>(cx[b], lb), cby = box_center<T>(cy[b], lb), cbz = box_center<T>(cz[b], lb);
    const int n = cnt[b], f = first[b];
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        typename Vec4<T>::type v{};
        if (i < n) v = pts[f + i];
        T acc[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
        for (uint32_t e = u_ptr[b]; e < u_ptr[b + 1]; ++e) {
            const int a = u_idx[e];
            const int la = lvl[a];
            const T ox = box_center<T>(cx[a], la) - cbx, oy = box_center<T>(cy[a], la) - cby,
                    oz = box_center<T>(cz[a], la) - cbz;
            const int na = cnt[a], fa = first[a];
            for (int c0 = 0; c0 < na; c0 += kLeafThreads) {
                __syncthreads();
                if (c0 + threadIdx.x < na) {
                    const auto w = pts[fa + c0 + threadIdx.x];
                    sx[threadIdx.x] = ox + w.x;
                    sy[threadIdx.x] = oy + w.y;
                    sz[threadIdx.x] = oz + w.z;
                    sq[threadIdx.x] = w.w;
                }
                __syncthreads();
                if (i < n) {
                    const int m = min(kLeafThreads, na - c0);
                    T p = 0, gx = 0, gy = 0, gz = 0;
                    for (int j = 0; j < m; ++j) lap_accum<T>(v.x - sx[j], v.y - sy[j], v.z - sz[j], sq[j], p, gx, gy, gz);
                    const T part[4] = {p, gx, gy, gz};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        T s, err;
                        two_sum<T>(acc[c], part[c], s, err);
                        acc[c] = s;
                        cmp[c] += err;
                    }
                }
            }
        }
        if (i < n) {
            double4 r = res[f + i];
            r.x += (double)acc[0] + (double)cmp[0];
            r.y += (double)acc[1] + (double)cmp[1];
            r.z += (double)acc[2] + (double)cmp[2];
            r.w += (double)acc[3] + (double)cmp[3];
            res[f + i] = r;
        }
    }
}

// Scatter to caller order with 1/(4 pi), coef and physical units.
template <typename TO>
__global__ void k_finalize(int64_t n, const double4 *__restrict__ res, const uint32_t *__restrict__ perm,
                           const int64_t *__restrict__ off, int S, const double *__restrict__ lo_side, double coef,
                           TO *pot, TO *grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= (int64_t)j) lo = mid; else hi = mid - 1;
    }
    const double side = lo_side[lo * 4 + 3];
    const double c1 = coef * kInv4Pi / side, c2 = c1 / side;
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

template <typename T>
cudaError_t evaluate_t(Plan &P, void *pot, void *grad, double *energy, cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    const int ns = P.ns;
    const T *surf = P.f64 ? (const T *)P.surf64 : (const T *)P.surf32;
    T *u = (T *)P.u_chk, *d = (T *)P.d_chk;
    const V4 *pts = (const V4 *)P.pts;
    double4 *res = (double4 *)P.res;
    // upward pass
    const size_t sm1 = sizeof(T) * ns;
    stage_begin(P, KIFMM_STAGE_P2M, s);
    ++g_launches, k_p2m<T><<<(unsigned)P.n_leaves, kLeafThreads, 0, s>>>(P.leaves, P.lvl, P.first, P.cnt, pts,
                                                                        surf, ns, u);
    stage_end(P, KIFMM_STAGE_P2M, s);
    stage_begin(P, KIFMM_STAGE_M2M, s);
    for (int l = P.max_level - 1; l >= 0; --l) {
        const int64_t ls = P.level_start[l], le = P.level_start[l + 1];
        ++g_launches, k_m2m<T><<<(unsigned)(le - ls), 128, sm1, s>>>(ls, P.child_first, P.nchild, P.cx, P.cy,
                                                                      P.cz, (const T *)P.m2m_t, ns, u);
    }
    stage_end(P, KIFMM_STAGE_M2M, s);
    KIFMM_CUDA_TRY(cudaGetLastError());
    // interactions
    stage_begin(P, KIFMM_STAGE_M2L, s);
    KIFMM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(T) * (size_t)P.nb * ns, s));
    const bool tensor = (P.desc.precision == KIFMM_MIXED_TF32 || P.desc.precision == KIFMM_MIXED_FP16);
    if (tensor) {
        KIFMM_CUDA_TRY(m2l_tensor(P, s));
    } else {
        for (int c = 0; c < 8; ++c) {
            const int64_t a = P.m2l_class_start[c], e = P.m2l_class_start[c + 1];
            if (e > a)
                ++g_launches, k_m2l_simt<T><<<grid_for(e - a, kM2LT), 256, 0, s>>>(
                                  P.m2l_targets, a, e, c, P.vdense, P.slot_off, (const T *)P.m2l_t, ns, u, d);
        }
    }
    stage_end(P, KIFMM_STAGE_M2L, s);
    if (P.n_x > 0) {
        stage_begin(P, KIFMM_STAGE_P2L, s);
        ++g_launches, k_p2l<T><<<(unsigned)P.nb, kLeafThreads, 0, s>>>(P.nx, P.xdense, P.lvl, P.cx, P.cy, P.cz,
                                                                        P.first, P.cnt, pts, surf, ns, d);
        stage_end(P, KIFMM_STAGE_P2L, s);
    }
    // downward pass
    stage_begin(P, KIFMM_STAGE_L2L, s);
    for (int l = 1; l <= P.max_level; ++l) {
        const int64_t ls = P.level_start[l], le = P.level_start[l + 1];
        ++g_launches, k_l2l<T><<<(unsigned)(le - ls), 128, sm1, s>>>(ls, P.parent, P.cx, P.cy, P.cz,
                                                                      (const T *)P.l2l_t, ns, d);
    }
    stage_end(P, KIFMM_STAGE_L2L, s);
    KIFMM_CUDA_TRY(cudaGetLastError());
    // leaves
    stage_begin(P, KIFMM_STAGE_LEAF, s);
    if (P.n_w > 0)
        ++g_launches, k_up_dens<T><<<(unsigned)P.nb, 128, 3 * sm1, s>>>(P.nb, P.wsrc_flag, (const T *)P.up_w_t,
                                                                         (const T *)P.up_v_t, ns, u,
                                                                         (T *)P.up_dens);
    ++g_launches, k_leaf_far<T><<<(unsigned)P.n_leaves, kLeafThreads, 3 * sm1, s>>>(
                      P.leaves, P.lvl, P.cx, P.cy, P.cz, P.first, P.cnt, pts, surf, ns, (const T *)P.dn_w_t,
                      (const T *)P.dn_v_t, d, P.w_ptr, P.w_idx, (const T *)P.up_dens, res);
    stage_end(P, KIFMM_STAGE_LEAF, s);
    stage_begin(P, KIFMM_STAGE_P2P, s);
    ++g_launches, k_p2p<T><<<(unsigned)P.n_leaves, kLeafThreads, 0, s>>>(P.leaves, P.lvl, P.cx, P.cy, P.cz,
                                                                        P.first, P.cnt, pts, P.u_ptr, P.u_idx,
                                                                        res);
    stage_end(P, KIFMM_STAGE_P2P, s);
    KIFMM_CUDA_TRY(cudaGetLastError());
    // outputs
    stage_begin(P, KIFMM_STAGE_OUT, s);
    if (pot || grad) {
        if (P.io_f64)
            ++g_launches, k_finalize<double><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, res, P.perm, P.sys_off_d, P.n_sys, P.lo_side, P.coef, (double *)pot,
                              (double *)grad);
        else
            ++g_launches, k_finalize<float><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, res, P.perm, P.sys_off_d, P.n_sys, P.lo_side, P.coef, (float *)pot,
                              (float *)grad);
    }
    if (energy) {
        ++g_launches, k_energy_chunks<T><<<(unsigned)P.n_energy_chunks, 256, 0, s>>>(P.energy_chunks, res, pts,
                                                                                   P.energy_partial);
        ++g_launches, k_energy_sum<<<grid_for(P.n_sys, 64), 64, 0, s>>>(P.energy_chunk_start, P.energy_partial,
                                                                         P.lo_side, P.coef, P.n_sys, energy);
    }
    stage_end(P, KIFMM_STAGE_OUT, s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_evaluate(Plan &P, void *pot, void *grad, double *energy, cudaStream_t s) {
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
