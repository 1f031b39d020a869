// Tree construction on the GPU (Sec. 2.2, first step: adaptive octree with
// at most M points per leaf; third step: the interaction lists).
//
//   per-system bounding cube -> 63-bit Morton keys -> stable LSD radix sort
//   of the key digits the octree reads (8-bit digits) -> octree level by
//   level (binary search of the octant boundaries inside each split node's
//   key range) -> colleagues, coarse adjacent leaves, U/V/W/X lists.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace kifmm {

namespace {

constexpr int kBlock = 256;
constexpr int kItems = 4;
constexpr int kTile = kBlock * kItems;  // radix-sort tile

__device__ __forceinline__ unsigned long long ord_of(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double unord(unsigned long long b) {
    b = (b & 0x8000000000000000ULL) ? (b & ~0x8000000000000000ULL) : ~b;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ int find_sys(const int64_t *off, int S, int64_t i) {
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void k_bbox_init(unsigned long long *bb, int S) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S * 6) bb[i] = (i % 6 < 3) ? ~0ULL : 0ULL;
}

// Per-system min/max of the positions; non-finite inputs raise a status.
// A block takes kBboxTile particles; minima and maxima are taken in the input
// type (FP32 inputs need no FP64 arithmetic, which this GPU runs at a small
// fraction of the FP32 rate) and become ordered 64-bit words once per warp.
constexpr int kBboxTile = 1024;
template <typename T>
__global__ void k_bbox(int64_t n, const T *__restrict__ xyz, const T *__restrict__ q,
                       const int64_t *__restrict__ off, int S, unsigned long long *bb, int *status) {
    __shared__ unsigned long long red[6][kBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kBboxTile;
    if (base >= n) return;
    const int64_t end = min(n, base + (int64_t)kBboxTile);
    const int s0 = find_sys(off, S, base), s1 = find_sys(off, S, end - 1);
    const T inf = (T)INFINITY;
    T mn[3] = {inf, inf, inf}, mx[3] = {-inf, -inf, -inf};
    bool bad = false;
    for (int64_t i = base + threadIdx.x; i < end; i += kBlock) {
        T v[3];
        for (int d = 0; d < 3; ++d) v[d] = xyz[3 * i + d];
        if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2]) || (q && !isfinite(q[i]))) {
            bad = true;
            continue;
        }
        if (s0 != s1) {
            int s = find_sys(off, S, i);
            for (int d = 0; d < 3; ++d) {
                atomicMin(&bb[s * 6 + d], ord_of((double)v[d]));
                atomicMax(&bb[s * 6 + 3 + d], ord_of((double)v[d]));
            }
            continue;
        }
        for (int d = 0; d < 3; ++d) {
            mn[d] = v[d] < mn[d] ? v[d] : mn[d];
            mx[d] = v[d] > mx[d] ? v[d] : mx[d];
        }
    }
    if (bad) set_status(status, KIFMM_ERR_NONFINITE);
    if (s0 != s1) return;
    // block reduction (single system): in T within each warp, then ordered words
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            const T a = __shfl_xor_sync(0xffffffffu, mn[d], o), c = __shfl_xor_sync(0xffffffffu, mx[d], o);
            mn[d] = a < mn[d] ? a : mn[d];
            mx[d] = c > mx[d] ? c : mx[d];
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < 3; ++d) {
            red[d][threadIdx.x >> 5] = mn[d] < inf ? ord_of((double)mn[d]) : ~0ULL;
            red[3 + d][threadIdx.x >> 5] = mx[d] > -inf ? ord_of((double)mx[d]) : 0ULL;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        int k = threadIdx.x;
        unsigned long long v = red[k][0];
        for (int w = 1; w < kBlock / 32; ++w) v = (k < 3) ? min(v, red[k][w]) : max(v, red[k][w]);
        if (k < 3) atomicMin(&bb[s0 * 6 + k], v); else atomicMax(&bb[s0 * 6 + k], v);
    }
}

// Root cube per system: lo = per-axis minimum, side = largest extent (1 if 0).
__global__ void k_bbox_final(const unsigned long long *bb, int S, double *lo_side, double *key_scale, double coef,
                             double *out_scale, float *inv_side_f) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double side = 0.0;
    for (int d = 0; d < 3; ++d) {
        double lo = unord(bb[s * 6 + d]), hi = unord(bb[s * 6 + 3 + d]);
        lo_side[s * 4 + d] = lo;
        side = fmax(side, hi - lo);
    }
    side = (side > 0.0) ? side : 1.0;
    lo_side[s * 4 + 3] = side;
    key_scale[s] = __ddiv_rn(2097152.0, side);  // once per system: FP64 division is slow
    inv_side_f[s] = (float)__ddiv_rn(1.0, side);
    // output scales of the unit-root results: potential coef / (4 pi side), gradient / side^2
    const double c1 = coef * kInv4Pi / side;
    out_scale[2 * s] = c1;
    out_scale[2 * s + 1] = c1 / side;
}

// Periodic cell [0, cell)^3: a coordinate wrapped into it (identity for a
// free-space plan, cell = 0).
__device__ __forceinline__ double wrap_cell(double x, double cell) {
    return cell > 0.0 ? x - cell * floor(x / cell) : x;
}

// The root cube of a periodic plan is the cell itself.
__global__ void k_periodic_root(double cell, double *lo_side, double *key_scale, double coef, double *out_scale,
                                float *inv_side_f) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    lo_side[0] = lo_side[1] = lo_side[2] = 0.0;
    lo_side[3] = cell;
    key_scale[0] = __ddiv_rn(2097152.0, cell);
    inv_side_f[0] = (float)__ddiv_rn(1.0, cell);
    const double c1 = coef * kInv4Pi / cell;
    out_scale[0] = c1;
    out_scale[1] = c1 / cell;
}

// Neutrality of a periodic cell (Sec. 2.4: the Coulomb lattice sum converges
// only for a neutral cell): qsum[0] += sum q, qsum[1] += sum |q|.
template <typename T>
__global__ void k_charge_sums(int64_t n, const T *__restrict__ q, double *qsum) {
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)q[i];
        a += v;
        b += fabs(v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&qsum[0], a);
        atomicAdd(&qsum[1], b);
    }
}
// rtol: 1e-12 for FP64 charges; 2^-24 for FP32 ones (a neutral set rounded
// to FP32 sums to at most that fraction of sum |q|).
__global__ void k_charge_check(const double *qsum, double rtol, int *status) {
    if (threadIdx.x == 0 && !(fabs(qsum[0]) <= rtol * qsum[1])) set_status(status, KIFMM_ERR_ARG);
}

__device__ __forceinline__ uint64_t spread3(uint64_t x) {
    x &= 0x1fffffULL;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

// 21-bit quantisation in FP64 without contraction: k = min(floor((x-lo)*s), 2^21-1),
// s = 2^21 / side (key_scale, correctly rounded); bits interleaved x-highest.
template <typename T>
__global__ void k_keys(int64_t n, const T *__restrict__ xyz, const int64_t *__restrict__ off, int S,
                       const double *__restrict__ lo_side, const double *__restrict__ key_scale, uint64_t *keys,
                       uint32_t *vals, uint64_t *keys_user, double cell) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = find_sys(off, S, i);
    const double sc = key_scale[s];
    const bool wrap = cell > 0.0;
    uint64_t k[3];
    for (int d = 0; d < 3; ++d) {
        // few FP64 operations (this GPU runs FP64 at a small fraction of the
        // FP32 rate): the floor comes with the conversion to an integer and
        // the clamp is integer arithmetic; the values equal floor() then a
        // clamp in FP64
        const double x = (double)xyz[3 * i + d];
        const double t = __dmul_rn(__dsub_rn(wrap ? wrap_cell(x, cell) : x, lo_side[s * 4 + d]), sc);
        const long long f = __double2ll_rd(t);
        k[d] = (f >= 2097151LL) ? 2097151ULL : (uint64_t)(f > 0LL ? f : 0LL);
    }
    uint64_t key = (spread3(k[0]) << 2) | (spread3(k[1]) << 1) | spread3(k[2]);
    keys[i] = key;
    keys_user[i] = key;
    vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value), 8-bit digits.  Digit source: the key
// (mode 0, bits [shift, shift+8)) or the system id of the value (mode 1), used
// for the most significant passes of batched sorts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t digit_of(uint64_t key, uint32_t val, int mode, int shift,
                                             const int64_t *off, int S) {
    if (mode == 0) return (uint32_t)((key >> shift) & 0xFF);
    return (uint32_t)((find_sys(off, S, val) >> shift) & 0xFF);
}

__global__ void k_rs_hist(int64_t n, const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                          int mode, int shift, const int64_t *off, int S, uint32_t *hist, int nblk) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const int64_t end = min(n, base + (int64_t)kTile);
    for (int64_t i = base + threadIdx.x; i < end; i += kBlock)
        atomicAdd(&h[digit_of(keys[i], vals[i], mode, shift, off, S)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * nblk + blockIdx.x] = h[d];
}

// Per digit (one block each): exclusive scan over the tiles' counts of that
// digit, in place ([digit][tile] layout), and the digit's total.
__global__ void __launch_bounds__(256) k_rs_dscan(uint32_t *hist, int nblk, uint32_t *dtot) {
    __shared__ uint32_t ws[8];
    uint32_t *h = hist + (int64_t)blockIdx.x * nblk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int c0 = 0; c0 < nblk; c0 += 256) {
        const int i = c0 + threadIdx.x;
        const uint32_t v = (i < nblk) ? h[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        uint32_t wb = 0, tot = 0;
        for (int w = 0; w < 8; ++w) {
            wb += (w < warp) ? ws[w] : 0u;
            tot += ws[w];
        }
        if (i < nblk) h[i] = carry + wb + x - v;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) dtot[blockIdx.x] = carry;
}

// Scatter with ranks stable in input order: rounds of 256 consecutive items,
// warp-level peer ranking, per-warp digit counts scanned across warps.  The
// digit bases are the exclusive scan of the digit totals plus this tile's
// offset within each digit.
__global__ void k_rs_scatter(int64_t n, const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t *kout, uint32_t *vout, int mode, int shift, const int64_t *off, int S,
                             const uint32_t *__restrict__ hist_scan, const uint32_t *__restrict__ dtot, int nblk) {
    static_assert(kBlock == 256, "one thread per digit");
    __shared__ uint32_t base_d[256];
    __shared__ uint32_t wcnt[kBlock / 32][256];
    __shared__ uint32_t ws8[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        const int d = threadIdx.x;
        const uint32_t v = dtot[d];
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws8[warp] = x;
        __syncthreads();
        uint32_t wb = 0;
        for (int w = 0; w < warp; ++w) wb += ws8[w];
        base_d[d] = wb + x - v + hist_scan[(int64_t)d * nblk + blockIdx.x];
    }
    const int64_t tile0 = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        for (int i = threadIdx.x; i < (kBlock / 32) * 256; i += kBlock) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t i = tile0 + (int64_t)r * kBlock + threadIdx.x;
        const bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0ULL;
        uint32_t val = valid ? vin[i] : 0u;
        uint32_t dig = valid ? digit_of(key, val, mode, shift, off, S) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const unsigned lt = (1u << lane) - 1u;
        const int rank_w = __popc(peers & lt);
        if (valid && rank_w == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        // per digit: exclusive scan across warps, then advance the running base
        for (int d = threadIdx.x; d < 256; d += kBlock) {
            uint32_t run = base_d[d];
            for (int w = 0; w < kBlock / 32; ++w) {
                uint32_t c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
            base_d[d] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wcnt[warp][dig] + rank_w;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 (three phases, recursive over block sums).
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

__global__ void k_scan_tiles(const uint32_t *__restrict__ in, uint32_t *out, int64_t n, uint32_t *sums) {
    __shared__ uint32_t ws[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t t = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        t += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = t;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < kScanBlock / 32) ? ws[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanBlock / 32) ws[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - t + (warp > 0 ? ws[warp - 1] : 0u);
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(uint32_t *out, int64_t n, const uint32_t *__restrict__ sums_scanned) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const uint32_t add = sums_scanned[blockIdx.x];
    for (int k = threadIdx.x; k < kScanTile; k += kScanBlock)
        if (base + k < n) out[base + k] += add;
}

// ---------------------------------------------------------------------------
// Octree
// ---------------------------------------------------------------------------
__global__ void k_roots(int S, const int64_t *off, int32_t *lvl, int32_t *cx, int32_t *cy, int32_t *cz,
                        int32_t *first, int32_t *cnt, int32_t *parent, int32_t *sys) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    lvl[s] = 0;
    cx[s] = cy[s] = cz[s] = 0;
    first[s] = (int32_t)off[s];
    cnt[s] = (int32_t)(off[s + 1] - off[s]);
    parent[s] = -1;
    sys[s] = s;
}

// For each node of one level: octant ranges of its keys and the number of
// non-empty octants if it splits (count > M and level < max depth).
// One warp per node; lanes 0..7 search in parallel for the end of octant o
// (first index in the node's range whose digit exceeds o).
// Nodes [ls, le) of one level.
__global__ void k_split(int64_t ls, int64_t le, int level, int leaf_cap, int max_depth,
                        const uint64_t *__restrict__ keys, const int32_t *__restrict__ first,
                        const int32_t *__restrict__ cnt, uint32_t *nchild_tmp, int32_t *rng) {
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t b = ls + j;
    if (b >= le) return;
    const bool split = cnt[b] > leaf_cap && level < max_depth;
    int64_t end = 0;
    const int64_t lo0 = first[b], hi0 = lo0 + cnt[b];
    if (split && lane < 8) {
        const int shift = 3 * (kMaxLevel - level);
        int64_t lo = lo0, hi = hi0;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int)((keys[mid] >> shift) & 7ULL) <= lane) lo = mid + 1; else hi = mid;
        }
        end = lo;
    }
    const int64_t start = __shfl_up_sync(0xffffffffu, end, 1);
    const int64_t s0 = (lane == 0) ? lo0 : start;
    const unsigned nonempty = __ballot_sync(0xffffffffu, split && lane < 8 && end > s0);
    if (split && lane < 8) {
        rng[j * 16 + 2 * lane] = (int32_t)s0;
        rng[j * 16 + 2 * lane + 1] = (int32_t)(end - s0);
    }
    if (lane == 0) nchild_tmp[j] = split ? (uint32_t)__popc(nonempty) : 0u;
}

// The children of the nodes [ls, le) of one level, numbered from le on in
// node order (the scan of the child counts) and octant order.
__global__ void k_emit(int64_t ls, int64_t le, const uint32_t *__restrict__ nchild_tmp,
                       const uint32_t *__restrict__ nchild_scan, const int32_t *__restrict__ rng, int32_t *lvl,
                       int32_t *cx, int32_t *cy, int32_t *cz, int32_t *first, int32_t *cnt, int32_t *parent,
                       int32_t *child_first, int32_t *nchild, int32_t *sys, int64_t cap, int *status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = ls + j;
    if (b >= le) return;
    const uint32_t nc = nchild_tmp[j];
    nchild[b] = (int32_t)nc;
    if (nc == 0) {
        child_first[b] = -1;
        return;
    }
    const int64_t c0 = le + nchild_scan[j];
    child_first[b] = (int32_t)c0;
    int k = 0;
    for (int o = 0; o < 8; ++o) {
        const int32_t f = rng[j * 16 + 2 * o], c = rng[j * 16 + 2 * o + 1];
        if (c == 0) continue;
        const int64_t ch = c0 + k++;
        if (ch >= cap) {
            set_status(status, KIFMM_ERR_CAPACITY);
            return;
        }
        lvl[ch] = lvl[b] + 1;
        cx[ch] = 2 * cx[b] + ((o >> 2) & 1);
        cy[ch] = 2 * cy[b] + ((o >> 1) & 1);
        cz[ch] = 2 * cz[b] + (o & 1);
        first[ch] = f;
        cnt[ch] = c;
        parent[ch] = (int32_t)b;
        sys[ch] = sys[b];
    }
}

// ---------------------------------------------------------------------------
// Every level of the octree at once, from the sorted keys (the levels the
// last tree had).  The adaptive octree of Sec. 2.2 splits a box while it holds
// more than M points; equivalently, a box of level l >= 1 is a particle i that starts a level-l
// key prefix (or its system's range) inside a level-(l-1) key segment of more
// than M particles, with l - 1 below the maximum depth.  Segment counts only
// shrink with the level, so every ancestor of that segment splits as well:
// the box exists with no further look up the tree.  Boxes are numbered level
// by level and, within a level, in particle order: the order of the
// level-by-level build (children grouped by parent, in octant order).
// Passes: counts per (level, particle tile); one block scans them into box
// offsets and level boundaries; the emit pass writes each box's own fields;
// the link pass finds parents and child ranges by binary search over the
// first particles of the neighbouring levels.
// ---------------------------------------------------------------------------
constexpr int kOsTile = 256;  // particles per block, one per thread

__device__ __forceinline__ uint32_t compact3(uint64_t x) {  // inverse of spread3
    x &= 0x1249249249249249ULL;
    x = (x | (x >> 2)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x >> 4)) & 0x100f00f00f00f00fULL;
    x = (x | (x >> 8)) & 0x1f0000ff0000ffULL;
    x = (x | (x >> 16)) & 0x1f00000000ffffULL;
    x = (x | (x >> 32)) & 0x1fffffULL;
    return (uint32_t)x;
}

// Shift of the level-l key prefix (the l leading octant digits).
__device__ __forceinline__ int prefix_shift(int l) { return 3 * (kMaxLevel + 1 - l); }

// Whether the level-(l-1) segment holding particle i (system range [s0, s1))
// has more than M particles: its start a is found within M places below i
// (or the segment already holds i - M .. i), then particle a + M decides.
__device__ __forceinline__ bool os_parent_splits(const uint64_t *__restrict__ keys, int64_t i, int64_t s0,
                                                 int64_t s1, int l, int M) {
    if (l == 1) return s1 - s0 > M;  // the parent is the root
    const int sh = prefix_shift(l - 1);
    const uint64_t pp = keys[i] >> sh;
    int64_t lo = max(s0, i - (int64_t)M), a;
    if ((keys[lo] >> sh) == pp) {
        if (i - lo >= M) return true;
        a = lo;  // lo is the system's first particle
    } else {
        int64_t hi = i;  // keys[lo] outside the segment, keys[hi] inside
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if ((keys[mid] >> sh) == pp) hi = mid; else lo = mid;
        }
        a = hi;
    }
    const int64_t j = a + M;
    return j < s1 && (keys[j] >> sh) == pp;
}

// The thread's particle: its key, its predecessor's and its system range.
struct OsPoint {
    bool valid;
    int sy;
    int64_t i, s0, s1;
    uint64_t key, prev;
};
__device__ __forceinline__ OsPoint os_point(int64_t n, const uint64_t *__restrict__ keys,
                                            const int64_t *__restrict__ off, int S) {
    OsPoint p;
    p.i = (int64_t)blockIdx.x * kOsTile + threadIdx.x;
    p.valid = p.i < n;
    p.key = p.valid ? keys[p.i] : 0ull;
    p.prev = (p.valid && p.i > 0) ? keys[p.i - 1] : 0ull;
    p.sy = p.valid ? find_sys(off, S, p.i) : 0;
    p.s0 = p.valid ? off[p.sy] : 0;
    p.s1 = p.valid ? off[p.sy + 1] : 0;
    return p;
}

// Bit l - 1 set: the particle is a box of level l (L <= kMaxLevel + 1 < 32).
// A particle that starts a level-l segment whose level-(l-1) segment holds at
// most M particles lies in a leaf of level l - 1 or coarser: no finer level
// can hold a box starting with it (its segments only shrink), so the levels
// below are not tested.
__device__ __forceinline__ uint32_t os_box_levels(const OsPoint &p, const uint64_t *__restrict__ keys, int L, int M,
                                                  int max_depth) {
    uint32_t f = 0;
    if (!p.valid) return f;
    for (int l = 1; l <= L && l - 1 < max_depth; ++l) {
        const int sh = prefix_shift(l);
        if (p.i > p.s0 && (p.key >> sh) == (p.prev >> sh)) continue;  // not a segment start
        if (!os_parent_splits(keys, p.i, p.s0, p.s1, l, M)) break;
        f |= 1u << (l - 1);
    }
    return f;
}

// Pass 1: boxes of levels 1 .. L per particle tile -> cnt[(l - 1) ntiles + tile].
__global__ void __launch_bounds__(kOsTile) k_os_count(int64_t n, const uint64_t *__restrict__ keys,
                                                      const int64_t *__restrict__ off, int S, int L, int M,
                                                      int max_depth, int ntiles, uint32_t *cnt) {
    const OsPoint p = os_point(n, keys, off, S);
    const uint32_t f = os_box_levels(p, keys, L, M, max_depth);
    for (int l = 1; l <= L; ++l) {
        const int c = __syncthreads_count((f >> (l - 1)) & 1u);
        if (threadIdx.x == 0) cnt[(size_t)(l - 1) * ntiles + blockIdx.x] = (uint32_t)c;
    }
}

// Pass 2 (one block): the counts cnt[(l - 1) ntiles + tile] become the first
// box index of each (level, tile) in first_idx (one exclusive scan over the
// level-major array: each warp sums a contiguous segment with coalesced loads,
// the warps' sums are scanned, each warp rescans its segment 32 at a time);
// level boundaries go to lb[0 .. L + 1] (level 0: the S roots), and fail is
// set when the boxes outgrow the arrays (then nothing else is written).
__global__ void __launch_bounds__(1024) k_os_scan(int L, int ntiles, int S, int64_t cap,
                                                  const uint32_t *__restrict__ cnt, uint32_t *__restrict__ first_idx,
                                                  int64_t *lb, int *fail) {
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t len = (int64_t)L * ntiles;
    const int64_t seg = ((len + 32 * 32 - 1) / (32 * 32)) * 32;  // per warp, a multiple of 32
    const int64_t w0 = min(len, warp * seg), w1 = min(len, w0 + seg);
    uint32_t sum = 0;
#pragma unroll 4
    for (int64_t k = w0 + lane; k < w1; k += 32) sum += cnt[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) ws[warp] = sum;
    __syncthreads();
    uint32_t before = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
        before += (w < warp) ? ws[w] : 0u;
        tot += ws[w];
    }
    int64_t run = (int64_t)S + before;  // boxes before this warp's segment
    for (int64_t k0 = w0; k0 < w1; k0 += 32) {
        const int64_t k = k0 + lane;
        const uint32_t v = k < w1 ? cnt[k] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (k < w1) {
            first_idx[k] = (uint32_t)(run + x - v);
            if (k % ntiles == 0) lb[k / ntiles + 1] = run + x - v;  // level k / ntiles + 1 starts here
        }
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (threadIdx.x == 0) {
        const int64_t total = (int64_t)S + tot;
        lb[0] = 0;
        if (ntiles == 0)
            for (int l = 1; l <= L; ++l) lb[l] = S;
        lb[L + 1] = total;
        *fail = total > cap || total > (int64_t)INT32_MAX;
    }
}

// End of the key segment that starts at particle i (prefix pf = keys[i] >> sh,
// system end s1): the first j > i with j = s1 or another prefix.  The whole
// warp probes 32 places per round, growing the stride 32-fold until a probe
// leaves the segment, then shrinking it 32-fold; in-segment probes always form
// a prefix of the lanes (sorted keys), so a ballot's count places the end.
// A segment of c particles takes about 2 log32(c) rounds instead of 2 log2(c)
// dependent loads.
__device__ __forceinline__ int64_t warp_segment_end(const uint64_t *__restrict__ keys, int64_t i, int64_t s1,
                                                   uint64_t pf, int sh, int lane) {
    int64_t lo = i, step = 1;  // keys[lo] is in the segment
    for (;;) {
        const int64_t pos = lo + step * (lane + 1);
        const bool in = pos < s1 && (keys[pos] >> sh) == pf;
        const int c = __popc(__ballot_sync(0xffffffffu, in));
        if (c < 32) {
            lo += step * c;
            break;
        }
        lo += 32 * step;
        step *= 32;
    }
    while (step > 1) {  // the end lies in (lo, lo + step]
        step = (step + 31) / 32;
        const int64_t pos = lo + step * (lane + 1);
        const bool in = pos < s1 && (keys[pos] >> sh) == pf;
        lo += step * __popc(__ballot_sync(0xffffffffu, in));
    }
    return lo + 1;
}

// Pass 3: each box's level, coordinates, particle range and system; its
// index is the tile's first box of the level plus the boxes of the level
// before it in the tile (ballots, then the warps' counts).
__global__ void __launch_bounds__(kOsTile) k_os_emit(int64_t n, const uint64_t *__restrict__ keys,
                                                     const int64_t *__restrict__ off, int S, int L, int M,
                                                     int max_depth, int ntiles, const uint32_t *__restrict__ base_idx,
                                                     const int *fail, int32_t *lvl, int32_t *cx, int32_t *cy,
                                                     int32_t *cz, int32_t *first, int32_t *cnt, int32_t *sys) {
    __shared__ uint32_t wc[kOsTile / 32];
    if (*fail) return;
    const OsPoint p = os_point(n, keys, off, S);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t f = os_box_levels(p, keys, L, M, max_depth);
    for (int l = 1; l <= L; ++l) {
        const bool box = (f >> (l - 1)) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, box);
        __syncthreads();  // wc free from the previous level
        if (lane == 0) wc[warp] = (uint32_t)__popc(m);
        __syncthreads();
        const int sh = prefix_shift(l);
        const uint64_t pf = p.key >> sh;
        // the segments' ends, one box of the warp at a time, all lanes probing
        int64_t hi = 0;
        for (unsigned pend = m; pend; pend &= pend - 1) {
            const int src = __ffs(pend) - 1;
            const int64_t e = warp_segment_end(keys, __shfl_sync(0xffffffffu, p.i, src),
                                               __shfl_sync(0xffffffffu, p.s1, src),
                                               __shfl_sync(0xffffffffu, pf, src), sh, lane);
            if (lane == src) hi = e;
        }
        if (!box) continue;
        uint32_t before = (uint32_t)__popc(m & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) before += wc[w];
        const int64_t b = (int64_t)base_idx[(size_t)(l - 1) * ntiles + blockIdx.x] + before;
        lvl[b] = l;
        cx[b] = (int32_t)compact3(pf >> 2);
        cy[b] = (int32_t)compact3(pf >> 1);
        cz[b] = (int32_t)compact3(pf);
        first[b] = (int32_t)p.i;
        cnt[b] = (int32_t)(hi - p.i);
        sys[b] = p.sy;
    }
}

// Index in [lo, hi) of the last a[k] <= x (lo - 1 if none).
__device__ __forceinline__ int64_t last_le(const int32_t *__restrict__ a, int64_t lo, int64_t hi, int32_t x) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

// Pass 4: parents (the last box of the level above whose first particle is
// at or before the box's) and child ranges (the boxes of the level below
// whose first particle lies in the box's range); the boxes of level L get
// none here (the level-by-level build continues from them if one splits).
__global__ void k_os_link(const int64_t *__restrict__ lb, int L, int M, int max_depth, const int *fail,
                          const int32_t *__restrict__ lvl, const int32_t *__restrict__ first,
                          const int32_t *__restrict__ cnt, int32_t *parent, int32_t *child_first, int32_t *nchild) {
    if (*fail) return;
    const int64_t nb = lb[L + 1];
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int l = lvl[b];
        const int32_t f = first[b], c = cnt[b];
        if (l >= 1) parent[b] = (int32_t)last_le(first, lb[l - 1], lb[l], f);
        if (l < L && l < max_depth && c > M) {
            const int64_t c0 = last_le(first, lb[l + 1], lb[l + 2], f - 1) + 1;
            const int64_t c1 = last_le(first, lb[l + 1], lb[l + 2], f + c - 1) + 1;
            child_first[b] = (int32_t)c0;
            nchild[b] = (int32_t)(c1 - c0);
        } else {
            child_first[b] = -1;
            nchild[b] = 0;
        }
    }
}

// Leaf centres in the caller's coordinates, C = lo + (c + 1/2) 2^-level side
// in FP64, as unevaluated sums C_hi + C_lo of two floats: one thread per
// (leaf, axis), so the few FP64 operations fill whole warps (this GPU runs
// FP64 at a small fraction of the FP32 rate, per warp instruction).
__global__ void k_leaf_centres(int64_t max_leaves, const uint32_t *__restrict__ n_leaves,
                               const int32_t *__restrict__ leaves, const int32_t *__restrict__ lvl,
                               const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                               const int32_t *__restrict__ cz, const int32_t *__restrict__ sys,
                               const double *__restrict__ lo_side, float2 *ctr) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t li = t / 3;
    const int d = (int)(t - 3 * li);
    if (li >= max_leaves || li >= (int64_t)*n_leaves) return;
    const int b = leaves[li], s = sys[b];
    const double w = ldexp(1.0, -lvl[b]);
    const int c = d == 0 ? cx[b] : d == 1 ? cy[b] : cz[b];
    const double C = fma((c + 0.5) * w, lo_side[s * 4 + 3], lo_side[s * 4 + d]);
    const float hi = (float)C;
    ctr[t] = make_float2(hi, (float)(C - (double)hi));
}

template <typename TI, typename TC>
__global__ void k_gather(int64_t max_leaves, const uint32_t *__restrict__ n_leaves,
                         const int32_t *__restrict__ leaves, const int32_t *__restrict__ first,
                         const int32_t *__restrict__ cnt, const int32_t *__restrict__ lvl,
                         const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                         const int32_t *__restrict__ cz, const int32_t *__restrict__ sys,
                         const double *__restrict__ lo_side, const uint32_t *__restrict__ perm,
                         const TI *__restrict__ xyz, const TI *__restrict__ q,
                         typename Vec4<TC>::type *pts, double cell, double *leaf_q2,
                         const float2 *__restrict__ ctr, const float *__restrict__ inv_side_f) {
    // one warp per leaf; the leaf count is read on the device (the grid
    // covers max_leaves)
    const int64_t li = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (li >= max_leaves || li >= (int64_t)*n_leaves) return;
    const int b = leaves[li];
    const int s = sys[b];
    if constexpr (sizeof(TC) == 4 && sizeof(TI) == 4) {
        if (cell == 0.0 && !leaf_q2) {
            // FP32 records from FP32 inputs in FP32 arithmetic: the leaf
            // centre comes as an unevaluated sum C_hi + C_lo of two floats
            // (k_leaf_centres); x - C_hi is exact for x next to C (Sterbenz),
            // so a record is still the caller's coordinate to about an ulp of
            // |x|
            const int lane = threadIdx.x & 31;
            const float2 c2 = lane < 3 ? ctr[3 * li + lane] : make_float2(0.f, 0.f);
            float ch[3], cl[3];
            for (int d = 0; d < 3; ++d) {
                ch[d] = __shfl_sync(0xffffffffu, c2.x, d);
                cl[d] = __shfl_sync(0xffffffffu, c2.y, d);
            }
            const float is = inv_side_f[s];
            const int n = cnt[b], f = first[b];
            for (int k = lane; k < n; k += 32) {
                const int64_t i = f + k;
                const uint32_t j = perm[i];
                float4 v;
                v.x = (xyz[3 * j] - ch[0] - cl[0]) * is;
                v.y = (xyz[3 * j + 1] - ch[1] - cl[1]) * is;
                v.z = (xyz[3 * j + 2] - ch[2] - cl[2]) * is;
                v.w = q ? (float)q[j] : 0.f;
                pts[i] = v;
            }
            return;
        }
    }
    const double side = lo_side[s * 4 + 3], inv_side = 1.0 / side;
    const double lo[3] = {lo_side[s * 4], lo_side[s * 4 + 1], lo_side[s * 4 + 2]};
    const double w = ldexp(1.0, -lvl[b]);
    // the leaf centre in the caller's coordinates: the offset x - C is then
    // exact (x lies next to C) and rounds only on the division, so a record
    // carries the caller's coordinate to about one unit in the last place of
    // |x|, not of |x - lo| (which is far larger for a particle near the origin
    // of a domain whose corner lies far from it)
    const double C[3] = {fma((cx[b] + 0.5) * w, side, lo[0]), fma((cy[b] + 0.5) * w, side, lo[1]),
                         fma((cz[b] + 0.5) * w, side, lo[2])};
    double q2 = 0.0;  // periodic cell: sum q |x - c_cell|^2 of the leaf, root units
    for (int k = threadIdx.x & 31; k < cnt[b]; k += 32) {
        const int64_t i = first[b] + k;
        const uint32_t j = perm[i];
        double r[3];
        // FP64 records keep the correctly rounded quotient (FP64 parity); FP32
        // records are rounded to FP32 anyway, so a reciprocal multiply will do
        for (int d = 0; d < 3; ++d) {
            const double x = wrap_cell((double)xyz[3 * j + d], cell);
            r[d] = sizeof(TC) == 8 ? (x - C[d]) / side : (x - C[d]) * inv_side;
        }
        typename Vec4<TC>::type v;
        v.x = (TC)r[0];
        v.y = (TC)r[1];
        v.z = (TC)r[2];
        v.w = q ? (TC)q[j] : TC(0);
        pts[i] = v;
        if (leaf_q2) {
            const double ex = (cx[b] + 0.5) * w + r[0] - 0.5, ey = (cy[b] + 0.5) * w + r[1] - 0.5,
                         ez = (cz[b] + 0.5) * w + r[2] - 0.5;
            q2 += (double)v.w * (ex * ex + ey * ey + ez * ez);
        }
    }
    if (leaf_q2) {
        for (int o = 16; o > 0; o >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
        if ((threadIdx.x & 31) == 0) leaf_q2[li] = q2;
    }
}

// Tree reuse test: one warp per leaf; every particle's leaf-relative offset
// (in FP64, in units of the root side) must lie within
// the leaf's half-width plus `margin` of its centre on every axis; otherwise
// (or for a non-finite coordinate) *moved is set.
template <typename TI>
__global__ void k_leaf_check(int64_t n_leaves, const int32_t *__restrict__ leaves, const int32_t *__restrict__ first,
                             const int32_t *__restrict__ cnt, const int32_t *__restrict__ lvl,
                             const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                             const int32_t *__restrict__ cz, const int32_t *__restrict__ sys,
                             const double *__restrict__ lo_side, const uint32_t *__restrict__ perm,
                             const TI *__restrict__ xyz, double margin, int *moved, double cell) {
    const int64_t li = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (li >= n_leaves) return;
    const int b = leaves[li];
    const int s = sys[b];
    const double inv_side = 1.0 / lo_side[s * 4 + 3];  // a tolerance test: no exact quotient needed
    const double lo[3] = {lo_side[s * 4], lo_side[s * 4 + 1], lo_side[s * 4 + 2]};
    const double w = ldexp(1.0, -lvl[b]);
    const double c[3] = {(cx[b] + 0.5) * w, (cy[b] + 0.5) * w, (cz[b] + 0.5) * w};
    const double lim = 0.5 * w + margin;
    bool bad = false;
    for (int k = threadIdx.x & 31; k < cnt[b]; k += 32) {
        const uint32_t j = perm[first[b] + k];
        for (int d = 0; d < 3; ++d) {
            const double r = (wrap_cell((double)xyz[3 * j + d], cell) - lo[d]) * inv_side - c[d];
            bad = bad || !(fabs(r) <= lim);  // also catches NaN
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(moved, 1);
}

// ---------------------------------------------------------------------------
// Lists
// ---------------------------------------------------------------------------
// Periodic cell (Sec. 2.4): a list entry is a box plus the image it is taken
// in, an image shift n in {-1, 0, 1}^3 stored as (n_x + 1) 9 + (n_y + 1) 3 +
// (n_z + 1) (13: the cell itself).  Shift arrays are null for a free-space
// plan, whose entries are all in the cell.
struct ListShifts {
    int8_t *coll, *coarse, *x, *u, *w;  // parallel to coll, coarse, xdense, u_idx, w_idx
};
__device__ __forceinline__ int shift_of(const int8_t *sh, int64_t i) { return sh ? (int)sh[i] : 13; }
// The shift of image s in boxes of `level` along each axis.
__device__ __forceinline__ void shift_boxes(int s, int level, int &ox, int &oy, int &oz) {
    ox = (s / 9 - 1) << level;
    oy = ((s / 3) % 3 - 1) << level;
    oz = (s % 3 - 1) << level;
}
// adjacent(box a in image sa, box at (lb, bx, by, bz))
__device__ __forceinline__ bool adjacent_img(int la, int ax, int ay, int az, int sa, int lb, int bx, int by, int bz) {
    int ox, oy, oz;
    shift_boxes(sa, la, ox, oy, oz);
    return boxes_adjacent(la, ax + ox, ay + oy, az + oz, lb, bx, by, bz);
}

// slot of offset d for octant class (ox,oy,oz): components range over
// [-2-o, 3-o]; the inner [-1,1]^3 is excluded.
// Closed form: lexicographic index in the 6^3 window minus the excluded inner
// 3^3 cells (at window offset 1 + o per axis) that precede it.
__device__ __forceinline__ int v_slot(int ox, int oy, int oz, int dx, int dy, int dz) {
    const int a = dx + 2 + ox, b = dy + 2 + oy, c = dz + 2 + oz;  // 0..5
    if (a < 0 || a > 5 || b < 0 || b > 5 || c < 0 || c > 5) return -1;
    const int a0 = 1 + ox, b0 = 1 + oy, c0 = 1 + oz;
    const bool ina = a >= a0 && a < a0 + 3, inb = b >= b0 && b < b0 + 3, inc = c >= c0 && c < c0 + 3;
    if (ina && inb && inc) return -1;
    int before = min(max(a - a0, 0), 3) * 9;
    if (ina) {
        before += min(max(b - b0, 0), 3) * 3;
        if (inb) before += min(max(c - c0, 0), 3);
    }
    return a * 36 + b * 6 + c - before;
}

// Colleagues and V list of b in one pass.  One warp per box: lane k < 27
// scans the children of the parent's colleague k (in that colleague's
// image); a child adjacent to (or equal to) b lands in its colleague slot,
// any other in its slot of b's octant-class table (V: children of the
// parent's colleagues not adjacent to b; each child has its own slot, and a
// slot fixes the source's offset, so the table needs no image shift).  In a
// periodic cell the root's colleagues are its 27 images (itself included).
// Returns the V count (the same on every lane).
__device__ __forceinline__ int dev_colleagues_v(int64_t b, int lane, int level, const int32_t *__restrict__ parent,
                                                const int32_t *__restrict__ child_first,
                                                const int32_t *__restrict__ nchild, const int32_t *__restrict__ cx,
                                                const int32_t *__restrict__ cy, const int32_t *__restrict__ cz,
                                                int32_t *coll, int32_t *vdense, const ListShifts &sh) {
    int32_t *cb = coll + b * kColl;
    // cb and the V table were set to -1 by memsets of the whole arrays
    if (level == 0) {
        if (sh.coll) {
            if (lane < kColl) {
                cb[lane] = (int32_t)b;
                sh.coll[b * kColl + lane] = (int8_t)lane;
            }
        } else if (lane == 0) {
            cb[13] = (int32_t)b;
        }
        return 0;
    }
    int cntv = 0;
    const int32_t c = (lane < kColl) ? coll[(int64_t)parent[b] * kColl + lane] : -1;
    if (c >= 0) {
        const int sc = shift_of(sh.coll, (int64_t)parent[b] * kColl + lane);
        int ox, oy, oz;
        shift_boxes(sc, level, ox, oy, oz);
        const int bx = cx[b], by = cy[b], bz = cz[b];
        const int px = bx & 1, py = by & 1, pz = bz & 1;
        int32_t *vb = vdense + b * kVSlots;
        const int32_t cf = child_first[c], nc = nchild[c];  // nc <= 8
        // (a fixed trip count: the children's coordinates load together)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k >= nc) continue;
            const int32_t ch = cf + k;
            const int dx = cx[ch] + ox - bx, dy = cy[ch] + oy - by, dz = cz[ch] + oz - bz;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) {
                const int slot = (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1);
                cb[slot] = ch;
                if (sh.coll) sh.coll[b * kColl + slot] = (int8_t)sc;
            } else {
                const int sl = v_slot(px, py, pz, dx, dy, dz);
                if (sl < 0) continue;  // unreachable: children of parent colleagues lie in the class window
                vb[sl] = ch;
                ++cntv;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cntv += __shfl_xor_sync(0xffffffffu, cntv, o);
    return cntv;
}

// Coarser-or-equal-level leaves adjacent to b: those of the parent that touch
// b (in the parent's order), then b's leaf colleagues (in slot order).  One
// warp per box; ballots keep the order.
// (coll is written by the colleague pass of the same launch: no read-only path)
__device__ __forceinline__ void dev_coarse(int64_t b, int lane, int level, const int32_t *__restrict__ parent,
                                           const int32_t *__restrict__ nchild, const int32_t *__restrict__ lvl,
                                           const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                                           const int32_t *__restrict__ cz, const int32_t *coll, int32_t *coarse,
                                           int32_t *ncoarse, int *status, const ListShifts &sh) {
    const unsigned below = (1u << lane) - 1u;
    int n = 0;
    int32_t *out = coarse + b * kMaxCoarse;
    if (level > 0) {
        const int32_t P = parent[b];
        const int np = ncoarse[P];  // <= kMaxCoarse < 32
        int32_t a = -1;
        int sa = 13;
        bool keep = false;
        if (lane < np) {
            a = coarse[(int64_t)P * kMaxCoarse + lane];
            sa = shift_of(sh.coarse, (int64_t)P * kMaxCoarse + lane);
            keep = adjacent_img(lvl[a], cx[a], cy[a], cz[a], sa, level, cx[b], cy[b], cz[b]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int pos = __popc(m & below);
            if (pos < kMaxCoarse) {
                out[pos] = a;
                if (sh.coarse) sh.coarse[b * kMaxCoarse + pos] = (int8_t)sa;
            }
        }
        n = __popc(m);
    }
    int32_t c = -1;
    int sc = 13;
    bool keep = false;
    if (lane < kColl && lane != 13) {
        c = coll[b * kColl + lane];
        keep = c >= 0 && nchild[c] == 0;
        if (keep) sc = shift_of(sh.coll, b * kColl + lane);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) {
        const int pos = n + __popc(m & below);
        if (pos < kMaxCoarse) {
            out[pos] = c;
            if (sh.coarse) sh.coarse[b * kMaxCoarse + pos] = (int8_t)sc;
        }
    }
    n += __popc(m);
    if (lane == 0) {
        if (n > kMaxCoarse) {
            set_status(status, KIFMM_ERR_CAPACITY);
            n = kMaxCoarse;
        }
        ncoarse[b] = n;
    }
}

// A leaf holding at most thr points: its W/X interactions are summed directly.
__device__ __forceinline__ bool direct_box(const int32_t *nchild, const int32_t *cnt, int thr, int32_t b) {
    return thr >= 0 && nchild[b] == 0 && cnt[b] <= thr;
}

// X list (coarser leaves adjacent to the parent but not to b; empty when b
// itself is a direct-sum leaf, see k_uw) in the parent's coarse order (a
// ballot), and the V and X counts.  One warp per box.
// (coarse and ncoarse of the parent come from the previous level's launch)
__device__ __forceinline__ void dev_x(int64_t b, int lane, int level, int thr, int cntv,
                                      const int32_t *__restrict__ parent, const int32_t *__restrict__ nchild,
                                      const int32_t *__restrict__ cnt, const int32_t *__restrict__ lvl,
                                      const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                                      const int32_t *__restrict__ cz, const int32_t *coarse, const int32_t *ncoarse,
                                      int32_t *nv, int32_t *xdense, int32_t *nx, const ListShifts &sh) {
    int cntx = 0;
    if (level > 0 && !direct_box(nchild, cnt, thr, (int32_t)b)) {
        const int32_t P = parent[b];
        const int np = ncoarse[P];
        int32_t a = -1;
        int sa = 13;
        bool keep = false;
        if (lane < np) {
            a = coarse[(int64_t)P * kMaxCoarse + lane];
            sa = shift_of(sh.coarse, (int64_t)P * kMaxCoarse + lane);
            keep = !adjacent_img(lvl[a], cx[a], cy[a], cz[a], sa, level, cx[b], cy[b], cz[b]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int pos = __popc(m & ((1u << lane) - 1u));
            xdense[b * kMaxCoarse + pos] = a;
            if (sh.x) sh.x[b * kMaxCoarse + pos] = (int8_t)sa;
        }
        cntx = __popc(m);
    }
    if (lane == 0) {
        nv[b] = cntv;
        nx[b] = cntx;
    }
}

// U and W of a leaf: U = {b} + coarse adjacent leaves + finer adjacent leaves
// found by descending b's non-leaf colleagues; a descendant that is not
// adjacent to b (while its parent is) goes to W, or to U when it is a
// direct-sum leaf.  When b itself is a direct-sum leaf, its X list (coarser
// leaves adjacent to the parent, not to b) goes to U as well.  Pass 0 counts,
// pass 1 fills.
__global__ void k_uw(int64_t nb, int pass, int thr, const int32_t *__restrict__ parent,
                     const int32_t *__restrict__ cnt, const int32_t *__restrict__ child_first,
                     const int32_t *__restrict__ nchild, const int32_t *__restrict__ lvl,
                     const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                     const int32_t *__restrict__ cz, const int32_t *__restrict__ coll,
                     const int32_t *__restrict__ coarse, const int32_t *__restrict__ ncoarse,
                     uint32_t *u_cnt, uint32_t *w_cnt, const uint32_t *__restrict__ u_ptr,
                     const uint32_t *__restrict__ w_ptr, int32_t *u_idx, int32_t *w_idx, int64_t u_cap,
                     int64_t w_cap, int *status, ListShifts sh) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    if (nchild[b] != 0) {
        if (pass == 0) u_cnt[b] = w_cnt[b] = 0;
        return;
    }
    const int lb = lvl[b], bx = cx[b], by = cy[b], bz = cz[b];
    uint32_t nu = 0, nw = 0;
    const uint32_t u0 = pass ? u_ptr[b] : 0, w0 = pass ? w_ptr[b] : 0;
    // pass 1 writes only inside the storage; the host sees a list that
    // outgrew it from the totals and builds the lists again
    auto put_u = [&](int32_t a, int sa) {
        if (pass && (int64_t)u0 + nu < u_cap) {
            u_idx[u0 + nu] = a;
            if (sh.u) sh.u[u0 + nu] = (int8_t)sa;
        }
        ++nu;
    };
    auto put_w = [&](int32_t a, int sa) {
        if (pass && (int64_t)w0 + nw < w_cap) {
            w_idx[w0 + nw] = a;
            if (sh.w) sh.w[w0 + nw] = (int8_t)sa;
        }
        ++nw;
    };
    put_u((int32_t)b, 13);
    for (int k = 0; k < ncoarse[b]; ++k) put_u(coarse[b * kMaxCoarse + k], shift_of(sh.coarse, b * kMaxCoarse + k));
    if (lb > 0 && direct_box(nchild, cnt, thr, (int32_t)b)) {
        const int32_t P = parent[b];
        for (int k = 0; k < ncoarse[P]; ++k) {
            const int32_t a = coarse[(int64_t)P * kMaxCoarse + k];
            const int sa = shift_of(sh.coarse, (int64_t)P * kMaxCoarse + k);
            if (adjacent_img(lvl[a], cx[a], cy[a], cz[a], sa, lb, bx, by, bz)) continue;
            put_u(a, sa);
        }
    }
    int32_t stack[8 * (kMaxLevel + 1)];
    for (int k = 0; k < kColl; ++k) {
        const int32_t c = coll[b * kColl + k];
        if (k == 13 || c < 0 || nchild[c] == 0) continue;
        const int sc = shift_of(sh.coll, b * kColl + k);  // every descendant is taken in this image
        int sp = 0;
        for (int32_t ch = child_first[c]; ch < child_first[c] + nchild[c]; ++ch) stack[sp++] = ch;
        while (sp > 0) {
            const int32_t a = stack[--sp];
            if (adjacent_img(lvl[a], cx[a], cy[a], cz[a], sc, lb, bx, by, bz)) {
                if (nchild[a] == 0) {
                    put_u(a, sc);
                } else {
                    if (sp + nchild[a] > 8 * (kMaxLevel + 1)) {
                        set_status(status, KIFMM_ERR_CAPACITY);
                        return;
                    }
                    for (int32_t ch = child_first[a]; ch < child_first[a] + nchild[a]; ++ch) stack[sp++] = ch;
                }
            } else if (direct_box(nchild, cnt, thr, a)) {
                put_u(a, sc);
            } else {
                put_w(a, sc);
            }
        }
    }
    if (pass == 0) {
        u_cnt[b] = nu;
        w_cnt[b] = nw;
    }
}

// W-list sources: the entry count is read on the device (w_ptr[nb]), capped
// by the storage.
__global__ void k_mark_w(int64_t cap, const uint32_t *__restrict__ w_total, const int32_t *__restrict__ w_idx,
                         int32_t *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cap && i < (int64_t)*w_total) flag[w_idx[i]] = 1;
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

size_t scan_tmp_needed(int64_t n) {
    size_t total = 0;
    int64_t m = n;
    while (m > 1) {
        m = (m + kScanTile - 1) / kScanTile;
        total += (size_t)m + 1;
    }
    return total + 4;
}

cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev,
                               uint32_t *tmp, size_t tmp_elems, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) KIFMM_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s));
        return cudaSuccess;
    }
    const int64_t nblk = (n + kScanTile - 1) / kScanTile;
    if ((size_t)nblk + 1 > tmp_elems) return cudaErrorInvalidValue;
    if (nblk == 1) {  // one tile: its sum is the total
        ++g_launches, k_scan_tiles<<<1, kScanBlock, 0, s>>>(in, out, n, total_dev ? total_dev : tmp);
        return cudaGetLastError();
    }
    uint32_t *sums = tmp;
    ++g_launches, k_scan_tiles<<<(unsigned)nblk, kScanBlock, 0, s>>>(in, out, n, sums);
    // the tile sums' own scan yields the grand total
    KIFMM_CUDA_TRY(exclusive_scan_u32(sums, sums, nblk, total_dev, tmp + nblk + 1, tmp_elems - nblk - 1, s));
    ++g_launches, k_scan_add<<<(unsigned)nblk, kScanBlock, 0, s>>>(out, n, sums);
    return cudaGetLastError();
}

// Partition keys (see Plan::part_list): mode 0 octant class of boxes with a
// V list (8: none), mode 1 leaves first then non-leaves by level, mode 2 W
// sources first, mode 3 level * 8 + octant (255: the roots).
__device__ __forceinline__ uint32_t part_key(int mode, int64_t b, const int32_t *__restrict__ nv,
                                             const int32_t *__restrict__ nchild, const int32_t *__restrict__ lvl,
                                             const int32_t *__restrict__ wflag, const int32_t *__restrict__ cx,
                                             const int32_t *__restrict__ cy, const int32_t *__restrict__ cz) {
    const uint32_t oct = (uint32_t)(4 * (cx[b] & 1) + 2 * (cy[b] & 1) + (cz[b] & 1));
    if (mode == 0) return (nv[b] > 0) ? oct : 8u;
    if (mode == 1) return (nchild[b] == 0) ? 0u : 1u + (uint32_t)lvl[b];
    if (mode == 2) return wflag[b] ? 0u : 1u;
    return (lvl[b] > 0) ? (uint32_t)lvl[b] * 8u + oct : 255u;
}

// All four partitions in one grid (blockIdx.y = mode): per-tile key
// histograms laid out [mode][key][tile] so that one exclusive scan serves all
// modes (mode m's positions come out offset by m * nb), plus key totals.
__global__ void k_part_hist(int64_t nb, int nblk, const int32_t *__restrict__ nv, const int32_t *__restrict__ nchild,
                            const int32_t *__restrict__ lvl, const int32_t *__restrict__ wflag,
                            const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                            const int32_t *__restrict__ cz, uint32_t *hist, uint32_t *counts) {
    __shared__ uint32_t h[256];
    const int mode = blockIdx.y;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const int64_t end = min(nb, base + (int64_t)kTile);
    for (int64_t b = base + threadIdx.x; b < end; b += kBlock)
        atomicAdd(&h[part_key(mode, b, nv, nchild, lvl, wflag, cx, cy, cz)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        hist[((int64_t)mode * 256 + d) * nblk + blockIdx.x] = h[d];
        if (h[d]) atomicAdd(&counts[mode * 256 + d], h[d]);
    }
}

// Stable scatter of box indices by key (ranks as in k_rs_scatter).
__global__ void k_part_scatter(int64_t nb, int nblk, const int32_t *__restrict__ nv,
                               const int32_t *__restrict__ nchild, const int32_t *__restrict__ lvl,
                               const int32_t *__restrict__ wflag, const int32_t *__restrict__ cx,
                               const int32_t *__restrict__ cy, const int32_t *__restrict__ cz,
                               const uint32_t *__restrict__ hist_scan, int32_t *out0, int32_t *out1, int32_t *out2,
                               int32_t *out3) {
    __shared__ uint32_t base_d[256];
    __shared__ uint32_t wcnt[kBlock / 32][256];
    const int mode = blockIdx.y;
    int32_t *out = mode == 0 ? out0 : mode == 1 ? out1 : mode == 2 ? out2 : out3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t shift = (uint32_t)(mode * nb);  // the joint scan's offset of this mode
    for (int d = threadIdx.x; d < 256; d += kBlock)
        base_d[d] = hist_scan[((int64_t)mode * 256 + d) * nblk + blockIdx.x] - shift;
    const int64_t tile0 = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        for (int i = threadIdx.x; i < (kBlock / 32) * 256; i += kBlock) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t b = tile0 + (int64_t)r * kBlock + threadIdx.x;
        const bool valid = b < nb;
        const uint32_t dig = valid ? part_key(mode, b, nv, nchild, lvl, wflag, cx, cy, cz) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int rank_w = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank_w == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += kBlock) {
            uint32_t run = base_d[d];
            for (int w = 0; w < kBlock / 32; ++w) {
                const uint32_t c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
            base_d[d] = run;
        }
        __syncthreads();
        if (valid) out[wcnt[warp][dig] + rank_w] = (int32_t)b;
        __syncthreads();
    }
}

__global__ void k_child8(int64_t nb, const int32_t *__restrict__ child_first, const int32_t *__restrict__ nchild,
                         const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                         const int32_t *__restrict__ cz, int32_t *child8) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int32_t *o = child8 + b * 8;
    for (int k = 0; k < 8; ++k) o[k] = -1;
    for (int32_t c = child_first[b]; c < child_first[b] + nchild[b]; ++c)
        o[4 * (cx[c] & 1) + 2 * (cy[c] & 1) + (cz[c] & 1)] = c;
}

static cudaError_t radix_pass(Plan &P, const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout,
                              int64_t n, int mode, int shift, cudaStream_t s) {
    const int nblk = (int)((n + kTile - 1) / kTile);
    if ((size_t)512 * nblk > P.hist_elems) {
        P.hist_elems = (size_t)512 * nblk;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.hist, sizeof(uint32_t) * P.hist_elems));
    }
    if (scan_tmp_needed((int64_t)256 * nblk) + 8 > P.scan_tmp_elems) {
        P.scan_tmp_elems = scan_tmp_needed((int64_t)256 * nblk) + 8;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.scan_tmp, sizeof(uint32_t) * P.scan_tmp_elems));
    }
    ++g_launches, k_rs_hist<<<nblk, kBlock, 0, s>>>(n, kin, vin, mode, shift, P.sys_off_d, P.n_sys, P.hist, nblk);
    uint32_t *dtot = P.hist + (size_t)256 * nblk;
    ++g_launches, k_rs_dscan<<<256, 256, 0, s>>>(P.hist, nblk, dtot);
    ++g_launches, k_rs_scatter<<<nblk, kBlock, 0, s>>>(n, kin, vin, kout, vout, mode, shift, P.sys_off_d, P.n_sys,
                                                       P.hist, dtot, nblk);
    return cudaGetLastError();
}

cudaError_t partition_boxes(Plan &P, cudaStream_t s) {
    const int64_t nb = P.nb;
    const int nblk = (int)((nb + kTile - 1) / kTile);
    const int64_t nh = (int64_t)4 * 256 * nblk;
    if ((size_t)2 * nh > P.hist_elems) {
        P.hist_elems = (size_t)2 * nh;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.hist, sizeof(uint32_t) * P.hist_elems));
    }
    if (scan_tmp_needed(nh) + 8 > P.scan_tmp_elems) {
        P.scan_tmp_elems = scan_tmp_needed(nh) + 8;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.scan_tmp, sizeof(uint32_t) * P.scan_tmp_elems));
    }
    ++g_launches, k_child8<<<grid_for(nb, 256), 256, 0, s>>>(nb, P.child_first, P.nchild, P.cx, P.cy, P.cz, P.child8);
    KIFMM_CUDA_TRY(cudaMemsetAsync(P.part_counts, 0, sizeof(uint32_t) * 4 * 256, s));
    const dim3 grid((unsigned)nblk, 4);
    ++g_launches, k_part_hist<<<grid, kBlock, 0, s>>>(nb, nblk, P.nv, P.nchild, P.lvl, P.wsrc_flag, P.cx, P.cy, P.cz,
                                                      P.hist, P.part_counts);
    KIFMM_CUDA_TRY(exclusive_scan_u32(P.hist, P.hist + nh, nh, nullptr, P.scan_tmp, P.scan_tmp_elems - 1, s));
    ++g_launches, k_part_scatter<<<grid, kBlock, 0, s>>>(nb, nblk, P.nv, P.nchild, P.lvl, P.wsrc_flag, P.cx, P.cy,
                                                         P.cz, P.hist + nh, P.part_list[0], P.part_list[1],
                                                         P.part_list[2], P.part_list[3]);
    // the four key histograms come back with set_sources' final
    // synchronisation (the gather reads the leaf count on the device)
    KIFMM_CUDA_TRY(cudaMemcpyAsync(P.rb->part_counts, P.part_counts, sizeof(P.rb->part_counts),
                                   cudaMemcpyDeviceToHost, s));
    P.m2l_targets = P.part_list[0];
    P.leaves = P.part_list[1];
    return cudaGetLastError();
}

void partition_finish(Plan &P) {
    for (int mode = 0; mode < 4; ++mode) {
        P.part_start[mode].assign(257, 0);
        for (int k = 0; k < 256; ++k) P.part_start[mode][k + 1] = P.part_start[mode][k] + P.rb->part_counts[mode][k];
    }
    for (int c = 0; c <= 8; ++c) P.m2l_class_start[c] = P.part_start[0][c];
    P.n_leaves = P.part_start[1][1];
}

// The fields of a box the lists depend on: level, coordinates, parent,
// child range, and whether it is a leaf summed directly (the small-leaf rule).
__device__ __forceinline__ void box_fields(int64_t b, int thr, const int32_t *lvl, const int32_t *cx,
                                           const int32_t *cy, const int32_t *cz, const int32_t *parent,
                                           const int32_t *nchild, const int32_t *child_first, const int32_t *cnt,
                                           int32_t (&f)[8]) {
    f[0] = lvl[b], f[1] = cx[b], f[2] = cy[b], f[3] = cz[b], f[4] = parent[b], f[5] = nchild[b],
    f[6] = child_first[b], f[7] = (nchild[b] == 0 && thr >= 0 && cnt[b] <= thr) ? 1 : 0;
}
__global__ void k_boxes_differ(int64_t nb, int thr, const int32_t *__restrict__ lvl, const int32_t *__restrict__ cx,
                               const int32_t *__restrict__ cy, const int32_t *__restrict__ cz,
                               const int32_t *__restrict__ parent, const int32_t *__restrict__ nchild,
                               const int32_t *__restrict__ child_first, const int32_t *__restrict__ cnt,
                               const int32_t *__restrict__ prev, int64_t cap, int *differs) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int32_t f[8];
    box_fields(b, thr, lvl, cx, cy, cz, parent, nchild, child_first, cnt, f);
    bool same = true;
#pragma unroll
    for (int k = 0; k < 8; ++k) same = same && (f[k] == prev[k * cap + b]);
    if (!same) *differs = 1;
}
__global__ void k_boxes_save(int64_t nb, int thr, const int32_t *__restrict__ lvl, const int32_t *__restrict__ cx,
                             const int32_t *__restrict__ cy, const int32_t *__restrict__ cz,
                             const int32_t *__restrict__ parent, const int32_t *__restrict__ nchild,
                             const int32_t *__restrict__ child_first, const int32_t *__restrict__ cnt,
                             int32_t *__restrict__ prev, int64_t cap) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int32_t f[8];
    box_fields(b, thr, lvl, cx, cy, cz, parent, nchild, child_first, cnt, f);
#pragma unroll
    for (int k = 0; k < 8; ++k) prev[k * cap + b] = f[k];
}

cudaError_t same_boxes(Plan &P, int *differs, cudaStream_t s) {
    KIFMM_CUDA_TRY(cudaMemsetAsync(P.tree_differs, 0, sizeof(int), s));
    if (P.nb > 0)
        ++g_launches, k_boxes_differ<<<grid_for(P.nb, 256), 256, 0, s>>>(
                          P.nb, P.direct_thr, P.lvl, P.cx, P.cy, P.cz, P.parent, P.nchild, P.child_first, P.cnt,
                          P.prev_tree, P.prev_cap, P.tree_differs);
    KIFMM_CUDA_TRY(cudaMemcpyAsync(differs, P.tree_differs, sizeof(int), cudaMemcpyDeviceToHost, s));
    return cudaStreamSynchronize(s);
}

cudaError_t save_boxes(Plan &P, cudaStream_t s) {
    if (P.nb > P.prev_cap) {
        const int64_t cap = P.nb + P.nb / 4 + 256;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.prev_tree, sizeof(int32_t) * 8 * cap));
        P.prev_cap = cap;
    }
    if (P.nb > 0)
        ++g_launches, k_boxes_save<<<grid_for(P.nb, 256), 256, 0, s>>>(P.nb, P.direct_thr, P.lvl, P.cx, P.cy, P.cz,
                                                                       P.parent, P.nchild, P.child_first, P.cnt,
                                                                       P.prev_tree, P.prev_cap);
    return cudaGetLastError();
}

// Octree levels whose split digits lie in the top `npass` 8-bit digits of the
// 63-bit key (level l is read from bits [63 - 3l, 66 - 3l)).
static int levels_sorted(int npass) { return (8 * npass - 1) / 3; }

// Stable LSD sort on the top `npass` key digits (then the system id, for
// batched sorts): equal top digits keep the incoming order.
static cudaError_t radix_sort(Plan &P, int64_t n, cudaStream_t s, int &cur, int npass) {
    const int nblk = (int)((n + kTile - 1) / kTile);
    struct Pass { int mode, shift; };
    std::vector<Pass> passes;
    for (int sh = 64 - 8 * npass; sh < 64; sh += 8) passes.push_back({0, sh});
    if (P.n_sys > 1) {
        for (int sh = 0; (1LL << sh) < P.n_sys; sh += 8) passes.push_back({1, sh});
    }
    (void)nblk;
    for (const Pass &ps : passes) {
        const int nxt = cur ^ 1;
        KIFMM_CUDA_TRY(radix_pass(P, P.keys[cur], P.vals[cur], P.keys[nxt], P.vals[nxt], n, ps.mode, ps.shift, s));
        cur = nxt;
    }
    return cudaSuccess;
}

static cudaError_t build_levels(Plan &P, cudaStream_t s, int lsort);

cudaError_t build_tree(Plan &P, const void *xyz, const void *q, cudaStream_t s) {
    const int64_t n = P.n;
    const int S = P.n_sys;
    if (P.sys_off_dev_h != P.sys_off_h) {
        KIFMM_CUDA_TRY(cudaMemcpyAsync(P.sys_off_d, P.sys_off_h.data(), sizeof(int64_t) * (S + 1),
                                       cudaMemcpyHostToDevice, s));
        P.sys_off_dev_h = P.sys_off_h;
    }
    ++g_launches, k_bbox_init<double><<<grid_for(S * 6, 128), 128, 0, s>>>(P.bbox_ord, S);
    const unsigned nt = grid_for(n, kTile);
    if (P.io_f64)
        ++g_launches, k_bbox<double><<<grid_for(n, kBboxTile), kBlock, 0, s>>>(n, (const double *)xyz,
                                             P.stokes ? nullptr : (const double *)q, P.sys_off_d, S,
                                             P.bbox_ord, P.status);
    else
        ++g_launches, k_bbox<float><<<grid_for(n, kBboxTile), kBlock, 0, s>>>(n, (const float *)xyz,
                                            P.stokes ? nullptr : (const float *)q, P.sys_off_d, S,
                                            P.bbox_ord, P.status);
    if (P.periodic) {
        // the root is the cell; the cell must be neutral
        ++g_launches, k_periodic_root<<<1, 32, 0, s>>>(P.cell, P.lo_side, P.key_scale, P.coef, P.out_scale,
                                                       P.inv_side_f);
        KIFMM_CUDA_TRY(cudaMemsetAsync(P.qsum, 0, 2 * sizeof(double), s));
        if (P.io_f64)
            ++g_launches, k_charge_sums<double><<<std::min<unsigned>(nt, 1024), 256, 0, s>>>(n, (const double *)q, P.qsum);
        else
            ++g_launches, k_charge_sums<float><<<std::min<unsigned>(nt, 1024), 256, 0, s>>>(n, (const float *)q, P.qsum);
        ++g_launches, k_charge_check<<<1, 32, 0, s>>>(P.qsum, P.io_f64 ? 1e-12 : 0x1p-24, P.status);
    } else {
        ++g_launches, k_bbox_final<<<grid_for(S, 128), 128, 0, s>>>(P.bbox_ord, S, P.lo_side, P.key_scale, P.coef,
                                                                    P.out_scale, P.inv_side_f);
    }
    if (P.io_f64)
        ++g_launches, k_keys<double><<<grid_for(n, 256), 256, 0, s>>>(n, (const double *)xyz, P.sys_off_d, S, P.lo_side,
                                                       P.key_scale, P.keys[0], P.vals[0], P.keys_user, P.cell);
    else
        ++g_launches, k_keys<float><<<grid_for(n, 256), 256, 0, s>>>(n, (const float *)xyz, P.sys_off_d, S, P.lo_side,
                                                      P.key_scale, P.keys[0], P.vals[0], P.keys_user, P.cell);
    KIFMM_CUDA_TRY(cudaGetLastError());
    // Sort only the key digits the octree will read: two levels below the
    // last tree's depth (or an estimate from N / M before the first tree),
    // capped by max_depth.  A node that must split below the sorted levels
    // sends the build back here for the remaining digits (a full stable sort
    // of the partly sorted keys: equal keys stay in caller order).
    int want = P.max_level > 0 ? P.max_level + 2
                               : (int)std::ceil(std::log((double)n / P.desc.leaf_cap + 1.0) / std::log(8.0)) + 2;
    want = std::max(1, std::min(want, P.desc.max_depth));
    int npass = 1;
    while (npass < 8 && levels_sorted(npass) < want) ++npass;
    for (;;) {
        int cur = 0;
        KIFMM_CUDA_TRY(radix_sort(P, n, s, cur, npass));
        if (cur != 0) {
            KIFMM_CUDA_TRY(cudaMemcpyAsync(P.keys[0], P.keys[1], sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
            KIFMM_CUDA_TRY(cudaMemcpyAsync(P.vals[0], P.vals[1], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        }
        cudaError_t e = build_levels(P, s, npass < 8 ? levels_sorted(npass) : kMaxLevel + 1);
        if (e == cudaErrorNotReady) {  // a node below the sorted levels must split
            npass = 8;
            continue;
        }
        KIFMM_CUDA_TRY(e);
        break;
    }
    P.sort_passes = npass;
    KIFMM_CUDA_TRY(cudaMemcpyAsync(P.perm, P.vals[0], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    return cudaGetLastError();  // the particle records follow once the leaves are listed
}

// Octree from sorted keys.  Nodes at level `lsort` cannot be split (their
// children's digit is not sorted): cudaErrorNotReady if one must.
//
// When the previous tree's level sizes are known, the levels it had are built
// at once (k_os_*: four launches, one synchronisation for the level
// boundaries); a deeper tree continues level by level from its last level.
// Otherwise each level needs its node count on the host (grid sizes,
// capacity, the end of the tree): a stream synchronisation per level.
static cudaError_t build_levels(Plan &P, cudaStream_t s, int lsort) {
    const int S = P.n_sys;
    const std::vector<int64_t> prev = P.level_start;  // the last build's level boundaries
    uint32_t *total_dev = P.scan_tmp + P.scan_tmp_elems - 1;
    // levels 1 .. lspec at once: every level the last tree had below its
    // roots, so that a tree of the same depth is complete at the one
    // synchronisation (a node at level lsort cannot be split from the sorted
    // digits).  The box arrays are sized for eight times twice the last
    // tree's level sizes; a tree that outgrows them is redone level by level.
    const int lspec = std::min((int)prev.size() - 1, lsort);
    const bool spec = lspec >= 2 && prev[1] == S;
    int64_t need = S;
    if (spec) {
        for (int l = 1; l < lspec; ++l) need += 8 * (2 * (prev[l + 1] - prev[l]) + 64);
        need += 8 * S;
        if (need > P.box_cap) {
            KIFMM_CUDA_TRY(grow_tree_arrays(P, need + 1024, 0));
            total_dev = P.scan_tmp + P.scan_tmp_elems - 1;
        }
    }
    bool spec_done = false;
    int64_t ls = 0, le = S;
    int level = 0;
    if (spec) {
        ++g_launches, k_roots<<<grid_for(S, 128), 128, 0, s>>>(S, P.sys_off_d, P.lvl, P.cx, P.cy, P.cz, P.first,
                                                                P.cnt, P.parent, P.sys);
        int64_t *lsd = P.spec_buf;  // lsd[l], lsd[l + 1]: level l's boxes
        const int64_t n = P.n;
        const int ntiles = (int)((n + kOsTile - 1) / kOsTile);
        const size_t need_cnt = 2 * (size_t)lspec * std::max(ntiles, 1);  // counts, then first indices
        if (need_cnt > P.os_cnt_elems) {
            P.os_cnt_elems = need_cnt;
            KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.os_cnt, sizeof(uint32_t) * P.os_cnt_elems));
        }
        const int M = P.desc.leaf_cap, D = P.desc.max_depth;
        if (ntiles > 0)
            ++g_launches, k_os_count<<<ntiles, kOsTile, 0, s>>>(n, P.keys[0], P.sys_off_d, S, lspec, M, D, ntiles,
                                                               P.os_cnt);
        uint32_t *first_idx = P.os_cnt + (size_t)lspec * std::max(ntiles, 1);
        ++g_launches, k_os_scan<<<1, 1024, 0, s>>>(lspec, ntiles, S, P.box_cap, P.os_cnt, first_idx, lsd,
                                                   P.spec_fail);
        if (ntiles > 0)
            ++g_launches, k_os_emit<<<ntiles, kOsTile, 0, s>>>(n, P.keys[0], P.sys_off_d, S, lspec, M, D, ntiles,
                                                              first_idx, P.spec_fail, P.lvl, P.cx, P.cy, P.cz,
                                                              P.first, P.cnt, P.sys);
        ++g_launches, k_os_link<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(need, 256),
                                                                                    (int64_t)P.num_sms * 8)),
                                  256, 0, s>>>(lsd, lspec, M, D, P.spec_fail, P.lvl, P.first, P.cnt, P.parent,
                                               P.child_first, P.nchild);
        KIFMM_CUDA_TRY(cudaGetLastError());
        std::vector<int64_t> lsh(lspec + 2);
        int fail = 0;
        KIFMM_CUDA_TRY(cudaMemcpyAsync(lsh.data(), lsd, sizeof(int64_t) * lsh.size(), cudaMemcpyDeviceToHost, s));
        KIFMM_CUDA_TRY(cudaMemcpyAsync(&fail, P.spec_fail, sizeof(int), cudaMemcpyDeviceToHost, s));
        KIFMM_CUDA_TRY(cudaStreamSynchronize(s));
        if (!fail) {
            // keep the non-empty levels; an empty one ends the tree
            int last = 0;
            while (last + 1 <= lspec && lsh[last + 2] > lsh[last + 1]) ++last;
            P.level_start.assign(lsh.begin(), lsh.begin() + last + 2);
            level = last;
            ls = lsh[last];
            le = lsh[last + 1];
            spec_done = (last < lspec);  // a level below lspec produced no children
            if (spec_done) {
                P.nb = le;
                P.max_level = level;
                return cudaGetLastError();
            }
        }
        if (fail) {
            level = 0;
            ls = 0;
            le = S;
        }
    }
    if (!spec || level == 0) {
        ++g_launches, k_roots<<<grid_for(S, 128), 128, 0, s>>>(S, P.sys_off_d, P.lvl, P.cx, P.cy, P.cz, P.first,
                                                                P.cnt, P.parent, P.sys);
        P.level_start.assign(1, 0);
        P.level_start.push_back(S);
    }
    while (true) {
        const int64_t m = le - ls;
        ++g_launches, k_split<<<grid_for(m, 4), 128, 0, s>>>(ls, le, level, P.desc.leaf_cap, P.desc.max_depth,
                                                             P.keys[0], P.first, P.cnt, P.tmp_nchild,
                                                             P.child_rng);
        uint32_t *scan_out = P.tmp_nchild + P.box_cap;
        KIFMM_CUDA_TRY(exclusive_scan_u32(P.tmp_nchild, scan_out, m, total_dev, P.scan_tmp,
                                          P.scan_tmp_elems - 1, s));
        uint32_t total = 0;
        KIFMM_CUDA_TRY(cudaMemcpyAsync(&total, total_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        KIFMM_CUDA_TRY(cudaStreamSynchronize(s));
        if (level >= lsort && total > 0) return cudaErrorNotReady;
        if (le + (int64_t)total > P.box_cap) {
            KIFMM_CUDA_TRY(grow_tree_arrays(P, 2 * (le + (int64_t)total) + 1024, le));
            scan_out = P.tmp_nchild + P.box_cap;
            total_dev = P.scan_tmp + P.scan_tmp_elems - 1;
            KIFMM_CUDA_TRY(exclusive_scan_u32(P.tmp_nchild, scan_out, m, total_dev, P.scan_tmp,
                                              P.scan_tmp_elems - 1, s));
        }
        ++g_launches, k_emit<<<grid_for(m, 128), 128, 0, s>>>(ls, le, P.tmp_nchild, scan_out, P.child_rng,
                                                              P.lvl, P.cx, P.cy, P.cz, P.first, P.cnt, P.parent,
                                                              P.child_first, P.nchild, P.sys, P.box_cap,
                                                              P.status);
        KIFMM_CUDA_TRY(cudaGetLastError());
        if (total == 0) break;
        ls = le;
        le = le + total;
        ++level;
        P.level_start.push_back(le);
    }
    P.nb = le;
    P.max_level = level;
    return cudaGetLastError();
}

cudaError_t check_leaves(Plan &P, const void *xyz, double skin, int *moved_dev, cudaStream_t s) {
    KIFMM_CUDA_TRY(cudaMemsetAsync(moved_dev, 0, sizeof(int), s));
    if (P.n_leaves == 0) return cudaSuccess;
    // the margin is skin half-widths of the finest level in the plan, so no
    // particle comes closer to any box of its lists than that box's own
    // surfaces allow for (a W-list box may be many levels finer than the leaf)
    const double margin = skin * ldexp(0.5, -P.max_level);
    const unsigned g = (unsigned)((P.n_leaves + 7) / 8);
    if (P.io_f64)
        ++g_launches, k_leaf_check<double><<<g, 256, 0, s>>>(P.n_leaves, P.leaves, P.first, P.cnt, P.lvl, P.cx,
                                                             P.cy, P.cz, P.sys, P.lo_side, P.perm,
                                                             (const double *)xyz, margin, moved_dev, P.cell);
    else
        ++g_launches, k_leaf_check<float><<<g, 256, 0, s>>>(P.n_leaves, P.leaves, P.first, P.cnt, P.lvl, P.cx,
                                                            P.cy, P.cz, P.sys, P.lo_side, P.perm,
                                                            (const float *)xyz, margin, moved_dev, P.cell);
    return cudaGetLastError();
}

// Stokeslet: the forces in sorted order, compute type; non-finite ones flagged.
template <typename TI, typename TC>
__global__ void k_gather_frc(int64_t n, const uint32_t *__restrict__ perm, const TI *__restrict__ f,
                             TC *__restrict__ frc, int *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    bool bad = false;
    for (int d = 0; d < 3; ++d) {
        const double v = (double)f[3 * (size_t)j + d];
        bad = bad || !isfinite(v);
        frc[3 * i + d] = (TC)v;
    }
    if (bad) set_status(status, KIFMM_ERR_NONFINITE);
}

// Leaf-relative particle records in the compute type (also used to refresh
// positions and charges with the tree frozen).
cudaError_t gather_particles(Plan &P, const void *xyz, const void *q_in, cudaStream_t s) {
    // Stokeslet plans: q_in holds forces [N][3], gathered on their own; the
    // records' weight is unused
    const void *q = P.stokes ? nullptr : q_in;
    if (P.stokes) {
        if (P.f64 && P.io_f64)
            ++g_launches, k_gather_frc<double, double><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, P.perm, (const double *)q_in, (double *)P.frc, P.status);
        else if (P.f64)
            ++g_launches, k_gather_frc<float, double><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, P.perm, (const float *)q_in, (double *)P.frc, P.status);
        else if (P.io_f64)
            ++g_launches, k_gather_frc<double, float><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, P.perm, (const double *)q_in, (float *)P.frc, P.status);
        else
            ++g_launches, k_gather_frc<float, float><<<grid_for(P.n, 256), 256, 0, s>>>(
                              P.n, P.perm, (const float *)q_in, (float *)P.frc, P.status);
    }
    P.fwd_valid = P.fwd_res_valid = false;  // new sources: the last evaluate's field no longer applies
    if (P.f64) {
        if (P.io_f64)
            ++g_launches, k_gather<double, double><<<grid_for(P.nb, 8), 256, 0, s>>>(
                P.nb, P.part_counts + 256, P.leaves, P.first, P.cnt, P.lvl, P.cx, P.cy, P.cz, P.sys, P.lo_side, P.perm,
                (const double *)xyz, (const double *)q, (double4 *)P.pts, P.cell, P.periodic ? P.leaf_q2 : nullptr, nullptr, nullptr);
        else
            ++g_launches, k_gather<float, double><<<grid_for(P.nb, 8), 256, 0, s>>>(
                P.nb, P.part_counts + 256, P.leaves, P.first, P.cnt, P.lvl, P.cx, P.cy, P.cz, P.sys, P.lo_side, P.perm,
                (const float *)xyz, (const float *)q, (double4 *)P.pts, P.cell, P.periodic ? P.leaf_q2 : nullptr, nullptr, nullptr);
    } else {
        if (P.io_f64)
            ++g_launches, k_gather<double, float><<<grid_for(P.nb, 8), 256, 0, s>>>(
                P.nb, P.part_counts + 256, P.leaves, P.first, P.cnt, P.lvl, P.cx, P.cy, P.cz, P.sys, P.lo_side, P.perm,
                (const double *)xyz, (const double *)q, (float4 *)P.pts, P.cell, P.periodic ? P.leaf_q2 : nullptr, nullptr, nullptr);
        else {
            if (!P.periodic)  // the FP32 path's leaf centres
                ++g_launches, k_leaf_centres<<<grid_for(3 * P.nb, 256), 256, 0, s>>>(
                    P.nb, P.part_counts + 256, P.leaves, P.lvl, P.cx, P.cy, P.cz, P.sys, P.lo_side, P.leaf_ctr);
            ++g_launches, k_gather<float, float><<<grid_for(P.nb, 8), 256, 0, s>>>(
                P.nb, P.part_counts + 256, P.leaves, P.first, P.cnt, P.lvl, P.cx, P.cy, P.cz, P.sys, P.lo_side, P.perm,
                (const float *)xyz, (const float *)q, (float4 *)P.pts, P.cell, P.periodic ? P.leaf_q2 : nullptr,
                P.leaf_ctr, P.inv_side_f);
        }
    }
    return cudaGetLastError();
}

// The list passes of one level, one warp per box: its colleagues and V list
// (one scan of the parent's colleagues' children), then its coarse adjacent
// leaves (which read its own colleagues), then its X list.  Everything else
// they read belongs to the previous level, so the passes need no grid-wide
// ordering.
__global__ void k_lists_level(int64_t ls, int64_t le, int level, int thr, const int32_t *__restrict__ parent,
                              const int32_t *__restrict__ child_first, const int32_t *__restrict__ nchild,
                              const int32_t *__restrict__ cnt, const int32_t *__restrict__ lvl,
                              const int32_t *__restrict__ cx, const int32_t *__restrict__ cy,
                              const int32_t *__restrict__ cz, int32_t *coll, int32_t *coarse, int32_t *ncoarse,
                              int32_t *vdense, int32_t *nv, int32_t *xdense, int32_t *nx,
                              unsigned long long *totals, int *status, ListShifts sh) {
    const int64_t b = ls + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    __shared__ unsigned long long blk_tot[2];
    if (threadIdx.x < 2) blk_tot[threadIdx.x] = 0;
    __syncthreads();
    if (b < le) {
        const int cntv =
            dev_colleagues_v(b, lane, level, parent, child_first, nchild, cx, cy, cz, coll, vdense, sh);
        __syncwarp();
        dev_coarse(b, lane, level, parent, nchild, lvl, cx, cy, cz, coll, coarse, ncoarse, status, sh);
        dev_x(b, lane, level, thr, cntv, parent, nchild, cnt, lvl, cx, cy, cz, coarse, ncoarse, nv, xdense, nx, sh);
        // V and X list totals: one global atomic per block, not per box (a
        // single address taking an atomic from every box serialises)
        if (lane == 0) {
            atomicAdd(&blk_tot[0], (unsigned long long)nv[b]);
            atomicAdd(&blk_tot[1], (unsigned long long)nx[b]);
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 && blk_tot[threadIdx.x]) atomicAdd(&totals[threadIdx.x], blk_tot[threadIdx.x]);
}

static ListShifts list_shifts(const Plan &P) {
    if (!P.periodic) return ListShifts{nullptr, nullptr, nullptr, nullptr, nullptr};
    return ListShifts{P.coll_sh, P.coarse_sh, P.x_sh, P.u_sh, P.w_sh};
}

cudaError_t build_lists(Plan &P, cudaStream_t s) {
    const int64_t nb = P.nb;
    KIFMM_CUDA_TRY(cudaMemsetAsync(P.coll, 0xFF, sizeof(int32_t) * kColl * nb, s));
    KIFMM_CUDA_TRY(cudaMemsetAsync(P.vdense, 0xFF, sizeof(int32_t) * kVSlots * nb, s));
    KIFMM_CUDA_TRY(cudaMemsetAsync(P.list_totals, 0, sizeof(unsigned long long) * 4, s));
    for (int l = 0; l <= P.max_level; ++l) {
        const int64_t ls = P.level_start[l], le = P.level_start[l + 1];
        const unsigned g = grid_for(le - ls, 8);  // warp per box, 8 per block
        ++g_launches, k_lists_level<<<g, 256, 0, s>>>(ls, le, l, P.direct_thr, P.parent, P.child_first, P.nchild,
                                                      P.cnt, P.lvl, P.cx, P.cy, P.cz, P.coll, P.coarse, P.ncoarse,
                                                      P.vdense, P.nv, P.xdense, P.nx, P.list_totals, P.status,
                                                      list_shifts(P));
        KIFMM_CUDA_TRY(cudaGetLastError());
    }
    const unsigned g = grid_for(nb, 128);
    ++g_launches, k_uw<<<g, 128, 0, s>>>(nb, 0, P.direct_thr, P.parent, P.cnt, P.child_first, P.nchild, P.lvl,
                                         P.cx, P.cy, P.cz, P.coll, P.coarse, P.ncoarse, P.u_cnt, P.w_cnt, nullptr,
                                         nullptr, nullptr, nullptr, 0, 0, P.status, list_shifts(P));
    // two scans, totals in the last two scratch words, then appended to the
    // offsets; the sizes come back to the host with set_sources' final
    // synchronisation (no round trip here: the fill pass writes only inside
    // the storage and flags a list that outgrew it)
    uint32_t *tot_u = P.scan_tmp + P.scan_tmp_elems - 1, *tot_w = P.scan_tmp + P.scan_tmp_elems - 2;
    KIFMM_CUDA_TRY(exclusive_scan_u32(P.u_cnt, P.u_ptr, nb, tot_u, P.scan_tmp, P.scan_tmp_elems - 2, s));
    KIFMM_CUDA_TRY(exclusive_scan_u32(P.w_cnt, P.w_ptr, nb, tot_w, P.scan_tmp, P.scan_tmp_elems - 2, s));
    KIFMM_CUDA_TRY(cudaMemcpyAsync(P.u_ptr + nb, tot_u, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    KIFMM_CUDA_TRY(cudaMemcpyAsync(P.w_ptr + nb, tot_w, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    KIFMM_CUDA_TRY(cudaMemcpyAsync(&P.rb->uw[0], tot_u, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    KIFMM_CUDA_TRY(cudaMemcpyAsync(&P.rb->uw[1], tot_w, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    KIFMM_CUDA_TRY(cudaMemcpyAsync(P.rb->vx, P.list_totals, sizeof(P.rb->vx), cudaMemcpyDeviceToHost, s));
    ++g_launches, k_uw<<<g, 128, 0, s>>>(nb, 1, P.direct_thr, P.parent, P.cnt, P.child_first, P.nchild, P.lvl,
                                         P.cx, P.cy, P.cz, P.coll, P.coarse, P.ncoarse, P.u_cnt, P.w_cnt, P.u_ptr,
                                         P.w_ptr, P.u_idx, P.w_idx, P.u_cap, P.w_cap, P.status, list_shifts(P));
    KIFMM_CUDA_TRY(cudaMemsetAsync(P.wsrc_flag, 0, sizeof(int32_t) * nb, s));
    if (P.w_cap > 0)
        ++g_launches, k_mark_w<<<grid_for(P.w_cap, 256), 256, 0, s>>>(P.w_cap, P.w_ptr + nb, P.w_idx, P.wsrc_flag);
    KIFMM_CUDA_TRY(cudaGetLastError());
    return cudaSuccess;
}

bool lists_finish(Plan &P) {
    P.n_u = P.rb->uw[0];
    P.n_w = P.rb->uw[1];
    P.n_v = (int64_t)P.rb->vx[0];
    P.n_x = (int64_t)P.rb->vx[1];
    return P.n_u <= P.u_cap && P.n_w <= P.w_cap;
}

cudaError_t grow_lists(Plan &P) {
    // grow the list storage (set_sources may allocate; evaluate never does)
    if (P.n_u > P.u_cap) {
        P.u_cap = P.n_u + P.n_u / 4 + 1024;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.u_idx, sizeof(int32_t) * P.u_cap));
        if (P.periodic) KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.u_sh, P.u_cap));
    }
    if (P.n_w > P.w_cap) {
        P.w_cap = P.n_w + P.n_w / 4 + 1024;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.w_idx, sizeof(int32_t) * P.w_cap));
        if (P.periodic) KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.w_sh, P.w_cap));
    }
    return cudaSuccess;
}

}  // namespace kifmm
