// M2L on the Blackwell tensor cores (tcgen05 / TMEM), mixed-precision modes.
//
// The V-list translations (Sec. 2.2: M2L between boxes in each other's far
// zone but not in their parents') are, for one octant class c of targets,
//     d(t) = sum_{s < 189} M_{off(c,s)} u(src(t, s))
// i.e. a sum over 189 slots of a [targets x K] x [K x N] product with gathered
// rows.  A CTA owns 128 targets of one class (one row each, M = 128) and all
// N = n_s check points (padded to a multiple of 16); the FP32 accumulator
// lives in TMEM (128 lanes x N columns).
//
// Precision (3xFP16): every operand x is split as x*sigma = hi + lo with hi,
// lo in FP16 and sigma a power of two (per tree level for the expansions, one
// for all operators); the product keeps hi*hi + hi*lo + lo*hi (the lo*lo term
// is below 2^-22 of the product) and the epilogue divides by sigma_A sigma_B.
//
// Pipeline (per CTA, 32 (PW + 9) threads, PW = 2 or 4 chosen by the tuner):
//   warps 0 .. PW-1  producers: cp.async (16 B, four threads per 64-byte
//              row) of the gathered A rows into a ring of shared-memory stages
//              laid out in the 64-byte swizzled K-major form; the slot's B
//              block (hi and lo halves adjacent) is stored in global memory
//              already in that form and arrives by one bulk (TMA) copy.
//              Completion is tracked by the stage's "full" mbarrier
//              (cp.async.mbarrier.arrive.noinc of the producer threads plus
//              the bulk copy's byte count).
//   warp PW    allocates TMEM; one thread issues tcgen05.mma for each stage
//              and frees the stage with tcgen05.commit on its "empty" barrier.
//   8 warps    drain: each V slot's partial accumulator is added in IEEE FP32
//              to running sums held in registers, then unscaled and stored.
// Every wait is bounded; on time-out the CTA records KIFMM_ERR_TIMEOUT, drains
// its own copies and MMAs (bounded), frees TMEM and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace kifmm {

namespace {

constexpr int kDrainWarps = 8;
// After a time-out the leader waits this many polls for its last bulk copy
// to land before the block's shared memory goes away (microseconds are
// enough; the barrier itself may never complete when other producers
// stopped before arriving).
constexpr long long kDrainPolls = 1LL << 18;
constexpr int kAccBufs = 3;         // per-slot partial accumulators in TMEM
constexpr int kKBlock = 32;         // FP16 elements per stage row (64 bytes)
constexpr int kRowBytes = 64;
// PW warps gather the A rows (each stage waits for their cp.async
// arrivals), then come the MMA warp and the drain warps.
constexpr int tc_threads(int pw, int tl) { return 32 * (pw + 1 + tl * kDrainWarps); }

struct TileArgs {
    const int32_t *targets;   // class-major target boxes
    const int4 *tiles;        // (class, begin, end, unused)
    const int32_t *vdense;    // [nb][189]
    const int *slot_off;      // [8][189]
    const __half *uh, *ul;    // [nb][kp] scaled expansions
    const __half *bhl;        // [316][kp/32][ncb][hi, lo][NT][32] scaled operators, K-block-major, 64-byte swizzled
    const int32_t *lvl;
    const float *level_unscale;  // 1 / (sigma_A(level) sigma_B)
    float *d;                 // [nb][ns]
    double *dbar;             // [nb] output column ns (the mean row), or nullptr
    int ns, kp, np, nstages;  // np: operator rows (output columns) incl. padding
    int ncb;                  // column blocks (np = ncb NT)
    long long wait_polls;     // bound of the pipeline's barrier waits (the clean-up waits keep kWaitIters)
    int *status;
};

// Byte offset of 16-byte chunk c of row r inside a 64-byte-swizzled tile.
__device__ __forceinline__ uint32_t swz64(int r, int c) {
    return (uint32_t)(r * kRowBytes + ((c ^ ((r >> 1) & 3)) << 4));
}

template <int NCH, int PW, int TL>
__global__ void __launch_bounds__(tc_threads(PW, TL), 1) k_m2l_tc(TileArgs a) {
    constexpr int NT = 32 * NCH;  // output columns of this CTA (MMA N)
    constexpr int kProdWarps = PW;
    constexpr int kRows = TL * kTcRows;  // target rows of the CTA: TL tiles of 128
    constexpr int kRowsPerThread = kRows / (8 * kProdWarps);
    constexpr int kMmaWarp = kProdWarps;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int kp = a.kp, NS = a.nstages;
    const int cb = blockIdx.y;  // column block: output columns [cb NT, (cb + 1) NT)
    const uint32_t a_bytes = kTcRows * kRowBytes;  // one tile, one of hi / lo
    const uint32_t b_bytes = (uint32_t)NT * kRowBytes;
    // stage: A hi, A lo of tile 0, (of tile 1,) then B hi, B lo; a multiple of 512
    const uint32_t stage_bytes = TL * 2 * a_bytes + 2 * b_bytes;
    __shared__ __align__(8) uint64_t full_bar[16], empty_bar[16], done_bar, accfull_bar[kAccBufs],
        accfree_bar[kAccBufs];
    __shared__ uint32_t tmem_base_s;
    __shared__ int32_t tgt_s[kRows];

    __shared__ volatile int abort_s;
    __shared__ volatile int abort_zero;  // never set: a wait on it runs to its bound

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 tile = a.tiles[blockIdx.x];
    const int cls = tile.x;
    // tiles holding targets (a CTA's second tile may be empty); uniform
    const int ntl = (TL == 2 && tile.z - tile.y > kTcRows) ? 2 : 1;
    if (threadIdx.x < kRows) {
        const int i = tile.y + threadIdx.x;
        tgt_s[threadIdx.x] = (i < tile.z) ? a.targets[i] : -1;
    }

    if (threadIdx.x == 0) {
        abort_s = 0;
        abort_zero = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 32 * kProdWarps + 1);  // producer cp.async arrivals + the bulk-copy leader
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        for (int b = 0; b < kAccBufs; ++b) {
            mbar_init(smem_u32(&accfull_bar[b]), 1);
            mbar_init(smem_u32(&accfree_bar[b]), kDrainWarps);  // lane 0 of each drain warp of one tile
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // TMEM columns: kAccBufs partial accumulators of NT columns each.
    constexpr uint32_t tmem_cols = (kAccBufs * NT <= 128) ? 128 : (kAccBufs * NT <= 256) ? 256 : 512;
    static_assert(kAccBufs * NT <= 512, "partial accumulators exceed TMEM");
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const int kblocks = kp / kKBlock;
    const int iters = kVSlots * kblocks;

    if (warp < kProdWarps) {
        // ---------------- producers ----------------
        // Thread t copies 16-byte chunk (t & 3) of rows (t >> 2) + 8 P i
        // (P producer warps), so each warp instruction reads eight whole
        // 64-byte rows; few producer threads keep the stage barrier's
        // arrival count low.  Row r belongs to tile r / 128.
        const int ch = threadIdx.x & 3, r0 = threadIdx.x >> 2;
        // row indices of the current and the next slot (the targets are
        // re-read from shared memory once per slot)
        int32_t src[kRowsPerThread], src_next[kRowsPerThread];
#pragma unroll
        for (int i = 0; i < kRowsPerThread; ++i) {
            const int32_t tg = tgt_s[r0 + 8 * kProdWarps * i];
            src[i] = -1;
            src_next[i] = (tg >= 0) ? a.vdense[(size_t)tg * kVSlots] : -1;
        }
        const bool leader = threadIdx.x == 0;
        int o_cur = 0, o_next = leader ? a.slot_off[cls * kVSlots] : 0, last_it = -1;
        for (int it = 0; it < iters; ++it) {
            const int stage = it % NS;
            const int s = it / kblocks, kb = it - s * kblocks;
            if (kb == 0) {
#pragma unroll
                for (int i = 0; i < kRowsPerThread; ++i) {
                    src[i] = src_next[i];
                    const int32_t tg = tgt_s[r0 + 8 * kProdWarps * i];
                    if (s + 1 < kVSlots) src_next[i] = (tg >= 0) ? a.vdense[(size_t)tg * kVSlots + s + 1] : -1;
                }
                if (leader) {
                    o_cur = o_next;
                    if (s + 1 < kVSlots) o_next = a.slot_off[cls * kVSlots + s + 1];
                }
            }
            if (!mbar_wait(smem_u32(&empty_bar[stage]), ((it / NS) & 1) ^ 1, &abort_s, a.wait_polls)) {
                set_status(a.status, KIFMM_ERR_TIMEOUT);
                abort_s = 1;
                break;
            }
            unsigned char *st = smem + (size_t)stage * stage_bytes;
            const uint32_t sA = smem_u32(st), sB = sA + TL * 2 * a_bytes;
            const uint32_t fb = smem_u32(&full_bar[stage]);
            if (leader) {
                // the hi and lo blocks of this (operator, K block, column
                // block) are adjacent in global and in shared memory: one copy
                const size_t boff = (((size_t)o_cur * kblocks + kb) * a.ncb + cb) * 2 * (size_t)NT * kKBlock;
                mbar_arrive_expect_tx(fb, 2 * b_bytes);
                bulk_g2s(sB, a.bhl + boff, 2 * b_bytes, fb);
                last_it = it;
            }
            const size_t koff = (size_t)kb * kKBlock + 8 * ch;
#pragma unroll
            for (int i = 0; i < kRowsPerThread; ++i) {
                const int r = r0 + 8 * kProdWarps * i;
                const int t = r / kTcRows, rr = r - t * kTcRows;
                const uint32_t tA = sA + (uint32_t)t * 2 * a_bytes;
                const size_t g = (size_t)(src[i] >= 0 ? src[i] : 0) * kp + koff;
                const uint32_t nbytes = (src[i] >= 0) ? 16u : 0u;
                cp_async16(tA + swz64(rr, ch), a.uh + g, nbytes);
                cp_async16(tA + a_bytes + swz64(rr, ch), a.ul + g, nbytes);
            }
            cp_async_arrive_noinc(fb);
        }
        cp_async_wait_all();
        if (leader && abort_s && last_it >= 0) {
            // the last bulk copy must land before the CTA's shared memory
            // goes away; the bounded wait outlasts it even when other
            // producers stopped before arriving on that stage
            (void)mbar_wait(smem_u32(&full_bar[last_it % NS]), (last_it / NS) & 1, &abort_zero, kDrainPolls);
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        // Partial accumulator u = s ntl + t (slot s, tile t) goes to buffer
        // u % kAccBufs (a fresh accumulator: the tensor core's FP32
        // accumulation rounds toward zero, so chains are kept to one slot
        // and summed by the drain warps in IEEE FP32).  Both tiles of a
        // stage read the same B block.
        if (lane == 0) {
            int it = 0;
            const uint32_t id = idesc_f16(NT);
            for (int s = 0; s < kVSlots && !abort_s; ++s) {
                uint32_t tacc[TL];
                bool ok = true;
                for (int t = 0; t < ntl; ++t) {
                    const int u = s * ntl + t, buf = u % kAccBufs;
                    if (u >= kAccBufs &&
                        !mbar_wait(smem_u32(&accfree_bar[buf]), ((u / kAccBufs) - 1) & 1, &abort_s, a.wait_polls)) {
                        ok = false;
                        break;
                    }
                    tacc[t] = tmem + (uint32_t)(buf * NT);
                }
                if (!ok) {
                    set_status(a.status, KIFMM_ERR_TIMEOUT);
                    abort_s = 1;
                    break;
                }
                tc_fence_after();
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int stage = it % NS;
                    if (!mbar_wait(smem_u32(&full_bar[stage]), (it / NS) & 1, &abort_s, a.wait_polls)) {
                        set_status(a.status, KIFMM_ERR_TIMEOUT);
                        abort_s = 1;
                        break;
                    }
                    fence_proxy_async();
                    tc_fence_after();
                    const uint32_t sA = smem_u32(smem + (size_t)stage * stage_bytes);
                    const uint32_t sB = sA + TL * 2 * a_bytes, sBl = sB + b_bytes;
                    for (int t = 0; t < ntl; ++t) {
                        const uint32_t tA = sA + (uint32_t)t * 2 * a_bytes, tAl = tA + a_bytes;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t dAh = sdesc_sw64(tA + 32 * kk), dAl = sdesc_sw64(tAl + 32 * kk);
                            const uint64_t dBh = sdesc_sw64(sB + 32 * kk);
                            const uint64_t dBl = sdesc_sw64(sBl + 32 * kk);
                            const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
                            // A_hi feeds two products: read once into the collector
                            mma_f16_fill(tacc[t], dAh, dBh, id, acc0);
                            mma_f16_lastuse(tacc[t], dAh, dBl, id, 1u);
                            mma_f16(tacc[t], dAl, dBh, id, 1u);
                        }
                    }
                    mma_commit(smem_u32(&empty_bar[stage]));
                }
                if (abort_s) break;
                for (int t = 0; t < ntl; ++t) mma_commit(smem_u32(&accfull_bar[(s * ntl + t) % kAccBufs]));
            }
            mma_commit(smem_u32(&done_bar));
        }
        __syncwarp();
    } else if (warp > kMmaWarp) {
        // ---------------- drain warps ----------------
        // kDrainWarps per tile.  Warp w may read TMEM lanes 32 (w % 4) ..
        // +31; two warps of a tile share each lane quadrant and split the NT
        // columns in halves.  The running sums stay in registers (IEEE FP32
        // adds of the per-slot partials).
        const int d = warp - kMmaWarp - 1;
        const int t = d / kDrainWarps;
        const int q = warp & 3, h = (d >> 2) & 1;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int c_base = h * (NT / 2);
        float acc[NT / 2];
#pragma unroll
        for (int j = 0; j < NT / 2; ++j) acc[j] = 0.f;
        bool ok = true;
        if (t < ntl) {
            for (int s = 0; s < kVSlots; ++s) {
                const int u = s * ntl + t, buf = u % kAccBufs;
                ok = mbar_wait(smem_u32(&accfull_bar[buf]), (u / kAccBufs) & 1, &abort_s, a.wait_polls);
                ok = __all_sync(0xffffffffu, ok);  // warp-uniform: tcgen05.ld is .sync.aligned
                if (!ok) {
                    set_status(a.status, KIFMM_ERR_TIMEOUT);
                    abort_s = 1;
                    break;
                }
                tc_fence_after();
                // (two tiles: eight columns per load, the running sums take
                // most of the registers)
                constexpr int LW = TL == 2 ? 8 : 16;
#pragma unroll
                for (int c = 0; c < NT / (2 * LW); ++c) {
                    float p[LW];
                    if constexpr (LW == 8)
                        tmem_ld8(tmem + lane_off + (uint32_t)(buf * NT + c_base + LW * c), p);
                    else
                        tmem_ld16(tmem + lane_off + (uint32_t)(buf * NT + c_base + LW * c), p);
#pragma unroll
                    for (int j = 0; j < LW; ++j) acc[LW * c + j] += p[j];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&accfree_bar[buf]));
            }
        }
        ok = ok && !abort_s && t < ntl;
        const int row = t * kTcRows + q * 32 + lane;
        const int32_t tb = tgt_s[row];
        if (ok && tb >= 0) {
            const float scale = a.level_unscale[a.lvl[tb]];
            const int col0 = cb * NT + c_base;
            float *out = a.d + (size_t)tb * a.ns + col0;
#pragma unroll
            for (int j = 0; j < NT / 2; ++j) {
                if (col0 + j < a.ns) out[j] = acc[j] * scale;
                else if (col0 + j == a.ns && a.dbar) a.dbar[tb] = (double)(acc[j] * scale);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        if (abort_s) {
            // bounded drain of in-flight MMAs (the done barrier completes when they do)
            for (long long i = 0; i < kWaitIters; ++i)
                if (mbar_try_wait(smem_u32(&done_bar), 0) || mbar_try_wait(smem_u32(&done_bar), 1)) break;
        }
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// max |u| per level, as float bits (non-negative floats order like integers).
// A warp per box; the block's maxima meet in shared memory first, so the
// few per-level words take one global atomic per block and level, not one
// per box.
__global__ void k_level_absmax(int64_t nb, int ns, const float *__restrict__ u, const int32_t *__restrict__ lvl,
                               unsigned *__restrict__ level_max) {
    __shared__ unsigned blk[kMaxLevel + 1];
    for (int l = threadIdx.x; l <= kMaxLevel; l += blockDim.x) blk[l] = 0u;
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (b < nb) {
        float m = 0.f;
        for (int k = threadIdx.x & 31; k < ns; k += 32) m = fmaxf(m, fabsf(u[(size_t)b * ns + k]));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&blk[lvl[b]], __float_as_uint(m));
    }
    __syncthreads();
    for (int l = threadIdx.x; l <= kMaxLevel; l += blockDim.x)
        if (blk[l]) atomicMax(&level_max[l], blk[l]);
}

__device__ __forceinline__ float pow2_scale_for(float maxabs) {
    if (!(maxabs > 0.f)) return 1.f;
    int e;
    frexpf(maxabs, &e);  // maxabs = m 2^e, m in [0.5, 1)
    return ldexpf(1.f, 14 - e);
}

__global__ void k_level_scale(int nlev, const unsigned *__restrict__ level_max, float sigma_b,
                              float *__restrict__ level_sigma, float *__restrict__ level_unscale) {
    const int l = threadIdx.x;
    if (l >= nlev) return;
    const float s = pow2_scale_for(__uint_as_float(level_max[l]));
    level_sigma[l] = s;
    level_unscale[l] = 1.f / (s * sigma_b);
}

// Compressed M2L projections: out[row][j] = sum_k in[row][k] M[j][k] for the
// rows listed in `rows` (all rows 0..nrows-1 when null).  M row-major
// [n_out][n_in].  A 64 x 64 output tile per block of 256 threads (4 x 4 per
// thread), K staged in shared memory 32 at a time.
__global__ void __launch_bounds__(256) k_rowmat(int64_t nrows, const int32_t *__restrict__ rows,
                                                const float *__restrict__ in, int ld_in, int n_in,
                                                const float *__restrict__ M, float *__restrict__ out, int ld_out,
                                                int n_out) {
    __shared__ float As[32][65], Bs[32][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < n_in; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 256) {
            const int r = e >> 5, k = e & 31;
            const int64_t rr = r0 + r;
            float v = 0.f;
            if (rr < nrows && k0 + k < n_in) {
                const int64_t row = rows ? rows[rr] : rr;
                v = in[row * ld_in + k0 + k];
            }
            As[k][r] = v;
            const int c = c0 + r;
            Bs[k][r] = (c < n_out && k0 + k < n_in) ? M[(size_t)c * n_in + k0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t rr = r0 + ty + 16 * i;
        if (rr >= nrows) continue;
        const int64_t row = rows ? rows[rr] : rr;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx + 16 * j;
            if (c < n_out) out[row * ld_out + c] = acc[i][j];
        }
    }
}

// hi/lo FP16 split of the scaled expansions, K padded with zeros; a warp per
// box (coalesced rows, no index division).
__global__ void k_split_u(int64_t nb, int ns, int kp, const float *__restrict__ u, const int32_t *__restrict__ lvl,
                          const float *__restrict__ level_sigma, __half *__restrict__ uh, __half *__restrict__ ul) {
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= nb) return;
    const float sg = level_sigma[lvl[b]];
    for (int k = threadIdx.x & 31; k < kp; k += 32) {
        const float x = (k < ns) ? u[(size_t)b * ns + k] * sg : 0.f;
        const __half h = __float2half_rn(x);
        uh[(size_t)b * kp + k] = h;
        ul[(size_t)b * kp + k] = __float2half_rn(x - __half2float(h));
    }
}

// Operator B[j][k] = M_o[j][k] (m2l_t is stored transposed, [o][k][ld], with
// the mean row as output j = ns when ld = ns + 1) split into FP16 hi/lo and
// stored K-block-major: block (o, kb, column block cb) holds the hi rows
// j = cb nt .. cb nt + nt - 1 and then the lo rows, 32 elements each, in the
// 64-byte swizzled K-major form (16-byte chunk c of row j at chunk position
// c ^ ((j >> 1) & 3)), so one linear copy of the block lands in shared memory
// ready for the tensor core.
__global__ void k_split_ops(int nops, int ns, int ld, int np, int nt, int kp, const float *__restrict__ m2l_t,
                            float sigma, __half *__restrict__ bhl) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nops * np * kp;
    if (idx >= total) return;
    const int kblocks = kp / kKBlock;
    const int64_t blk = idx / ((int64_t)np * kKBlock);  // o * kblocks + kb
    const int rem = (int)(idx - blk * np * kKBlock);
    const int o = (int)(blk / kblocks), kb = (int)(blk - (int64_t)o * kblocks);
    const int j = rem / kKBlock, pos = rem % kKBlock;   // pos: swizzled position in the row
    const int c = (pos >> 3) ^ ((j >> 1) & 3), e = pos & 7;
    const int k = kb * kKBlock + c * 8 + e;
    const float x = (j < ld && k < ns) ? m2l_t[((size_t)o * ns + k) * ld + j] * sigma : 0.f;
    const __half h = __float2half_rn(x);
    const int cb = j / nt, jj = j - cb * nt;
    const size_t out = ((size_t)blk * (np / nt) + cb) * 2 * (size_t)nt * kKBlock + (size_t)jj * kKBlock + pos;
    bhl[out] = h;
    bhl[out + (size_t)nt * kKBlock] = __float2half_rn(x - __half2float(h));
}

__global__ void k_absmax_f32(int64_t n, const float *__restrict__ x, unsigned *out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <int PW, int TL>
cudaError_t set_smem_attr_v(int nt, int bytes) {
    switch (nt) {
        case 32: return cudaFuncSetAttribute(k_m2l_tc<1, PW, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        case 64: return cudaFuncSetAttribute(k_m2l_tc<2, PW, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        case 96: return cudaFuncSetAttribute(k_m2l_tc<3, PW, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        case 128: return cudaFuncSetAttribute(k_m2l_tc<4, PW, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        case 160: return cudaFuncSetAttribute(k_m2l_tc<5, PW, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        default: return cudaErrorNotSupported;
    }
}
cudaError_t set_smem_attr(int nt, int bytes) {
    KIFMM_CUDA_TRY((set_smem_attr_v<2, 1>(nt, bytes)));
    KIFMM_CUDA_TRY((set_smem_attr_v<4, 1>(nt, bytes)));
    return set_smem_attr_v<2, 2>(nt, bytes);
}

// Kernel variants the tuner chooses between: (producer warps, tiles per
// CTA).  Two tiles take 608 threads and 96 registers, so two producer warps.
constexpr int kVariants[3][2] = {{2, 1}, {4, 1}, {2, 2}};

}  // namespace

struct TcState {
    int np = 0, kp = 0, nstages = 0;
    int nt = 0, ncb = 0;      // output columns per CTA (MMA N), column blocks (np = nt ncb)
    float sigma_b = 1.f;
    int pw = 2;               // producer warps
    int tl = 1;               // target tiles (of 128) per CTA, sharing each B block
    int n_tiles[2] = {0, 0};  // CTAs (entries of tiles) for 1 and 2 tiles per CTA
    size_t stage_bytes(int t) const { return (size_t)t * 2 * kTcRows * kRowBytes + 2 * (size_t)nt * kRowBytes; }
    int nstages_max(int t) const { return (int)std::min<size_t>(16, (227 * 1024 - 4096) / stage_bytes(t)); }
    __half *bhl = nullptr;    // operators, hi and lo blocks interleaved per (o, kb, cb)
    __half *uh = nullptr, *ul = nullptr;
    int64_t u_cap = 0;
    unsigned *level_max = nullptr;
    float *level_sigma = nullptr, *level_unscale = nullptr;
    int4 *tiles = nullptr;
    int64_t tiles_cap = 0;
    std::vector<int4> tiles_h;
    size_t smem = 0;
    int n_in = 0, n_out = 0, ld = 0;  // operator inputs, outputs (mean excluded), stored columns
    int4 *tiles_pin = nullptr;        // pinned staging of tiles_h (a pageable copy stalls the stream)
    size_t tiles_pin_cap = 0;
    cudaEvent_t tiles_copied = nullptr;  // the last upload from tiles_pin
    ~TcState() {
        if (tiles_copied) {
            cudaEventSynchronize(tiles_copied);
            cudaEventDestroy(tiles_copied);
        }
        if (tiles_pin) cudaFreeHost(tiles_pin);
    }
};

static TcState &tc_state(Plan &P) {
    if (!P.m2l_tc) P.m2l_tc = new TcState();
    return *(TcState *)P.m2l_tc;
}

int m2l_tensor_stages(const Plan &P) { return P.m2l_tc ? ((const TcState *)P.m2l_tc)->nstages : 0; }
int m2l_tensor_producers(const Plan &P) { return P.m2l_tc ? ((const TcState *)P.m2l_tc)->pw : 0; }
int m2l_tensor_tiles_per_cta(const Plan &P) { return P.m2l_tc ? ((const TcState *)P.m2l_tc)->tl : 0; }

bool m2l_tensor_pin(Plan &P, int producers, int tiles, int stages) {
    if (!P.m2l_tc) return false;
    TcState &S = *(TcState *)P.m2l_tc;
    bool known = false;
    for (const auto &v : kVariants) known = known || (v[0] == producers && v[1] == tiles);
    if (!known || stages < 2 || stages > S.nstages_max(tiles)) return false;
    S.pw = producers;
    S.tl = tiles;
    S.nstages = stages;
    P.tuned_m2l = true;
    return true;
}

void m2l_tensor_release(Plan &P) {
    if (P.m2l_tc) {
        delete (TcState *)P.m2l_tc;
        P.m2l_tc = nullptr;
    }
}

// Plan time: FP16 hi/lo operators with one power-of-two scale.
cudaError_t m2l_tensor_setup(Plan &P) {
    TcState &S = tc_state(P);
    // Dense: u (ns values) -> d (ns values + the mean row).  Compressed: the
    // rr-value projection of u -> rl values + the mean row.
    const bool comp = P.m2l_rl > 0;
    const float *ops = comp ? P.m2l_c : (const float *)P.m2l_t;
    S.n_in = comp ? P.m2l_rr : P.ns;
    S.n_out = comp ? P.m2l_rl : P.ns;
    S.ld = comp ? P.m2l_rl + 1 : P.op_ld;
    // Output columns per CTA: at most 160 (three partial accumulators fit
    // TMEM; the drain warps keep 80 running sums each in registers); larger
    // surfaces (p >= 7) are split into column blocks over blockIdx.y.
    const int np0 = round_up(S.n_out + 1, 32);  // room for the mean row (FP32-based modes)
    S.ncb = (np0 + 159) / 160;
    S.nt = round_up((np0 + S.ncb - 1) / S.ncb, 32);
    S.np = S.nt * S.ncb;
    S.kp = round_up(S.n_in, kKBlock);
    if (S.nt > 160 || S.nstages_max(2) < 2) return cudaErrorNotSupported;
    S.tl = 1;
    S.nstages = S.nstages_max(1);
    S.smem = (size_t)S.nstages_max(1) * S.stage_bytes(1) + 1024;  // the largest any variant takes
    unsigned *dmax = nullptr;
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&dmax, sizeof(unsigned)));
    KIFMM_CUDA_TRY(cudaMemset(dmax, 0, sizeof(unsigned)));
    const int64_t nm = (int64_t)kNumM2L * S.n_in * S.ld;
    ++g_launches, k_absmax_f32<<<256, 256>>>(nm, ops, dmax);
    unsigned mbits = 0;
    KIFMM_CUDA_TRY(cudaMemcpy(&mbits, dmax, sizeof(unsigned), cudaMemcpyDeviceToHost));
    float mx;
    memcpy(&mx, &mbits, sizeof(float));
    int e = 0;
    std::frexp(mx, &e);
    S.sigma_b = std::ldexp(1.0f, 14 - e);
    const size_t nb = (size_t)kNumM2L * S.np * S.kp;
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&S.bhl, 2 * sizeof(__half) * nb));
    ++g_launches, k_split_ops<<<(unsigned)((nb + 255) / 256), 256>>>(kNumM2L, S.n_in, S.ld, S.np, S.nt, S.kp, ops,
                                                                     S.sigma_b, S.bhl);
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&S.level_max, sizeof(unsigned) * 32));
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&S.level_sigma, sizeof(float) * 32));
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&S.level_unscale, sizeof(float) * 32));
    KIFMM_CUDA_TRY(set_smem_attr(S.nt, (int)S.smem));
    return cudaDeviceSynchronize();
}

// After set_sources: tiles of 128 targets within each octant class (one per
// CTA), then tiles of 256 (two per CTA, the second possibly short or empty).
cudaError_t m2l_tensor_tiles(Plan &P, cudaStream_t s) {
    TcState &S = tc_state(P);
    S.tiles_h.clear();
    for (int t = 1; t <= 2; ++t) {
        const int64_t rows = (int64_t)t * kTcRows;
        for (int c = 0; c < 8; ++c)
            for (int64_t b = P.m2l_class_start[c]; b < P.m2l_class_start[c + 1]; b += rows)
                S.tiles_h.push_back(make_int4(c, (int)b, (int)std::min<int64_t>(b + rows, P.m2l_class_start[c + 1]), 0));
        S.n_tiles[t - 1] = (int)S.tiles_h.size() - (t == 2 ? S.n_tiles[0] : 0);
    }
    if ((int64_t)S.tiles_h.size() > S.tiles_cap) {
        S.tiles_cap = (int64_t)S.tiles_h.size() + 64;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&S.tiles, sizeof(int4) * S.tiles_cap));
    }
    // the staging buffer may still feed the previous upload (set_sources on
    // another stream)
    if (S.tiles_copied) KIFMM_CUDA_TRY(cudaEventSynchronize(S.tiles_copied));
    else KIFMM_CUDA_TRY(cudaEventCreateWithFlags(&S.tiles_copied, cudaEventDisableTiming));
    if (S.tiles_h.size() > S.tiles_pin_cap) {
        if (S.tiles_pin) cudaFreeHost(S.tiles_pin);
        S.tiles_pin = nullptr;
        S.tiles_pin_cap = 0;
        KIFMM_CUDA_TRY(cudaMallocHost((void **)&S.tiles_pin, sizeof(int4) * (S.tiles_h.size() + 64)));
        S.tiles_pin_cap = S.tiles_h.size() + 64;
    }
    std::copy(S.tiles_h.begin(), S.tiles_h.end(), S.tiles_pin);
    if (!S.tiles_h.empty()) {
        KIFMM_CUDA_TRY(cudaMemcpyAsync(S.tiles, S.tiles_pin, sizeof(int4) * S.tiles_h.size(),
                                       cudaMemcpyHostToDevice, s));
        KIFMM_CUDA_TRY(cudaEventRecord(S.tiles_copied, s));
    }
    if (P.nb > S.u_cap) {
        S.u_cap = P.list_cap;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&S.uh, sizeof(__half) * S.u_cap * S.kp));
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&S.ul, sizeof(__half) * S.u_cap * S.kp));
    }
    return cudaGetLastError();
}

cudaError_t m2l_tensor(Plan &P, cudaStream_t s) {
    TcState &S = tc_state(P);
    if (S.tiles_h.empty()) return cudaSuccess;  // no V-list targets
    const int nlev = P.max_level + 1;
    const bool comp = P.m2l_rl > 0;
    const float *u = (const float *)P.u_chk;
    if (comp) {  // project every box's check potential onto the right basis
        ++g_launches, k_rowmat<<<dim3((unsigned)((P.nb + 63) / 64), (unsigned)((S.n_in + 63) / 64)), 256, 0, s>>>(
            P.nb, nullptr, u, P.ns, P.ns, P.m2l_wc, (float *)P.u_c, S.n_in, S.n_in);
        u = (const float *)P.u_c;
    }
    KIFMM_CUDA_TRY(cudaMemsetAsync(S.level_max, 0, sizeof(unsigned) * 32, s));
    ++g_launches, k_level_absmax<<<(unsigned)((P.nb + 7) / 8), 256, 0, s>>>(P.nb, S.n_in, u, P.lvl, S.level_max);
    ++g_launches, k_level_scale<<<1, 32, 0, s>>>(nlev, S.level_max, S.sigma_b, S.level_sigma, S.level_unscale);
    ++g_launches, k_split_u<<<(unsigned)((P.nb + 7) / 8), 256, 0, s>>>(P.nb, S.n_in, S.kp, u, P.lvl,
                                                                       S.level_sigma, S.uh, S.ul);
    TileArgs a;
    a.targets = P.m2l_targets;
    a.tiles = S.tiles;
    a.vdense = P.vdense;
    a.slot_off = P.slot_off;
    a.uh = S.uh;
    a.ul = S.ul;
    a.bhl = S.bhl;
    a.ncb = S.ncb;
    a.wait_polls = P.m2l_wait_polls > 0 ? P.m2l_wait_polls : kWaitIters;
    a.lvl = P.lvl;
    a.level_unscale = S.level_unscale;
    a.d = comp ? (float *)P.d_c : (float *)P.d_chk;
    a.dbar = (S.ld > S.n_out) ? P.dbar : nullptr;
    a.ns = S.n_out;
    a.kp = S.kp;
    a.np = S.np;
    a.status = P.status;
    auto launch_v = [&](auto pwc, auto tlc, int nst) -> cudaError_t {
        constexpr int PW = decltype(pwc)::value, TL = decltype(tlc)::value;
        const int n = S.n_tiles[TL - 1];
        if (n == 0) return cudaSuccess;
        a.nstages = nst;
        a.tiles = S.tiles + (TL == 2 ? S.n_tiles[0] : 0);
        const dim3 grid((unsigned)n, (unsigned)S.ncb);
        const size_t smem = (size_t)nst * S.stage_bytes(TL) + 1024;
        const int thr = tc_threads(PW, TL);
        switch (S.nt) {
            case 32: ++g_launches, k_m2l_tc<1, PW, TL><<<grid, thr, smem, s>>>(a); break;
            case 64: ++g_launches, k_m2l_tc<2, PW, TL><<<grid, thr, smem, s>>>(a); break;
            case 96: ++g_launches, k_m2l_tc<3, PW, TL><<<grid, thr, smem, s>>>(a); break;
            case 128: ++g_launches, k_m2l_tc<4, PW, TL><<<grid, thr, smem, s>>>(a); break;
            case 160: ++g_launches, k_m2l_tc<5, PW, TL><<<grid, thr, smem, s>>>(a); break;
            default: return cudaErrorNotSupported;
        }
        return cudaGetLastError();
    };
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    using I1 = std::integral_constant<int, 1>;
    auto launch_with = [&](int pw, int tl, int nst) -> cudaError_t {
        if (tl == 2) return launch_v(I2{}, I2{}, nst);
        return pw == 4 ? launch_v(I4{}, I1{}, nst) : launch_v(I2{}, I1{}, nst);
    };
    if (!P.tuned_m2l) {
        // untuned: two tiles per CTA (each operator block read once for 256
        // targets) when that still gives every SM a CTA, else one
        const bool two = S.n_tiles[1] >= P.num_sms;
        S.pw = 2;
        S.tl = two ? 2 : 1;
        S.nstages = two ? std::min(3, S.nstages_max(2)) : S.nstages_max(1);
    }
    if (!P.tuned_m2l && tuning_wanted(P, s)) {
        // producer warps x tiles per CTA x pipeline depth (2 .. the
        // shared-memory maximum, at most five depths)
        float best = 1e30f;
        int pick = S.nstages, pick_pw = S.pw, pick_tl = S.tl;
        KIFMM_CUDA_TRY(launch_with(S.pw, S.tl, S.nstages));  // warm the caches first
        for (const auto &v : kVariants) {
            const int mx = S.nstages_max(v[1]);
            for (int nst = mx; nst >= std::max(2, mx - 4); --nst) {
                cudaError_t e = cudaSuccess;
                float ms = 1e30f;
                for (int rep = 0; rep < 2; ++rep)  // best of two
                    ms = std::min(ms, time_launch(s, [&] { e = launch_with(v[0], v[1], nst); }));
                KIFMM_CUDA_TRY(e);
                if (ms < best) {
                    best = ms;
                    pick = nst;
                    pick_pw = v[0];
                    pick_tl = v[1];
                }
            }
        }
        S.nstages = pick;
        S.pw = pick_pw;
        S.tl = pick_tl;
        P.tuned_m2l = true;
    }
    KIFMM_CUDA_TRY(launch_with(S.pw, S.tl, S.nstages));
    if (comp) {  // back to the mean-free check potential of every target
        const int64_t nt = P.m2l_class_start[8];
        ++g_launches, k_rowmat<<<dim3((unsigned)((nt + 63) / 64), (unsigned)((P.ns + 63) / 64)), 256, 0, s>>>(
            nt, P.m2l_targets, (const float *)P.d_c, S.n_out, S.n_out, P.m2l_ul, (float *)P.d_chk, P.ns, P.ns);
    }
    return cudaGetLastError();
}

}  // namespace kifmm
