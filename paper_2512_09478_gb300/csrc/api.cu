// C ABI of the KIFMM library: plan lifecycle, argument validation, workspace
// management, orchestration of the tree build and of the evaluation passes,
// and host-side introspection for tests.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.h"

using kifmm::Plan;

struct kifmm_plan {
    Plan P;
};

namespace kifmm {

thread_local long long g_launches = 0;

void stage_begin(Plan &P, int stage, cudaStream_t s) {
    if (!P.prof) return;
    if (P.ev_used + 2 > P.ev_pool.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            P.ev_pool.push_back(e);
        }
    }
    const int i = (int)P.ev_used;
    P.ev_used += 2;
    cudaEventRecord(P.ev_pool[i], s);
    P.ev_pending.push_back({stage, i});
}

void stage_end(Plan &P, int stage, cudaStream_t s) {
    if (!P.prof) return;
    for (auto it = P.ev_pending.rbegin(); it != P.ev_pending.rend(); ++it)
        if (it->first == stage) {
            cudaEventRecord(P.ev_pool[it->second + 1], s);
            return;
        }
}

static cudaError_t profile_collect(Plan &P) {
    for (const auto &pe : P.ev_pending) {
        KIFMM_CUDA_TRY(cudaEventSynchronize(P.ev_pool[pe.second + 1]));
        float ms = 0.f;
        KIFMM_CUDA_TRY(cudaEventElapsedTime(&ms, P.ev_pool[pe.second], P.ev_pool[pe.second + 1]));
        P.prof_ms[pe.first] += ms;
        P.prof_calls[pe.first] += 1;
    }
    P.ev_pending.clear();
    P.ev_used = 0;
    return cudaSuccess;
}

LeafTiling leaf_tiling_candidate(int c) {
    // variants: 0 = (1, 4), 1 = (2, 4), 2 = (1, 2), 3 = (2, 2), 4 = (1, 1), 5 = (2, 1) as (TPL, G)
    static const int fam[kLeafTilingCandidates][6] = {
        {0, 1, 4, 4, 4, 4}, {0, 2, 4, 4, 4, 5}, {0, 1, 3, 3, 5, 5},
        {0, 1, 4, 4, 5, 5}, {4, 4, 4, 4, 4, 4}, {2, 2, 4, 4, 4, 4},
        {0, 2, 2, 4, 4, 4}, {0, 1, 2, 4, 4, 4}};
    LeafTiling t{};
    for (int i = 0; i < kLeafBuckets; ++i) t.set(i, fam[c][i < 4 ? i : (i < 8 ? 4 : 5)]);
    return t;
}

bool tuning_wanted(const Plan &P, cudaStream_t s) {
    if (!P.desc.autotune) return false;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st == cudaStreamCaptureStatusNone;
}

cudaError_t plan_alloc(Plan &P, void **ptr, size_t bytes) {
    if (*ptr) {
        for (auto it = P.owned.begin(); it != P.owned.end(); ++it)
            if (it->ptr == *ptr) {
                cudaFree(it->ptr);
                P.owned.erase(it);
                break;
            }
        *ptr = nullptr;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) return e;
    P.owned.push_back({p, bytes});
    *ptr = p;
    return cudaSuccess;
}

cudaError_t plan_grow(Plan &P, void **ptr, size_t bytes, size_t keep_bytes) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) return e;
    if (*ptr && keep_bytes) {
        e = cudaMemcpy(p, *ptr, keep_bytes, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) {
            cudaFree(p);
            return e;
        }
    }
    if (*ptr) {
        for (auto it = P.owned.begin(); it != P.owned.end(); ++it)
            if (it->ptr == *ptr) {
                cudaFree(it->ptr);
                P.owned.erase(it);
                break;
            }
    }
    P.owned.push_back({p, bytes});
    *ptr = p;
    return cudaSuccess;
}

// Per-node arrays used while the octree is built.
cudaError_t grow_tree_arrays(Plan &P, int64_t cap, int64_t keep) {
    KIFMM_CUDA_TRY(cudaDeviceSynchronize());
    int32_t **arrs[] = {&P.lvl, &P.cx, &P.cy, &P.cz, &P.first, &P.cnt, &P.parent, &P.child_first, &P.nchild, &P.sys};
    for (int32_t **a : arrs)
        KIFMM_CUDA_TRY(plan_grow(P, (void **)a, sizeof(int32_t) * cap, sizeof(int32_t) * keep));
    KIFMM_CUDA_TRY(plan_grow(P, (void **)&P.tmp_nchild, sizeof(uint32_t) * 2 * cap, sizeof(uint32_t) * keep));
    KIFMM_CUDA_TRY(plan_grow(P, (void **)&P.child_rng, sizeof(int32_t) * 16 * cap, sizeof(int32_t) * 16 * keep));
    P.box_cap = cap;
    const size_t need = scan_tmp_needed(2 * cap) + 8;
    if (need > P.scan_tmp_elems) {
        P.scan_tmp_elems = need;
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.scan_tmp, sizeof(uint32_t) * need));
    }
    return cudaSuccess;
}

// Per-box arrays sized after the tree is known.
static cudaError_t ensure_box_arrays(Plan &P) {
    if (P.nb <= P.list_cap) return cudaSuccess;
    const int64_t cap = P.nb + P.nb / 4 + 256;
    const size_t esz = P.f64 ? sizeof(double) : sizeof(float);
    struct A { void **p; size_t bytes; };
    const A arrs[] = {
        {(void **)&P.coll, sizeof(int32_t) * kColl * cap},
        {(void **)&P.coarse, sizeof(int32_t) * kMaxCoarse * cap},
        {(void **)&P.ncoarse, sizeof(int32_t) * cap},
        {(void **)&P.vdense, sizeof(int32_t) * kVSlots * cap},
        {(void **)&P.nv, sizeof(int32_t) * cap},
        {(void **)&P.xdense, sizeof(int32_t) * kMaxCoarse * cap},
        {(void **)&P.nx, sizeof(int32_t) * cap},
        {(void **)&P.u_ptr, sizeof(uint32_t) * (cap + 1)},
        {(void **)&P.w_ptr, sizeof(uint32_t) * (cap + 1)},
        {(void **)&P.u_cnt, sizeof(uint32_t) * cap},
        {(void **)&P.w_cnt, sizeof(uint32_t) * cap},
        {(void **)&P.part_list[0], sizeof(int32_t) * cap},
        {(void **)&P.part_list[1], sizeof(int32_t) * cap},
        {(void **)&P.part_list[2], sizeof(int32_t) * cap},
        {(void **)&P.part_list[3], sizeof(int32_t) * cap},
        {(void **)&P.child8, sizeof(int32_t) * 8 * cap},
        {(void **)&P.wsrc_flag, sizeof(int32_t) * cap},
        {(void **)&P.leaf_ctr, sizeof(float2) * 3 * cap},
        {&P.u_chk, esz * P.ns * cap},
        {&P.d_chk, esz * P.ns * cap},
        {&P.up_dens, esz * P.ns * cap},
        {&P.tmp_chk, esz * P.ns * cap},
        {&P.dn_dens, esz * P.ns * cap},
        {&P.adj_e1, esz * P.ns * cap},
        {&P.adj_e2, esz * P.ns * cap},
        {(void **)&P.dbar, sizeof(double) * cap},
        {&P.u_c, sizeof(float) * (size_t)P.m2l_rr * cap},
        {&P.d_c, sizeof(float) * (size_t)P.m2l_rl * cap},
        {(void **)&P.leaf_vlist, sizeof(int2) * kLeafTiles * (cap + P.desc.n_max / 8 + 64)},
        {(void **)&P.leaf_vcnt, sizeof(int32_t) * 16},
    };
    for (const A &a : arrs) KIFMM_CUDA_TRY(plan_alloc(P, a.p, a.bytes));
    if (P.periodic) {
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.coll_sh, (size_t)kColl * cap));
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.coarse_sh, (size_t)kMaxCoarse * cap));
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.x_sh, (size_t)kMaxCoarse * cap));
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.leaf_q2, sizeof(double) * cap));
    }
    P.list_cap = cap;
    P.leaf_item_cap = cap + P.desc.n_max / 8 + 64;
    return cudaSuccess;
}


}  // namespace kifmm

using namespace kifmm;

static kifmm_status from_cuda(cudaError_t e) {
    return e == cudaSuccess ? KIFMM_OK : KIFMM_ERR_CUDA;
}

#define API_CUDA(expr)                          \
    do {                                        \
        cudaError_t e_ = (expr);                \
        if (e_ != cudaSuccess) {                \
            (void)cudaGetLastError();           \
            return KIFMM_ERR_CUDA;              \
        }                                       \
    } while (0)

extern "C" {

static kifmm_status set_sources_impl(Plan &P, const void *xyz, const void *q, cudaStream_t s);

const char *kifmm_status_string(kifmm_status s) {
    switch (s) {
        case KIFMM_OK: return "ok";
        case KIFMM_ERR_ARG: return "invalid argument";
        case KIFMM_ERR_CAPACITY: return "capacity exceeded";
        case KIFMM_ERR_CUDA: return "CUDA runtime error";
        case KIFMM_ERR_NONFINITE: return "non-finite position or charge";
        case KIFMM_ERR_TIMEOUT: return "device wait timed out";
        case KIFMM_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

kifmm_status kifmm_lr_stride(double k_dem, double k_lr, int64_t *stride) {
    if (!stride || !(k_dem > 0.0) || !(k_lr > 0.0) || !std::isfinite(k_dem) || !std::isfinite(k_lr))
        return KIFMM_ERR_ARG;
    const double r = std::sqrt(k_dem / k_lr);  // may overflow to inf for extreme ratios
    *stride = (r >= 9.0e18) ? (int64_t)9000000000000000000LL : std::max<int64_t>(1, (int64_t)std::floor(r));
    return KIFMM_OK;
}

kifmm_status kifmm_plan_create(const kifmm_plan_desc *desc, kifmm_plan **out) {
    if (!desc || !out) return KIFMM_ERR_ARG;
    *out = nullptr;
    const kifmm_plan_desc &d = *desc;
    if (d.p < 2 || d.p > 10 || d.leaf_cap < 1 || d.max_depth < 1 || d.max_depth > kMaxLevel) return KIFMM_ERR_ARG;
    if (d.precision != KIFMM_FP64 && d.precision != KIFMM_FP32 && d.precision != KIFMM_MIXED_FP16)
        return KIFMM_ERR_ARG;
    if (d.n_max < 1 || d.n_max > (int64_t)0x7fffffff || d.n_systems_max < 1) return KIFMM_ERR_ARG;
    if (d.dtype != KIFMM_DTYPE_F32 && d.dtype != KIFMM_DTYPE_F64) return KIFMM_ERR_ARG;
    if (!(d.pinv_eps >= 0.0) || d.pinv_eps >= 1.0) return KIFMM_ERR_ARG;
    if (!(d.m2l_eps >= 0.0) || d.m2l_eps >= 1.0) return KIFMM_ERR_ARG;
    if (d.m2l_eps > 0.0 && d.precision != KIFMM_MIXED_FP16) return KIFMM_ERR_ARG;
    if (!(d.cell >= 0.0) || !std::isfinite(d.cell)) return KIFMM_ERR_ARG;
    if (d.kernel != KIFMM_KERNEL_LAPLACE && d.kernel != KIFMM_KERNEL_STOKESLET) return KIFMM_ERR_ARG;
    if (d.reuse_lists != 0 && d.reuse_lists != 1) return KIFMM_ERR_ARG;
    if (d.kernel == KIFMM_KERNEL_STOKESLET &&
        (d.precision == KIFMM_MIXED_FP16 || d.m2l_eps != 0.0 || d.cell != 0.0 || d.p > 8))
        return KIFMM_ERR_ARG;
    if (d.cell > 0.0 && d.n_systems_max != 1) return KIFMM_ERR_ARG;  // one periodic cell per plan
    kifmm_plan *pl = new (std::nothrow) kifmm_plan();
    if (!pl) return KIFMM_ERR_CUDA;
    Plan &P = pl->P;
    P.desc = d;
    P.p = d.p;
    P.nsurf = 6 * (d.p - 1) * (d.p - 1) + 2;
    P.stokes = d.kernel == KIFMM_KERNEL_STOKESLET;
    P.ns = P.stokes ? 3 * P.nsurf : P.nsurf;
    P.f64 = (d.precision == KIFMM_FP64);
    P.io_f64 = (d.dtype == KIFMM_DTYPE_F64);
    P.coef = (d.coef == 0.0) ? 1.0 : d.coef;
    // FP32 arithmetic cannot resolve the modes below ~1e-9 sigma_max: keeping
    // them only inflates the composite operators (at p = 8 their entries grow
    // ~30x and so does the FP32 rounding of every translation).
    P.eps = (d.pinv_eps != 0.0) ? d.pinv_eps : (P.f64 ? 1e-12 : 1e-9);
    P.direct_thr = (d.direct_max < 0) ? -1 : (d.direct_max == 0 ? P.nsurf : d.direct_max);
    P.leaf_tile = leaf_tiling_candidate(0);
    P.periodic = d.cell > 0.0;
    P.cell = d.cell;
    auto fail = [&](kifmm_status st) {
        kifmm_plan_destroy(pl);
        (void)cudaGetLastError();
        return st;
    };
    if (cudaGetDevice(&P.device) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, P.device);
    std::string err;
    cudaError_t e = build_operators(P, err);
    if (e == cudaErrorInvalidValue) return fail(KIFMM_ERR_ARG);
    if (e != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    if (d.precision == KIFMM_MIXED_FP16) {
        e = m2l_tensor_setup(P);
        if (e == cudaErrorNotSupported) return fail(KIFMM_ERR_ARG);
        if (e != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    }
    // workspace for n_max particles
    const int64_t n = d.n_max;
    P.n_cap = n;
    P.sys_cap = d.n_systems_max;
    const size_t esz = P.f64 ? sizeof(double) : sizeof(float);
    const int64_t nblk = (n + 4095) / 4096;
    P.hist_elems = (size_t)512 * nblk;
    struct A { void **p; size_t bytes; };
    const A arrs[] = {
        {(void **)&P.keys[0], sizeof(uint64_t) * n},   {(void **)&P.keys[1], sizeof(uint64_t) * n},
        {(void **)&P.vals[0], sizeof(uint32_t) * n},   {(void **)&P.vals[1], sizeof(uint32_t) * n},
        {(void **)&P.keys_user, sizeof(uint64_t) * n}, {(void **)&P.perm, sizeof(uint32_t) * n},
        {&P.pts, esz * 4 * n},                         {(void **)&P.res, sizeof(double) * 4 * n},
        {&P.w_sorted, esz * n},
        {&P.g_sorted, esz * 3 * n},
        {(void **)&P.adj_hg, sizeof(double) * 4 * n},
        {(void **)&P.adj_pd, sizeof(double) * 4 * n},
        {(void **)&P.adj_pot, sizeof(double) * n},
        {&P.gemm_part, esz * 8 * kSplitTargets * (size_t)(P.ns + 1)},
        {(void **)&P.sys_off_d, sizeof(int64_t) * (P.sys_cap + 1)},
        {(void **)&P.lo_side, sizeof(double) * 4 * P.sys_cap},
        {(void **)&P.key_scale, sizeof(double) * P.sys_cap},
        {(void **)&P.inv_side_f, sizeof(float) * P.sys_cap},
        {(void **)&P.out_scale, sizeof(double) * 2 * P.sys_cap},
        {(void **)&P.bbox_ord, sizeof(unsigned long long) * 6 * P.sys_cap},
        {(void **)&P.hist, sizeof(uint32_t) * P.hist_elems},
        {(void **)&P.status, sizeof(int)},
        {(void **)&P.moved, sizeof(int)},
        {(void **)&P.spec_buf, sizeof(int64_t) * 32},
        {(void **)&P.spec_fail, sizeof(int)},
        {(void **)&P.part_counts, sizeof(uint32_t) * 4 * 256},
        {(void **)&P.list_totals, sizeof(unsigned long long) * 4},
        {(void **)&P.energy_chunk_start, sizeof(int32_t) * (P.sys_cap + 1)},
        {(void **)&P.qsum, sizeof(double) * 2},
        {&P.frc, P.stokes ? esz * 3 * n : 8},
        {(void **)&P.pshift, sizeof(double)},
        {(void **)&P.tree_differs, sizeof(int)},
    };
    for (const A &a : arrs)
        if (plan_alloc(P, a.p, a.bytes) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    if (cudaEventCreateWithFlags(&P.leaf_fork, cudaEventDisableTiming) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    for (int v = 0; v < kLeafTiles; ++v)
        if (cudaStreamCreateWithFlags(&P.leaf_streams[v], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&P.leaf_join[v], cudaEventDisableTiming) != cudaSuccess)
            return fail(KIFMM_ERR_CUDA);
    const int64_t box0 = 12 * (n / (d.leaf_cap + 1)) + 64LL * P.sys_cap + 1024;
    if (grow_tree_arrays(P, box0, 0) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    P.scan_tmp_elems = std::max(P.scan_tmp_elems, scan_tmp_needed((int64_t)256 * nblk) + 8);
    if (plan_alloc(P, (void **)&P.scan_tmp, sizeof(uint32_t) * P.scan_tmp_elems) != cudaSuccess)
        return fail(KIFMM_ERR_CUDA);
    if (cudaMemset(P.status, 0, sizeof(int)) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    if (cudaMallocHost((void **)&P.rb, sizeof(Plan::Readback)) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    *out = pl;
    return KIFMM_OK;
}

kifmm_status kifmm_plan_destroy(kifmm_plan *pl) {
    if (!pl) return KIFMM_ERR_ARG;
    cudaDeviceSynchronize();
    m2l_tensor_release(pl->P);
    for (auto &b : pl->P.owned) cudaFree(b.ptr);
    pl->P.owned.clear();
    if (pl->P.rb) cudaFreeHost(pl->P.rb);
    for (cudaEvent_t e : pl->P.ev_pool) cudaEventDestroy(e);
    if (pl->P.leaf_fork) cudaEventDestroy(pl->P.leaf_fork);
    for (int v = 0; v < kLeafTiles; ++v) {
        if (pl->P.leaf_join[v]) cudaEventDestroy(pl->P.leaf_join[v]);
        if (pl->P.leaf_streams[v]) cudaStreamDestroy(pl->P.leaf_streams[v]);
    }
    delete pl;
    return KIFMM_OK;
}

kifmm_status kifmm_set_sources(kifmm_plan *pl, int n_systems, const int64_t *sys_offsets, const void *xyz,
                               const void *q, kifmm_stream_t stream) {
    if (!pl || !sys_offsets || !xyz || !q) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (n_systems < 1) return KIFMM_ERR_ARG;
    if (n_systems > P.sys_cap) return KIFMM_ERR_CAPACITY;
    if (sys_offsets[0] != 0) return KIFMM_ERR_ARG;
    for (int s = 0; s < n_systems; ++s)
        if (sys_offsets[s + 1] <= sys_offsets[s]) return KIFMM_ERR_ARG;
    const int64_t n = sys_offsets[n_systems];
    if (n > P.n_cap) return KIFMM_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    P.last_stream = s;
    P.has_sources = false;
    P.n = n;
    P.n_sys = n_systems;
    P.sys_off_h.assign(sys_offsets, sys_offsets + n_systems + 1);
    const long long l0 = g_launches;
    stage_begin(P, KIFMM_STAGE_TREE, s);
    kifmm_status rc = set_sources_impl(P, xyz, q, s);
    stage_end(P, KIFMM_STAGE_TREE, s);
    P.launches += g_launches - l0;
    return rc;
}

static kifmm_status set_sources_impl(Plan &P, const void *xyz, const void *q, cudaStream_t s) {
    const int n_systems = P.n_sys;
    const int64_t *sys_offsets = P.sys_off_h.data();
    API_CUDA(cudaMemsetAsync(P.status, 0, sizeof(int), s));
    // Non-finite inputs still quantise to valid keys, so the tree and lists
    // build regardless; the status is read once at the end.
    API_CUDA(build_tree(P, xyz, q, s));
    API_CUDA(ensure_box_arrays(P));
    // the lists (and the box partitions) depend on the boxes alone: when the
    // new tree has the boxes the lists were built for, they are kept
    P.lists_reused = false;
    if (P.desc.reuse_lists && P.prev_nb == P.nb && P.prev_sys_off == P.sys_off_h) {
        int differs = 1;
        API_CUDA(same_boxes(P, &differs, s));
        P.lists_reused = (differs == 0);
    }
    if (!P.lists_reused) {
        P.prev_nb = -1;  // recorded below once the build has succeeded
        API_CUDA(build_lists(P, s));
        API_CUDA(partition_boxes(P, s));
        if (P.desc.reuse_lists) API_CUDA(save_boxes(P, s));
    }
    API_CUDA(gather_particles(P, xyz, q, s));
    // energy chunks (sorted order never mixes systems; they depend on the
    // system offsets only)
    if (P.energy_off_h != P.sys_off_h) {
        std::vector<int64_t> ch;
        std::vector<int32_t> start(n_systems + 1, 0);
        for (int sy = 0; sy < n_systems; ++sy) {
            start[sy] = (int32_t)(ch.size() / 2);
            for (int64_t a = sys_offsets[sy]; a < sys_offsets[sy + 1]; a += 4096) {
                ch.push_back(a);
                ch.push_back(std::min(a + 4096, sys_offsets[sy + 1]));
            }
        }
        start[n_systems] = (int32_t)(ch.size() / 2);
        const int64_t nch = (int64_t)ch.size() / 2;
        if (nch > P.n_energy_chunks) {
            API_CUDA(plan_alloc(P, (void **)&P.energy_chunks, sizeof(int64_t) * 2 * nch));
            API_CUDA(plan_alloc(P, (void **)&P.energy_partial, sizeof(double) * nch));
        }
        P.n_energy_chunks = nch;
        API_CUDA(cudaMemcpyAsync(P.energy_chunks, ch.data(), sizeof(int64_t) * ch.size(), cudaMemcpyHostToDevice, s));
        API_CUDA(cudaMemcpyAsync(P.energy_chunk_start, start.data(), sizeof(int32_t) * start.size(),
                                 cudaMemcpyHostToDevice, s));
        P.energy_off_h = P.sys_off_h;
    }
    // the one synchronisation after the octree levels: the status word and,
    // for new lists, their sizes and the partition counts
    API_CUDA(cudaMemcpyAsync(&P.rb->status, P.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    API_CUDA(cudaStreamSynchronize(s));
    const int st = P.rb->status;
    if (!P.lists_reused) {
        if (!lists_finish(P)) {
            // a U or W list outgrew its storage: grow it and build again
            // (the totals of this build bound the next one exactly)
            API_CUDA(grow_lists(P));
            return set_sources_impl(P, xyz, q, s);
        }
        partition_finish(P);
    }
    if (st != 0) return (kifmm_status)st;
    // tiles of the tensor-core M2L (kept lists: the same tiles)
    if (P.desc.precision == KIFMM_MIXED_FP16 && !P.lists_reused) API_CUDA(m2l_tensor_tiles(P, s));
    if (!P.lists_reused) {
        P.prev_nb = P.nb;
        P.prev_sys_off = P.sys_off_h;
    }
    P.has_sources = true;
    return KIFMM_OK;
}

kifmm_status kifmm_evaluate(kifmm_plan *pl, void *pot, void *grad, double *energy, kifmm_stream_t stream) {
    if (!pl) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (P.stokes && (grad || energy)) return KIFMM_ERR_ARG;  // Stokeslet: velocities in pot only
    if (!P.has_sources) return KIFMM_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    P.last_stream = s;
    const long long l0 = g_launches;
    cudaError_t e = run_evaluate(P, pot, grad, energy, s);
    P.launches += g_launches - l0;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return KIFMM_ERR_CUDA;
    }
    return KIFMM_OK;
}

kifmm_status kifmm_clump_reduce(kifmm_plan *pl, int64_t n_clumps, const int64_t *clump_offsets, const void *xyz,
                                const void *q, const void *grad, const void *ref, void *force, void *torque,
                                kifmm_stream_t stream) {
    if (!pl || n_clumps < 0) return KIFMM_ERR_ARG;
    if (n_clumps > 0 && (!clump_offsets || !xyz || !q || !grad || !ref || !force || !torque)) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (P.stokes) return KIFMM_ERR_ARG;  // forces from charges: the Laplace kernel only
    cudaStream_t s = (cudaStream_t)stream;
    P.last_stream = s;
    return from_cuda(run_clump_reduce(P, n_clumps, clump_offsets, xyz, q, grad, ref, force, torque, s));
}

kifmm_status kifmm_backward(kifmm_plan *pl, const void *dL_dpot, const void *dL_dgrad, const double *dL_denergy,
                            const void *grad, void *dq, void *dx, kifmm_stream_t stream) {
    if (!pl || (!dL_dpot && !dL_dgrad && !dL_denergy)) return KIFMM_ERR_ARG;
    if (pl->P.periodic || pl->P.stokes) return KIFMM_ERR_ARG;  // not built for these plans
    if (dx && (dL_dpot || dL_denergy) && !grad) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!P.has_sources) return KIFMM_ERR_STATE;
    // the Hessian and energy terms read the last evaluate's field
    if ((dL_dgrad || dL_denergy) && !P.fwd_valid) return KIFMM_ERR_STATE;
    if (dL_denergy && !P.fwd_res_valid) return KIFMM_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    P.last_stream = s;
    const long long l0 = g_launches;
    cudaError_t e = run_backward(P, dL_dpot, dL_dgrad, dL_denergy, grad, dq, dx, s);
    P.launches += g_launches - l0;
    return from_cuda(e);
}

kifmm_status kifmm_update_sources(kifmm_plan *pl, const void *xyz, const void *q, kifmm_stream_t stream) {
    if (!pl || !xyz || !q) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!P.has_sources) return KIFMM_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    P.last_stream = s;
    const long long l0 = g_launches;
    stage_begin(P, KIFMM_STAGE_TREE, s);
    cudaError_t e = gather_particles(P, xyz, q, s);
    stage_end(P, KIFMM_STAGE_TREE, s);
    P.launches += g_launches - l0;
    return from_cuda(e);
}

kifmm_status kifmm_refresh_sources(kifmm_plan *pl, const void *xyz, const void *q, double skin, int *reused,
                                   kifmm_stream_t stream) {
    if (!pl || !xyz || !q || !(skin >= 0.0 && skin <= 1.0)) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!P.has_sources) return KIFMM_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    P.last_stream = s;
    const long long l0 = g_launches;
    stage_begin(P, KIFMM_STAGE_TREE, s);
    int moved = 1;
    kifmm_status rc = KIFMM_OK;
    cudaError_t e = check_leaves(P, xyz, skin, P.moved, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&moved, P.moved, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        rc = from_cuda(e);
    } else if (!moved) {
        rc = from_cuda(gather_particles(P, xyz, q, s));
    } else {
        // same systems, new tree: the full set_sources pass
        P.has_sources = false;
        rc = set_sources_impl(P, xyz, q, s);
    }
    stage_end(P, KIFMM_STAGE_TREE, s);
    P.launches += g_launches - l0;
    if (reused) *reused = (rc == KIFMM_OK && !moved) ? 1 : 0;
    return rc;
}

kifmm_status kifmm_get_device_status(kifmm_plan *pl, int *code) {
    if (!pl || !code) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    API_CUDA(cudaStreamSynchronize(P.last_stream));
    int st = 0;
    API_CUDA(cudaMemcpy(&st, P.status, sizeof(int), cudaMemcpyDeviceToHost));
    API_CUDA(cudaMemset(P.status, 0, sizeof(int)));
    *code = st;
    return KIFMM_OK;
}

kifmm_status kifmm_profile_enable(kifmm_plan *pl, int enable) {
    if (!pl) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!enable && P.prof) API_CUDA(profile_collect(P));
    P.prof = enable != 0;
    return KIFMM_OK;
}

kifmm_status kifmm_profile_read(kifmm_plan *pl, kifmm_profile_t *out) {
    if (!pl || !out) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    API_CUDA(profile_collect(P));
    for (int k = 0; k < KIFMM_STAGE_COUNT; ++k) {
        out->ms[k] = P.prof_ms[k];
        out->calls[k] = P.prof_calls[k];
        P.prof_ms[k] = 0.0;
        P.prof_calls[k] = 0;
    }
    out->launches = P.launches;
    P.launches = 0;
    return KIFMM_OK;
}

kifmm_status kifmm_set_m2l_wait_bound(kifmm_plan *pl, int64_t polls) {
    if (!pl || polls < 0) return KIFMM_ERR_ARG;
    if (pl->P.desc.precision != KIFMM_MIXED_FP16) return KIFMM_ERR_ARG;
    pl->P.m2l_wait_polls = polls;
    return KIFMM_OK;
}

kifmm_status kifmm_set_m2l_tuning(kifmm_plan *pl, int producers, int tiles, int stages) {
    if (!pl) return KIFMM_ERR_ARG;
    return m2l_tensor_pin(pl->P, producers, tiles, stages) ? KIFMM_OK : KIFMM_ERR_ARG;
}

kifmm_status kifmm_get_tuning(kifmm_plan *pl, kifmm_tuning_t *out) {
    if (!pl || !out) return KIFMM_ERR_ARG;
    const Plan &P = pl->P;
    out->tuned = (P.tuned_leaf ? 1 : 0) | (P.tuned_m2l ? 2 : 0);
    out->m2l_stages = m2l_tensor_stages(P);
    out->m2l_producers = m2l_tensor_producers(P);
    out->m2l_tiles = m2l_tensor_tiles_per_cta(P);
    out->m2l_rank_out = P.m2l_rl;
    out->m2l_rank_in = P.m2l_rr;
    for (int i = 0; i < kLeafBuckets; ++i) {
        out->leaf_tpl[i] = leaf_tile_tpl(P.leaf_tile.get(i));
        out->leaf_groups[i] = leaf_tile_groups(P.leaf_tile.get(i));
    }
    return KIFMM_OK;
}

kifmm_status kifmm_tree_info(kifmm_plan *pl, kifmm_tree_info_t *info) {
    if (!pl || !info) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!P.has_sources) return KIFMM_ERR_STATE;
    info->n_particles = P.n;
    info->n_boxes = P.nb;
    info->max_level = P.max_level;
    info->n_systems = P.n_sys;
    info->n_u = P.n_u;
    info->n_v = P.n_v;
    info->n_w = P.n_w;
    info->n_x = P.n_x;
    info->sort_passes = P.sort_passes;
    info->lists_reused = P.lists_reused ? 1 : 0;
    return KIFMM_OK;
}

kifmm_status kifmm_copy_keys(kifmm_plan *pl, uint64_t *keys, int64_t *perm, double *lo_side) {
    if (!pl) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!P.has_sources) return KIFMM_ERR_STATE;
    API_CUDA(cudaDeviceSynchronize());
    if (keys) API_CUDA(cudaMemcpy(keys, P.keys_user, sizeof(uint64_t) * P.n, cudaMemcpyDeviceToHost));
    if (perm) {
        std::vector<uint32_t> p(P.n);
        API_CUDA(cudaMemcpy(p.data(), P.perm, sizeof(uint32_t) * P.n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < P.n; ++i) perm[i] = p[i];
    }
    if (lo_side) API_CUDA(cudaMemcpy(lo_side, P.lo_side, sizeof(double) * 4 * P.n_sys, cudaMemcpyDeviceToHost));
    return KIFMM_OK;
}

kifmm_status kifmm_copy_tree(kifmm_plan *pl, int64_t *sys, int64_t *level, int64_t *coord, int64_t *first,
                             int64_t *count, int64_t *parent) {
    if (!pl) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!P.has_sources) return KIFMM_ERR_STATE;
    API_CUDA(cudaDeviceSynchronize());
    const int64_t nb = P.nb;
    std::vector<int32_t> t(nb);
    auto get = [&](const int32_t *src, int64_t *dst, int stride, int off) -> cudaError_t {
        cudaError_t e = cudaMemcpy(t.data(), src, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        for (int64_t b = 0; b < nb; ++b) dst[b * stride + off] = t[b];
        return cudaSuccess;
    };
    if (sys) API_CUDA(get(P.sys, sys, 1, 0));
    if (level) API_CUDA(get(P.lvl, level, 1, 0));
    if (coord) {
        API_CUDA(get(P.cx, coord, 3, 0));
        API_CUDA(get(P.cy, coord, 3, 1));
        API_CUDA(get(P.cz, coord, 3, 2));
    }
    if (first) API_CUDA(get(P.first, first, 1, 0));
    if (count) API_CUDA(get(P.cnt, count, 1, 0));
    if (parent) API_CUDA(get(P.parent, parent, 1, 0));
    return KIFMM_OK;
}

kifmm_status kifmm_copy_expansions(kifmm_plan *pl, double *u, double *d, double *res) {
    if (!pl) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!P.has_sources) return KIFMM_ERR_STATE;
    API_CUDA(cudaDeviceSynchronize());
    const size_t m = (size_t)P.nb * P.ns;
    auto get = [&](const void *src, double *dst) -> cudaError_t {
        if (P.f64) return cudaMemcpy(dst, src, sizeof(double) * m, cudaMemcpyDeviceToHost);
        std::vector<float> t(m);
        cudaError_t e = cudaMemcpy(t.data(), src, sizeof(float) * m, cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < m; ++i) dst[i] = t[i];
        return e;
    };
    if (u) API_CUDA(get(P.u_chk, u));
    if (d) {
        API_CUDA(get(P.d_chk, d));
        if (!P.f64) {
            // FP32-based modes store the mean separately: return the whole check potential
            std::vector<double> dbar((size_t)P.nb);
            API_CUDA(cudaMemcpy(dbar.data(), P.dbar, sizeof(double) * P.nb, cudaMemcpyDeviceToHost));
            for (int64_t b = 0; b < P.nb; ++b)
                for (int k = 0; k < P.ns; ++k) d[(size_t)b * P.ns + k] += dbar[(size_t)b];
        }
    }
    if (res) API_CUDA(cudaMemcpy(res, P.res, sizeof(double) * 4 * P.n, cudaMemcpyDeviceToHost));
    return KIFMM_OK;
}

// Lists as (box, image) pairs per node, sorted; the image of a V-list entry
// follows from its slot's offset (the slot table stores the box only).
static kifmm_status list_pairs(Plan &P, int kind, std::vector<std::vector<std::pair<int64_t, int>>> &lists) {
    API_CUDA(cudaDeviceSynchronize());
    const int64_t nb = P.nb;
    lists.assign(nb, {});
    if (kind == 0 || kind == 2) {
        std::vector<uint32_t> p(nb + 1);
        const int64_t tot = (kind == 0) ? P.n_u : P.n_w;
        std::vector<int32_t> ix(std::max<int64_t>(tot, 1));
        std::vector<int8_t> sh(std::max<int64_t>(tot, 1), 13);
        API_CUDA(cudaMemcpy(p.data(), kind == 0 ? P.u_ptr : P.w_ptr, sizeof(uint32_t) * (nb + 1),
                            cudaMemcpyDeviceToHost));
        if (tot) {
            API_CUDA(cudaMemcpy(ix.data(), kind == 0 ? P.u_idx : P.w_idx, sizeof(int32_t) * tot,
                                cudaMemcpyDeviceToHost));
            const int8_t *dsh = kind == 0 ? P.u_sh : P.w_sh;
            if (P.periodic) API_CUDA(cudaMemcpy(sh.data(), dsh, tot, cudaMemcpyDeviceToHost));
        }
        for (int64_t b = 0; b < nb; ++b)
            for (uint32_t e = p[b]; e < p[b + 1]; ++e) lists[b].push_back({ix[e], sh[e]});
    } else if (kind == 1) {
        std::vector<int32_t> v((size_t)nb * kVSlots), slot(8 * kVSlots), lv(nb), c3(3 * (size_t)nb);
        API_CUDA(cudaMemcpy(v.data(), P.vdense, sizeof(int32_t) * v.size(), cudaMemcpyDeviceToHost));
        API_CUDA(cudaMemcpy(slot.data(), P.slot_off, sizeof(int32_t) * slot.size(), cudaMemcpyDeviceToHost));
        API_CUDA(cudaMemcpy(lv.data(), P.lvl, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost));
        API_CUDA(cudaMemcpy(c3.data(), P.cx, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost));
        API_CUDA(cudaMemcpy(c3.data() + nb, P.cy, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost));
        API_CUDA(cudaMemcpy(c3.data() + 2 * nb, P.cz, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost));
        const std::vector<int> offs = m2l_offset_list();
        for (int64_t b = 0; b < nb; ++b)
            for (int sl = 0; sl < kVSlots; ++sl) {
                const int32_t a = v[(size_t)b * kVSlots + sl];
                if (a < 0) continue;
                const int cls = ((c3[b] & 1) << 2) | ((c3[nb + b] & 1) << 1) | (c3[2 * nb + b] & 1);
                const int o = slot[cls * kVSlots + sl];
                int img = 0;
                for (int d = 0; d < 3; ++d) {
                    const int64_t diff = (int64_t)c3[d * nb + b] + offs[3 * o + d] - c3[d * nb + a];
                    img = 3 * img + (int)(diff >> lv[b]) + 1;  // the image shift, in cells
                }
                lists[b].push_back({a, img});
            }
    } else {
        std::vector<int32_t> x((size_t)nb * kMaxCoarse), nx(nb);
        std::vector<int8_t> xs((size_t)nb * kMaxCoarse, 13);
        API_CUDA(cudaMemcpy(x.data(), P.xdense, sizeof(int32_t) * x.size(), cudaMemcpyDeviceToHost));
        API_CUDA(cudaMemcpy(nx.data(), P.nx, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost));
        if (P.periodic) API_CUDA(cudaMemcpy(xs.data(), P.x_sh, xs.size(), cudaMemcpyDeviceToHost));
        for (int64_t b = 0; b < nb; ++b)
            for (int k = 0; k < nx[b]; ++k)
                lists[b].push_back({x[(size_t)b * kMaxCoarse + k], xs[(size_t)b * kMaxCoarse + k]});
    }
    for (auto &l : lists) std::sort(l.begin(), l.end());
    return KIFMM_OK;
}

kifmm_status kifmm_copy_list_images(kifmm_plan *pl, int kind, int64_t *ptr, int64_t *idx, int64_t *img) {
    if (!pl || !ptr || kind < 0 || kind > 3) return KIFMM_ERR_ARG;
    Plan &P = pl->P;
    if (!P.has_sources) return KIFMM_ERR_STATE;
    std::vector<std::vector<std::pair<int64_t, int>>> lists;
    const kifmm_status st = list_pairs(P, kind, lists);
    if (st != KIFMM_OK) return st;
    ptr[0] = 0;
    for (int64_t b = 0; b < P.nb; ++b) {
        ptr[b + 1] = ptr[b] + (int64_t)lists[b].size();
        for (size_t k = 0; k < lists[b].size(); ++k) {
            if (idx) idx[ptr[b] + k] = lists[b][k].first;
            if (img) img[ptr[b] + k] = lists[b][k].second;
        }
    }
    return KIFMM_OK;
}

kifmm_status kifmm_copy_list(kifmm_plan *pl, int kind, int64_t *ptr, int64_t *idx) {
    return kifmm_copy_list_images(pl, kind, ptr, idx, nullptr);
}

}  // extern "C"
