// Internal declarations of the KIFMM library: the plan object and the host
// launchers implemented in the .cu translation units.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/kifmm.h"

namespace kifmm {

constexpr int kMaxLevel = 20;       // 21-bit quantisation per axis
constexpr int kNumM2L = 316;        // offsets in {-3..3}^3 minus {-1..1}^3
constexpr int kVSlots = 189;        // V-list slots per octant class (6^3 - 3^3)
constexpr int kMaxCoarse = 26;      // coarser-or-equal adjacent leaves of a box
constexpr int kColl = 27;           // colleague slots (3^3, centre = self)
constexpr int kSplitTargets = 4096; // targets of a gathered GEMM the slot-split form may take (up to 8 slots)

// Leaf-kernel tiles (variants): id -> (targets per lane TPL, source groups
// G); a pass covers (32 / G) TPL targets.  The table maps the number of
// targets still to cover, in buckets of 8 (the last bucket: more than 120),
// to the variant of the next pass.
constexpr int kLeafTiles = 6;
constexpr int kLeafBuckets = 16;
constexpr int kLeafTilingCandidates = 8;
__host__ __device__ constexpr int leaf_tile_tpl(int id) { return id % 2 + 1; }
__host__ __device__ constexpr int leaf_tile_groups(int id) { return id < 2 ? 4 : (id < 4 ? 2 : 1); }
struct LeafTiling {
    unsigned long long packed;  // 4 bits per bucket
    __host__ __device__ int get(int bucket) const { return (int)((packed >> (4 * bucket)) & 15ULL); }
    __host__ __device__ int for_targets(int r) const { return get((r - 1) >> 3 < kLeafBuckets ? (r - 1) >> 3 : kLeafBuckets - 1); }
    void set(int bucket, int id) {
        packed = (packed & ~(15ULL << (4 * bucket))) | ((unsigned long long)id << (4 * bucket));
    }
};
__host__ __device__ inline int leaf_variant(const LeafTiling &t, int n) { return t.for_targets(n > 0 ? n : 1); }
// Candidate c of the tuner (c = 0 is the default): the variant for up to 8,
// 16, 24, 32, 64 and more remaining targets.
LeafTiling leaf_tiling_candidate(int c);

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Device-side status codes share the kifmm_status numbering.
struct Plan {
    kifmm_plan_desc desc{};
    int device = 0;
    int p = 0, ns = 0;        // surface order, expansion length (surface points x components)
    int nsurf = 0;            // surface points, 6 (p - 1)^2 + 2
    bool stokes = false;      // Stokeslet kernel: 3-vector sources, densities and outputs
    void *frc = nullptr;      // Stokeslet: [N][3] forces in sorted order, compute type
    bool f64 = false;         // compute type is double (FP64 mode)
    int io_f64 = 0;           // caller dtype is double
    double coef = 1.0;
    double eps = 1e-12;
    int direct_thr = -1;      // W/X of leaves with at most this many points go to U (-1: none)
    LeafTiling leaf_tile{};   // leaf-kernel tiles (tuned when desc.autotune)
    bool tuned_leaf = false, tuned_m2l = false;
    int num_sms = 0;

    // ---- operators (device) ----
    double *surf64 = nullptr;   // [ns*3] unit-cube surface points
    float *surf32 = nullptr;
    // Composite translation operators in "check-potential" form, stored
    // transposed ([o][k][j]) in the compute type:
    void *m2m_t = nullptr;      // [8][ns][ns]   u(child)  -> u(parent)
    void *l2l_t = nullptr;      // [8][ns][op_ld]   d(parent) -> d(child)
    void *m2l_t = nullptr;      // [316][ns][op_ld] u(source) -> d(target)
    // FP32-based modes: l2l_t and m2l_t are mean-free over their outputs,
    // stored [blk][k][ns + 1] with the mean row in column ns (op_ld = ns + 1;
    // ns otherwise); d is then the mean-free part and dbar (FP64, per box)
    // the mean of the downward check potential.
    int op_ld = 0;
    double *dbar = nullptr;     // [nb]
    // Two-step pseudo-inverses for leaf evaluation: dens = V (W chk),
    // W = diag(sinv) U^T, both stored transposed ([k][j]).
    void *up_w_t = nullptr, *up_v_t = nullptr;
    void *dn_w_t = nullptr, *dn_v_t = nullptr;
    // Adjoint operators, read as [k][j] by the gathered GEMM: M2M^T, L2L^T,
    // M2L^T (indexed by the offset of the adjoint's source), and the leaf
    // pseudo-inverse factors W_up, V_up, W_dn, V_dn row-major.
    void *adj_m2m = nullptr, *adj_l2l = nullptr, *adj_m2l = nullptr, *adj_pinv = nullptr;
    void *w_sorted = nullptr;   // [N] adjoint weights in sorted order
    // Adjoint of a loss on the gradient / the energy: dipoles dL/dgrad in
    // sorted order and root units [N][3]; per particle the Hessian term and
    // the dipoles' near field (double4 each) and the forward potential; per
    // box the transposed pass's scratch (kept apart from the forward's
    // equivalent densities, which the Hessian term reads).
    void *g_sorted = nullptr;
    double *adj_hg = nullptr, *adj_pd = nullptr, *adj_pot = nullptr;
    void *adj_e1 = nullptr, *adj_e2 = nullptr;
    // Periodic cell (desc.cell > 0): image shifts of the list entries
    // (int8, (n_x + 1) 9 + (n_y + 1) 3 + (n_z + 1), 13 = the cell itself),
    // the far-image operator on the root (compute type, stored [k][j] like
    // the other composites), the root's second-moment functional g (FP64:
    // the trace of the root's equivalent density's second moment is g . u),
    // the per-leaf particle second moments and the uniform potential term.
    bool periodic = false;
    double cell = 0.0;
    int8_t *coll_sh = nullptr, *coarse_sh = nullptr, *x_sh = nullptr, *u_sh = nullptr, *w_sh = nullptr;
    double *far_t = nullptr;     // FP64 in every mode
    double *far_g = nullptr;
    double *m2m64 = nullptr;     // FP32-based periodic plans: FP64 copy of the M2M composites
    double *u_root64 = nullptr;  // ... and the root's upward check potential from them, FP64
    double *leaf_q2 = nullptr;   // [leaf cap]
    double *qsum = nullptr;      // [2]: sum q, sum |q| (neutrality)
    double *pshift = nullptr;    // [1]: uniform potential term (root units)
    bool fwd_valid = false;     // the last evaluate ran on the current sources (densities)
    bool fwd_res_valid = false; // ... and res still holds its field (no backward since)
    // Tensor-core M2L operands (mixed modes), built lazily.
    void *m2l_tc = nullptr;     // layout owned by the tensor-core kernel
    float *m2l_tc_scale = nullptr;
    int *slot_off = nullptr;    // [8][189] V slot -> M2L offset index (-1 unused)
    // Compressed M2L (desc.m2l_eps > 0, tensor-core mode): d = U C_o W u with
    // C_o = U^T K0_o V (plus the mean row m_o^T V), W = V^T P_up.
    int m2l_rl = 0, m2l_rr = 0; // left rank (outputs, mean excluded), right rank (inputs)
    float *m2l_c = nullptr;     // [316][rr][rl + 1] C_o^T with the mean row in column rl
    float *m2l_wc = nullptr;    // [rr][ns] W: check potential -> compressed input
    float *m2l_ul = nullptr;    // [ns][rl] U: compressed output -> mean-free check potential
    void *u_c = nullptr, *d_c = nullptr;  // [box cap][rr], [box cap][rl]

    // ---- capacities ----
    int64_t n_cap = 0, box_cap = 0, u_cap = 0, w_cap = 0;
    int sys_cap = 0;

    // ---- particles ----
    uint64_t *keys[2] = {nullptr, nullptr};
    uint32_t *vals[2] = {nullptr, nullptr};
    uint64_t *keys_user = nullptr;  // keys in caller order (introspection)
    uint32_t *perm = nullptr;       // sorted -> caller index
    void *pts = nullptr;            // [N] {dx, dy, dz, q} leaf-relative, compute type
    double *near_pot = nullptr;     // scratch accumulators (FP64 final sums)
    int64_t *sys_off_d = nullptr;   // [S+1]
    double *lo_side = nullptr;      // [S][4]
    double *key_scale = nullptr;    // [S] 2^21 / side
    float *inv_side_f = nullptr;    // [S] 1 / side (FP64 quotient rounded to FP32)
    float2 *leaf_ctr = nullptr;     // [leaf][3] leaf centres (FP64) as unevaluated sums hi + lo of two floats
    double *out_scale = nullptr;    // [S][2] coef / (4 pi side), coef / (4 pi side^2)
    unsigned long long *bbox_ord = nullptr;  // [S][6]
    uint32_t *scan_tmp = nullptr;   // scan scratch
    size_t scan_tmp_elems = 0;
    uint32_t *hist = nullptr;       // radix histograms
    size_t hist_elems = 0;

    // ---- tree (canonical order: level, system, Morton prefix) ----
    int32_t *lvl = nullptr, *cx = nullptr, *cy = nullptr, *cz = nullptr;
    int32_t *first = nullptr, *cnt = nullptr, *parent = nullptr, *child_first = nullptr,
            *nchild = nullptr, *sys = nullptr;
    uint32_t *tmp_nchild = nullptr;   // per node scratch
    int32_t *child_rng = nullptr;     // [box][16] scratch: (first, count) per octant
    std::vector<int64_t> level_start;  // host: level l owns [level_start[l], level_start[l+1])
    int64_t nb = 0, n = 0;
    int n_sys = 0, max_level = 0;
    int sort_passes = 8;  // 8-bit key digits the last build sorted (from the top)
    long long m2l_wait_polls = 0;  // tensor-core M2L barrier-wait bound (0: the default)
    // The boxes the lists were last built for: level, coordinates, parent,
    // child range and direct-sum flag per box ([8][prev_cap] int32).  A new
    // tree with the same boxes has the same lists, so set_sources keeps them.
    int32_t *prev_tree = nullptr;
    int64_t prev_nb = -1, prev_cap = 0;
    std::vector<int64_t> prev_sys_off;
    int *tree_differs = nullptr;
    bool lists_reused = false;
    std::vector<int64_t> sys_off_h;
    // Offsets already on the device and those the energy chunks were built
    // for: unchanged systems skip both uploads (a pageable copy would stall
    // the stream).
    std::vector<int64_t> sys_off_dev_h, energy_off_h;

    // ---- lists ----
    int32_t *coll = nullptr;         // [nb][27]
    int32_t *coarse = nullptr;       // [nb][26] coarser-or-equal adjacent leaves
    int32_t *ncoarse = nullptr;      // [nb]
    int32_t *vdense = nullptr;       // [nb][189] source box per slot, -1 if none
    int32_t *nv = nullptr;           // [nb]
    int32_t *xdense = nullptr;       // [nb][26]
    int32_t *nx = nullptr;           // [nb]
    uint32_t *u_ptr = nullptr, *w_ptr = nullptr;  // [nb+1]
    int32_t *u_idx = nullptr, *w_idx = nullptr;
    uint32_t *u_cnt = nullptr, *w_cnt = nullptr;  // [nb] scratch
    int64_t n_u = 0, n_v = 0, n_w = 0, n_x = 0;
    // M2L work: targets grouped by octant class
    int32_t *m2l_targets = nullptr;  // [nb] boxes with a V list, class-major
    int64_t m2l_class_start[9] = {0};
    int32_t *leaves = nullptr;       // [nb] leaf indices
    int64_t n_leaves = 0;
    int2 *leaf_vlist = nullptr;      // [kLeafTiles][leaf_item_cap] (leaf, first target) passes per variant
    int32_t *leaf_vcnt = nullptr;    // [16]: passes per variant [0, 8), then each variant's next-pass counter
    int64_t leaf_item_cap = 0;       // bound on passes: every pass but a leaf's last covers >= 8 targets
    // the leaf-kernel variants run concurrently: forked from the caller's
    // stream onto these and joined back (event-ordered, so capturable)
    cudaStream_t leaf_streams[kLeafTiles] = {};
    cudaEvent_t leaf_fork = nullptr, leaf_join[kLeafTiles] = {};
    int32_t *wsrc_flag = nullptr;    // [nb] 1 if the box is in some W list
    uint32_t *part_counts = nullptr; // [4][256]
    // What set_sources reads back at its final synchronisation (pinned host
    // memory): the status word, the list sizes and the partition counts.
    struct Readback {
        int status;
        uint32_t uw[2];                 // U and W list entries
        unsigned long long vx[4];       // V and X list entries
        uint32_t part_counts[4][256];
    } *rb = nullptr;
    unsigned long long *list_totals = nullptr;  // [4] V and X list sizes
    // Box lists grouped by a small key (stable, canonical order within a key):
    //   0: octant class of boxes with a V list (8 = none)
    //   1: leaves (key 0), then non-leaves by level (key 1 + level)
    //   2: boxes in some W list (key 0)
    //   3: boxes below the root by level * 8 + octant (L2L groups)
    int32_t *part_list[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<int64_t> part_start[4];  // host: exclusive prefix of the key counts (257 entries)
    int32_t *child8 = nullptr;       // [nb][8] child in each octant, -1 if none
    void *tmp_chk = nullptr;         // [nb][ns] pseudo-inverse scratch
    void *gemm_part = nullptr;       // [8][kSplitTargets][ns + 1] slot partials of the slot-split gathered GEMM
    void *dn_dens = nullptr;         // [nb][ns] normalised downward densities of leaves
    int64_t list_cap = 0;            // boxes the per-box list/expansion arrays hold

    // ---- expansions (compute type) ----
    void *u_chk = nullptr;   // [nb][ns] upward check potentials
    void *d_chk = nullptr;   // [nb][ns] downward check potentials
    void *up_dens = nullptr; // [nb][ns] normalised upward densities (W sources)

    // ---- results in sorted order ----
    double *res = nullptr;   // [N][4] pot, gx, gy, gz (normalised units, FP64 final)
    // energy reduction: chunks of sorted particles that never straddle systems
    int64_t *energy_chunks = nullptr;     // [n_chunks][2] (begin, end)
    int32_t *energy_chunk_start = nullptr; // [S+1]
    double *energy_partial = nullptr;     // [n_chunks]
    int64_t n_energy_chunks = 0;

    // ---- profiling ----
    bool prof = false;
    int64_t launches = 0;
    std::vector<cudaEvent_t> ev_pool;             // created lazily
    std::vector<std::pair<int, int>> ev_pending;  // (stage, event index of the start)
    size_t ev_used = 0;
    double prof_ms[KIFMM_STAGE_COUNT] = {0};
    int64_t prof_calls[KIFMM_STAGE_COUNT] = {0};

    // ---- status ----
    int *status = nullptr;   // device status word
    int *moved = nullptr;    // device flag of the tree reuse test
    int64_t *spec_buf = nullptr;  // [32] all-levels octree build: level boundaries
    int *spec_fail = nullptr;     // the all-levels build outgrew the box arrays
    uint32_t *os_cnt = nullptr;   // [levels][particle tiles] box counts, then box offsets
    size_t os_cnt_elems = 0;
    cudaStream_t last_stream = nullptr;
    bool has_sources = false;

    std::vector<DevBuf> owned;
};

// allocation helpers (tracked, freed with the plan).  plan_alloc replaces
// *ptr (freeing a previous tracked buffer); plan_grow keeps the first
// keep_bytes of the old contents.
cudaError_t plan_alloc(Plan &P, void **ptr, size_t bytes);
cudaError_t plan_grow(Plan &P, void **ptr, size_t bytes, size_t keep_bytes);
cudaError_t grow_tree_arrays(Plan &P, int64_t new_cap, int64_t keep);

// Stage bracketing (no-ops unless profiling is enabled).
void stage_begin(Plan &P, int stage, cudaStream_t s);
void stage_end(Plan &P, int stage, cudaStream_t s);
inline void count_launch(Plan &P, int64_t k = 1) { P.launches += k; }

// ---- tree.cu ----
cudaError_t build_tree(Plan &P, const void *xyz, const void *q, cudaStream_t s);
cudaError_t build_lists(Plan &P, cudaStream_t s);
cudaError_t partition_boxes(Plan &P, cudaStream_t s);
// after the final synchronisation of set_sources: list sizes and partition
// offsets from the read-back counts; false when a list outgrew its storage
// (grown here; the caller builds the lists again)
bool lists_finish(Plan &P);
cudaError_t grow_lists(Plan &P);
void partition_finish(Plan &P);
// tree.cu: *differs = 0 when the current boxes equal the saved ones
// (synchronises the stream); save_boxes records the current boxes.
cudaError_t same_boxes(Plan &P, int *differs, cudaStream_t s);
cudaError_t save_boxes(Plan &P, cudaStream_t s);
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev,
                               uint32_t *tmp, size_t tmp_elems, cudaStream_t s);
size_t scan_tmp_needed(int64_t n);

// ---- operators.cu ----
cudaError_t build_operators(Plan &P, std::string &err);
// operators.cu: unit-cube surface points [n_s][3], lexicographic.
std::vector<double> unit_surface(int p);
// operators.cu: the 316 M2L offsets d (3 ints each), {-3..3}^3 minus {-1..1}^3.
std::vector<int> m2l_offset_list();
// periodic.cu: far-image matrix of a periodic cell of side L (host FP64).
cudaError_t far_image_operator(int p, double L, double *T);

// ---- m2l_tc.cu (mixed modes) ----
// tree.cu: *moved_dev = 1 if some particle lies outside its leaf by more than
// skin half-widths of the finest level (refresh_sources' reuse test); enqueues only.
cudaError_t check_leaves(Plan &P, const void *xyz, double skin, int *moved_dev, cudaStream_t s);
cudaError_t m2l_tensor_setup(Plan &P);
cudaError_t m2l_tensor_tiles(Plan &P, cudaStream_t s);
cudaError_t m2l_tensor(Plan &P, cudaStream_t s);
void m2l_tensor_release(Plan &P);

// ---- fmm.cu ----
// Autotuning: true when desc.autotune asks for it, something is still
// untuned and the stream is not being captured (tuning synchronises).
bool tuning_wanted(const Plan &P, cudaStream_t s);
bool m2l_tensor_pin(Plan &P, int producers, int tiles, int stages);  // false: no such variant
int m2l_tensor_tiles_per_cta(const Plan &P);  // its target tiles per CTA (0: none)
int m2l_tensor_producers(const Plan &P);  // its producer warps (0: none)
int m2l_tensor_stages(const Plan &P);  // current pipeline depth of the tensor-core M2L (0: none)
// Device time of one launch sequence on stream s, in ms (synchronises).
template <class F>
float time_launch(cudaStream_t s, F &&launch) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    launch();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

cudaError_t run_evaluate(Plan &P, void *pot, void *grad, double *energy, cudaStream_t s);
cudaError_t run_backward(Plan &P, const void *w, const void *g, const double *dLdU, const void *grad, void *dq,
                         void *dx, cudaStream_t s);
cudaError_t gather_particles(Plan &P, const void *xyz, const void *q, cudaStream_t s);
cudaError_t run_clump_reduce(Plan &P, int64_t n_clumps, const int64_t *offs, const void *xyz,
                             const void *q, const void *grad, const void *ref, void *force,
                             void *torque, cudaStream_t s);

}  // namespace kifmm
