/*
 * kifmm.h - C ABI of the GB300 (sm_103a) kernel-independent fast multipole
 * library for long-range 1/r forces in discrete-element simulations.
 *
 * The method is the kernel-independent FMM outlined in Sec. 2.2 of the paper
 * (an adaptive octree with at most M points per leaf; fine-to-coarse M2M;
 * M2L between boxes in each other's far zone but not in their parents';
 * coarse-to-fine L2L; far field plus near field at the leaves; densities on
 * equivalent surfaces and translation matrices computed from the kernel),
 * applied to the sum of Eq. 1 with the Laplace kernel normalised as in Eq. 3:
 *
 *     pot_i  = coef * sum_{j, |x_i - x_j| > 0} q_j / (4 pi |x_i - x_j|)
 *     grad_i = gradient of pot_i with respect to x_i
 *
 * coef = 1 gives Eq. 3 units, 1/eps0 SI Coulomb, -4 pi G gravity with masses as
 * charges (Eq. 4 read as attraction).  The force on particle i is
 * F_i = -q_i grad_i and the long-range energy is U = 1/2 sum_i q_i pot_i
 * (Sec. 2.4).
 *
 * Conventions for every call:
 *  - Pointers marked "device" address memory on the plan's CUDA device,
 *    contiguous, row-major, in the plan's dtype (float or double).  The
 *    caller owns them; the library never frees or retains them past the call.
 *  - Pointers marked "host" address ordinary host memory.
 *  - The plan owns its workspace, operators and tree.  A plan is not
 *    thread-safe; calls on one plan must be serialised by the caller.
 *  - Work is enqueued on the given stream; nothing returns before its
 *    arguments are validated.  Argument errors are returned at once.  Errors
 *    detected on the device (non-finite input, capacity, timeout) are recorded
 *    in a device status word read by kifmm_get_device_status.
 *  - No C++ exception crosses this interface.
 */
#ifndef KIFMM_H
#define KIFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *kifmm_stream_t;

typedef enum {
    KIFMM_OK = 0,
    KIFMM_ERR_ARG = 1,       /* invalid argument (null pointer, bad size or mode) */
    KIFMM_ERR_CAPACITY = 2,  /* more particles or systems than the plan was made for */
    KIFMM_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    KIFMM_ERR_NONFINITE = 4, /* a position or charge is NaN or infinite */
    KIFMM_ERR_TIMEOUT = 5,   /* a bounded device wait ran out */
    KIFMM_ERR_STATE = 6      /* call out of order (e.g. evaluate before set_sources) */
} kifmm_status;

/* Value 2 is not a precision: a 3xTF32 tensor-core M2L would give the same
 * accuracy as the 3xFP16 one (both operand halves carry 11 significant bits)
 * at half the tensor rate, and single TF32 or BF16 operands (or a BF16 split)
 * do not reach the FP32 path's accuracy, so only the 3xFP16 split is offered.
 * plan_create returns KIFMM_ERR_ARG for 2. */
typedef enum {
    KIFMM_FP64 = 0,       /* every stage in double precision (parity path) */
    KIFMM_FP32 = 1,       /* single precision, SIMT M2L ("plain FP32")         */
    KIFMM_MIXED_FP16 = 3  /* M2L on tensor cores, 3xFP16 split with power-of-two
                             scaling, FP32 accumulate                         */
} kifmm_precision;

typedef enum { KIFMM_DTYPE_F32 = 0, KIFMM_DTYPE_F64 = 1 } kifmm_dtype;

/* Plan description.  Zero-initialise and set the fields you need. */
typedef struct {
    int p;               /* surface order: points per cube edge, 2 <= p <= 10;
                            n_s = 6 (p - 1)^2 + 2 points per surface          */
    int leaf_cap;        /* M: a box splits while it holds more than M points  */
    int max_depth;       /* deepest octree level, 1 <= max_depth <= 20          */
    int precision;       /* kifmm_precision                                    */
    double coef;         /* multiplies 1/(4 pi r); 0 is read as 1              */
    int64_t n_max;       /* largest total particle count over all systems      */
    int n_systems_max;   /* largest number of independent systems per call     */
    int dtype;           /* kifmm_dtype of xyz, q, pot, grad, forces           */
    double pinv_eps;     /* relative SVD truncation of the check-to-equivalent
                            pseudo-inverse; 0 selects 1e-12 in FP64 mode and
                            1e-9 in the FP32-based modes.  In FP64 mode it must
                            not lie within a factor 1.1 of any
                            sigma_i / sigma_max (KIFMM_ERR_ARG otherwise).    */
    int autotune;        /* 1: on the first evaluate (outside stream capture),
                            time the candidate leaf-kernel tilings and
                            tensor-core M2L pipeline depths on the live tree
                            and keep the fastest (synchronises once; results
                            may then differ from an untuned plan's in the
                            last FP32 bits).  0: fixed defaults.             */
    int direct_max;      /* a W/X interaction whose finer box (the W member,
                            or the owner of the X list) is a leaf holding at
                            most this many points is summed directly, as a
                            U-list (P2P) entry: the original KIFMM's cost rule
                            for the adaptive lists (Sec. 2.2).  0 selects n_s;
                            a negative value keeps every W/X interaction.      */
    double m2l_eps;      /* compressed M2L (tensor-core modes only; 0: dense).
                            The 316 M2L matrices K_o (downward check surface
                            from the source's upward equivalent surface, Sec.
                            2.2's operators computed from the kernel) are
                            replaced by low-rank forms on two shared bases: U,
                            the leading left singular vectors of their
                            mean-free forms side by side, and V, the leading
                            right singular vectors of the matrices stacked.
                            Ranks: the singular values above m2l_eps * sigma_0,
                            rounded up to fill 32-wide tensor-core tiles (the
                            left rank leaves one column for the mean), then
                            lowered while the cut would split a cluster of
                            equal values (within a factor 1.001).  Each M2L is
                            then (U U^T K0_o + 1 m_o^T) V V^T.  A value >= 1
                            or not finite is KIFMM_ERR_ARG, as is any nonzero
                            value in the FP64 and FP32 modes.               */
    double cell;         /* 0: free space.  > 0: periodic boundary conditions
                            (Sec. 2.4): the particles live in the cubic cell
                            [0, cell)^3 (positions outside are wrapped into
                            it), repeated over Z^3.  The cell is the root box;
                            the lists run over the cell and its 26 nearest
                            images (entries carry an image shift), farther
                            images act on the root through one far-image
                            operator (kifmm_far_image_operator), and the
                            potential gets the uniform second-moment term of
                            the conducting-boundary lattice sum.  The cell
                            must be neutral (|sum q| <= 1e-12 sum |q| for
                            double charges, 2^-24 sum |q| for float ones: a
                            neutral set rounded to float; else set_sources
                            returns KIFMM_ERR_ARG); one system
                            per plan (n_systems_max = 1); kifmm_backward is
                            not available (KIFMM_ERR_ARG).  In the FP32-based
                            modes that uniform term carries the FP32 error of
                            the root's upward expansion amplified by the
                            pseudo-inverse (a constant offset of every
                            potential; gradients, forces and the energy of a
                            neutral cell do not depend on it).              */
    int kernel;          /* kifmm_kernel: the kernel of the sum of Eq. 1      */
    int reuse_lists;     /* 0: every set_sources builds the U/V/W/X lists and
                            box partitions.  1: set_sources compares the boxes
                            of the new tree (level, integer coordinates,
                            parent, child range, small-leaf flag) with those
                            the lists were last built for and keeps the lists
                            when they are equal (the lists are a function of
                            the boxes alone, so the outputs are bit-identical
                            to a rebuild); kifmm_tree_info reports which.   */
} kifmm_plan_desc;

/* Kernels of Eq. 1.  The Laplace kernel is the default (1/(4 pi r) times
 * coef, Eq. 3; scalar charges; outputs potential, gradient, energy).  The
 * Stokeslet, G(r) = (I / |r| + r r^T / |r|^3) / (8 pi) times coef (coef =
 * 1 / mu: the velocity of point forces in Stokes flow, Sec. 2.4), is the
 * tensor-kernel form Eq. 1 admits: set_sources takes forces [N, 3] in place
 * of q, evaluate writes velocities [N, 3] to pot (grad and energy must be
 * NULL).  Same tree, lists, surfaces and pseudo-inverse rules, with 3-vector
 * densities on the surfaces.  Stokeslet plans run in KIFMM_FP64 or
 * KIFMM_FP32, free space, with no compressed M2L, clump reduce or adjoint
 * (KIFMM_ERR_ARG). */
typedef enum { KIFMM_KERNEL_LAPLACE = 0, KIFMM_KERNEL_STOKESLET = 1 } kifmm_kernel;

typedef struct kifmm_plan kifmm_plan;

/*
 * Create a plan: validate desc, allocate workspace for n_max particles,
 * build the unit surfaces (Sec. 2.2, equivalent surfaces), compute the FP64
 * pseudo-inverses of the check-from-equivalent matrices on the GPU (one-sided
 * Jacobi SVD, truncated at pinv_eps) and the M2M, L2L and 316 M2L translation
 * matrices (Sec. 2.2: matrices computed automatically for the kernel), and
 * synchronise.  This is the per-setup precompute of Sec. 2.4.
 * out (host): receives the plan.  Returns KIFMM_ERR_ARG for a bad desc or an
 * ambiguous truncation threshold, KIFMM_ERR_CUDA if allocation fails.
 */
kifmm_status kifmm_plan_create(const kifmm_plan_desc *desc, kifmm_plan **out);

/* Free the plan and all device memory it owns (synchronises its device). */
kifmm_status kifmm_plan_destroy(kifmm_plan *plan);

/*
 * Load particles and build the tree (Sec. 2.2, first and third steps): per
 * system bounding cube, 63-bit Morton keys, stable radix sort of the key
 * digits the octree reads (two levels below the previous tree's depth, all
 * digits if the tree turns out deeper), adaptive octree (split while
 * count > leaf_cap and level < max_depth), U/V/W/X lists.  Particles come out
 * grouped by leaf in Morton order; within a leaf their order is unspecified.
 * n_systems: number of independent systems (1 <= n_systems <= n_systems_max).
 * sys_offsets (host): n_systems + 1 ascending int64 offsets, sys_offsets[0] = 0;
 *   system s owns particles [sys_offsets[s], sys_offsets[s+1]), at least one.
 * xyz (device): [N, 3] positions; q (device): [N] charges (masses for gravity);
 *   N = sys_offsets[n_systems] <= n_max.  Both are read during this call only;
 *   the plan keeps sorted copies.
 * Synchronises the stream (the tree size is data dependent).  Returns
 * KIFMM_ERR_NONFINITE if a position or charge is not finite.
 */
kifmm_status kifmm_set_sources(kifmm_plan *plan, int n_systems, const int64_t *sys_offsets,
                               const void *xyz, const void *q, kifmm_stream_t stream);

/*
 * Refresh positions and charges with the tree and lists frozen.  The paper
 * recomputes long-range forces only every S steps (Eq. 2) and builds the tree
 * once at setup (Sec. 2.4); this call keeps the last set_sources' particle
 * order, boxes and lists and only rewrites the leaf-relative particle records,
 * so that evaluate and backward see the new positions.  Particles that left
 * their leaf stay assigned to it (accuracy degrades with the distance moved;
 * exactness of the pair coverage does not).  xyz (device, [N,3]) and q
 * (device, [N]) must hold the same particles in the same order as the last
 * set_sources.  Never allocates or synchronises (capturable in a CUDA graph).
 */
kifmm_status kifmm_update_sources(kifmm_plan *plan, const void *xyz, const void *q, kifmm_stream_t stream);

/*
 * Refresh with a validity test: keep the tree when it still fits, rebuild it
 * when it does not (the tree reuse between long-range evaluations of Sec. 2.4
 * and Eq. 2, with a Verlet-style skin).  The test runs on the device: every
 * particle, taken in the last set_sources' root cube, must lie inside its leaf
 * grown on every side by skin times the half-width of the finest leaf level
 * in the plan.  That bound keeps each particle inside the 1.05 h surfaces of
 * its own leaf for skin <= 0.05 and keeps the separation of every V, W and X
 * pair, so a reused tree has the accuracy of a fresh one (the default 0.05).
 * If the test passes, this is kifmm_update_sources; otherwise it is
 * kifmm_set_sources with the same systems (a new root cube and tree).
 * xyz (device, [N,3]) and q (device, [N]): the same particles in the same
 *   order as the last set_sources, in the plan's dtype.
 * skin: in [0, 1]; 0 requires every particle inside its own leaf.
 * reused (host, may be NULL): set to 1 if the tree was kept, else 0.
 * Synchronises the stream once (the decision is taken on the host), so it is
 * not capturable in a CUDA graph.  A non-finite coordinate fails the test and
 * the rebuild returns KIFMM_ERR_NONFINITE.  Returns KIFMM_ERR_STATE before
 * the first set_sources and KIFMM_ERR_ARG for a skin outside [0, 1].
 */
kifmm_status kifmm_refresh_sources(kifmm_plan *plan, const void *xyz, const void *q, double skin, int *reused,
                                   kifmm_stream_t stream);

/*
 * Evaluate the long-range field on every particle (Sec. 2.2 passes; Sec. 2.4
 * per-step evaluation): P2M, M2M, M2L (V list), P2L (X list), L2L, L2P,
 * M2P (W list), P2P (U list).
 * pot (device, [N] or NULL), grad (device, [N, 3] or NULL): outputs in the
 *   caller's particle order, coef applied, self-interaction excluded.
 * energy (device, [n_systems] doubles, or NULL): U_s = 1/2 sum_{i in s} q_i pot_i.
 * Enqueues work only; never allocates; never synchronises.
 */
kifmm_status kifmm_evaluate(kifmm_plan *plan, void *pot, void *grad, double *energy,
                            kifmm_stream_t stream);

/*
 * Rigid-clump aggregation (Sec. 2.3-2.4): charges sit on pebbles, forces are
 * applied per pebble and summed into the clump force and the torque about the
 * clump reference point:
 *   F_c = sum_{k in c} F_k,  tau_c = sum_{k in c} (x_k - X_c) x F_k,
 *   F_k = -q_k grad_k.
 * clump_offsets (device): n_clumps + 1 ascending int64 offsets into the
 *   caller's particle order; xyz, q, grad (device): [N,3], [N], [N,3] as passed
 *   to set_sources / returned by evaluate; ref (device): [n_clumps, 3] X_c;
 *   force, torque (device): [n_clumps, 3] outputs.  Accumulates in FP64.
 */
kifmm_status kifmm_clump_reduce(kifmm_plan *plan, int64_t n_clumps, const int64_t *clump_offsets,
                                const void *xyz, const void *q, const void *grad, const void *ref,
                                void *force, void *torque, kifmm_stream_t stream);

/*
 * Adjoint of evaluate with the tree frozen (not in the paper; it makes the
 * evaluation differentiable, e.g. for a loss on the forces of Sec. 2.3-2.4).
 * With pot = A(x) q and grad = G(x) q the FMM operators and a loss L with
 * w = dL/dpot, g = dL/dgrad and u_s = dL/dU_s (U_s the energy of system s):
 *   dq_j = (A^T w)_j + (G^T g)_j + u_s (pot_j + (A^T q)_j) / 2,
 *   dx_k = w'_k grad_k + H_k g_k + q_k grad_{x_k}(A^T w' + G^T g)_k,
 * with w' = w + u_s q / 2 and H_k the Hessian of the field at x_k; computed
 * by the transposed passes (G^T g: the dipoles g on the same surfaces, lists
 * and translation operators) and, for H g and the explicit energy term, from
 * the last evaluate's equivalent densities and potentials.  No other
 * intermediate is stored.
 * dL_dpot (device, [N] or NULL), dL_dgrad (device, [N, 3] or NULL),
 * dL_denergy (device, [n_systems] doubles or NULL): at least one is given.
 * grad (device, [N, 3]): the forward gradient (coef applied); needed for dx
 *   when dL_dpot or dL_denergy is given.
 * dq (device, [N] or NULL), dx (device, [N, 3] or NULL): outputs, caller order.
 * KIFMM_ERR_STATE when dL_dgrad or dL_denergy is given but no evaluate ran on
 * the current sources (set_sources / update_sources / refresh_sources since),
 * and when dL_denergy is given and another backward ran after that evaluate
 * (the energy term reads the evaluate's potentials, which a backward
 * overwrites).  The forward's equivalent densities are kept, so several
 * backward calls with dL_dpot / dL_dgrad may follow one evaluate; the
 * expansions (kifmm_copy_expansions) then show the transposed pass.  Never
 * allocates.
 */
kifmm_status kifmm_backward(kifmm_plan *plan, const void *dL_dpot, const void *dL_dgrad, const double *dL_denergy,
                            const void *grad, void *dq, void *dx, kifmm_stream_t stream);

/*
 * Long-range energy U = 1/2 sum_i q_i pot_i without allocating anything.
 * The paper has no counterpart: this is a convenience for callers that cannot
 * allocate device memory where they need the energy — a DEM step recorded into
 * a CUDA graph (cudaMalloc cannot be captured), an application whose device
 * memory belongs to its own pool, a time-critical loop that must not enter an
 * allocator.  It sums q_i pot_i over all n entries in the caller's order with
 * a fixed-chunk two-stage scheme (FP64 partial sums of 4096 entries, then one
 * ordered sum of the partials), so its result is deterministic and equal to
 * the energy output of kifmm_evaluate up to rounding (evaluate sums FP64
 * internal potentials per system; this call sums the pot it is given, so in
 * FP32 the two differ at the level of FP32 rounding of pot).  Given the
 * particles of several systems it returns their total energy.  The partial
 * sums live in a fixed array of 16384 doubles (128 KiB) in the library's
 * device image; every GPU that loads the library keeps that array until the
 * process exits.
 * n: number of particles, at most 67,108,864 (16384 chunks of 4096); larger n
 *   returns KIFMM_ERR_CAPACITY without launching anything.
 * dtype: kifmm_dtype of q and pot.  q, pot (device, [n]): charges and the
 *   potential returned by kifmm_evaluate.  energy (device, one double): output.
 * No cudaMalloc/cudaFree or other allocation happens.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.  All calls
 * on a device share the array and it keeps the last call's partials: every
 * partial a call reads is written earlier in the same call, so nothing needs
 * clearing, but calls that overlap on the GPU (different streams, no ordering)
 * race on it.
 */
kifmm_status kifmm_energy_noalloc(int64_t n, int dtype, const void *q, const void *pot, double *energy,
                                  kifmm_stream_t stream);

/* Synchronise the last stream used by the plan and read (then clear) the
 * device status word.  code (host) receives a kifmm_status value. */
kifmm_status kifmm_get_device_status(kifmm_plan *plan, int *code);

/* Static description of a status code. */
const char *kifmm_status_string(kifmm_status status);

/*
 * Long-range force computation stride (Eq. 2): S ~ sqrt(k_DEM / k_LR), the
 * number of DEM time steps over which one long-range evaluation may be
 * reused, since the Rayleigh time step scales with the square root of the
 * stiffness.  The forces must be recomputed at least once every S steps, so
 * the approximation is rounded down: S = max(1, floor(sqrt(k_dem / k_lr))).
 * k_dem: the largest contact stiffness; k_lr: the largest stiffness of the
 * long-range interaction (both > 0 and finite, same units).  stride (host)
 * receives S.  Host only: needs no device and no plan.  KIFMM_ERR_ARG for a
 * non-positive or non-finite stiffness or a NULL stride.
 */
kifmm_status kifmm_lr_stride(double k_dem, double k_lr, int64_t *stride);

/*
 * Far-image operator of a periodic cell (Sec. 2.4: periodic boundary
 * conditions, which the paper allows for neutral cells only), the plan-time
 * building block of a periodic evaluation.  With the cell of side `cell` as
 * the root box (half-width h = cell / 2), T[j][k] is the potential, with the
 * kernel 1/(4 pi r) of Eq. 3, at the root's downward check point
 * 1.05 h S_j due to a unit charge at its upward equivalent point
 * 1.05 h S_k repeated over every image cell n with max |n_i| >= 2 (the
 * images a periodic evaluation's lists, which run over the cell and its 26
 * neighbours, do not reach).  S is the unit surface of order p (n_s =
 * 6 (p - 1)^2 + 2 points, lexicographic, as everywhere in this library).
 * The sum converges only conditionally; it is taken as Ewald's sum with the
 * conducting boundary minus the 27 nearest images, so applied to a density
 * that sums to zero (a neutral cell) it is the conducting-boundary far
 * field.  T (host, [n_s][n_s] row-major doubles) receives the matrix.
 * Host only, FP64, about a second at p = 6: needs no device and no plan.
 * KIFMM_ERR_ARG for p outside 2..10, a non-positive or non-finite cell, or
 * a NULL T.
 */
kifmm_status kifmm_far_image_operator(int p, double cell, double *T);

/* ------------------------------------------------------------------------
 * Profiling.  When enabled, every stage of set_sources / evaluate is
 * bracketed by CUDA events recorded on the call's stream (no extra
 * synchronisation), and every kernel launch is counted.  kifmm_profile_read
 * synchronises, returns the device time accumulated per stage since the
 * last read (or enable) and resets the accumulators.
 * ------------------------------------------------------------------------ */
typedef enum {
    KIFMM_STAGE_TREE = 0,  /* set_sources: bbox, keys, sort, octree, lists  */
    KIFMM_STAGE_P2M = 1,
    KIFMM_STAGE_M2M = 2,
    KIFMM_STAGE_M2L = 3,
    KIFMM_STAGE_P2L = 4,
    KIFMM_STAGE_L2L = 5,
    KIFMM_STAGE_LEAF = 6,  /* equivalent-density solves, L2P, M2P         */
    KIFMM_STAGE_P2P = 7,
    KIFMM_STAGE_OUT = 8,   /* scatter to caller order, energy             */
    KIFMM_STAGE_COUNT = 9
} kifmm_stage;

typedef struct {
    double ms[KIFMM_STAGE_COUNT]; /* summed device milliseconds per stage  */
    int64_t calls[KIFMM_STAGE_COUNT]; /* bracketed occurrences per stage   */
    int64_t launches;             /* kernels launched by the library       */
} kifmm_profile_t;

/* enable (host): 1 to record, 0 to stop. */
kifmm_status kifmm_profile_enable(kifmm_plan *plan, int enable);
/* out (host): accumulated times since the last read; resets them. */
kifmm_status kifmm_profile_read(kifmm_plan *plan, kifmm_profile_t *out);

/* Tile shapes in use (no counterpart in the paper: the M2L and P2P tile
 * shapes are chosen by an autotuner on the live tree).  tuned: bit 0 leaf kernel,
 * bit 1 tensor-core M2L.  m2l_stages: shared-memory pipeline depth of the
 * tensor-core M2L (0 when the plan has none).  Leaf kernel: a leaf is
 * covered by passes; with r of its targets still to cover, bucket
 * min((r - 1) / 8, 15) selects leaf_tpl targets per lane and leaf_groups
 * source groups for the next pass, which covers 32 / groups * tpl targets;
 * each (tpl, groups) variant is its own kernel.  m2l_rank_out/in: the ranks
 * a compressed M2L (desc.m2l_eps) chose at plan creation.
 * Host memory; no device work. */
typedef struct {
    int tuned;
    int m2l_stages;
    int leaf_tpl[16];
    int leaf_groups[16];
    int m2l_rank_out;    /* compressed M2L: left rank (outputs, without the
                            mean column); 0 for a dense M2L               */
    int m2l_rank_in;     /* compressed M2L: right rank (inputs); 0 if dense  */
    int m2l_producers;   /* tensor-core M2L: warps gathering the source rows
                            (0 when the plan has none)                      */
    int m2l_tiles;       /* tensor-core M2L: tiles of 128 targets per CTA that
                            share each operator block (1 or 2; 0: none)     */
} kifmm_tuning_t;
kifmm_status kifmm_get_tuning(kifmm_plan *plan, kifmm_tuning_t *out);

/* Pins the tensor-core M2L variant instead of tuning it (a known-good choice
 * replayed, or each variant tested): producers 2 or 4 warps, tiles 1 or 2
 * (two tiles take two producer warps), stages 2 .. the shared-memory
 * maximum for that tile count.  Every variant computes bit-identical
 * results.  KIFMM_ERR_ARG for other values or a plan without the
 * tensor-core M2L (FP64, FP32, Stokeslet).  Host only; no device work. */
kifmm_status kifmm_set_m2l_tuning(kifmm_plan *plan, int producers, int tiles, int stages);

/* Bound, in polls, of every barrier wait of the tensor-core M2L's pipeline
 * (0: the default, about 2^24).  Every wait of that kernel is bounded: on
 * time-out its blocks record KIFMM_ERR_TIMEOUT in the device status
 * (kifmm_get_device_status), wait for their own copies in flight (with the
 * default bound), free their tensor memory and return, so that the context
 * stays usable; that evaluate's outputs are then not valid.  A tiny bound
 * makes the waits run out on purpose (the time-out path's test).
 * KIFMM_ERR_ARG for a negative bound or a plan without the tensor-core M2L.
 * Host only; no device work. */
kifmm_status kifmm_set_m2l_wait_bound(kifmm_plan *plan, int64_t polls);

/* ------------------------------------------------------------------------
 * Introspection (tests and tools).  All outputs are host buffers sized by
 * the caller from kifmm_tree_info; nodes are in canonical order (system,
 * level, Morton prefix within the level).
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_particles;
    int64_t n_boxes;
    int max_level;
    int n_systems;
    int64_t n_u, n_v, n_w, n_x; /* total list entries */
    int sort_passes;            /* 8-bit key digits the last build's radix sort
                                   processed (from the most significant one) */
    int lists_reused;           /* 1: the last set_sources found the boxes its
                                   lists were built for (reuse_lists plans
                                   only) and kept the lists and box
                                   partitions; 0: built them                   */
} kifmm_tree_info_t;

kifmm_status kifmm_tree_info(kifmm_plan *plan, kifmm_tree_info_t *info);

/* keys (host, [N] uint64): Morton keys in the caller's order;
 * perm (host, [N] int64): perm[i] = caller index of the i-th sorted particle
 *   (grouped by leaf; the order within a leaf is unspecified);
 * lo_side (host, [n_systems, 4] double): root cube lo xyz and side. */
kifmm_status kifmm_copy_keys(kifmm_plan *plan, uint64_t *keys, int64_t *perm, double *lo_side);

/* Per node (host, [n_boxes] int64 each, NULL to skip): system, level, integer
 * coordinates (3 per node), first sorted particle, count, parent (-1 root). */
kifmm_status kifmm_copy_tree(kifmm_plan *plan, int64_t *sys, int64_t *level, int64_t *coord,
                             int64_t *first, int64_t *count, int64_t *parent);

/* Expansions after the last evaluate, in root-normalised units of the
 * kernel 1/r: u (host, [n_boxes, n_s]) upward check potentials, d (host,
 * [n_boxes, n_s]) downward check potentials, res (host, [N, 4]) potential and
 * gradient per sorted particle (NULL to skip).  All double. */
kifmm_status kifmm_copy_expansions(kifmm_plan *plan, double *u, double *d, double *res);

/* One list kind (0 = U, 1 = V, 2 = W, 3 = X) as CSR over nodes:
 * ptr (host, [n_boxes + 1]), idx (host, [n_kind]); sources of each node are
 * sorted ascending. */
kifmm_status kifmm_copy_list(kifmm_plan *plan, int kind, int64_t *ptr, int64_t *idx);

/* The same with the image of every entry (periodic plans; all 13 in free
 * space): img (host, [n_kind]) receives (n_x + 1) 9 + (n_y + 1) 3 + (n_z + 1)
 * for the image shift n in {-1, 0, 1}^3 of the source box; entries sorted by
 * (box, image).  ptr, idx as kifmm_copy_list. */
kifmm_status kifmm_copy_list_images(kifmm_plan *plan, int kind, int64_t *ptr, int64_t *idx, int64_t *img);

#ifdef __cplusplus
}
#endif

#endif /* KIFMM_H */
