/*
 * KIFMM oracle: plain FP64 CPU reference for the kernel-independent fast
 * multipole evaluation of 1/r long-range forces.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links, includes or
 * calls this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * What it computes, in the order of the paper's outline of the method
 * (Sec. 2.2) and of the original KIFMM (Ying, Biros & Zorin 2004, cited in
 * Sec. 2.2):
 *   - direct O(N^2) sum of the Laplace potential and gradient (Sec. 1, Eq. 1,
 *     normalised as in Eq. 3);
 *   - Morton keys of the quantised positions and the adaptive octree with at
 *     most M points per leaf (Sec. 2.2, first step);
 *   - U, V, W, X interaction lists classified pair by pair from their
 *     geometric definitions (Sec. 2.2, third step: "not in the far zone of the
 *     parent but in the far zones of the descendants");
 *   - the upward pass (check-surface evaluation, then equivalent-density
 *     solve), M2L, P2L, the downward pass and the leaf evaluation
 *     (Sec. 2.2 steps two to four, equivalent densities of Sec. 2.2).
 * Everything is double precision, written as straight loops, parallel over
 * boxes or targets with OpenMP.  Compile with -ffp-contract=off so that the
 * Morton quantisation is the IEEE expression as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_BITS 21

/* ---------------------------------------------------------------------- */
/* Kernel: K(x, y) = 1 / (4 pi |x - y|), zero when x == y (Eq. 3 units).   */
/* grad_x K(x, y) = -(x - y) / (4 pi |x - y|^3).                           */
/* ---------------------------------------------------------------------- */
static inline double lap_pot(double dx, double dy, double dz) {
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return 0.0;
    return 1.0 / (4.0 * ORC_PI * sqrt(r2));
}

static inline void lap_pot_grad(double dx, double dy, double dz, double q, double *p, double *g) {
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return;
    double r = sqrt(r2);
    double k = q / (4.0 * ORC_PI * r);
    double k3 = k / r2;
    p[0] += k;
    g[0] -= dx * k3;
    g[1] -= dy * k3;
    g[2] -= dz * k3;
}

/*
 * Direct sum (Eq. 1 with the Laplace kernel, Eq. 3 normalisation):
 *   pot_i  = sum_{j, r_ij > 0} q_j / (4 pi r_ij)
 *   grad_i = -sum_{j, r_ij > 0} q_j (x_i - y_j) / (4 pi r_ij^3)
 * for targets xt[nt,3] over sources ys[ns,3] with charges qs[ns].
 */
void orc_direct(int64_t ns, const double *ys, const double *qs, int64_t nt, const double *xt,
                double *pot, double *grad) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        double p = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < ns; ++j)
            lap_pot_grad(xt[3 * i] - ys[3 * j], xt[3 * i + 1] - ys[3 * j + 1],
                         xt[3 * i + 2] - ys[3 * j + 2], qs[j], &p, g);
        pot[i] = p;
        if (grad) {
            grad[3 * i] = g[0];
            grad[3 * i + 1] = g[1];
            grad[3 * i + 2] = g[2];
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Morton keys.  The root cube is [lo, lo + side]^3 with lo the per-axis    */
/* minimum and side the largest extent (1 if all points coincide).  Each   */
/* coordinate is quantised to 21 bits, k = min(floor((x - lo) * s), 2^21-1) */
/* with s = 2^21 / side, and the bits are interleaved x-highest, so the     */
/* 3-bit digit of a level is the octant 4x + 2y + z.                        */
/* ---------------------------------------------------------------------- */
void orc_bbox(int64_t n, const double *x, double *lo, double *side) {
    double mn[3], mx[3];
    for (int d = 0; d < 3; ++d) { mn[d] = x[d]; mx[d] = x[d]; }
    for (int64_t i = 1; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            double v = x[3 * i + d];
            if (v < mn[d]) mn[d] = v;
            if (v > mx[d]) mx[d] = v;
        }
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        lo[d] = mn[d];
        if (mx[d] - mn[d] > s) s = mx[d] - mn[d];
    }
    *side = (s > 0.0) ? s : 1.0;
}

void orc_morton(int64_t n, const double *x, const double *lo, double side, uint64_t *keys) {
    const double s = 2097152.0 / side; /* 2^21 / side */
    const uint64_t kmax = (1ULL << ORC_BITS) - 1ULL;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k[3];
        for (int d = 0; d < 3; ++d) {
            double t = (x[3 * i + d] - lo[d]) * s;
            double f = floor(t);
            uint64_t v = (f >= (double)kmax) ? kmax : (uint64_t)f;
            k[d] = v;
        }
        uint64_t key = 0;
        for (int b = 0; b < ORC_BITS; ++b) {
            key |= ((k[0] >> b) & 1ULL) << (3 * b + 2);
            key |= ((k[1] >> b) & 1ULL) << (3 * b + 1);
            key |= ((k[2] >> b) & 1ULL) << (3 * b);
        }
        keys[i] = key;
    }
}

/* ---------------------------------------------------------------------- */
/* Interaction lists by pair-wise classification (Ying, Biros & Zorin 2004 */
/* adaptive lists; the paper describes the V list in Sec. 2.2).           */
/* Boxes are closed cubes [c, c+1] * 2^-level in integer coordinates.     */
/* Two boxes are adjacent when their closed cubes intersect and neither   */
/* contains the other.                                                     */
/* ---------------------------------------------------------------------- */
static int box_adjacent(int la, const int64_t *a, int lb, const int64_t *b) {
    int L = la > lb ? la : lb;
    int intersect = 1, a_in_b = 1, b_in_a = 1;
    for (int d = 0; d < 3; ++d) {
        int64_t alo = a[d] << (L - la), ahi = (a[d] + 1) << (L - la);
        int64_t blo = b[d] << (L - lb), bhi = (b[d] + 1) << (L - lb);
        if (!(alo <= bhi && blo <= ahi)) intersect = 0;
        if (!(blo <= alo && ahi <= bhi)) a_in_b = 0;
        if (!(alo <= blo && bhi <= ahi)) b_in_a = 0;
    }
    return intersect && !a_in_b && !b_in_a;
}

/* Far enough apart that no list can relate them: the gap on some axis   */
/* exceeds twice the larger box width.                                    */
static int box_far(int la, const int64_t *a, int lb, const int64_t *b) {
    int L = la > lb ? la : lb;
    int64_t wa = 1LL << (L - la), wb = 1LL << (L - lb);
    int64_t w = wa > wb ? wa : wb;
    for (int d = 0; d < 3; ++d) {
        int64_t alo = a[d] * wa, ahi = alo + wa, blo = b[d] * wb, bhi = blo + wb;
        int64_t gap = (alo > bhi) ? alo - bhi : ((blo > ahi) ? blo - ahi : 0);
        if (gap > 2 * w) return 1;
    }
    return 0;
}

/*
 * List of target box t (kind: 0 = U, 1 = V, 2 = W, 3 = X), all sources in
 * canonical node order.  Writes up to cap entries to out and returns the
 * full count.
 *   U(t): t a leaf; leaves s adjacent to t, and t itself.
 *   V(t): s at the level of t, s != t, not adjacent to t, parent(s) equal or
 *         adjacent to parent(t).
 *   W(t): t a leaf; level(s) > level(t), s not adjacent to t, parent(s)
 *         adjacent to t.
 *   X(t): s a leaf; level(t) > level(s), t not adjacent to s, parent(t)
 *         adjacent to s.
 */
int64_t orc_list_of(int64_t nb, const int32_t *level, const int64_t *coord, const int32_t *parent,
                    const int32_t *isleaf, int kind, int64_t t, int64_t *out, int64_t cap) {
    int64_t cnt = 0;
    const int lt = level[t];
    const int64_t *ct = coord + 3 * t;
    for (int64_t s = 0; s < nb; ++s) {
        const int ls = level[s];
        const int64_t *cs = coord + 3 * s;
        int in = 0;
        if (box_far(lt, ct, ls, cs)) continue;
        if (kind == 0) {
            in = isleaf[t] && isleaf[s] && (s == t || box_adjacent(lt, ct, ls, cs));
        } else if (kind == 1) {
            if (ls == lt && s != t && parent[s] >= 0 && parent[t] >= 0 &&
                !box_adjacent(lt, ct, ls, cs)) {
                int64_t ps = parent[s], pt = parent[t];
                in = (ps == pt) || box_adjacent(level[ps], coord + 3 * ps, level[pt], coord + 3 * pt);
            }
        } else if (kind == 2) {
            if (isleaf[t] && ls > lt && !box_adjacent(lt, ct, ls, cs)) {
                int64_t ps = parent[s];
                in = box_adjacent(level[ps], coord + 3 * ps, lt, ct);
            }
        } else {
            if (isleaf[s] && lt > ls && parent[t] >= 0 && !box_adjacent(lt, ct, ls, cs)) {
                int64_t pt = parent[t];
                in = box_adjacent(level[pt], coord + 3 * pt, ls, cs);
            }
        }
        if (in) {
            if (cnt < cap) out[cnt] = s;
            ++cnt;
        }
    }
    return cnt;
}

/* Counts of one list kind for every target (first pass of CSR assembly). */
void orc_list_counts(int64_t nb, const int32_t *level, const int64_t *coord, const int32_t *parent,
                     const int32_t *isleaf, int kind, int64_t *counts) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nb; ++t)
        counts[t] = orc_list_of(nb, level, coord, parent, isleaf, kind, t, NULL, 0);
}

/* Fill pass: ptr is the exclusive scan of the counts. */
void orc_list_fill(int64_t nb, const int32_t *level, const int64_t *coord, const int32_t *parent,
                   const int32_t *isleaf, int kind, const int64_t *ptr, int64_t *idx) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nb; ++t)
        orc_list_of(nb, level, coord, parent, isleaf, kind, t, idx + ptr[t], ptr[t + 1] - ptr[t]);
}

/* ---------------------------------------------------------------------- */
/* KIFMM evaluation (Sec. 2.2).                                           */
/* ---------------------------------------------------------------------- */
typedef struct {
    /* tree (canonical order: level, then Morton prefix) */
    int64_t nb;
    const int32_t *level;
    const int64_t *coord;  /* [nb,3] integer box coordinates at its level */
    const int32_t *parent; /* -1 for the root */
    const int32_t *isleaf;
    const int64_t *first;  /* first sorted particle */
    const int64_t *count;
    const int64_t *child_first; /* children are contiguous */
    const int64_t *nchild;
    int32_t max_level;
    double lo[3], side;
    /* particles in sorted order */
    const double *x;
    const double *q;
    /* lists (CSR) */
    const int64_t *u_ptr, *u_idx, *v_ptr, *v_idx, *w_ptr, *w_idx, *x_ptr, *x_idx;
    /* operators on the unit box (half-width 1) */
    int ns;
    const double *surf;     /* [ns,3] unit surface points in [-1,1]^3 */
    double a_ue, a_uc, a_de, a_dc;
    const double *m2m;      /* [8][ns][ns]  K(UC_parent, UE_child)   */
    const double *m2l;      /* [316][ns][ns] K(DC_target, UE_source) */
    const double *l2l;      /* [8][ns][ns]  K(DC_child, DE_parent)   */
    const double *up_u, *up_sinv, *up_v; /* pinv K(UC,UE) = V diag(sinv) U^T */
    const double *dn_u, *dn_sinv, *dn_v; /* pinv K(DC,DE)                    */
    /* work / outputs */
    double *q_up;  /* [nb,ns] upward equivalent densities   */
    double *d_chk; /* [nb,ns] downward check potentials     */
    double *q_dn;  /* [nb,ns] downward equivalent densities */
    double *pot;   /* [N]   sorted order */
    double *grad;  /* [N,3] sorted order */
} orc_fmm;

static void box_center(const orc_fmm *f, int64_t b, double *c, double *h) {
    double w = f->side / (double)(1LL << f->level[b]);
    for (int d = 0; d < 3; ++d) c[d] = f->lo[d] + ((double)f->coord[3 * b + d] + 0.5) * w;
    *h = 0.5 * w;
}

/* Equivalent-density solve: out = h * V diag(sinv) U^T chk (pinv of the    */
/* unit-box check-from-equivalent matrix, scaled by the homogeneity of 1/r).*/
static void solve_density(int ns, const double *u, const double *sinv, const double *v, double h,
                          const double *chk, double *out) {
    double *t = (double *)malloc(sizeof(double) * (size_t)ns);
    for (int i = 0; i < ns; ++i) {
        double s = 0.0;
        for (int j = 0; j < ns; ++j) s += u[j * ns + i] * chk[j];
        t[i] = s * sinv[i];
    }
    for (int k = 0; k < ns; ++k) {
        double s = 0.0;
        for (int i = 0; i < ns; ++i) s += v[k * ns + i] * t[i];
        out[k] = h * s;
    }
    free(t);
}

static int oct_of(const orc_fmm *f, int64_t b) {
    return (int)(4 * (f->coord[3 * b] & 1) + 2 * (f->coord[3 * b + 1] & 1) + (f->coord[3 * b + 2] & 1));
}

static int m2l_offset_index(int dx, int dy, int dz) {
    /* offsets d in {-3..3}^3 minus {-1..1}^3, enumerated lexicographically */
    int idx = 0;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b)
            for (int c = -3; c <= 3; ++c) {
                if (a >= -1 && a <= 1 && b >= -1 && b <= 1 && c >= -1 && c <= 1) continue;
                if (a == dx && b == dy && c == dz) return idx;
                ++idx;
            }
    return -1;
}

/* Upward pass: P2M at leaves, M2M bottom-up (check evaluation + solve). */
static void upward(orc_fmm *f) {
    const int ns = f->ns;
    for (int lev = f->max_level; lev >= 0; --lev) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t b = 0; b < f->nb; ++b) {
            if (f->level[b] != lev) continue;
            double c[3], h;
            box_center(f, b, c, &h);
            double *chk = (double *)calloc((size_t)ns, sizeof(double));
            if (f->isleaf[b]) {
                /* P2M: potential of the box's particles on its upward check surface */
                for (int j = 0; j < ns; ++j) {
                    double y[3];
                    for (int d = 0; d < 3; ++d) y[d] = c[d] + f->a_uc * h * f->surf[3 * j + d];
                    double s = 0.0;
                    for (int64_t i = f->first[b]; i < f->first[b] + f->count[b]; ++i)
                        s += lap_pot(y[0] - f->x[3 * i], y[1] - f->x[3 * i + 1], y[2] - f->x[3 * i + 2]) * f->q[i];
                    chk[j] = s;
                }
            } else {
                /* M2M: children's equivalent densities on the parent's check surface */
                for (int64_t ci = 0; ci < f->nchild[b]; ++ci) {
                    int64_t ch = f->child_first[b] + ci;
                    const double *mat = f->m2m + (size_t)oct_of(f, ch) * ns * ns;
                    const double *qc = f->q_up + (size_t)ch * ns;
                    for (int j = 0; j < ns; ++j) {
                        double s = 0.0;
                        for (int k = 0; k < ns; ++k) s += mat[j * ns + k] * qc[k];
                        chk[j] += s / h;
                    }
                }
            }
            solve_density(ns, f->up_u, f->up_sinv, f->up_v, h, chk, f->q_up + (size_t)b * ns);
            free(chk);
        }
    }
}

/* M2L (V list) and P2L (X list) into the downward check potentials. */
static void interactions(orc_fmm *f) {
    const int ns = f->ns;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < f->nb; ++b) {
        double c[3], h;
        box_center(f, b, c, &h);
        double *chk = f->d_chk + (size_t)b * ns;
        for (int64_t e = f->v_ptr[b]; e < f->v_ptr[b + 1]; ++e) {
            int64_t a = f->v_idx[e];
            int o = m2l_offset_index((int)(f->coord[3 * a] - f->coord[3 * b]),
                                     (int)(f->coord[3 * a + 1] - f->coord[3 * b + 1]),
                                     (int)(f->coord[3 * a + 2] - f->coord[3 * b + 2]));
            const double *mat = f->m2l + (size_t)o * ns * ns;
            const double *qa = f->q_up + (size_t)a * ns;
            for (int j = 0; j < ns; ++j) {
                double s = 0.0;
                for (int k = 0; k < ns; ++k) s += mat[j * ns + k] * qa[k];
                chk[j] += s / h;
            }
        }
        for (int64_t e = f->x_ptr[b]; e < f->x_ptr[b + 1]; ++e) {
            int64_t a = f->x_idx[e];
            for (int j = 0; j < ns; ++j) {
                double y[3];
                for (int d = 0; d < 3; ++d) y[d] = c[d] + f->a_dc * h * f->surf[3 * j + d];
                double s = 0.0;
                for (int64_t i = f->first[a]; i < f->first[a] + f->count[a]; ++i)
                    s += lap_pot(y[0] - f->x[3 * i], y[1] - f->x[3 * i + 1], y[2] - f->x[3 * i + 2]) * f->q[i];
                chk[j] += s;
            }
        }
    }
}

/* Downward pass: L2L top-down, then the downward equivalent-density solve. */
static void downward(orc_fmm *f) {
    const int ns = f->ns;
    for (int lev = 0; lev <= f->max_level; ++lev) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t b = 0; b < f->nb; ++b) {
            if (f->level[b] != lev) continue;
            double c[3], h;
            box_center(f, b, c, &h);
            double *chk = f->d_chk + (size_t)b * ns;
            int64_t p = f->parent[b];
            if (p >= 0) {
                double cp[3], hp;
                box_center(f, p, cp, &hp);
                const double *mat = f->l2l + (size_t)oct_of(f, b) * ns * ns;
                const double *qp = f->q_dn + (size_t)p * ns;
                for (int j = 0; j < ns; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < ns; ++k) s += mat[j * ns + k] * qp[k];
                    chk[j] += s / hp;
                }
            }
            solve_density(ns, f->dn_u, f->dn_sinv, f->dn_v, h, chk, f->q_dn + (size_t)b * ns);
        }
    }
}

/* Leaf evaluation: L2P, M2P (W list) and P2P (U list). */
static void leaves(orc_fmm *f) {
    const int ns = f->ns;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < f->nb; ++b) {
        if (!f->isleaf[b]) continue;
        double c[3], h;
        box_center(f, b, c, &h);
        for (int64_t i = f->first[b]; i < f->first[b] + f->count[b]; ++i) {
            const double *xi = f->x + 3 * i;
            double p = 0.0, g[3] = {0.0, 0.0, 0.0};
            /* L2P: downward equivalent density on the DE surface */
            const double *qd = f->q_dn + (size_t)b * ns;
            for (int k = 0; k < ns; ++k) {
                double y[3];
                for (int d = 0; d < 3; ++d) y[d] = c[d] + f->a_de * h * f->surf[3 * k + d];
                lap_pot_grad(xi[0] - y[0], xi[1] - y[1], xi[2] - y[2], qd[k], &p, g);
            }
            /* M2P: upward equivalent densities of W-list boxes */
            for (int64_t e = f->w_ptr[b]; e < f->w_ptr[b + 1]; ++e) {
                int64_t a = f->w_idx[e];
                double ca[3], ha;
                box_center(f, a, ca, &ha);
                const double *qa = f->q_up + (size_t)a * ns;
                for (int k = 0; k < ns; ++k) {
                    double y[3];
                    for (int d = 0; d < 3; ++d) y[d] = ca[d] + f->a_ue * ha * f->surf[3 * k + d];
                    lap_pot_grad(xi[0] - y[0], xi[1] - y[1], xi[2] - y[2], qa[k], &p, g);
                }
            }
            /* P2P: particles of U-list leaves (self excluded by r > 0) */
            for (int64_t e = f->u_ptr[b]; e < f->u_ptr[b + 1]; ++e) {
                int64_t a = f->u_idx[e];
                for (int64_t j = f->first[a]; j < f->first[a] + f->count[a]; ++j)
                    lap_pot_grad(xi[0] - f->x[3 * j], xi[1] - f->x[3 * j + 1], xi[2] - f->x[3 * j + 2],
                                 f->q[j], &p, g);
            }
            f->pot[i] = p;
            f->grad[3 * i] = g[0];
            f->grad[3 * i + 1] = g[1];
            f->grad[3 * i + 2] = g[2];
        }
    }
}

void orc_fmm_evaluate(orc_fmm *f) {
    memset(f->d_chk, 0, sizeof(double) * (size_t)f->nb * (size_t)f->ns);
    upward(f);
    interactions(f);
    downward(f);
    leaves(f);
}

int orc_fmm_struct_size(void) { return (int)sizeof(orc_fmm); }
