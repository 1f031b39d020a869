"""KIFMM oracle: plain FP64 CPU reference of the long-range force evaluation.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline / reference legs import this module; the GPU library
never does, and the two share no code (inputs come from ``workloads``).

It follows the paper's outline of the kernel-independent FMM (Sec. 2.2): an
adaptive octree with at most M points per leaf, an upward pass producing
equivalent densities on surfaces around each box, M2L between boxes in each
other's far zone but not in their parents', a downward pass, and the leaf
evaluation of far field plus near field.  The details the paper leaves open
are taken from the original KIFMM (Ying, Biros & Zorin 2004, cited in
Sec. 2.2) and fixed as follows:

* Kernel: K(x, y) = 1/(4 pi |x - y|), the normalisation of Eq. 3; pairs at
  zero distance contribute nothing.  Outputs are pot_i = sum_j K q_j and its
  gradient; the physical potential is ``coef`` times that (coef = 1 gives
  Eq. 3 units, 1/eps0 SI Coulomb, -4 pi G gravity with masses as charges,
  which is Eq. 4 read as attractive).
* Surfaces: box centre c, half-width h, points c + alpha h (-1 + 2 (i,j,k)/(p-1))
  with at least one index on the boundary, lexicographic; n_s = 6(p-1)^2 + 2.
  alpha = 1.05 (upward equivalent, downward check), 2.95 (upward check,
  downward equivalent).
* Pseudo-inverse: SVD, singular values below eps * sigma_max dropped; the
  threshold must not lie within a factor 1.1 of any sigma_i / sigma_max (gap
  check), so that any backward-stable SVD truncates the same modes.  It is
  applied as V (Sigma^-1 (U^T b)), never as an explicit matrix.
* Tree: root cube from the per-axis minimum and the largest extent; 21-bit
  quantisation, Morton order x-highest; stable sort; split while
  count > M and level < max_depth; only non-empty children exist; canonical
  node order (level, Morton prefix).
* Lists: U, V, W, X of the adaptive KIFMM, classified from their definitions;
  a W/X interaction whose finer box is a leaf with at most n_s points is
  summed directly (moved to U), the original KIFMM's cost rule.
* Compressed M2L (optional; the operators are matrices computed from the
  kernel, Sec. 2.2, so a low-rank form of them is another such matrix): the
  316 M2L matrices share a left basis (the leading left singular vectors of
  their mean-free forms side by side) and a right basis (the leading right
  singular vectors of the full matrices stacked), truncated at eps * sigma_0
  with the ranks rounded up to fill 32-wide tiles (the left rank leaves one
  slot for the mean) and lowered off any cluster of equal singular values;
  each matrix is replaced by its projection (U U^T K0 + 1 m^T) V V^T.
* Tensor kernel: the direct sum of Stokeslets (point forces in Stokes flow),
  the kind of vector/tensor kernel Eq. 1 admits, and the KIFMM with it (the
  same tree, lists, surfaces and regularised pseudo-inverses; 3-vector
  densities).
* Periodic sums (Sec. 2.4): a neutral cubic cell repeated over Z^3, summed
  by Ewald's split with the conducting boundary (the mean potential of the
  cell is zero); a charged cell is refused, the paper's neutrality condition.
  The periodic KIFMM takes the cell as the root, runs the lists over the
  cell and its 26 neighbouring images, brings the farther images in through
  one operator on the root's equivalent density, and corrects the potential
  by the second-moment trace that density does not carry.

Parity status: every function here is pinned by tests under tests/ against
closed forms, invariants or brute force (see the test module docstrings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

ALPHA_UE = 1.05
ALPHA_UC = 2.95
ALPHA_DE = 2.95
ALPHA_DC = 1.05
BITS = 21


def build() -> str:
    """Compile the oracle's C core (gcc, OpenMP, no FMA contraction)."""
    return _lib()._name


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        out_dir = os.path.join(_HERE, "_build")
        os.makedirs(out_dir, exist_ok=True)
        so = os.path.join(out_dir, "liborc.so")
        src = os.path.join(_HERE, "kifmm_oracle.c")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                                   "-ffp-contract=off", src, "-o", tmp, "-lm"])
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.orc_direct.argtypes = [I64, P, P, I64, P, P, P]
        lib.orc_bbox.argtypes = [I64, P, P, P]
        lib.orc_morton.argtypes = [I64, P, P, ctypes.c_double, P]
        lib.orc_list_counts.argtypes = [I64, P, P, P, P, ctypes.c_int, P]
        lib.orc_list_fill.argtypes = [I64, P, P, P, P, ctypes.c_int, P, P]
        lib.orc_list_of.argtypes = [I64, P, P, P, P, ctypes.c_int, I64, P, I64]
        lib.orc_list_of.restype = I64
        lib.orc_fmm_evaluate.argtypes = [P]
        lib.orc_fmm_struct_size.restype = ctypes.c_int
        _LIB = lib
        return lib


def _p(a):
    return a.ctypes.data if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Direct sum (Sec. 1: all pairs; Eq. 1 with the Laplace kernel, Eq. 3 units)
# ---------------------------------------------------------------------------
def direct(x, q, targets=None):
    """pot, grad at ``targets`` (default: the sources) from all sources,
    zero-distance pairs excluded."""
    lib = _lib()
    x = _f64(x).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    t = x if targets is None else _f64(targets).reshape(-1, 3)
    pot = np.empty(t.shape[0])
    grad = np.empty((t.shape[0], 3))
    lib.orc_direct(x.shape[0], _p(x), _p(q), t.shape[0], _p(t), _p(pot), _p(grad))
    return pot, grad


# ---------------------------------------------------------------------------
# Morton keys and the adaptive octree (Sec. 2.2, first step)
# ---------------------------------------------------------------------------
def bbox(x):
    lib = _lib()
    x = _f64(x).reshape(-1, 3)
    lo = np.empty(3)
    side = np.empty(1)
    lib.orc_bbox(x.shape[0], _p(x), _p(lo), _p(side))
    return lo, float(side[0])


def morton(x, lo, side):
    lib = _lib()
    x = _f64(x).reshape(-1, 3)
    lo = _f64(lo)
    keys = np.empty(x.shape[0], dtype=np.uint64)
    lib.orc_morton(x.shape[0], _p(x), _p(lo), float(side), _p(keys))
    return keys


def deinterleave(prefix: int, level: int):
    """Integer box coordinates (x, y, z) of a Morton prefix of ``level`` digits."""
    c = [0, 0, 0]
    for b in range(level):
        digit = (prefix >> (3 * b)) & 7
        c[0] |= ((digit >> 2) & 1) << b
        c[1] |= ((digit >> 1) & 1) << b
        c[2] |= (digit & 1) << b
    return c


def build_tree(keys_sorted, leaf_cap: int, max_depth: int):
    """Adaptive octree over sorted keys: a box splits while it holds more than
    ``leaf_cap`` points and its level is below ``max_depth``; only non-empty
    children are created.  Nodes come out in canonical (level, prefix) order
    with each node's children contiguous."""
    keys_sorted = np.asarray(keys_sorted, dtype=np.uint64)
    n = keys_sorted.shape[0]
    level, prefix, first, count, parent = [0], [0], [0], [n], [-1]
    child_first, nchild = [], []
    begin = 0
    while begin < len(level):
        end = len(level)
        for b in range(begin, end):
            lev = level[b]
            if count[b] > leaf_cap and lev < max_depth:
                shift = np.uint64(3 * (BITS - lev - 1))
                lo_i = first[b]
                sub = keys_sorted[lo_i:lo_i + count[b]]
                digits = ((sub >> shift) & np.uint64(7)).astype(np.int64)
                child_first.append(len(level))
                nc = 0
                for o in range(8):
                    a = int(np.searchsorted(digits, o, side="left"))
                    e = int(np.searchsorted(digits, o, side="right"))
                    if e > a:
                        level.append(lev + 1)
                        prefix.append((prefix[b] << 3) | o)
                        first.append(lo_i + a)
                        count.append(e - a)
                        parent.append(b)
                        nc += 1
                nchild.append(nc)
            else:
                child_first.append(-1)
                nchild.append(0)
        begin = end
    nb = len(level)
    coord = np.array([deinterleave(prefix[b], level[b]) for b in range(nb)], dtype=np.int64).reshape(nb, 3)
    tree = {
        "level": np.array(level, dtype=np.int32),
        "prefix": np.array(prefix, dtype=np.uint64),
        "coord": coord,
        "first": np.array(first, dtype=np.int64),
        "count": np.array(count, dtype=np.int64),
        "parent": np.array(parent, dtype=np.int32),
        "child_first": np.array(child_first, dtype=np.int64),
        "nchild": np.array(nchild, dtype=np.int64),
    }
    tree["isleaf"] = (tree["nchild"] == 0).astype(np.int32)
    tree["nb"] = nb
    tree["max_level"] = int(tree["level"].max())
    return tree


def sort_and_tree(x, leaf_cap: int, max_depth: int):
    """Root cube, keys, stable sort (ties by input index) and the octree."""
    lo, side = bbox(x)
    keys = morton(x, lo, side)
    perm = np.argsort(keys, kind="stable")
    tree = build_tree(keys[perm], leaf_cap, max_depth)
    tree.update(lo=lo, side=side, keys=keys, perm=perm)
    return tree


# ---------------------------------------------------------------------------
# Interaction lists (Sec. 2.2, third step; adaptive U/V/W/X of Ying et al.)
# ---------------------------------------------------------------------------
LIST_KINDS = {"U": 0, "V": 1, "W": 2, "X": 3}


def lists(tree):
    """CSR lists {kind: (ptr, idx)} for every node, sources in node order."""
    lib = _lib()
    nb = tree["nb"]
    args = (nb, _p(tree["level"]), _p(tree["coord"]), _p(tree["parent"]), _p(tree["isleaf"]))
    out = {}
    for name, k in LIST_KINDS.items():
        counts = np.empty(nb, dtype=np.int64)
        lib.orc_list_counts(*args, k, _p(counts))
        ptr = np.zeros(nb + 1, dtype=np.int64)
        np.cumsum(counts, out=ptr[1:])
        idx = np.empty(int(ptr[-1]), dtype=np.int64)
        lib.orc_list_fill(*args, k, _p(ptr), _p(idx))
        out[name] = (ptr, idx)
    return out


def direct_threshold(ns: int, direct_max: int = 0) -> int:
    """Particle count up to which a W/X box is evaluated directly: n_s by
    default (direct_max = 0), none when direct_max < 0."""
    if direct_max < 0:
        return -1
    return ns if direct_max == 0 else int(direct_max)


def effective_lists(tree, lst, thr: int):
    """Lists as evaluated: a W or X interaction whose finer box (the W member,
    or the X list's owner) is a leaf holding at most ``thr`` particles is
    evaluated directly, so its source moves to the U list.

    This is the original KIFMM's cost rule (Ying, Biros & Zorin 2004, the
    adaptive lists cited in Sec. 2.2): M2P costs n_s evaluations per target
    and P2L n_s per source, so a box with fewer points than its equivalent
    surface is cheaper, and exact, to sum point by point.  The rule is the
    same from both sides of a pair (A in W(B) iff B in X(A)), so U stays
    symmetric and X stays the transpose of W."""
    if thr < 0:
        return lst
    nb = tree["nb"]
    leaf = tree["isleaf"].astype(bool)
    cnt = tree["count"]
    small = leaf & (cnt <= thr)

    def rows(kind):
        ptr, idx = lst[kind]
        return [idx[ptr[b]:ptr[b + 1]] for b in range(nb)]

    U, V, W, X = (rows(k) for k in "UVWX")
    U2, W2, X2 = [], [], []
    for b in range(nb):
        w_keep = [a for a in W[b] if not small[a]]
        w_move = [a for a in W[b] if small[a]]
        x_move = list(X[b]) if small[b] else []
        x_keep = [] if small[b] else list(X[b])
        U2.append(sorted(list(U[b]) + w_move + x_move))
        W2.append(w_keep)
        X2.append(x_keep)

    def csr(r):
        ptr = np.zeros(nb + 1, dtype=np.int64)
        ptr[1:] = np.cumsum([len(v) for v in r])
        idx = np.array([a for v in r for a in v], dtype=np.int64)
        return ptr, idx

    return {"U": csr(U2), "V": lst["V"], "W": csr(W2), "X": csr(X2)}


def list_of(tree, kind: str, t: int):
    """One target's list (used to check sampled boxes of large trees)."""
    lib = _lib()
    nb = tree["nb"]
    args = (nb, _p(tree["level"]), _p(tree["coord"]), _p(tree["parent"]), _p(tree["isleaf"]))
    n = lib.orc_list_of(*args, LIST_KINDS[kind], t, None, 0)
    out = np.empty(max(n, 1), dtype=np.int64)
    lib.orc_list_of(*args, LIST_KINDS[kind], t, _p(out), n)
    return out[:n]


# ---------------------------------------------------------------------------
# Surfaces and translation operators (Sec. 2.2: densities on equivalent
# surfaces; operators are matrices computed automatically for the kernel)
# ---------------------------------------------------------------------------
def surface(p: int):
    """Unit-cube surface grid: (-1 + 2 (i,j,k)/(p-1)) with at least one index
    on the boundary, lexicographic in (i, j, k)."""
    pts = []
    for i in range(p):
        for j in range(p):
            for k in range(p):
                if i in (0, p - 1) or j in (0, p - 1) or k in (0, p - 1):
                    pts.append((-1 + 2 * i / (p - 1), -1 + 2 * j / (p - 1), -1 + 2 * k / (p - 1)))
    return np.array(pts, dtype=np.float64)


def kernel_matrix(targets, sources):
    d = targets[:, None, :] - sources[None, :, :]
    r = np.sqrt(np.sum(d * d, axis=-1))
    with np.errstate(divide="ignore"):
        k = np.where(r > 0, 1.0 / (4.0 * np.pi * r), 0.0)
    return k


def m2l_offsets():
    """The 316 relative positions d in {-3..3}^3 minus {-1..1}^3, in
    lexicographic order (index = position in this list)."""
    out = []
    for a in range(-3, 4):
        for b in range(-3, 4):
            for c in range(-3, 4):
                if -1 <= a <= 1 and -1 <= b <= 1 and -1 <= c <= 1:
                    continue
                out.append((a, b, c))
    return np.array(out, dtype=np.int64)


def child_offset(o: int):
    """Centre of child octant o = 4x + 2y + z of a half-width-1 parent."""
    return np.array([0.5 if (o >> 2) & 1 else -0.5, 0.5 if (o >> 1) & 1 else -0.5,
                     0.5 if o & 1 else -0.5])


class PinvGapError(ValueError):
    pass


def svd_pinv_factors(k, eps: float):
    """Truncated SVD pseudo-inverse factors (U, sinv, V) with pinv = V diag(sinv) U^T."""
    u, s, vh = np.linalg.svd(k)
    rel = s / s[0]
    near = np.logical_and(rel > eps / 1.1, rel < eps * 1.1)
    if np.any(near):
        raise PinvGapError(f"singular value within a factor 1.1 of eps={eps:g}: {rel[near]}")
    sinv = np.where(rel >= eps, 1.0 / s, 0.0)
    return np.ascontiguousarray(u), sinv, np.ascontiguousarray(vh.T), s


def operators(p: int, eps: float = 1e-12):
    """Unit-box (half-width 1) matrices; a box of half-width h scales them by 1/h."""
    S = surface(p)
    ns = S.shape[0]
    ops = {"p": p, "ns": ns, "surf": S, "eps": eps}
    ops["up"] = svd_pinv_factors(kernel_matrix(ALPHA_UC * S, ALPHA_UE * S), eps)
    ops["dn"] = svd_pinv_factors(kernel_matrix(ALPHA_DC * S, ALPHA_DE * S), eps)
    ops["m2m"] = np.stack([kernel_matrix(ALPHA_UC * S, child_offset(o) + 0.5 * ALPHA_UE * S)
                           for o in range(8)])
    ops["l2l"] = np.stack([kernel_matrix(child_offset(o) + 0.5 * ALPHA_DC * S, ALPHA_DE * S)
                           for o in range(8)])
    ops["m2l"] = np.stack([kernel_matrix(ALPHA_DC * S, 2.0 * d + ALPHA_UE * S) for d in m2l_offsets()])
    return ops


def operators_perturbed(p: int, seed: int, eps: float = 1e-12):
    """The operators of ``operators(p, eps)`` recomputed as another correct
    FP64 implementation might: every pseudo-inverse from its check-from-
    equivalent matrix plus a random perturbation of norm 2^-53 ||K|| (the
    backward error of any backward-stable SVD), every translation matrix
    with each entry moved by up to one unit in its last place (the rounding
    of one kernel evaluation).  Running the KIFMM with these and with the
    unperturbed operators measures the rounding floor of the method itself:
    how far two correct FP64 evaluations of it can lie apart."""
    rng = np.random.default_rng(seed)
    ops = dict(operators(p, eps))
    S = ops["surf"]
    unit = 2.0 ** -53

    def pert(k):
        e = rng.standard_normal(k.shape)
        return k + unit * np.linalg.norm(k, 2) * e / np.linalg.norm(e, 2)

    ops["up"] = svd_pinv_factors(pert(kernel_matrix(ALPHA_UC * S, ALPHA_UE * S)), eps)
    ops["dn"] = svd_pinv_factors(pert(kernel_matrix(ALPHA_DC * S, ALPHA_DE * S)), eps)
    for k in ("m2m", "l2l", "m2l"):
        a = np.asarray(ops[k])
        ops[k] = a * (1.0 + 2.0 * unit * rng.uniform(-1.0, 1.0, size=a.shape))
    return ops


M2L_GAP = 1.001


def compress_rank(sig, eps: float, tile: int = 32, mean_slot: int = 0) -> int:
    """Rank kept from descending singular values ``sig``: the count above
    eps * sig[0], rounded up so that rank + mean_slot is a multiple of
    ``tile`` (at most len(sig)), then lowered while the cut would split a
    cluster of equal values (sig[r-1] <= M2L_GAP * sig[r])."""
    sig = np.asarray(sig, dtype=np.float64)
    n = sig.shape[0]
    r0 = int(np.sum(sig > eps * sig[0]))
    r = min(n, tile * ((r0 + mean_slot + tile - 1) // tile) - mean_slot)
    while 1 < r < n and sig[r - 1] <= M2L_GAP * sig[r]:
        r -= 1
    return r


def compress_m2l(ops, eps: float, tile: int = 32):
    """Operators with every M2L matrix K_o (DC <- UE + 2 d_o, on equivalent
    densities) replaced by its projection onto the shared bases:
    K_o -> (U U^T K0_o + 1 m_o^T) V V^T, where m_o is the mean of K_o over its
    outputs (rows), K0_o = K_o - 1 m_o^T, U = leading left singular vectors of
    [K0_1 ... K0_316] (rank r_L, mean_slot 1) and V = leading right singular
    vectors of [K_1; ...; K_316] (rank r_R).  Returns (ops', info) with the
    ranks and both singular value lists."""
    K = np.asarray(ops["m2l"], dtype=np.float64)
    m = K.mean(axis=1)
    K0 = K - m[:, None, :]
    u_l, s_l, _ = np.linalg.svd(np.concatenate(list(K0), axis=1), full_matrices=False)
    _, s_r, vh_r = np.linalg.svd(np.concatenate(list(K), axis=0), full_matrices=False)
    r_l = compress_rank(s_l, eps, tile, 1)
    r_r = compress_rank(s_r, eps, tile, 0)
    U = u_l[:, :r_l]
    V = vh_r[:r_r].T
    Kh = (np.einsum("ij,ojk->oik", U @ U.T, K0) + np.ones((1, K.shape[1], 1)) * m[:, None, :]) @ (V @ V.T)
    out = dict(ops)
    out["m2l"] = np.ascontiguousarray(Kh)
    return out, {"r_l": r_l, "r_r": r_r, "s_l": s_l, "s_r": s_r, "U": U, "V": V}


# ---------------------------------------------------------------------------
# KIFMM evaluation
# ---------------------------------------------------------------------------
class _Fmm(ctypes.Structure):
    _fields_ = [
        ("nb", ctypes.c_int64),
        ("level", ctypes.c_void_p), ("coord", ctypes.c_void_p), ("parent", ctypes.c_void_p),
        ("isleaf", ctypes.c_void_p), ("first", ctypes.c_void_p), ("count", ctypes.c_void_p),
        ("child_first", ctypes.c_void_p), ("nchild", ctypes.c_void_p),
        ("max_level", ctypes.c_int32),
        ("lo", ctypes.c_double * 3), ("side", ctypes.c_double),
        ("x", ctypes.c_void_p), ("q", ctypes.c_void_p),
        ("u_ptr", ctypes.c_void_p), ("u_idx", ctypes.c_void_p),
        ("v_ptr", ctypes.c_void_p), ("v_idx", ctypes.c_void_p),
        ("w_ptr", ctypes.c_void_p), ("w_idx", ctypes.c_void_p),
        ("x_ptr", ctypes.c_void_p), ("x_idx", ctypes.c_void_p),
        ("ns", ctypes.c_int),
        ("surf", ctypes.c_void_p),
        ("a_ue", ctypes.c_double), ("a_uc", ctypes.c_double),
        ("a_de", ctypes.c_double), ("a_dc", ctypes.c_double),
        ("m2m", ctypes.c_void_p), ("m2l", ctypes.c_void_p), ("l2l", ctypes.c_void_p),
        ("up_u", ctypes.c_void_p), ("up_sinv", ctypes.c_void_p), ("up_v", ctypes.c_void_p),
        ("dn_u", ctypes.c_void_p), ("dn_sinv", ctypes.c_void_p), ("dn_v", ctypes.c_void_p),
        ("q_up", ctypes.c_void_p), ("d_chk", ctypes.c_void_p), ("q_dn", ctypes.c_void_p),
        ("pot", ctypes.c_void_p), ("grad", ctypes.c_void_p),
    ]


def kifmm(x, q, p: int = 6, leaf_cap: int = 64, max_depth: int = 20, eps: float = 1e-12,
          ops=None, tree=None, lst=None, direct_max: int = 0):
    """Potential and gradient (user order, Eq. 3 units) of every particle from
    all others, by the KIFMM.  ``lst`` (if given) holds the lists as
    classified; W/X interactions of small leaves are then moved to U by
    effective_lists (threshold from direct_threshold(n_s, direct_max)).
    Returns (pot, grad, info) where info holds the tree, the lists as
    evaluated and the intermediate densities (canonical node order)."""
    lib = _lib()
    x = _f64(x).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    n = x.shape[0]
    if tree is None:
        tree = sort_and_tree(x, leaf_cap, max_depth)
    if lst is None:
        lst = lists(tree)
    if ops is None:
        ops = operators(p, eps)
    lst = effective_lists(tree, lst, direct_threshold(ops["ns"], direct_max))
    perm = tree["perm"]
    xs = np.ascontiguousarray(x[perm])
    qsrt = np.ascontiguousarray(q[perm])
    nb, ns = tree["nb"], ops["ns"]
    q_up = np.zeros((nb, ns))
    d_chk = np.zeros((nb, ns))
    q_dn = np.zeros((nb, ns))
    pot_s = np.zeros(n)
    grad_s = np.zeros((n, 3))
    keep = [xs, qsrt]
    f = _Fmm()
    f.nb = nb
    for name in ("level", "coord", "parent", "isleaf", "first", "count", "child_first", "nchild"):
        arr = np.ascontiguousarray(tree[name])
        keep.append(arr)
        setattr(f, name, arr.ctypes.data)
    f.max_level = tree["max_level"]
    for d in range(3):
        f.lo[d] = tree["lo"][d]
    f.side = tree["side"]
    f.x, f.q = xs.ctypes.data, qsrt.ctypes.data
    for name in ("U", "V", "W", "X"):
        ptr, idx = lst[name]
        idx = idx if idx.size else np.zeros(1, dtype=np.int64)
        keep += [ptr, idx]
        setattr(f, name.lower() + "_ptr", ptr.ctypes.data)
        setattr(f, name.lower() + "_idx", idx.ctypes.data)
    f.ns = ns
    mats = {k: np.ascontiguousarray(ops[k]) for k in ("surf", "m2m", "m2l", "l2l")}
    keep += list(mats.values())
    f.surf, f.m2m, f.m2l, f.l2l = (mats[k].ctypes.data for k in ("surf", "m2m", "m2l", "l2l"))
    f.a_ue, f.a_uc, f.a_de, f.a_dc = ALPHA_UE, ALPHA_UC, ALPHA_DE, ALPHA_DC
    uu, us, uv, _ = ops["up"]
    du, ds, dv, _ = ops["dn"]
    keep += [uu, us, uv, du, ds, dv]
    f.up_u, f.up_sinv, f.up_v = uu.ctypes.data, us.ctypes.data, uv.ctypes.data
    f.dn_u, f.dn_sinv, f.dn_v = du.ctypes.data, ds.ctypes.data, dv.ctypes.data
    f.q_up, f.d_chk, f.q_dn = q_up.ctypes.data, d_chk.ctypes.data, q_dn.ctypes.data
    f.pot, f.grad = pot_s.ctypes.data, grad_s.ctypes.data
    assert ctypes.sizeof(f) == lib.orc_fmm_struct_size()
    lib.orc_fmm_evaluate(ctypes.byref(f))
    pot = np.empty(n)
    grad = np.empty((n, 3))
    pot[perm] = pot_s
    grad[perm] = grad_s
    info = {"tree": tree, "lists": lst, "ops": ops, "q_up": q_up, "d_chk": d_chk, "q_dn": q_dn}
    return pot, grad, info


# ---------------------------------------------------------------------------
# Derived quantities
# ---------------------------------------------------------------------------
def energy(q, pot, coef: float = 1.0):
    """Long-range potential energy U = 1/2 coef sum_i q_i pot_i (Sec. 2.4)."""
    return 0.5 * coef * float(np.dot(np.asarray(q, dtype=np.float64), np.asarray(pot, dtype=np.float64)))


def forces(q, grad, coef: float = 1.0):
    """Per-particle force F_i = -coef q_i grad_i (Eq. 3 for coef = 1)."""
    return -coef * np.asarray(q, dtype=np.float64)[:, None] * np.asarray(grad, dtype=np.float64)


def clump_reduce(x, q, grad, offsets, ref, coef: float = 1.0):
    """Clump force and torque (Sec. 2.4): sums over each clump's pebbles of
    F_k and (x_k - X_c) x F_k about the reference point X_c."""
    x = _f64(x).reshape(-1, 3)
    f = forces(q, grad, coef)
    ref = _f64(ref).reshape(-1, 3)
    nc = ref.shape[0]
    F = np.zeros((nc, 3))
    T = np.zeros((nc, 3))
    for c in range(nc):
        for k in range(int(offsets[c]), int(offsets[c + 1])):
            F[c] += f[k]
            T[c] += np.cross(x[k] - ref[c], f[k])
    return F, T


# ---------------------------------------------------------------------------
# Tensor kernel (Eq. 1 allows vector and tensor kernels; Stokes flow is the
# paper's example of one with its own periodic constraints, Sec. 2.4)
# ---------------------------------------------------------------------------
def stokeslet_direct(x, f, targets=None, mu: float = 1.0):
    """Velocity u(t) = sum_j G(t - x_j) f_j of point forces f_j at x_j, with the
    Stokeslet G(r) = (I / |r| + r r^T / |r|^3) / (8 pi mu); pairs at zero
    distance excluded.  x [N,3], f [N,3]; targets default to the sources."""
    x = _f64(x).reshape(-1, 3)
    f = _f64(f).reshape(-1, 3)
    t = x if targets is None else _f64(targets).reshape(-1, 3)
    u = np.zeros((t.shape[0], 3))
    for i in range(t.shape[0]):
        d = t[i][None, :] - x                      # [N, 3]
        r2 = np.sum(d * d, axis=1)
        ok = r2 > 0.0
        r = np.sqrt(r2[ok])
        dd, ff = d[ok], f[ok]
        u[i] = np.sum(ff / r[:, None], axis=0) + np.sum(dd * (np.sum(dd * ff, axis=1) / r ** 3)[:, None], axis=0)
    return u / (8.0 * np.pi * mu)


def stokeslet_matrix(targets, sources, mu: float = 1.0):
    """[3 nt, 3 ns] matrix of the Stokeslet: block (i, j) is G(t_i - s_j)
    (zero at zero distance); row 3 i + a, column 3 j + b."""
    t = _f64(targets).reshape(-1, 3)
    s = _f64(sources).reshape(-1, 3)
    d = t[:, None, :] - s[None, :, :]
    r2 = np.sum(d * d, axis=-1)
    ok = r2 > 0.0
    r = np.sqrt(np.where(ok, r2, 1.0))
    g = np.eye(3)[None, None, :, :] / r[:, :, None, None] + d[:, :, :, None] * d[:, :, None, :] / \
        (r ** 3)[:, :, None, None]
    g = np.where(ok[:, :, None, None], g, 0.0) / (8.0 * np.pi * mu)
    return g.transpose(0, 2, 1, 3).reshape(3 * t.shape[0], 3 * s.shape[0])


def kifmm_stokes(x, f, p: int = 6, leaf_cap: int = 64, max_depth: int = 20, eps: float = 1e-12,
                 mu: float = 1.0, direct_max: int = 0):
    """Velocities u_i = sum_{j != i} G(x_i - x_j) f_j by the KIFMM with the
    Stokeslet (Sec. 2.2's method for a tensor kernel of Eq. 1): the tree and
    lists of the Laplace oracle; every surface point carries a 3-vector
    density (3 n_s unknowns); the operators are Stokeslet matrices between
    the same surfaces, with the same regularised pseudo-inverses.  The
    Stokeslet is homogeneous of degree -1 like 1/r, so unit-box operators
    scale by 1/h.  The passes follow the Laplace oracle: P2M and M2M into
    upward check velocities and densities, M2L (V) and P2L (X) into downward
    check velocities, L2L, then L2P, M2P (W) and P2P (U) at the leaves."""
    x = _f64(x).reshape(-1, 3)
    f = _f64(f).reshape(-1, 3)
    tree = sort_and_tree(x, leaf_cap, max_depth)
    S = surface(p)
    ns = S.shape[0]
    lst = effective_lists(tree, lists(tree), direct_threshold(ns, direct_max))
    K = lambda t, s: stokeslet_matrix(t, s, mu)
    up = svd_pinv_factors(K(ALPHA_UC * S, ALPHA_UE * S), eps)
    dn = svd_pinv_factors(K(ALPHA_DC * S, ALPHA_DE * S), eps)
    pinv = lambda fac: fac[2] @ np.diag(fac[1]) @ fac[0].T
    P_up, P_dn = pinv(up), pinv(dn)
    m2m = [K(ALPHA_UC * S, child_offset(o) + 0.5 * ALPHA_UE * S) for o in range(8)]
    l2l = [K(child_offset(o) + 0.5 * ALPHA_DC * S, ALPHA_DE * S) for o in range(8)]
    offs = m2l_offsets()
    m2l = {tuple(d): K(ALPHA_DC * S, 2.0 * d + ALPHA_UE * S) for d in offs}
    perm = tree["perm"]
    xs, fs = x[perm], f[perm]
    nb = tree["nb"]
    level, coord, first, count = tree["level"], tree["coord"], tree["first"], tree["count"]
    w = tree["side"] / 2.0 ** level
    centre = tree["lo"][None, :] + (coord + 0.5) * w[:, None]
    half = 0.5 * w
    octant = 4 * (coord[:, 0] & 1) + 2 * (coord[:, 1] & 1) + (coord[:, 2] & 1)
    isleaf = tree["child_first"] < 0
    pts = lambda b: slice(int(first[b]), int(first[b] + count[b]))
    q_up = np.zeros((nb, 3 * ns))
    d_chk = np.zeros((nb, 3 * ns))
    q_dn = np.zeros((nb, 3 * ns))
    for lev in range(int(level.max()), -1, -1):           # upward
        for b in np.nonzero(level == lev)[0]:
            if isleaf[b]:
                chk = K(centre[b] + ALPHA_UC * half[b] * S, xs[pts(b)]) @ fs[pts(b)].ravel()
            else:
                chk = np.zeros(3 * ns)
                for c in range(int(tree["child_first"][b]), int(tree["child_first"][b] + tree["nchild"][b])):
                    chk += m2m[octant[c]] @ q_up[c] / half[b]
            q_up[b] = half[b] * (P_up @ chk)
    V, X, W, U = (lst[k] for k in "VXWU")
    for b in range(nb):                                     # M2L, P2L
        for a in V[1][V[0][b]:V[0][b + 1]]:
            d_chk[b] += m2l[tuple(coord[a] - coord[b])] @ q_up[a] / half[b]
        for a in X[1][X[0][b]:X[0][b + 1]]:
            d_chk[b] += K(centre[b] + ALPHA_DC * half[b] * S, xs[pts(a)]) @ fs[pts(a)].ravel()
    for lev in range(int(level.max()) + 1):                 # downward
        for b in np.nonzero(level == lev)[0]:
            pb = tree["parent"][b]
            if pb >= 0:
                d_chk[b] += l2l[octant[b]] @ q_dn[pb] / half[pb]
            q_dn[b] = half[b] * (P_dn @ d_chk[b])
    u = np.zeros((x.shape[0], 3))
    for b in np.nonzero(isleaf)[0]:                         # L2P, M2P, P2P
        xt = xs[pts(b)]
        ub = K(xt, centre[b] + ALPHA_DE * half[b] * S) @ q_dn[b]
        for a in W[1][W[0][b]:W[0][b + 1]]:
            ub += K(xt, centre[a] + ALPHA_UE * half[a] * S) @ q_up[a]
        for a in U[1][U[0][b]:U[0][b + 1]]:
            ub += K(xt, xs[pts(a)]) @ fs[pts(a)].ravel()
        u[perm[pts(b)]] = ub.reshape(-1, 3)
    return u


# ---------------------------------------------------------------------------
# Periodic sums (Sec. 2.4: periodic boundary conditions; the lattice sum of
# the Coulomb kernel converges only for a neutral cell)
# ---------------------------------------------------------------------------
class NotNeutralError(ValueError):
    pass


def check_neutral(q, rtol: float = 1e-12):
    """The cell's total charge must vanish (relative to sum |q|) for the
    periodic Coulomb sum to exist without a neutralising background."""
    q = _f64(q).reshape(-1)
    tot, mag = float(np.sum(q)), float(np.sum(np.abs(q)))
    if abs(tot) > rtol * max(mag, 1e-300):
        raise NotNeutralError(f"cell charge {tot:.3e} is not zero (sum |q| = {mag:.3e})")


def ewald(x, q, L: float, alpha: float = None, real_shells: int = 2, kmax: int = None):
    """Potential and gradient (Eq. 3 units, K = 1/(4 pi r)) at every particle of
    a neutral cubic cell [0, L)^3 repeated over Z^3, self term excluded, by
    Ewald's split into a real-space sum (erfc(alpha r) / r over the images
    within `real_shells` cells) and a reciprocal-space sum over k = 2 pi m / L,
    0 < |m_i| <= kmax, with the conducting ("tin-foil") boundary: the sum
    taken over growing spheres of images converges to this result when the
    cell's dipole moment vanishes.  alpha defaults to 6 / L; kmax to the
    shell where exp(-k^2 / (4 alpha^2)) drops below 1e-17."""
    x = _f64(x).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    check_neutral(q)
    L = float(L)
    a = 6.0 / L if alpha is None else float(alpha)
    if kmax is None:
        kmax = int(np.ceil(a * L * np.sqrt(4.0 * 39.2) / (2.0 * np.pi)))  # exp(-39.2) ~ 1e-17
    n = x.shape[0]
    pot = np.zeros(n)
    grad = np.zeros((n, 3))
    from math import pi, sqrt
    from scipy.special import erfc
    # real space
    rng = range(-real_shells, real_shells + 1)
    shifts = np.array([(i, j, k) for i in rng for j in rng for k in rng], dtype=np.float64) * L
    for i in range(n):
        d = x[i][None, None, :] - x[None, :, :] + shifts[:, None, :]   # [images, j, 3]
        r = np.sqrt(np.sum(d * d, axis=-1))
        self0 = np.zeros_like(r, dtype=bool)
        self0[np.all(shifts == 0.0, axis=1), i] = True
        r_ok = np.where(self0, 1.0, r)
        ec = erfc(a * r_ok)
        term = np.where(self0, 0.0, ec / r_ok)
        pot[i] += np.sum(term * q[None, :])
        # d/dx_i of erfc(a r)/r = -(erfc(a r)/r^2 + 2a/sqrt(pi) exp(-a^2 r^2)/r) * d/r
        g = np.where(self0, 0.0, (ec / r_ok ** 2 + 2.0 * a / sqrt(pi) * np.exp(-(a * r_ok) ** 2) / r_ok) / r_ok)
        grad[i] -= np.sum((g * q[None, :])[:, :, None] * d, axis=(0, 1))
    # reciprocal space
    m = np.arange(-kmax, kmax + 1, dtype=np.float64)
    M = np.stack(np.meshgrid(m, m, m, indexing="ij"), axis=-1).reshape(-1, 3)
    M = M[np.any(M != 0.0, axis=1)]
    k = 2.0 * pi / L * M
    k2 = np.sum(k * k, axis=1)
    w = (4.0 * pi / L ** 3) * np.exp(-k2 / (4.0 * a * a)) / k2            # [K]
    phase = x @ k.T                                                       # [n, K]
    c = (q[:, None] * np.cos(phase)).sum(axis=0)                         # C(k) = sum_j q_j cos(k.x_j)
    sn = (q[:, None] * np.sin(phase)).sum(axis=0)                        # S(k) = sum_j q_j sin(k.x_j)
    # sum_j q_j cos(k.(x_i - x_j)) = cos(k.x_i) C + sin(k.x_i) S
    pot += (np.cos(phase) * c[None, :] + np.sin(phase) * sn[None, :]) @ w
    # gradient: -k sin(k.(x_i - x_j)) summed = -k (sin(k.x_i) C - cos(k.x_i) S)
    fac = (np.sin(phase) * c[None, :] - np.cos(phase) * sn[None, :]) * w[None, :]
    grad -= fac @ k
    # self term of the Gaussian screening charge
    pot -= 2.0 * a / sqrt(pi) * q
    return pot / (4.0 * pi), grad / (4.0 * pi)


def _adjacent(la, ca, lb, cb):
    """Closed cubes of boxes (level la, integer coordinates ca [K,3]) and
    (lb, cb) intersect and neither contains the other (vectorised)."""
    la, lb = np.broadcast_arrays(np.asarray(la, np.int64), np.asarray(lb, np.int64))
    ca, cb = np.broadcast_arrays(np.asarray(ca, np.int64), np.asarray(cb, np.int64))
    L = np.maximum(la, lb)
    sa = (np.int64(1) << (L - la))[..., None]
    sb = (np.int64(1) << (L - lb))[..., None]
    alo, ahi, blo, bhi = ca * sa, (ca + 1) * sa, cb * sb, (cb + 1) * sb
    inter = np.all((alo <= bhi) & (blo <= ahi), axis=-1)
    a_in_b = np.all((blo <= alo) & (ahi <= bhi), axis=-1)
    b_in_a = np.all((alo <= blo) & (bhi <= ahi), axis=-1)
    return inter & ~a_in_b & ~b_in_a


def periodic_lists(tree):
    """U/V/W/X lists of every box of a tree whose root is the periodic cell,
    over the boxes of the cell and of its 26 neighbouring images: entries
    (box, image shift n in {-1, 0, 1}^3).  The definitions are those of the
    free-space lists applied to the tiling; an image box's parent is the
    parent's image, and the root's images are its colleagues (so its own
    lists hold only what its children cannot cover).  Images beyond the
    neighbours never enter: they act through the far-image operator."""
    nb, level, coord = tree["nb"], tree["level"].astype(np.int64), tree["coord"].astype(np.int64)
    parent, isleaf = tree["parent"], tree["isleaf"].astype(bool)
    shifts = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)], np.int64)
    src = np.repeat(np.arange(nb), 27)
    n = np.tile(np.arange(27), nb)
    ls = level[src]
    cs = coord[src] + shifts[n] * (np.int64(1) << ls)[:, None]
    ps = np.where(parent[src] >= 0, parent[src], 0)
    lps = level[ps]
    cps = coord[ps] + shifts[n] * (np.int64(1) << lps)[:, None]
    has_p = parent[src] >= 0
    out = {k: [] for k in "UVWX"}
    for t in range(nb):
        lt, ct = level[t], coord[t]
        adj = _adjacent(lt, ct[None, :], ls, cs)
        same = (src == t) & (n == 13)
        u = isleaf[t] & isleaf[src] & (same | adj)
        v = np.zeros_like(u)
        w = np.zeros_like(u)
        x = np.zeros_like(u)
        if parent[t] >= 0:
            pt = parent[t]
            par_eq = (ps == pt) & (n == 13) & has_p
            par_adj = _adjacent(level[pt], coord[pt][None, :], lps, cps) & has_p
            v = (ls == lt) & ~same & ~adj & (par_eq | par_adj)
            x = isleaf[src] & (lt > ls) & ~adj & _adjacent(level[pt], coord[pt][None, :], ls, cs)
        if isleaf[t]:
            w = (ls > lt) & ~adj & has_p & _adjacent(lt, ct[None, :], lps, cps)
        for k, m in zip("UVWX", (u, v, w, x)):
            out[k].append(np.stack([src[m], n[m]], axis=1))
    return out, shifts


def _lap_pot_grad(t, s, q):
    """pot, grad at targets t from charges q at s, K = 1/(4 pi r), r = 0 skipped."""
    d = t[:, None, :] - s[None, :, :]
    r2 = np.sum(d * d, axis=-1)
    ok = r2 > 0.0
    inv = np.where(ok, 1.0 / np.sqrt(np.where(ok, r2, 1.0)), 0.0)
    pot = (inv * q[None, :]).sum(axis=1)
    grad = -np.einsum("tsd,ts->td", d, inv ** 3 * q[None, :])
    return pot / (4.0 * np.pi), grad / (4.0 * np.pi)


def far_image_operator(p: int, L: float, alpha: float = None, real_shells: int = 5):
    """T[j, k]: potential (Eq. 3 units) on the root's downward check point j
    of a unit charge on its upward equivalent point k repeated over every image
    cell n with max|n_i| >= 2: the Ewald sum of the charge (no k = 0 term, so a
    uniform background; the backgrounds cancel on a neutral density) minus its
    27 nearest images, each written as -erf(alpha r) / r so the difference is
    smooth where the two surfaces meet."""
    from scipy.special import erf, erfc
    S = surface(p)
    h = 0.5 * L
    y = ALPHA_DC * h * S
    z = ALPHA_UE * h * S
    a = 3.0 / L if alpha is None else float(alpha)
    r = y[:, None, :] - z[None, :, :]
    T = np.zeros((S.shape[0], S.shape[0]))
    rng_ = range(-real_shells, real_shells + 1)
    for i in rng_:
        for j in rng_:
            for k in rng_:
                d = r + L * np.array([i, j, k], dtype=np.float64)
                dist = np.sqrt(np.sum(d * d, axis=-1))
                near = max(abs(i), abs(j), abs(k)) <= 1
                if near:
                    safe = np.where(dist > 0, dist, 1.0)
                    T += np.where(dist > 0, -erf(a * safe) / safe, -2.0 * a / np.sqrt(np.pi))
                else:
                    T += erfc(a * dist) / dist
    kmax = int(np.ceil(a * L * np.sqrt(4.0 * 39.2) / (2.0 * np.pi)))
    m = np.arange(-kmax, kmax + 1, dtype=np.float64)
    M = np.stack(np.meshgrid(m, m, m, indexing="ij"), axis=-1).reshape(-1, 3)
    M = M[np.any(M != 0.0, axis=1)]
    kv = 2.0 * np.pi / L * M
    k2 = np.sum(kv * kv, axis=1)
    wk = (4.0 * np.pi / L ** 3) * np.exp(-k2 / (4.0 * a * a)) / k2
    py, pz = y @ kv.T, z @ kv.T
    T += (np.cos(py) * wk) @ np.cos(pz).T + (np.sin(py) * wk) @ np.sin(pz).T
    return T / (4.0 * np.pi)


def periodic_tree(x, L: float, leaf_cap: int, max_depth: int):
    """The tree of a periodic cell [0, L)^3: the same rules as sort_and_tree
    with the cell itself as the root cube (x already wrapped into it)."""
    x = _f64(x).reshape(-1, 3)
    lo = np.zeros(3)
    keys = morton(x, lo, L)
    perm = np.argsort(keys, kind="stable")
    tree = build_tree(keys[perm], leaf_cap, max_depth)
    tree.update(lo=lo, side=float(L), keys=keys, perm=perm)
    return tree


def kifmm_periodic(x, q, L: float, p: int = 6, leaf_cap: int = 64, max_depth: int = 20, eps: float = 1e-12,
                   ops=None):
    """Potential and gradient (Eq. 3 units) of a neutral cubic cell [0, L)^3
    repeated over Z^3 by the KIFMM: the tree's root is the cell; the lists run
    over the cell and its 26 neighbouring images (periodic_lists); the images
    beyond them reach the root's downward check potential through one
    operator on its upward equivalent density (far_image_operator).  The
    rest are the free-space passes with image shifts.  The result converges
    to oracle.ewald (conducting boundary) as p grows."""
    x = np.mod(_f64(x).reshape(-1, 3), L)
    q = _f64(q).reshape(-1)
    check_neutral(q)
    tree = periodic_tree(x, L, leaf_cap, max_depth)
    perm = tree["perm"]
    if ops is None:
        ops = operators(p, eps)
    S, ns = ops["surf"], ops["ns"]
    uu, us, uv, _ = ops["up"]
    du, ds, dv, _ = ops["dn"]
    P_up, P_dn = uv @ np.diag(us) @ uu.T, dv @ np.diag(ds) @ du.T
    lst, shifts = periodic_lists(tree)
    m2l_index = {tuple(d): i for i, d in enumerate(m2l_offsets())}
    xs, qs = x[perm], q[perm]
    nb = tree["nb"]
    level, coord, first, count = tree["level"], tree["coord"].astype(np.int64), tree["first"], tree["count"]
    w = L / 2.0 ** level
    centre = (coord + 0.5) * w[:, None]
    half = 0.5 * w
    octant = 4 * (coord[:, 0] & 1) + 2 * (coord[:, 1] & 1) + (coord[:, 2] & 1)
    isleaf = tree["isleaf"].astype(bool)
    sl = lambda b: slice(int(first[b]), int(first[b] + count[b]))
    q_up = np.zeros((nb, ns))
    d_chk = np.zeros((nb, ns))
    q_dn = np.zeros((nb, ns))
    for lev in range(int(level.max()), -1, -1):           # upward (inside the cell)
        for b in np.nonzero(level == lev)[0]:
            if isleaf[b]:
                chk = kernel_matrix(centre[b] + ALPHA_UC * half[b] * S, xs[sl(b)]) @ qs[sl(b)]
            else:
                chk = np.zeros(ns)
                for c in range(int(tree["child_first"][b]), int(tree["child_first"][b] + tree["nchild"][b])):
                    chk += ops["m2m"][octant[c]] @ q_up[c] / half[b]
            q_up[b] = half[b] * (P_up @ chk)
    d_chk[0] += far_image_operator(p, L) @ q_up[0]         # images beyond the neighbours
    for b in range(nb):                                     # M2L (V), P2L (X) with image shifts
        for a, ni in lst["V"][b]:
            off = coord[a] + shifts[ni] * (1 << int(level[a])) - coord[b]
            d_chk[b] += ops["m2l"][m2l_index[tuple(off)]] @ q_up[a] / half[b]
        for a, ni in lst["X"][b]:
            d_chk[b] += kernel_matrix(centre[b] + ALPHA_DC * half[b] * S, xs[sl(a)] + L * shifts[ni]) @ qs[sl(a)]
    for lev in range(int(level.max()) + 1):                 # downward
        for b in np.nonzero(level == lev)[0]:
            pb = tree["parent"][b]
            if pb >= 0:
                d_chk[b] += ops["l2l"][octant[b]] @ q_dn[pb] / half[pb]
            q_dn[b] = half[b] * (P_dn @ d_chk[b])
    pot = np.zeros(x.shape[0])
    grad = np.zeros((x.shape[0], 3))
    for b in np.nonzero(isleaf)[0]:                         # L2P, M2P (W), P2P (U)
        xt = xs[sl(b)]
        pb_, gb = _lap_pot_grad(xt, centre[b] + ALPHA_DE * half[b] * S, q_dn[b])
        for a, ni in lst["W"][b]:
            pa, ga = _lap_pot_grad(xt, centre[a] + L * shifts[ni] + ALPHA_UE * half[a] * S, q_up[a])
            pb_, gb = pb_ + pa, gb + ga
        for a, ni in lst["U"][b]:
            pa, ga = _lap_pot_grad(xt, xs[sl(a)] + L * shifts[ni], qs[sl(a)])
            pb_, gb = pb_ + pa, gb + ga
        pot[perm[sl(b)]] = pb_
        grad[perm[sl(b)]] = gb
    # The root's equivalent density reproduces the cell's exterior field, not
    # the trace of its second moment sum q |x - c|^2, which the conducting-
    # boundary sum also sees (de Leeuw, Perram & Smith): the difference is a
    # uniform potential 2 pi / (3 V) (Q2(particles) - Q2(density)).
    c = np.full(3, 0.5 * L)
    z = c + ALPHA_UE * (0.5 * L) * S
    q2 = np.sum(qs * np.sum((xs - c) ** 2, axis=1)) - np.sum(q_up[0] * np.sum((z - c) ** 2, axis=1))
    pot += (2.0 * np.pi / (3.0 * L ** 3)) * q2 / (4.0 * np.pi)
    return pot, grad


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 in FP64 over all entries."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))
