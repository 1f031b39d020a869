"""Pins of the oracle's Morton keys, adaptive octree (Sec. 2.2, first step:
leaves hold at most M points) and U/V/W/X lists (Sec. 2.2, third step)
against hand-derived examples, brute-force coverage and invariants."""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import generators as G


def test_morton_hand_keys():
    """With lo = 0 and side = 1, x = k / 2^21 quantises to k exactly; bits
    interleave x-highest, so (1,0,0) -> 4, (0,1,0) -> 2, (0,0,1) -> 1 and
    bit b of x lands at 3b + 2."""
    s = 2.0 ** 21
    pts = np.array([[0, 0, 0], [1, 1, 1], [1 / s, 0, 0], [0, 1 / s, 0], [0, 0, 1 / s],
                    [2 / s, 0, 0], [3 / s, 5 / s, 6 / s]], dtype=float)
    lo, side = O.bbox(pts)
    assert side == 1.0 and np.all(lo == 0)
    keys = O.morton(pts, lo, side)
    assert keys[0] == 0
    assert keys[1] == (1 << 63) - 1  # max corner clamps to all ones
    assert keys[2] == 4 and keys[3] == 2 and keys[4] == 1
    assert keys[5] == 1 << 5
    # x=3 (bits 0,1), y=5 (bits 0,2), z=6 (bits 1,2)
    want = (1 << 2) | (1 << 5) | (1 << 1) | (1 << 7) | (1 << 3) | (1 << 6)
    assert keys[6] == want


def test_morton_power_of_two_scaling_invariance():
    rng = np.random.default_rng(1)
    x = rng.uniform(-3, 7, size=(2000, 3))
    lo, side = O.bbox(x)
    k1 = O.morton(x, lo, side)
    y = 8.0 * x + 0.0
    lo2, side2 = O.bbox(y)
    assert np.array_equal(k1, O.morton(y, lo2, side2))


def test_tree_hand_example():
    """Three points; M = 1.  p1 and p3 share octant 0 down to level 3 and
    separate at level 4 (x = 2^-4 quantises to 2^17, so x bit 17 is p3's only
    set bit); p2 is the max corner alone in octant 7 of the root."""
    pts = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.0625, 0.0, 0.0]])
    t = O.sort_and_tree(pts, 1, 20)
    assert list(t["level"]) == [0, 1, 1, 2, 3, 4, 4]
    assert list(t["count"]) == [3, 2, 1, 2, 2, 1, 1]
    assert list(t["parent"]) == [-1, 0, 0, 1, 3, 4, 4]
    assert list(t["isleaf"]) == [0, 0, 1, 0, 0, 1, 1]
    assert list(t["coord"][2]) == [1, 1, 1]
    assert list(t["coord"][6]) == [1, 0, 0]
    assert list(t["perm"]) == [0, 2, 1]


def _tree_invariants(t, n, M, D):
    lev, cnt, first = t["level"], t["count"], t["first"]
    assert np.all(np.diff(lev) >= 0)
    for b in range(t["nb"]):
        if t["nchild"][b]:
            ch = np.arange(t["child_first"][b], t["child_first"][b] + t["nchild"][b])
            assert np.all(t["parent"][ch] == b)
            assert cnt[ch].sum() == cnt[b]
            assert first[ch[0]] == first[b]
            assert cnt[b] > M and lev[b] < D
        else:
            assert cnt[b] <= M or lev[b] == D
        assert cnt[b] > 0
    leaves = np.nonzero(t["isleaf"])[0]
    order = leaves[np.argsort(first[leaves])]
    assert np.array_equal(np.cumsum(cnt[order])[:-1], first[order][1:])
    assert cnt[leaves].sum() == n
    # canonical order: (level, prefix) strictly increasing
    key = [(int(l), int(p)) for l, p in zip(lev, t["prefix"])]
    assert key == sorted(key) and len(set(key)) == len(key)


@pytest.mark.parametrize("shape", ["uniform", "plummer"])
def test_tree_invariants(shape):
    if shape == "uniform":
        x, _ = G.uniform_charges(5000, 11)
    else:
        x, _ = G.plummer(5000, 11)
    t = O.sort_and_tree(x, 24, 8)
    _tree_invariants(t, 5000, 24, 8)
    assert t["max_level"] <= 8


def test_uniform_grid_lists_hand_counts():
    """One point at the centre of each of the 64 level-2 cells, M = 1: a full
    level-2 tree.  A corner box has 8 U boxes (its 2x2x2 block) and 64 - 8 V
    boxes; box (1,1,1) has 27 U boxes and 64 - 27 V boxes; W and X are empty."""
    c = (np.arange(4) + 0.5) / 4
    x = np.array([[a, b, d] for a in c for b in c for d in c])
    t = O.sort_and_tree(x, 1, 20)
    assert t["nb"] == 1 + 8 + 64 and t["max_level"] == 2
    L = O.lists(t)
    idx = {tuple(t["coord"][b]): b for b in range(t["nb"]) if t["level"][b] == 2}
    def n(kind, b):
        ptr, _ = L[kind]
        return ptr[b + 1] - ptr[b]
    assert n("U", idx[(0, 0, 0)]) == 8 and n("V", idx[(0, 0, 0)]) == 56
    assert n("U", idx[(1, 1, 1)]) == 27 and n("V", idx[(1, 1, 1)]) == 37
    assert L["W"][1].size == 0 and L["X"][1].size == 0
    # level-1 boxes have no V list (their parent, the root, has no colleagues)
    assert all(n("V", b) == 0 for b in range(1, 9))


def _ancestors(t, b):
    out = []
    while b >= 0:
        out.append(b)
        b = t["parent"][b]
    return out


def _leaf_of_particle(t):
    leaf = np.empty(int(t["count"][0]), dtype=np.int64)
    for b in np.nonzero(t["isleaf"])[0]:
        leaf[t["first"][b]:t["first"][b] + t["count"][b]] = b
    return leaf


def _descendant_leaves(t, b):
    if t["isleaf"][b]:
        return [b]
    out = []
    for c in range(t["child_first"][b], t["child_first"][b] + t["nchild"][b]):
        out += _descendant_leaves(t, c)
    return out


@pytest.mark.parametrize("thr", [-1, 6, 56])
@pytest.mark.parametrize("shape,n,M", [("plummer", 1500, 8), ("uniform", 900, 6), ("clustered", 700, 4)])
def test_lists_cover_every_pair_exactly_once(shape, n, M, thr):
    """Every ordered (target leaf, source leaf) pair is accounted for exactly
    once by U(B), W(B) (source inside a W box) or V/X of an ancestor-or-self
    of B (source inside that box): the sum then counts each interaction once.
    Holds for the lists as classified (thr = -1) and as evaluated, with W/X
    interactions of leaves holding at most thr points moved to U."""
    if shape == "plummer":
        x, _ = G.plummer(n, 5)
    elif shape == "uniform":
        x, _ = G.uniform_charges(n, 5)
    else:
        rng = np.random.default_rng(5)
        x = np.concatenate([rng.normal(0, 0.01, size=(n // 2, 3)), rng.uniform(-1, 1, size=(n - n // 2, 3))])
    t = O.sort_and_tree(x, M, 20)
    raw = O.lists(t)
    L = O.effective_lists(t, raw, thr)
    leaves = np.nonzero(t["isleaf"])[0]
    pos = {b: i for i, b in enumerate(leaves)}
    desc = {b: _descendant_leaves(t, b) for b in range(t["nb"])}

    def members(kind, b):
        ptr, idx = L[kind]
        return idx[ptr[b]:ptr[b + 1]]

    for B in leaves:
        cover = np.zeros(len(leaves), dtype=np.int64)
        for A in members("U", B):
            cover[pos[A]] += 1
        for A in members("W", B):
            for a in desc[A]:
                cover[pos[a]] += 1
        for Bp in _ancestors(t, B):
            for kind in ("V", "X"):
                for A in members(kind, Bp):
                    for a in desc[A]:
                        cover[pos[a]] += 1
        assert np.all(cover == 1), (B, np.nonzero(cover != 1)[0][:10])
    assert raw["W"][1].size > 0 or shape == "uniform"
    # every U entry is a leaf, and a moved entry is a W/X pair of a small leaf
    assert np.all(t["isleaf"][L["U"][1]] == 1)
    small = (t["isleaf"] == 1) & (t["count"] <= thr)
    for b in range(t["nb"]):
        Wr = set(members_raw("W", raw, b))
        Xr = set(members_raw("X", raw, b))
        moved = set(L["U"][1][L["U"][0][b]:L["U"][0][b + 1]]) - set(members_raw("U", raw, b))
        assert moved == {a for a in Wr if small[a]} | (Xr if small[b] else set())


def members_raw(kind, L, b):
    ptr, idx = L[kind]
    return [int(a) for a in idx[ptr[b]:ptr[b + 1]]]


@pytest.mark.parametrize("thr", [-1, 8, 56])
def test_lists_duality(thr):
    """U and V are symmetric relations and X is the transpose of W, for the
    lists as classified and as evaluated (the direct-sum rule is the same
    from both sides of a W/X pair)."""
    x, _ = G.plummer(1200, 9)
    t = O.sort_and_tree(x, 8, 20)
    L = O.effective_lists(t, O.lists(t), thr)

    def pairs(kind):
        ptr, idx = L[kind]
        return {(b, int(a)) for b in range(t["nb"]) for a in idx[ptr[b]:ptr[b + 1]]}

    U, V, W, X = (pairs(k) for k in "UVWX")
    assert U == {(a, b) for b, a in U}
    assert V == {(a, b) for b, a in V}
    assert X == {(a, b) for b, a in W}
    assert len(W) > 0 or thr >= 8
    # V members are never adjacent: offsets stay within the 316 M2L offsets
    offs = {tuple(d) for d in O.m2l_offsets()}
    for b, a in V:
        assert tuple(t["coord"][a] - t["coord"][b]) in offs


def _boxes_by_segments(keys, M, D):
    """The octree's boxes read off the sorted keys level by level, with no
    recursion: a box of level l >= 1 starts where the level-l key prefix
    changes, inside a level-(l-1) run of equal prefixes longer than M, at a
    level l - 1 below the maximum depth D (runs only shrink with the level,
    so every coarser run around it is longer than M too).  Returns the
    (level, first, count) of every box in level-major, then key order."""
    keys = np.asarray(keys, dtype=np.uint64)
    n = keys.size
    out = [(0, 0, n)]

    def runs(p):
        start = np.ones(n, dtype=bool)
        start[1:] = p[1:] != p[:-1]
        first = np.flatnonzero(start)
        length = np.diff(np.append(first, n))
        return start, np.repeat(length, length)   # run length seen from every point

    prev_len = np.full(n, n)
    for l in range(1, O.BITS + 1):
        p = keys >> np.uint64(3 * (O.BITS - l))
        start, length = runs(p)
        box = start & (prev_len > M) & (l - 1 < D)
        if not box.any():
            break
        out += [(l, int(i), int(length[i])) for i in np.flatnonzero(box)]
        prev_len = length
    return out


@pytest.mark.parametrize("case", ["uniform", "plummer", "clustered"])
@pytest.mark.parametrize("M,D", [(1, 20), (8, 20), (32, 4), (200, 20)])
def test_tree_equals_the_segment_rule(case, M, D):
    """The oracle's level-by-level octree (split while more than M points and
    above depth D) has exactly the boxes of the segment rule, in the same
    order, with the same counts."""
    rng = np.random.default_rng(11)
    x = {"uniform": lambda: G.uniform_charges(3000, 3)[0],
         "plummer": lambda: G.plummer(3000, 4)[0],
         "clustered": lambda: np.concatenate([rng.normal(0, 1e-4, (600, 3)), rng.uniform(-1, 1, (600, 3))])}[case]()
    t = O.sort_and_tree(x, M, D)
    want = _boxes_by_segments(t["keys"][t["perm"]], M, D)
    got = list(zip(t["level"].tolist(), t["first"].tolist(), t["count"].tolist()))
    assert got == want
