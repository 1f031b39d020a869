"""Pins of the oracle's periodic Coulomb sum (Ewald summation with the
conducting boundary; the cell must be neutral, Sec. 2.4).

* Madelung constants of rock salt and caesium chloride (textbook values,
  e.g. Kittel, Introduction to Solid State Physics, ch. 3: 1.747565 and
  1.762675; here to 13 digits).
* Independence of the splitting parameter alpha; invariance under a common
  translation and under moving a particle by a lattice vector.
* The plain image sum over growing spheres of cells (written out below, no
  Ewald split): for a neutral cell without dipole moment its gradient
  converges to Ewald's and its potential to Ewald's plus the constant
  (2 pi / 3V) sum_j q_j |x_j - c|^2 (de Leeuw, Perram & Smith 1980, the paper's
  reference for the neutrality condition), c the centre of the sphere.
* The gradient is the derivative of the potential (central differences).
* A charged cell is refused.
* The periodic KIFMM (cell as the root, lists over the 26 neighbouring
  images, one far-image operator, the second-moment trace correction)
  converges to the Ewald sum as p grows, on uniform and clustered cells.
* Its lists cover every (target leaf, source leaf, neighbouring image) pair
  exactly once (brute-force count), on uniform, clustered and one-leaf trees.
"""
import numpy as np
import pytest

from oracle import oracle as O

M_NACL = 1.747564594633182   # per nearest-neighbour distance
M_CSCL = 1.762674773070989


def test_madelung_rock_salt():
    na = [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    cl = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
    x = np.array(na + cl, dtype=float)          # cubic cell 2, nearest neighbours 1 apart
    q = np.array([1.0] * 4 + [-1.0] * 4)
    pot, grad = O.ewald(x, q, 2.0)
    assert np.allclose(pot * 4 * np.pi, -q * M_NACL, rtol=0, atol=1e-12)
    assert np.abs(grad).max() < 1e-12          # every ion sits at a centre of symmetry


def test_madelung_caesium_chloride():
    x = np.array([(0.0, 0.0, 0.0), (0.5, 0.5, 0.5)])
    q = np.array([1.0, -1.0])
    pot, grad = O.ewald(x, q, 1.0)
    r0 = np.sqrt(3.0) / 2.0
    assert np.allclose(pot * 4 * np.pi * r0, -q * M_CSCL, rtol=0, atol=1e-12)
    assert np.abs(grad).max() < 1e-12


def _neutral(n, seed, L=1.0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, size=(n, 3))
    q = rng.normal(size=n)
    q -= q.mean()
    return x, q


def test_splitting_parameter_does_not_matter():
    x, q = _neutral(12, 5)
    ref = O.ewald(x, q, 1.0, alpha=6.0)
    for a in (4.5, 8.0):
        pot, grad = O.ewald(x, q, 1.0, alpha=a)
        assert O.rel_l2(pot, ref[0]) < 1e-12 and O.rel_l2(grad, ref[1]) < 1e-12, a


def test_translation_and_lattice_shifts():
    x, q = _neutral(10, 6, L=2.5)
    pot, grad = O.ewald(x, q, 2.5)
    t = np.array([0.37, -1.1, 2.2])
    p2, g2 = O.ewald(np.mod(x + t, 2.5), q, 2.5)
    assert O.rel_l2(p2, pot) < 1e-12 and O.rel_l2(g2, grad) < 1e-12
    y = x.copy()
    y[3] += np.array([2.5, 0.0, -2.5])
    p3, g3 = O.ewald(y, q, 2.5)
    assert O.rel_l2(p3, pot) < 1e-12 and O.rel_l2(g3, grad) < 1e-12


def _sphere_sum(x, q, L, R):
    """sum_j q_j / (4 pi |x_i - x_j + L s|) over cells s with |s| <= R (self excluded)."""
    n = int(np.ceil(R))
    r = np.arange(-n, n + 1)
    S = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(float)
    S = S[np.linalg.norm(S, axis=1) <= R]
    pot = np.zeros(len(x))
    grad = np.zeros((len(x), 3))
    for i in range(len(x)):
        d = x[i][None, None, :] - x[None, :, :] + L * S[:, None, :]
        rr = np.linalg.norm(d, axis=-1)
        rr[np.all(S == 0, axis=1), i] = np.inf
        pot[i] = np.sum(q[None, :] / rr)
        grad[i] = -np.sum((q[None, :] / rr ** 3)[:, :, None] * d, axis=(0, 1))
    return pot / (4 * np.pi), grad / (4 * np.pi)


def test_sphere_of_images_converges_to_ewald():
    rng = np.random.default_rng(3)
    L = 1.0
    c = np.full(3, 0.5 * L)
    h = rng.uniform(0, L, size=(4, 3))
    x = np.concatenate([h, 2 * c - h])           # inversion pairs: zero dipole
    q = np.array([1.0, -1.0, 2.0, -2.0] * 2)
    pe, ge = O.ewald(x, q, L)
    shift = (2 * np.pi / (3 * L ** 3)) * np.sum(q * np.sum((x - c) ** 2, axis=1)) / (4 * np.pi)
    errs = []
    for R in (8, 16):
        ps, gs = _sphere_sum(x, q, L, R)
        errs.append(O.rel_l2(gs, ge))
        assert O.rel_l2(ps, pe - shift) < 2e-4, R
    assert errs[1] < errs[0] / 8 and errs[1] < 1e-5, errs


def test_gradient_is_the_derivative_of_the_potential():
    x, q = _neutral(8, 11)
    _, grad = O.ewald(x, q, 1.0)
    h = 1e-5
    for i in (0, 5):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (O.ewald(xp, q, 1.0)[0][i] - O.ewald(xm, q, 1.0)[0][i]) / (2 * h)
            assert abs(fd - grad[i, d]) <= 1e-7 * (1.0 + abs(grad[i, d])), (i, d)


def test_charged_cell_is_refused():
    x = np.array([(0.1, 0.2, 0.3), (0.6, 0.5, 0.4)])
    with pytest.raises(O.NotNeutralError):
        O.ewald(x, np.array([1.0, -0.5]), 1.0)
    O.check_neutral(np.array([1.0, -1.0, 0.5, -0.5]))


# ---------------------------------------------------------------------------
# The periodic KIFMM (oracle.kifmm_periodic) against the Ewald sum
# ---------------------------------------------------------------------------
def test_periodic_kifmm_converges_to_ewald():
    x, q = _neutral(300, 1)
    pe, ge = O.ewald(x, q, 1.0)
    e = {}
    for p in (4, 6):
        pp, gp = O.kifmm_periodic(x, q, 1.0, p=p, leaf_cap=32)
        e[p] = (O.rel_l2(pp, pe), O.rel_l2(gp, ge))
    assert max(e[4]) < 2e-3 and max(e[6]) < 3e-5, e
    assert e[6][0] < e[4][0] / 10 and e[6][1] < e[4][1] / 10, e
    # a single leaf: the 27 nearest images directly, the rest through the
    # far-image operator alone
    pp, gp = O.kifmm_periodic(x, q, 1.0, p=6, leaf_cap=400)
    assert O.rel_l2(pp, pe) < 3e-5 and O.rel_l2(gp, ge) < 3e-5


def test_periodic_kifmm_adaptive_tree_with_images():
    from workloads import generators as G
    xp, _ = G.plummer(400, 3)
    x = np.mod(0.5 + 0.05 * xp, 1.0)               # a cluster in the cell, wrapped
    q = np.random.default_rng(12).normal(size=400)
    q -= q.mean()
    lo = np.zeros(3)
    keys = O.morton(x, lo, 1.0)
    perm = np.argsort(keys, kind="stable")
    tree = O.build_tree(keys[perm], 16, 20)
    lst, shifts = O.periodic_lists(tree)
    assert sum(len(w) for w in lst["W"]) > 0 and sum(len(v) for v in lst["X"]) > 0
    assert any((u[:, 1] != 13).any() for u in lst["U"] if len(u))   # image neighbours occur
    for kind in "UVWX":                                             # no entry twice
        for e in lst[kind]:
            assert len({(int(a), int(n)) for a, n in e}) == len(e)
    pe, ge = O.ewald(x, q, 1.0)
    pp, gp = O.kifmm_periodic(x, q, 1.0, p=6, leaf_cap=16)
    assert O.rel_l2(pp, pe) < 3e-5 and O.rel_l2(gp, ge) < 5e-5


def test_periodic_kifmm_refuses_a_charged_cell():
    x = np.array([(0.1, 0.2, 0.3), (0.6, 0.5, 0.4)])
    with pytest.raises(O.NotNeutralError):
        O.kifmm_periodic(x, np.array([1.0, 0.5]), 1.0, p=4)


def _periodic_tree(x, M):
    lo = np.zeros(3)
    keys = O.morton(x, lo, 1.0)
    perm = np.argsort(keys, kind="stable")
    return O.build_tree(keys[perm], M, 20)


@pytest.mark.parametrize("shape,n,M", [("uniform", 400, 8), ("cluster", 500, 6), ("one_leaf", 50, 64)])
def test_periodic_lists_cover_every_image_pair_exactly_once(shape, n, M):
    """Every (target leaf B in the cell, source leaf A, image shift s with
    s in {-1, 0, 1}^3) is accounted for exactly once: by U(B), by a W(B) box
    whose image holds A's image, or by V/X of an ancestor-or-self of B; images
    farther away belong to the far-image operator alone."""
    rng = np.random.default_rng(31)
    if shape == "cluster":
        from workloads import generators as G
        xp, _ = G.plummer(n, 4)
        x = np.mod(0.3 + 0.04 * xp, 1.0)
    else:
        x = rng.uniform(0, 1, size=(n, 3))
    t = _periodic_tree(x, M)
    lst, _ = O.periodic_lists(t)
    leaves = np.nonzero(t["isleaf"])[0]
    pos = {int(b): i for i, b in enumerate(leaves)}

    def desc(b):
        if t["isleaf"][b]:
            return [int(b)]
        out = []
        for c in range(t["child_first"][b], t["child_first"][b] + t["nchild"][b]):
            out += desc(c)
        return out

    for B in leaves:
        cover = np.zeros((len(leaves), 27), dtype=np.int64)
        for A, s in lst["U"][B]:
            cover[pos[int(A)], s] += 1
        for A, s in lst["W"][B]:
            for a in desc(A):
                cover[pos[a], s] += 1
        b = int(B)
        while b >= 0:
            for kind in ("V", "X"):
                for A, s in lst[kind][b]:
                    for a in desc(A):
                        cover[pos[a], s] += 1
            b = int(t["parent"][b])
        assert np.all(cover == 1), (int(B), np.argwhere(cover != 1)[:5])
