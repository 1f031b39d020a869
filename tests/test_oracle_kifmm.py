"""Pins of the oracle's surfaces, translation operators and KIFMM evaluation
(Sec. 2.2) against closed forms, brute force and invariants:

* surface counts and geometry;
* the pseudo-inverse reproduces check potentials, and an equivalent density
  fitted to one source reproduces its far field (the defining property of the
  equivalent surface, Sec. 2.2);
* a tree that is a single leaf is the direct sum;
* the error against the direct sum falls as the surface order p grows;
* Newton's third law holds to the FMM error, U = 1/2 sum q phi, and the
  result is invariant (to rounding) under 2^k scaling and axis permutation.
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import generators as G


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_surface_counts(p):
    S = O.surface(p)
    assert S.shape == (6 * (p - 1) ** 2 + 2, 3)
    assert np.allclose(np.max(np.abs(S), axis=1), 1.0)
    assert len({tuple(r) for r in S}) == S.shape[0]
    # lexicographic in (i, j, k)
    grid = np.rint((S + 1) * (p - 1) / 2).astype(int)
    keys = grid[:, 0] * p * p + grid[:, 1] * p + grid[:, 2]
    assert np.all(np.diff(keys) > 0)


def test_pinv_reproduces_check_potential():
    ops = O.operators(6)
    S = ops["surf"]
    K = O.kernel_matrix(O.ALPHA_UC * S, O.ALPHA_UE * S)
    u, sinv, v, s = ops["up"]
    rng = np.random.default_rng(2)
    src = rng.uniform(-1, 1, size=(20, 3))
    b = O.kernel_matrix(O.ALPHA_UC * S, src) @ rng.normal(size=20)
    dens = v @ (sinv * (u.T @ b))
    assert np.linalg.norm(K @ dens - b) < 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("p,tol", [(4, 5e-3), (6, 5e-5), (8, 2e-6)])
def test_equivalent_density_far_field(p, tol):
    """A unit source inside the unit box, fitted on the upward check surface,
    is reproduced at points beyond that surface (distance 3 to 6)."""
    ops = O.operators(p)
    S = ops["surf"]
    u, sinv, v, _ = ops["up"]
    rng = np.random.default_rng(p)
    y = rng.uniform(-1, 1, size=(1, 3))
    b = O.kernel_matrix(O.ALPHA_UC * S, y)[:, 0]
    dens = v @ (sinv * (u.T @ b))
    d = rng.normal(size=(200, 3))
    far = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(3.2, 6, size=(200, 1))
    exact = 1.0 / (4 * np.pi * np.linalg.norm(far - y, axis=1))
    approx = O.kernel_matrix(far, O.ALPHA_UE * S) @ dens
    assert np.max(np.abs(approx - exact) / exact) < tol


def test_gap_check_rejects_ambiguous_threshold():
    S = O.surface(6)
    K = O.kernel_matrix(O.ALPHA_UC * S, O.ALPHA_UE * S)
    s = np.linalg.svd(K, compute_uv=False)
    with pytest.raises(O.PinvGapError):
        O.svd_pinv_factors(K, s[40] / s[0])


def test_single_leaf_is_direct_sum():
    x, q = G.uniform_charges(50, 21)
    pot, grad, info = O.kifmm(x, q, p=4, leaf_cap=64)
    assert info["tree"]["nb"] == 1
    pd, gd = O.direct(x, q)
    assert O.rel_l2(pot, pd) < 1e-14 and O.rel_l2(grad, gd) < 1e-14


@pytest.mark.parametrize("shape", ["uniform", "plummer"])
def test_error_falls_with_p(shape):
    if shape == "uniform":
        x, q = G.uniform_charges(3000, 31)
        M = 32
    else:
        x, _ = G.plummer(3000, 31)
        q = np.random.default_rng(31).normal(size=3000)
        M = 16
    pd, gd = O.direct(x, q)
    errs = []
    tree = O.sort_and_tree(x, M, 20)
    lst = O.lists(tree)
    for p in (4, 6, 8):
        pot, grad, _ = O.kifmm(x, q, p=p, tree=tree, lst=lst)
        errs.append((O.rel_l2(pot, pd), O.rel_l2(grad, gd)))
    for a, b in zip(errs, errs[1:]):
        assert b[0] < a[0] / 5 and b[1] < a[1] / 5
    assert errs[0][0] < 1e-3 and errs[0][1] < 1e-2
    assert errs[1][0] < 3e-5 and errs[1][1] < 1e-4


def test_newton_energy_and_invariances():
    x, q = G.uniform_charges(2500, 41)
    pot, grad, info = O.kifmm(x, q, p=6, leaf_cap=32)
    pd, gd = O.direct(x, q)
    err = O.rel_l2(grad, gd)
    F = O.forces(q, grad)
    net = np.linalg.norm(F.sum(axis=0)) / np.abs(F).sum()
    assert net < 10 * err
    assert O.energy(q, pot) == pytest.approx(O.energy(q, pd), rel=10 * O.rel_l2(pot, pd))
    # 2^k scaling: same tree, potential scales by 2^-k and gradient by 2^-2k
    pot2, grad2, info2 = O.kifmm(4.0 * x + 1.0, q, p=6, leaf_cap=32)
    assert np.array_equal(info2["tree"]["prefix"], info["tree"]["prefix"])
    assert O.rel_l2(4.0 * pot2, pot) < 1e-12 and O.rel_l2(16.0 * grad2, grad) < 1e-12
    # axis permutation (x, y, z) -> (y, z, x): the cube surfaces map onto themselves
    perm = [1, 2, 0]
    pot3, grad3, _ = O.kifmm(x[:, perm], q, p=6, leaf_cap=32)
    assert O.rel_l2(pot3, pot) < 1e-12 and O.rel_l2(grad3, grad[:, perm]) < 1e-12


def test_clump_reduce_brute_force():
    """Clump force and torque are the sums over pebbles of F_k and
    (x_k - X_c) x F_k; with the whole system made of clumps, the net force and
    torque vanish for the exact pair forces (Newton's third law, central
    forces)."""
    x, q, off, centres = G.clumps(40, 3, charges_per_clump=4)
    pd, gd = O.direct(x, q)
    F, T = O.clump_reduce(x, q, gd, off, centres)
    f = O.forces(q, gd)
    c = 7
    sl = slice(off[c], off[c + 1])
    np.testing.assert_allclose(F[c], f[sl].sum(axis=0), rtol=1e-13)
    np.testing.assert_allclose(T[c], np.cross(x[sl] - centres[c], f[sl]).sum(axis=0), rtol=1e-12)
    scale = np.abs(f).sum()
    assert np.linalg.norm(F.sum(axis=0)) < 1e-12 * scale
    # total torque about the origin: sum_c (T_c + X_c x F_c) = sum_k x_k x F_k = 0
    Ttot = T.sum(axis=0) + np.cross(centres, F).sum(axis=0)
    assert np.linalg.norm(Ttot) < 1e-10 * scale * np.abs(x).max()


def test_perturbed_operators_are_rounding_level():
    """operators_perturbed (the parity tests' rounding floor) moves every
    translation entry by about one unit in the last place, keeps the
    pseudo-inverse factors those of a matrix within 2^-53 ||K|| of K (the
    truncated rank is unchanged), and moves the KIFMM output far less than
    the method's own error: a rounding floor, not a different method."""
    p = 6
    a, b = O.operators(p), O.operators_perturbed(p, 1)
    for k in ("m2m", "l2l", "m2l"):
        rel = np.abs(b[k] - a[k]) / np.abs(a[k])
        # the drawn relative move (at most 2^-52) plus the rounding of the product
        assert rel.max() <= 2.0 ** -52 + 2.0 ** -53 and rel.max() > 0
    for k in ("up", "dn"):
        assert np.count_nonzero(a[k][1]) == np.count_nonzero(b[k][1])
        assert np.allclose(b[k][3], a[k][3], rtol=0, atol=1e-14 * a[k][3][0])
    x, q = G.uniform_charges(1500, 5)
    p0, g0, _ = O.kifmm(x, q, p=p, leaf_cap=32)
    p1, g1, _ = O.kifmm(x, q, p=p, leaf_cap=32, ops=b)
    pd, gd = O.direct(x, q)
    floor_p, floor_g = O.rel_l2(p1, p0), O.rel_l2(g1, g0)
    assert 0 < floor_p < 1e-12 and 0 < floor_g < 1e-12
    assert floor_p < 1e-6 * O.rel_l2(p0, pd) and floor_g < 1e-6 * O.rel_l2(g0, gd)
