"""Pins of the oracle's Stokeslet direct sum (the tensor kernel of Stokes
flow; Eq. 1 admits vector and tensor kernels).

* One point force: the closed form along and across the force (velocity
  F / (4 pi mu r) along it, F / (8 pi mu r) across).
* A sphere of radius a carrying a uniform traction (total force F) moves the
  fluid inside it uniformly, u = F / (6 pi mu a) (the Stokes drag relation);
  checked with a Fibonacci quadrature of the sphere.
* The flow is divergence free away from the forces (central differences).
* Lorentz reciprocity: f_a . u(x_a; f_b at x_b) = f_b . u(x_b; f_a at x_a).
* Scaling u(lambda x) = u(x) / lambda; linearity in the forces; far field of
  a cluster tends to a single Stokeslet of the total force.
* The KIFMM with the Stokeslet: one leaf is the direct sum; the error against
  the direct sum falls tenfold from p = 4 to p = 6; the adaptive W and X
  passes hold the same bar on a clustered (Plummer) set; the method is exactly
  homogeneous of degree -1.
"""
import numpy as np

from oracle import oracle as O


def test_single_point_force_closed_form():
    F = np.array([[0.0, 0.0, 2.0]])
    x = np.zeros((1, 3))
    mu = 0.7
    t = np.array([[0.0, 0.0, 1.5], [1.5, 0.0, 0.0], [0.0, -0.5, 0.0]])
    u = O.stokeslet_direct(x, F, targets=t, mu=mu)
    assert np.allclose(u[0], [0.0, 0.0, 2.0 / (4 * np.pi * mu * 1.5)], rtol=1e-14, atol=0)
    assert np.allclose(u[1], [0.0, 0.0, 2.0 / (8 * np.pi * mu * 1.5)], rtol=1e-14, atol=0)
    assert np.allclose(u[2], [0.0, 0.0, 2.0 / (8 * np.pi * mu * 0.5)], rtol=1e-14, atol=0)


def _fibonacci_sphere(n):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)


def test_uniform_traction_sphere_moves_its_interior_rigidly():
    a, mu, n = 1.3, 1.0, 8000
    F = np.array([1.0, 0.3, -0.2])
    x = a * _fibonacci_sphere(n)
    f = np.tile(F / n, (n, 1))
    t = a * np.array([[0.0, 0.0, 0.0], [0.3, 0.2, -0.1], [0.1, -0.5, 0.2], [0.0, 0.0, 0.6]])
    u = O.stokeslet_direct(x, f, targets=t, mu=mu)
    ex = F / (6 * np.pi * mu * a)
    assert np.abs(u - ex).max() < 1e-5 * np.linalg.norm(ex)


def test_divergence_free():
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, size=(40, 3))
    f = rng.normal(size=(40, 3))
    p = np.array([[2.0, 0.5, -1.5]])
    h = 1e-4
    div = 0.0
    for d in range(3):
        e = np.zeros((1, 3))
        e[0, d] = h
        div += (O.stokeslet_direct(x, f, p + e)[0, d] - O.stokeslet_direct(x, f, p - e)[0, d]) / (2 * h)
    scale = np.abs(O.stokeslet_direct(x, f, p)).max()
    assert abs(div) < 1e-7 * scale


def test_reciprocity_scaling_linearity_far_field():
    rng = np.random.default_rng(5)
    xa, xb = rng.normal(size=(1, 3)), rng.normal(size=(1, 3))
    fa, fb = rng.normal(size=(1, 3)), rng.normal(size=(1, 3))
    lhs = fa[0] @ O.stokeslet_direct(xb, fb, xa)[0]
    rhs = fb[0] @ O.stokeslet_direct(xa, fa, xb)[0]
    assert abs(lhs - rhs) < 1e-14 * max(abs(lhs), 1e-300)
    x = rng.uniform(-1, 1, size=(30, 3))
    f = rng.normal(size=(30, 3))
    t = rng.uniform(-1, 1, size=(5, 3)) + 3.0
    u = O.stokeslet_direct(x, f, t)
    assert np.allclose(O.stokeslet_direct(2.5 * x, f, 2.5 * t), u / 2.5, rtol=1e-13, atol=0)
    g = rng.normal(size=(30, 3))
    assert np.allclose(O.stokeslet_direct(x, 2 * f - g, t), 2 * u - O.stokeslet_direct(x, g, t),
                       rtol=1e-12, atol=1e-14)
    # far away the cluster acts as one Stokeslet of its total force: error O(size / distance)
    errs = []
    for R in (50.0, 500.0):
        far = np.array([[R, 0.3 * R, -0.2 * R]])
        one = O.stokeslet_direct(np.zeros((1, 3)), f.sum(axis=0, keepdims=True), far)
        errs.append(np.linalg.norm(O.stokeslet_direct(x, f, far) - one) / np.linalg.norm(one))
    assert errs[1] < errs[0] / 5 and errs[1] < 1e-2


# ---------------------------------------------------------------------------
# The KIFMM with the Stokeslet (oracle.kifmm_stokes) against the direct sum
# ---------------------------------------------------------------------------
def test_kifmm_stokes_single_leaf_is_the_direct_sum():
    rng = np.random.default_rng(21)
    x, f = rng.uniform(0, 1, (300, 3)), rng.normal(size=(300, 3))
    u = O.kifmm_stokes(x, f, p=4, leaf_cap=400)
    assert O.rel_l2(u, O.stokeslet_direct(x, f)) < 1e-13


def test_kifmm_stokes_converges_with_surface_order():
    rng = np.random.default_rng(2)
    x, f = rng.uniform(0, 1, (1500, 3)), rng.normal(size=(1500, 3))
    ud = O.stokeslet_direct(x, f)
    e4 = O.rel_l2(O.kifmm_stokes(x, f, p=4, leaf_cap=32), ud)
    e6 = O.rel_l2(O.kifmm_stokes(x, f, p=6, leaf_cap=32), ud)
    assert e4 < 2e-3 and e6 < 1e-4 and e6 < e4 / 10, (e4, e6)


def test_kifmm_stokes_adaptive_lists_and_scaling():
    from workloads import generators as G
    x, _ = G.plummer(1200, 5)
    f = np.random.default_rng(6).normal(size=(1200, 3))
    t = O.sort_and_tree(x, 16, 20)
    lst = O.lists(t)
    assert lst["W"][1].size > 0 and lst["X"][1].size > 0
    ud = O.stokeslet_direct(x, f)
    # every W/X interaction through M2P / P2L (none moved to the direct sum)
    assert O.rel_l2(O.kifmm_stokes(x, f, p=4, leaf_cap=16, direct_max=-1), ud) < 3e-3
    # homogeneity of degree -1: the whole method scales exactly
    u1 = O.kifmm_stokes(x[:600], f[:600], p=4, leaf_cap=16)
    u2 = O.kifmm_stokes(2.0 * x[:600], f[:600], p=4, leaf_cap=16)
    assert O.rel_l2(u2, u1 / 2.0) < 1e-11
