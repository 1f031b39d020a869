"""Pins of the oracle's direct sum (Sec. 1 all-pairs sum; Eq. 1 with the
Laplace kernel normalised as in Eq. 3) against closed forms and invariants
that do not reuse the oracle's own formula."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_two_charges_eq3():
    """Two like charges repel with |F| = q1 q2 / (4 pi r^2) along the line
    joining them (Eq. 3)."""
    g = _load("two_charges.json")
    x = np.array(g["x"], dtype=float)
    q = np.array(g["q"], dtype=float)
    pot, grad = O.direct(x, q)
    np.testing.assert_allclose(pot, g["pot"], rtol=1e-15)
    F = O.forces(q, grad)
    np.testing.assert_allclose(F, g["force"], rtol=1e-15, atol=1e-18)
    # repulsion: the force on particle 0 points away from particle 1
    assert np.dot(F[0], x[0] - x[1]) > 0


def test_cube_corners_closed_form():
    """Eight unit charges on the corners of a unit cube: by symmetry each feels
    the same potential and a force along the outward body diagonal; the
    values sum 3 edge, 3 face-diagonal and 1 body-diagonal neighbours."""
    g = _load("cube_corners.json")
    x = np.array(g["x"], dtype=float)
    q = np.ones(8)
    pot, grad = O.direct(x, q)
    np.testing.assert_allclose(pot, g["pot_each"], rtol=1e-14)
    F = O.forces(q, grad)
    centre = np.full(3, 0.5)
    for i in range(8):
        outward = (x[i] - centre) / np.linalg.norm(x[i] - centre)
        np.testing.assert_allclose(np.linalg.norm(F[i]), g["force_mag"], rtol=1e-14)
        np.testing.assert_allclose(np.dot(F[i], outward), g["force_mag"], rtol=1e-14)


def test_shell_potential_at_centre():
    """Charges anywhere on a sphere of radius R give exactly Q/(4 pi R) at the
    centre (every source is at distance R)."""
    rng = np.random.default_rng(3)
    d = rng.normal(size=(500, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    R = 2.5
    q = rng.uniform(0.1, 1.0, size=500)
    pot, grad = O.direct(R * d, q, targets=np.zeros((1, 3)))
    np.testing.assert_allclose(pot[0], q.sum() / (4 * np.pi * R), rtol=1e-13)


def test_newton_third_law_exact():
    """sum_i q_i grad_i = 0: the pair forces cancel (direct sum, to rounding)."""
    rng = np.random.default_rng(4)
    x = rng.uniform(size=(700, 3))
    q = rng.normal(size=700)
    pot, grad = O.direct(x, q)
    F = O.forces(q, grad)
    scale = np.abs(F).sum(axis=0)
    assert np.all(np.abs(F.sum(axis=0)) < 1e-12 * scale)


def test_energy_is_pair_sum_and_symmetry():
    """U = 1/2 sum q_i phi_i equals the sum over unordered pairs, and the
    potential at i from a unit charge at j equals that at j from i."""
    rng = np.random.default_rng(5)
    x = rng.uniform(size=(60, 3))
    q = rng.normal(size=60)
    pot, _ = O.direct(x, q)
    U = O.energy(q, pot)
    pair = 0.0
    for i in range(60):
        for j in range(i + 1, 60):
            pair += q[i] * q[j] / (4 * np.pi * np.linalg.norm(x[i] - x[j]))
    np.testing.assert_allclose(U, pair, rtol=1e-13)
    e = np.zeros(60)
    e[7] = 1.0
    p7, _ = O.direct(x, e)
    e[:] = 0.0
    e[19] = 1.0
    p19, _ = O.direct(x, e)
    assert p7[19] == pytest.approx(p19[7], rel=1e-15)


def test_coincident_points_contribute_nothing():
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    q = np.array([1.0, 5.0, 2.0])
    pot, grad = O.direct(x, q)
    assert np.all(np.isfinite(pot)) and np.all(np.isfinite(grad))
    np.testing.assert_allclose(pot[0], 2.0 / (4 * np.pi), rtol=1e-15)
    np.testing.assert_allclose(pot[2], 6.0 / (4 * np.pi), rtol=1e-15)


def test_gravity_reading_is_attractive():
    """Eq. 4 read as attraction: coef = -4 pi G turns the 1/(4 pi r) sum into
    -G sum m_j / r, and the force pulls each mass towards the other."""
    G = 1.0
    x = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    m = np.array([3.0, 5.0])
    pot, grad = O.direct(x, m)
    coef = -4 * np.pi * G
    np.testing.assert_allclose(coef * pot[0], -G * 5.0 / 2.0, rtol=1e-15)
    F = O.forces(m, grad, coef)
    np.testing.assert_allclose(F[0], [G * 3 * 5 / 4.0, 0, 0], rtol=1e-15)
    assert F[0][0] > 0 and F[1][0] < 0
