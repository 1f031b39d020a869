"""Pins of the oracle's compressed M2L (low-rank M2L matrices on shared bases).

* compress_rank: the threshold count, the tile rounding with and without the
  mean slot, the cap at n and the lowering off clusters, on hand-made lists.
* The bases are singular vectors of the right stacks: the squared singular
  values equal the eigenvalues of the Gram matrices (another LAPACK routine),
  and the projection errors equal the discarded energy (Eckart-Young).
* Full rank reproduces the dense operators and the dense KIFMM.
* Truncated ranks change the result by an amount that shrinks with eps and
  stays within the budget, against the direct sum.
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import generators as G


def test_compress_rank_rules():
    s = np.array([1.0, 0.5, 0.2, 0.1, 0.05, 0.01, 0.005, 0.001])
    assert O.compress_rank(s, 0.03, tile=1) == 5          # values above 0.03
    assert O.compress_rank(s, 0.03, tile=4) == 8          # 5 -> 8
    assert O.compress_rank(s, 0.03, tile=4, mean_slot=1) == 7   # 5 + 1 -> 8, minus the slot
    assert O.compress_rank(s, 0.3, tile=2) == 2           # 2 -> 2
    assert O.compress_rank(s, 0.3, tile=32) == 8          # capped at n
    t = np.array([1.0, 0.5, 0.3, 0.3, 0.3, 0.1, 0.05, 0.01])
    assert O.compress_rank(t, 0.4, tile=4) == 2           # 2 -> 4 would split the 0.3 triplet -> 2
    assert O.compress_rank(t, 0.2, tile=4) == 8           # 5 -> 8 is n: no cut
    assert O.compress_rank(t, 0.2, tile=3) == 6           # 5 -> 6, cut between 0.1 and 0.05: kept
    u = np.array([1.0, 0.5, 0.5 / 1.0005, 0.2])           # within the 1.001 cluster width
    assert O.compress_rank(u, 0.6, tile=2) == 1           # 1 -> 2 splits the pair -> 1


@pytest.fixture(scope="module")
def ops6():
    ops = O.operators(6)
    return ops, O.compress_m2l(ops, 1e-5)


def test_bases_are_singular_vectors_of_the_stacks(ops6):
    ops, (_, info) = ops6
    K = ops["m2l"]
    m = K.mean(axis=1)
    K0 = K - m[:, None, :]
    # eigenvalues of the Gram matrices (eigvalsh, not svd) = squared singular values
    gl = np.sort(np.linalg.eigvalsh(np.einsum("oij,okj->ik", K0, K0)))[::-1]
    gr = np.sort(np.linalg.eigvalsh(np.einsum("oji,ojk->ik", K, K)))[::-1]
    top = gl[0]
    assert np.allclose(info["s_l"] ** 2, gl, rtol=1e-9, atol=1e-12 * top)
    assert np.allclose(info["s_r"] ** 2, gr, rtol=1e-9, atol=1e-12 * gr[0])
    U, V, rl, rr = info["U"], info["V"], info["r_l"], info["r_r"]
    assert U.shape == (ops["ns"], rl) and V.shape == (ops["ns"], rr)
    # Eckart-Young: what the projections leave out is the discarded energy
    el = sum(np.linalg.norm(k0 - U @ (U.T @ k0)) ** 2 for k0 in K0)
    er = sum(np.linalg.norm(k - (k @ V) @ V.T) ** 2 for k in K)
    assert el == pytest.approx(np.sum(info["s_l"][rl:] ** 2), rel=1e-6)
    assert er == pytest.approx(np.sum(info["s_r"][rr:] ** 2), rel=1e-6)
    # the mean-free left basis is orthogonal to the constant vector
    assert np.abs(U.T @ np.ones(ops["ns"])).max() < 1e-8   # eps_mach sigma_0 / sigma_r at the cut
    # p = 6, eps = 1e-5: ranks fill 128- and 96-wide tiles (126 + mean and 94 after
    # lowering off the clusters at the cut)
    assert (rl, rr) == (126, 94)


def test_full_rank_is_the_dense_operator():
    ops = O.operators(4)
    ops_c, info = O.compress_m2l(ops, 1e-14)
    assert info["r_l"] == ops["ns"] and info["r_r"] == ops["ns"]
    rel = np.linalg.norm(ops_c["m2l"] - ops["m2l"]) / np.linalg.norm(ops["m2l"])
    assert rel < 1e-12
    x, q = G.uniform_charges(600, 3)
    pot_d, grad_d, _ = O.kifmm(x, q, p=4, leaf_cap=16, ops=ops)
    pot_c, grad_c, _ = O.kifmm(x, q, p=4, leaf_cap=16, ops=ops_c)
    assert O.rel_l2(pot_c, pot_d) < 1e-11 and O.rel_l2(grad_c, grad_d) < 1e-11


def test_truncation_error_shrinks_with_eps():
    ops = O.operators(4)
    x, q = G.uniform_charges(1500, 5)
    pd, gd = O.direct(x, q)
    pot_d, grad_d, _ = O.kifmm(x, q, p=4, leaf_cap=16, ops=ops)
    diffs = []
    for eps in (1e-2, 1e-3, 1e-4):
        ops_c, info = O.compress_m2l(ops, eps, tile=4)
        assert info["r_l"] < ops["ns"] and info["r_r"] < ops["ns"]
        pot_c, grad_c, _ = O.kifmm(x, q, p=4, leaf_cap=16, ops=ops_c)
        diffs.append((O.rel_l2(pot_c, pot_d), O.rel_l2(grad_c, grad_d)))
        # within eps-sized budget of the dense method, against the direct sum
        assert O.rel_l2(grad_c, gd) <= O.rel_l2(grad_d, gd) + 30 * eps
    assert diffs[0][0] > diffs[1][0] > diffs[2][0] > 0
    assert diffs[0][1] > diffs[1][1] > diffs[2][1] > 0
