"""Periodic boundary conditions on the GPU (Sec. 2.4: a neutral cubic cell
repeated over Z^3), through the C ABI, against the oracle:

* the tree of the cell and its U/V/W/X lists with image shifts: bit-exact
  against oracle.periodic_lists (every entry a (box, image) pair);
* FP64: potentials and gradients against oracle.kifmm_periodic (the same
  method: lists over the cell and its 26 nearest images, the far-image
  operator on the root, the uniform second-moment term): within 10x the
  periodic method's measured rounding floor
  (parity_helpers.periodic_rounding_floor), never looser than 1e-12; uniform
  and clustered cells, p = 4 and 6, two cell sides;
* the mixed path (FP32 data, tensor-core M2L) against the Ewald sum
  (oracle.ewald, conducting boundary): gradients within the method's own
  error at p = 6 plus the FP32 floor; potentials with their mean removed (the
  FP32-based modes leave the uniform term's FP32 error in the mean, which
  gradients, forces and a neutral cell's energy do not see);
* positions outside the cell are wrapped; a charged cell is refused.

Plans take direct_max = -1: the oracle's periodic method keeps every W/X
interaction as classified.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from workloads import generators as G
from parity_helpers import periodic_rounding_floor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_09478_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def _neutral(n, seed, L=1.0):
    """n (even) points uniform in the cell, charges +1 and -1 in equal numbers
    (neutral exactly, in any precision)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, L, size=(n, 3))
    q = rng.permutation(np.repeat([1.0, -1.0], n // 2))
    return x, q


def _cluster(n, seed, L=1.0):
    xp, _ = G.plummer(n, seed)
    x = np.mod(0.5 * L + 0.05 * L * xp, L)
    q = np.random.default_rng(seed + 9).normal(size=n)
    return x, q - q.mean()


def _plan(n, L, p, M, precision="fp64", dtype=torch.float64):
    from paper_2512_09478_gb300 import Plan
    return Plan(p=p, leaf_cap=M, max_depth=20, precision=precision, n_max=n, dtype=dtype, cell=L, direct_max=-1)


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("case,n,M", [("uniform", 600, 16), ("cluster", 500, 8), ("one_leaf", 60, 64)])
def test_periodic_tree_and_lists_bit_exact(case, n, M):
    x, q = _cluster(n, 4) if case == "cluster" else _neutral(n, 5)
    plan = _plan(n, 1.0, 4, M)
    plan.set_sources(_dev(x), _dev(q))
    t = O.periodic_tree(x, 1.0, M, 20)
    g = plan.tree()
    assert g["level"].shape[0] == t["nb"]
    for name in ("level", "first", "count", "parent"):
        assert np.array_equal(g[name], t[name]), name
    lst, _ = O.periodic_lists(t)
    for kind in "UVWX":
        ptr, idx, img = plan.list_images(kind)
        for b in range(t["nb"]):
            mine = sorted(zip(idx[ptr[b]:ptr[b + 1]].tolist(), img[ptr[b]:ptr[b + 1]].tolist()))
            want = sorted((int(a), int(s)) for a, s in lst[kind][b])
            assert mine == want, (kind, b, mine[:6], want[:6])
    if case == "cluster":
        assert sum(len(w) for w in lst["W"]) > 0 and sum(len(v) for v in lst["X"]) > 0
    assert any((np.asarray(u)[:, 1] != 13).any() for u in lst["U"] if len(u))


@pytest.mark.parametrize("case,n,M,p,L", [("uniform", 2000, 32, 4, 1.0), ("uniform", 2000, 32, 6, 2.5),
                                          ("cluster", 1500, 16, 6, 1.0), ("one_leaf", 60, 64, 6, 1.0)])
def test_periodic_fp64_matches_oracle(case, n, M, p, L):
    x, q = _cluster(n, 7, L) if case == "cluster" else _neutral(n, 6, L)
    pot_o, grad_o = O.kifmm_periodic(x, q, L, p=p, leaf_cap=M)
    bar_p, bar_g = periodic_rounding_floor(x, q, L, p, M, pot_o, grad_o)
    plan = _plan(n, L, p, M)
    plan.set_sources(_dev(x), _dev(q))
    pot, grad, energy = plan.evaluate(want_energy=True)
    assert plan.device_status() == 0
    e_p = O.rel_l2(pot.cpu().numpy(), pot_o)
    e_g = O.rel_l2(grad.cpu().numpy(), grad_o)
    print("periodic fp64 %s p=%d L=%g: pot %.2e (bar %.2e) grad %.2e (bar %.2e)" % (case, p, L, e_p, bar_p, e_g, bar_g))
    assert e_p <= bar_p and e_g <= bar_g
    assert abs(energy.item() - O.energy(q, pot_o)) <= 0.5 * np.linalg.norm(q) * bar_p * np.linalg.norm(pot_o)


def test_periodic_positions_are_wrapped():
    x, q = _neutral(800, 8)
    shift = np.random.default_rng(3).integers(-2, 3, size=x.shape).astype(np.float64)
    plan = _plan(800, 1.0, 4, 16)
    plan.set_sources(_dev(x), _dev(q))
    pot0, grad0, _ = plan.evaluate()
    plan.set_sources(_dev(x + shift), _dev(q))     # the same particles, other images
    pot1, grad1, _ = plan.evaluate()
    assert O.rel_l2(pot1.cpu().numpy(), pot0.cpu().numpy()) < 1e-13
    assert O.rel_l2(grad1.cpu().numpy(), grad0.cpu().numpy()) < 1e-13


def test_periodic_charged_cell_is_refused():
    from paper_2512_09478_gb300 import KifmmError, Plan
    x, q = _neutral(300, 9)
    q[0] += 0.5
    plan = _plan(300, 1.0, 4, 16)
    with pytest.raises(KifmmError) as e:
        plan.set_sources(_dev(x), _dev(q))
    assert e.value.code == 1
    with pytest.raises(KifmmError) as e:        # one cell per plan
        Plan(p=4, leaf_cap=16, n_max=10, n_systems_max=2, cell=1.0)
    assert e.value.code == 1


@pytest.mark.parametrize("precision", ["mixed_fp16", "fp32"])
def test_periodic_reduced_precision_vs_ewald(precision):
    """The FP32-based paths against the Ewald sum over the FP32 inputs: the
    gradient within 1.1x the FP64 periodic method's own error plus 1e-6; the
    potential, mean removed, within 1.1x plus 1e-6."""
    x, q = _neutral(1200, 10)
    x32 = x.astype(np.float32).astype(np.float64)
    q32 = q                      # +-1: exact in FP32
    pe, ge = O.ewald(x32, q32, 1.0)
    pot_o, grad_o = O.kifmm_periodic(x32, q32, 1.0, p=6, leaf_cap=32)
    plan = _plan(1200, 1.0, 6, 32, precision, torch.float32)
    plan.set_sources(_dev(x32, torch.float32), _dev(q32, torch.float32))
    pot, grad, _ = plan.evaluate()
    assert plan.device_status() == 0
    pot, grad = pot.double().cpu().numpy(), grad.double().cpu().numpy()
    centre = lambda a: a - a.mean()
    e_g, e_go = O.rel_l2(grad, ge), O.rel_l2(grad_o, ge)
    e_p, e_po = O.rel_l2(centre(pot), centre(pe)), O.rel_l2(centre(pot_o), centre(pe))
    print("periodic %s vs Ewald: grad %.2e (fp64 method %.2e), pot-mean %.2e (%.2e)" % (precision, e_g, e_go, e_p, e_po))
    assert e_g <= 1.1 * e_go + 1e-6
    assert e_p <= 1.1 * e_po + 1e-6


def test_periodic_lists_kept_with_reuse_lists():
    """A periodic plan with reuse_lists keeps its image-shifted lists for a
    tree with the same boxes; its lists and outputs equal those of a plan that
    builds them every time and runs the same calls."""
    from paper_2512_09478_gb300 import Plan
    x, q = _neutral(1200, 12)
    jitter = np.random.default_rng(13).uniform(-1e-9, 1e-9, size=x.shape)
    mk = lambda reuse: Plan(p=4, leaf_cap=16, max_depth=20, precision="fp64", n_max=len(x), dtype=torch.float64,
                            cell=1.0, direct_max=-1, reuse_lists=reuse)
    plain, plan = mk(False), mk(True)
    for xs, reused in ((x, 0), (np.mod(x + jitter, 1.0), 1)):
        for pl in (plain, plan):
            pl.set_sources(_dev(xs), _dev(q))
        assert plan.tree_info()["lists_reused"] == reused
        pot, grad, _ = plan.evaluate()
        pp, gp, _ = plain.evaluate()
        assert torch.equal(pot, pp) and torch.equal(grad, gp)
        for kind in "UVWX":
            a, b = plan.list_images(kind), plain.list_images(kind)
            assert all(np.array_equal(u, v) for u, v in zip(a, b)), kind
    assert plan.device_status() == 0
