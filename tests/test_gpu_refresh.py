"""Tree reuse with a validity test (kifmm_refresh_sources), through the C ABI.

* The keep/rebuild decision matches the one taken on the CPU from the
  oracle's tree (the leaf of every particle, the finest level, the root cube).
* A kept tree gives exactly what update_sources gives; a rebuilt one gives
  what a fresh set_sources gives (same tree, results within rounding).
* Accuracy after small motions: within the method's error of a fresh tree,
  against the FP64 direct sum.
* Non-finite input and argument errors are reported.
* set_sources keeps the lists when the rebuilt tree has the same boxes: the
  outputs and lists equal a fresh plan's bit for bit; other boxes rebuild them.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from workloads import generators as G

pytestmark = pytest.mark.gpu

SKIN = 0.05


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_09478_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def _plan(n, precision="fp64", p=4, M=32, dtype=torch.float64, reuse_lists=False):
    from paper_2512_09478_gb300 import Plan
    return Plan(p=p, leaf_cap=M, max_depth=20, precision=precision, n_max=n, dtype=dtype, reuse_lists=reuse_lists)


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def _leaf_geometry(x, M):
    """Per particle (user order): its leaf's centre and half-width in root
    units, from the oracle's tree; plus the finest level and the root cube."""
    t = O.sort_and_tree(x, M, 20)
    n = len(x)
    centre = np.empty((n, 3))
    half = np.empty(n)
    for b in np.nonzero(t["child_first"] < 0)[0]:
        w = 2.0 ** -int(t["level"][b])
        idx = t["perm"][t["first"][b]:t["first"][b] + t["count"][b]]
        centre[idx] = (t["coord"][b] + 0.5) * w
        half[idx] = 0.5 * w
    return centre, half, int(t["level"].max()), t["lo"], t["side"]


def _keeps(x_old, x_new, M, skin):
    """The decision the device must take: every new position, in the old root
    cube, within its leaf's half-width plus skin finest-level half-widths."""
    centre, half, lmax, lo, side = _leaf_geometry(x_old, M)
    r = (np.asarray(x_new) - lo) / side - centre
    return bool(np.all(np.abs(r) <= (half + skin * 0.5 * 2.0 ** -lmax)[:, None]))


def _margin(x, M, skin=SKIN):
    _, _, lmax, _, side = _leaf_geometry(x, M)
    return skin * 0.5 * side * 2.0 ** -lmax


@pytest.mark.parametrize("precision,dtype", [("fp64", torch.float64), ("fp32", torch.float32),
                                             ("mixed_fp16", torch.float32)])
def test_small_motion_keeps_tree_and_equals_update_sources(precision, dtype):
    x, q = G.uniform_charges(4096, 31)
    M = 32
    x2 = x + np.random.default_rng(32).uniform(-0.2, 0.2, size=x.shape) * _margin(x, M)
    q2 = q * 1.5
    assert _keeps(x, x2, M, SKIN)
    plan = _plan(len(x), precision=precision, M=M, dtype=dtype)
    plan.set_sources(_dev(x, dtype), _dev(q, dtype))
    plan.evaluate()
    info0 = plan.tree_info()
    assert plan.refresh_sources(_dev(x2, dtype), _dev(q2, dtype), skin=SKIN) is True
    assert plan.tree_info() == info0
    pot_r, grad_r, _ = plan.evaluate()
    pot_r, grad_r = pot_r.cpu().numpy(), grad_r.cpu().numpy()
    plan.update_sources(_dev(x2, dtype), _dev(q2, dtype))
    pot_u, grad_u, _ = plan.evaluate()
    assert np.array_equal(pot_r, pot_u.cpu().numpy())
    assert np.array_equal(grad_r, grad_u.cpu().numpy())
    assert plan.device_status() == 0


def test_reused_tree_accuracy_matches_fresh_tree():
    """Motions of 0.9 of the skin: the kept tree's error against the direct
    sum stays within 1.2x that of a tree built for the new positions."""
    x, q = G.uniform_charges(4096, 41)
    M = 32
    x2 = x + np.random.default_rng(42).uniform(-0.9, 0.9, size=x.shape) * _margin(x, M) / np.sqrt(3.0)
    assert _keeps(x, x2, M, SKIN)
    pd, gd = O.direct(x2, q)
    plan = _plan(len(x), p=6, M=M)
    plan.set_sources(_dev(x), _dev(q))
    assert plan.refresh_sources(_dev(x2), _dev(q), skin=SKIN) is True
    pot_r, grad_r, _ = plan.evaluate()
    fresh = _plan(len(x), p=6, M=M)
    fresh.set_sources(_dev(x2), _dev(q))
    pot_f, grad_f, _ = fresh.evaluate()
    e_pr, e_gr = O.rel_l2(pot_r.cpu().numpy(), pd), O.rel_l2(grad_r.cpu().numpy(), gd)
    e_pf, e_gf = O.rel_l2(pot_f.cpu().numpy(), pd), O.rel_l2(grad_f.cpu().numpy(), gd)
    assert e_pr <= 1.2 * e_pf + 1e-12, (e_pr, e_pf)
    assert e_gr <= 1.2 * e_gf + 1e-12, (e_gr, e_gf)


def test_skin_decides_between_keep_and_rebuild():
    """One particle put half a margin outside its leaf (toward the root's
    centre): kept with skin 0.05, rebuilt with skin 0."""
    x, q = G.uniform_charges(3000, 51)
    M = 16
    centre, half, lmax, lo, side = _leaf_geometry(x, M)
    i = 123
    ax = 1
    sgn = 1.0 if centre[i, ax] < 0.5 else -1.0
    x2 = x.copy()
    x2[i, ax] = lo[ax] + side * (centre[i, ax] + sgn * (half[i] + 0.5 * SKIN * 0.5 * 2.0 ** -lmax))
    assert _keeps(x, x2, M, SKIN) and not _keeps(x, x2, M, 0.0)
    plan = _plan(len(x), M=M)
    plan.set_sources(_dev(x), _dev(q))
    assert plan.refresh_sources(_dev(x2), _dev(q), skin=SKIN) is True
    plan.set_sources(_dev(x), _dev(q))
    assert plan.refresh_sources(_dev(x2), _dev(q), skin=0.0) is False
    # unchanged positions keep the tree even without a skin
    assert plan.refresh_sources(_dev(x2), _dev(q), skin=0.0) is True


def test_large_motion_rebuilds_like_set_sources():
    x, q = G.uniform_charges(4096, 61)
    M = 32
    rng = np.random.default_rng(62)
    x2 = x.copy()
    x2[rng.choice(len(x), 40, replace=False)] = rng.uniform(0, 1, size=(40, 3))
    assert not _keeps(x, x2, M, SKIN)
    plan = _plan(len(x), M=M)
    plan.set_sources(_dev(x), _dev(q))
    plan.evaluate()
    assert plan.refresh_sources(_dev(x2), _dev(q), skin=SKIN) is False
    pot_r, grad_r, _ = plan.evaluate()
    fresh = _plan(len(x), M=M)
    fresh.set_sources(_dev(x2), _dev(q))
    pot_f, grad_f, _ = fresh.evaluate()
    # the same tree (the sorted digit count may differ: it follows each plan's last depth)
    strip = lambda d: {k: v for k, v in d.items() if k not in ("sort_passes", "lists_reused")}
    assert strip(plan.tree_info()) == strip(fresh.tree_info())
    k1, p1, l1 = plan.keys()
    k2, p2, l2 = fresh.keys()
    assert np.array_equal(k1, k2) and np.array_equal(l1, l2)
    # same particles per leaf (the order inside a leaf depends on how many key
    # digits each plan sorted)
    g = plan.tree()
    isleaf = ~np.isin(np.arange(len(g["level"])), g["parent"])
    for f, c in zip(g["first"][isleaf], g["count"][isleaf]):
        assert np.array_equal(np.sort(p1[f:f + c]), np.sort(p2[f:f + c]))
    assert O.rel_l2(pot_r.cpu().numpy(), pot_f.cpu().numpy()) <= 1e-14
    assert O.rel_l2(grad_r.cpu().numpy(), grad_f.cpu().numpy()) <= 1e-14
    # and the new tree is the oracle's
    t = O.sort_and_tree(x2, M, 20)
    assert np.array_equal(k1, t["keys"])


def test_refresh_with_several_systems():
    """Two systems: a motion in the second one only rebuilds both (one tree
    per plan), and the kept case leaves every system's tree alone."""
    x1, q1 = G.uniform_charges(1500, 71)
    x2, q2 = G.uniform_charges(2500, 72)
    x = np.concatenate([x1, x2 + 5.0])
    q = np.concatenate([q1, q2])
    off = [0, 1500, 4000]
    from paper_2512_09478_gb300 import Plan
    plan = Plan(p=4, leaf_cap=32, max_depth=20, precision="fp64", n_max=len(x), n_systems_max=2,
                dtype=torch.float64)
    plan.set_sources(_dev(x), _dev(q), sys_offsets=off)
    info0 = plan.tree_info()
    assert plan.refresh_sources(_dev(x), _dev(q * 2), skin=SKIN) is True
    assert plan.tree_info() == info0
    xm = x.copy()
    xm[3000] = [5.0, 5.0, 5.0]
    xm[3001] = [6.0, 6.0, 6.0]
    assert plan.refresh_sources(_dev(xm), _dev(q), skin=SKIN) is False
    pot, _, energy = plan.evaluate(want_energy=True)
    fresh = Plan(p=4, leaf_cap=32, max_depth=20, precision="fp64", n_max=len(x), n_systems_max=2,
                 dtype=torch.float64)
    fresh.set_sources(_dev(xm), _dev(q), sys_offsets=off)
    pot_f, _, energy_f = fresh.evaluate(want_energy=True)
    # the same tree (the sorted digit count may differ: it follows each plan's last depth)
    strip = lambda d: {k: v for k, v in d.items() if k not in ("sort_passes", "lists_reused")}
    assert strip(plan.tree_info()) == strip(fresh.tree_info())
    assert O.rel_l2(pot.cpu().numpy(), pot_f.cpu().numpy()) <= 1e-14
    assert O.rel_l2(energy.cpu().numpy(), energy_f.cpu().numpy()) <= 1e-14


def test_refresh_errors():
    from paper_2512_09478_gb300 import KifmmError
    x, q = G.uniform_charges(300, 81)
    plan = _plan(len(x), M=16)
    with pytest.raises(KifmmError) as e:
        plan.refresh_sources(_dev(x), _dev(q))
    assert e.value.code == 6                      # before set_sources
    plan.set_sources(_dev(x), _dev(q))
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(KifmmError) as e:
            plan.refresh_sources(_dev(x), _dev(q), skin=bad)
        assert e.value.code == 1
    xn = x.copy()
    xn[17, 2] = np.nan
    with pytest.raises(KifmmError) as e:
        plan.refresh_sources(_dev(xn), _dev(q))
    assert e.value.code == 4                      # non-finite: rebuild reports it
    with pytest.raises(KifmmError) as e:
        plan.evaluate()
    assert e.value.code == 6                      # and the plan holds no sources


def test_changed_system_offsets_are_uploaded():
    """A plan reuses the uploaded system offsets (and energy chunks) while they
    are unchanged; new offsets must reach the device: the same particles split
    differently give each system's energy as a fresh plan does."""
    from paper_2512_09478_gb300 import Plan
    x, q = G.uniform_charges(4000, 91)
    mk = lambda: Plan(p=4, leaf_cap=32, max_depth=20, precision="fp64", n_max=len(x), n_systems_max=3,
                      dtype=torch.float64)
    plan = mk()
    for off in ([0, 1500, 4000], [0, 1500, 4000], [0, 2500, 4000], [0, 1000, 3000, 4000]):
        plan.set_sources(_dev(x), _dev(q), sys_offsets=off)
        pot, _, energy = plan.evaluate(want_energy=True)
        fresh = mk()
        fresh.set_sources(_dev(x), _dev(q), sys_offsets=off)
        pot_f, _, energy_f = fresh.evaluate(want_energy=True)
        assert energy.shape[0] == len(off) - 1
        assert O.rel_l2(energy.cpu().numpy(), energy_f.cpu().numpy()) <= 1e-14, off
        assert O.rel_l2(pot.cpu().numpy(), pot_f.cpu().numpy()) <= 1e-14, off


@pytest.mark.parametrize("precision,dtype", [("fp64", torch.float64), ("mixed_fp16", torch.float32)])
def test_set_sources_keeps_lists_of_unchanged_boxes(precision, dtype):
    """With reuse_lists, a rebuilt tree with the same boxes (level,
    coordinates, parent, children, small-leaf flag) keeps its lists and box
    partitions.  A plan with the flag and one without run the same sequence of
    set_sources calls (so that they sort the same key digits): their lists and
    outputs are bit-identical at every step, kept lists or not.  A tree whose
    boxes changed builds them again, and then equals a fresh plan's within
    rounding (the particle order inside a leaf follows the sorted digits)."""
    x, q = G.uniform_charges(6000, 91)
    M = 32
    jitter = np.random.default_rng(92).uniform(-1e-9, 1e-9, size=x.shape)
    x2 = x.copy()   # particles moved into one corner: other boxes
    x2[:200] = np.random.default_rng(93).uniform(0, 0.2, size=(200, 3))
    plain = _plan(len(x), precision=precision, M=M, dtype=dtype)
    plan = _plan(len(x), precision=precision, M=M, dtype=dtype, reuse_lists=True)
    for xs, reused in ((x, 0), (x + jitter, 1), (x, 1), (x2, 0), (x2 + jitter, 1)):
        for pl in (plain, plan):
            pl.set_sources(_dev(xs, dtype), _dev(q, dtype))
        assert plain.tree_info()["lists_reused"] == 0
        assert plan.tree_info()["lists_reused"] == reused
        pot, grad, _ = plan.evaluate()
        pp, gp, _ = plain.evaluate()
        assert torch.equal(pot, pp) and torch.equal(grad, gp)
        for kind in "UVWX":
            a, b = plan.list(kind), plain.list(kind)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    fresh = _plan(len(x), precision=precision, M=M, dtype=dtype)
    fresh.set_sources(_dev(x2 + jitter, dtype), _dev(q, dtype))
    pf, gf, _ = fresh.evaluate()
    tol = 1e-14 if dtype == torch.float64 else 1e-6
    assert O.rel_l2(pot.double().cpu().numpy(), pf.double().cpu().numpy()) <= tol
    assert O.rel_l2(grad.double().cpu().numpy(), gf.double().cpu().numpy()) <= tol
    assert plan.device_status() == 0
