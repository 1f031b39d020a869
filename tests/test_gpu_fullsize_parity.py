"""Element-wise parity at full size, on the DEM Coulomb packing (p = 6, leaf
cap 128, the benchmark's configuration): 125k spheres (the profiling case)
and the whole 1M packing.

* FP64 GPU path vs oracle.kifmm on every particle: potentials and gradients
  within rel-L2 1e-12.  Keys, tree and the sort's leaf membership are
  compared bit for bit.  The tree is built twice on one plan, so the second build runs the
  path that reuses the previous tree's level sizes, and the sort covers only
  the key digits the octree reads (asserted).
* The benchmarked mixed path (FP32 data, 3xFP16 tensor-core M2L, autotuned
  tiles) vs oracle.kifmm on the same FP32-rounded inputs with the FP32 modes'
  pseudo-inverse truncation (1e-9): the same method, so what remains is
  FP32 rounding.  Bar: the plain FP32 SIMT path's own distance to the oracle
  (the FP32 floor of this formulation) times 1.5, plus 1e-7.

Branch coverage: the gathered-GEMM launcher picks big tiles, big tiles with
the child slots split over blocks (M2M levels of 2432..4096 parents), small
split tiles and small plain tiles by level size; the test asserts from the
tree which of them this workload exercises (all four at 1M).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from workloads import generators as G

pytestmark = pytest.mark.gpu

SMS = 152
SPLIT_TARGETS = 4096


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_09478_gb300 import build as B
    B.build()
    G.build()
    O.build()
    torch.cuda.set_device(0)


_CACHE = {}


def _packing(n):
    if n not in _CACHE:
        x, q, _ = G.dem_coulomb(n, 1001)
        _CACHE[n] = (x, q / 1e-12)  # Eq. 3 units, charges of order one
    return _CACHE[n]


def ggemm_branch(total, nslots, ld):
    """The gathered-GEMM launcher's tile choice for `total` targets (the rule
    of ggemm_classes on a 152-SM GPU)."""
    big_blocks = -(-total // 64) * -(-ld // 160)
    if big_blocks >= 2 * SMS:
        return "big"
    splittable = 1 < nslots <= 8 and total <= SPLIT_TARGETS
    if splittable and big_blocks * nslots >= 2 * SMS:
        return "big_split"
    small_blocks = -(-total // 16) * -(-ld // 32)
    if splittable and small_blocks < 16 * SMS:
        return "small_split"
    return "small"


def _branches(tree, ns):
    lvl, parent = tree["level"], tree["parent"]
    seen = set()
    for l in range(int(lvl.max()) + 1):
        parents = np.unique(parent[(lvl == l + 1)]) if l < lvl.max() else np.array([])
        if parents.size:
            seen.add(("m2m", ggemm_branch(parents.size, 8, ns)))
        if l >= 1:
            seen.add(("l2l", ggemm_branch(int((lvl == l).sum()), 1, ns)))
    return seen


def _fp64_run(x, q):
    from paper_2512_09478_gb300 import Plan
    plan = Plan(p=6, leaf_cap=128, max_depth=20, precision="fp64", n_max=len(x), dtype=torch.float64,
                autotune=True)
    xt = torch.tensor(x, device="cuda")
    qt = torch.tensor(q, device="cuda")
    plan.set_sources(xt, qt)
    first_passes = plan.tree_info()["sort_passes"]
    plan.set_sources(xt, qt)   # the second build reuses the first tree's level sizes
    pot, grad, energy = plan.evaluate(want_energy=True)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return plan, first_passes, pot.cpu().numpy(), grad.cpu().numpy(), energy.item()


@pytest.mark.parametrize("n", [125_000, 1_000_000])
def test_fp64_elementwise_vs_oracle(n):
    x, q = _packing(n)
    plan, first_passes, pot, grad, energy = _fp64_run(x, q)
    t = O.sort_and_tree(x, 128, 20)
    lst = O.lists(t)
    # structure, bit for bit
    keys, perm, _ = plan.keys()
    assert np.array_equal(keys, t["keys"])
    g = plan.tree()
    for name in ("level", "first", "count", "parent"):
        assert np.array_equal(g[name], t[name]), name
    for b in np.nonzero(t["child_first"] < 0)[0]:
        f, c = int(t["first"][b]), int(t["count"][b])
        assert np.array_equal(np.sort(perm[f:f + c]), np.sort(t["perm"][f:f + c]))
    info = plan.tree_info()
    assert info["sort_passes"] < 8 and first_passes < 8   # the partial sort ran, both builds
    sizes = np.bincount(t["level"])
    assert sizes.max() > 1024
    br = _branches(t, 153)
    print("n=%d levels %s sort passes %d branches %s" % (n, sizes.tolist(), info["sort_passes"], sorted(br)))
    if n == 1_000_000:
        assert ("m2m", "big_split") in br and ("m2m", "small_split") in br
        assert ("l2l", "big") in br and ("l2l", "small") in br
    # every particle against the oracle
    pot_o, grad_o, _ = O.kifmm(x, q, p=6, leaf_cap=128, tree=t, lst=lst)
    e_p, e_g = O.rel_l2(pot, pot_o), O.rel_l2(grad, grad_o)
    print("n=%d fp64 vs oracle: pot %.2e grad %.2e" % (n, e_p, e_g))
    assert e_p <= 1e-12 and e_g <= 1e-12
    assert abs(energy - O.energy(q, pot_o)) <= 0.5 * np.linalg.norm(q) * 1e-12 * np.linalg.norm(pot_o)


def _reduced_run(x32, q32, precision):
    from paper_2512_09478_gb300 import Plan
    plan = Plan(p=6, leaf_cap=128, max_depth=20, precision=precision, n_max=len(x32), dtype=torch.float32,
                autotune=True)
    xt = torch.tensor(x32, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q32, dtype=torch.float32, device="cuda")
    plan.set_sources(xt, qt)
    plan.evaluate()              # the first evaluate tunes the tiles
    pot, grad, _ = plan.evaluate()
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return pot.double().cpu().numpy(), grad.double().cpu().numpy()


@pytest.mark.parametrize("n", [125_000, 1_000_000])
def test_mixed_vs_same_method_oracle(n):
    x, q = _packing(n)
    x32 = x.astype(np.float32).astype(np.float64)
    q32 = q.astype(np.float32).astype(np.float64)
    t = O.sort_and_tree(x32, 128, 20)
    lst = O.lists(t)
    # the FP32-based modes truncate the pseudo-inverse at 1e-9 (FP32 cannot
    # resolve the modes below it): the oracle with that truncation is the
    # same method
    pot_o, grad_o, _ = O.kifmm(x32, q32, p=6, leaf_cap=128, tree=t, lst=lst, eps=1e-9)
    pot_m, grad_m = _reduced_run(x32, q32, "mixed_fp16")
    pot_f, grad_f = _reduced_run(x32, q32, "fp32")
    e = {k: (O.rel_l2(a, pot_o), O.rel_l2(b, grad_o)) for k, (a, b) in
         {"mixed": (pot_m, grad_m), "fp32": (pot_f, grad_f)}.items()}
    print("n=%d vs oracle (pinv 1e-9): mixed pot %.2e grad %.2e | fp32 pot %.2e grad %.2e"
          % (n, *e["mixed"], *e["fp32"]))
    assert e["mixed"][0] <= 1.5 * e["fp32"][0] + 1e-7
    assert e["mixed"][1] <= 1.5 * e["fp32"][1] + 1e-7
    # the FP32 floor itself: a few 1e-6 (potential) and 1e-5 (gradient)
    assert e["fp32"][0] < 5e-6 and e["fp32"][1] < 2e-5
