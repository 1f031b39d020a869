"""The Stokeslet kernel on the GPU (the tensor kernel Eq. 1 admits; Stokes
flow, Sec. 2.4), through the C ABI, against the oracle:

* FP64 velocities against oracle.kifmm_stokes (the same tree, lists,
  surfaces and pseudo-inverse rules with 3-vector densities), element by
  element: within 10x the method's rounding floor measured on the oracle
  (its change under a re-rounding of the input, x -> a x + b, undone exactly
  by the kernel's homogeneity), never looser than 1e-12.  The Stokeslet's
  check-from-equivalent matrices keep a near-null direction (the normal
  density, singular values down to 4e-11 of the largest at p = 6), so at p = 6
  two correct FP64 evaluations differ by ~3e-8;
* a single leaf equals the direct sum; W and X lists (a Plummer cloud);
* FP32 against the direct sum within 1.1x the FP64 method's error plus the
  FP32 floor;
* exact linearity in the forces; calls a Stokeslet plan does not support
  are refused.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from workloads import generators as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_09478_gb300 import build as B
    B.build()
    O.build()
    torch.cuda.set_device(0)


def _plan(n, p, M, precision="fp64", dtype=torch.float64):
    from paper_2512_09478_gb300 import Plan
    return Plan(p=p, leaf_cap=M, max_depth=20, precision=precision, n_max=n, dtype=dtype, kernel="stokeslet")


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def _stokes_floor(x, f, p, M, u_o):
    fl = 0.0
    for a, b in ((3.0, 0.1234567), (0.7, -0.3141592)):
        fl = max(fl, O.rel_l2(a * O.kifmm_stokes(a * x + b, f, p=p, leaf_cap=M), u_o))
    return max(1e-12, 10 * fl)


CASES = {
    "uniform": lambda n: (G.uniform_charges(n, 3)[0], np.random.default_rng(4).normal(size=(n, 3))),
    "plummer": lambda n: (G.plummer(n, 5)[0], np.random.default_rng(6).normal(size=(n, 3))),
}


@pytest.mark.parametrize("case,n,M,p", [("uniform", 1500, 32, 4), ("uniform", 1500, 32, 6),
                                        ("plummer", 1200, 16, 4)])
def test_stokes_fp64_matches_oracle(case, n, M, p):
    x, f = CASES[case](n)
    u_o = O.kifmm_stokes(x, f, p=p, leaf_cap=M)
    bar = _stokes_floor(x, f, p, M, u_o)
    plan = _plan(n, p, M)
    plan.set_sources(_dev(x), _dev(f))
    u, grad, energy = plan.evaluate()
    assert grad is None and energy is None and tuple(u.shape) == (n, 3)
    assert plan.device_status() == 0
    e = O.rel_l2(u.cpu().numpy(), u_o)
    print("stokes fp64 %s p=%d: %.2e (bar %.2e)" % (case, p, e, bar))
    assert e <= bar
    if case == "plummer":
        info = plan.tree_info()
        assert info["n_w"] > 0 and info["n_x"] > 0


def test_stokes_single_leaf_is_the_direct_sum():
    x, f = CASES["uniform"](100)
    plan = _plan(100, 4, 128)
    plan.set_sources(_dev(x), _dev(f))
    u, _, _ = plan.evaluate()
    assert plan.tree_info()["n_boxes"] == 1
    assert O.rel_l2(u.cpu().numpy(), O.stokeslet_direct(x, f)) < 1e-14


def test_stokes_is_linear_in_the_forces():
    x, f = CASES["uniform"](1500)
    plan = _plan(1500, 4, 32)
    plan.set_sources(_dev(x), _dev(f))
    u1 = plan.evaluate()[0].clone()
    plan.set_sources(_dev(x), _dev(2.0 * f))
    u2 = plan.evaluate()[0]
    assert torch.equal(u2, 2.0 * u1)   # scaling by 2 is exact through every stage


def test_stokes_fp32_vs_direct_sum():
    x, f = CASES["uniform"](3000)
    x32 = x.astype(np.float32).astype(np.float64)
    f32 = f.astype(np.float32).astype(np.float64)
    ud = O.stokeslet_direct(x32, f32)
    e64 = O.rel_l2(O.kifmm_stokes(x32, f32, p=6, leaf_cap=32), ud)
    plan = _plan(3000, 6, 32, "fp32", torch.float32)
    plan.set_sources(_dev(x32, torch.float32), _dev(f32, torch.float32))
    u, _, _ = plan.evaluate()
    assert plan.device_status() == 0
    e = O.rel_l2(u.double().cpu().numpy(), ud)
    print("stokes fp32 vs direct: %.2e (fp64 method %.2e)" % (e, e64))
    assert e <= 1.1 * e64 + 1e-5


def test_stokes_refuses_what_it_does_not_support():
    from paper_2512_09478_gb300 import KifmmError, Plan
    for kw in (dict(precision="mixed_fp16"), dict(cell=1.0), dict(p=9)):
        args = dict(p=4, leaf_cap=16, n_max=100, kernel="stokeslet")
        args.update(kw)
        with pytest.raises(KifmmError) as e:
            Plan(**args)
        assert e.value.code == 1
    x, f = CASES["uniform"](200)
    plan = _plan(200, 4, 16)
    plan.set_sources(_dev(x), _dev(f))
    with pytest.raises(KifmmError) as e:
        plan.evaluate(grad=torch.empty(200, 3, dtype=torch.float64, device="cuda"))
    assert e.value.code == 1
    u, _, _ = plan.evaluate()
    with pytest.raises(KifmmError) as e:
        plan.backward(torch.ones(200, dtype=torch.float64, device="cuda"), u)
    assert e.value.code == 1


def test_stokes_lists_kept_with_reuse_lists():
    """A Stokeslet plan with reuse_lists keeps its lists for a tree with the
    same boxes; its velocities equal those of a plan that builds them every
    time and runs the same calls, bit for bit."""
    from paper_2512_09478_gb300 import Plan
    x, f = CASES["uniform"](1500)
    jitter = np.random.default_rng(14).uniform(-1e-9, 1e-9, size=x.shape)
    mk = lambda reuse: Plan(p=4, leaf_cap=32, max_depth=20, precision="fp64", n_max=len(x), dtype=torch.float64,
                            kernel="stokeslet", reuse_lists=reuse)
    plain, plan = mk(False), mk(True)
    for xs, reused in ((x, 0), (x + jitter, 1)):
        for pl in (plain, plan):
            pl.set_sources(_dev(xs), _dev(f))
        assert plan.tree_info()["lists_reused"] == reused
        u, _, _ = plan.evaluate()
        up, _, _ = plain.evaluate()
        assert torch.equal(u, up)
    assert plan.device_status() == 0
