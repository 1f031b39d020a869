"""The tensor-core M2L's kernel variants (producer warps, one or two target
tiles of 128 per CTA sharing each operator block, pipeline depth) compute the
same sums in the same order: every variant's potentials and gradients are
bit-identical to the default's, through the C ABI.  Cases: a uniform set and
a Plummer cloud (W/X lists, many levels, classes whose last CTA holds a short
or empty second tile), p = 4, 6 and 8 (two output-column blocks).  The
default variant itself is checked against the oracle and the FP32 path by
the parity tests.  Pinning a variant the plan does not have is refused."""
import numpy as np
import pytest
import torch

from workloads import generators as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_09478_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


VARIANTS = [(2, 1, 2), (2, 1, 4), (4, 1, 3), (4, 1, 6), (2, 2, 2), (2, 2, 3), (2, 2, 4)]


def _run(x, q, p, M, variant):
    from paper_2512_09478_gb300 import Plan
    plan = Plan(p=p, leaf_cap=M, max_depth=20, precision="mixed_fp16", n_max=len(x), dtype=torch.float32)
    if variant is not None:
        pw, tl, ns = variant
        if ns > 4 and p >= 8:
            ns = 4
        plan.set_m2l_tuning(pw, tl, ns)
        assert plan.tuning()["m2l_producers"] == pw and plan.tuning()["m2l_tiles"] == tl
    plan.set_sources(torch.tensor(x, dtype=torch.float32, device="cuda"),
                     torch.tensor(q, dtype=torch.float32, device="cuda"))
    pot, grad, _ = plan.evaluate()
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    info = plan.tree_info()
    return pot.cpu().numpy(), grad.cpu().numpy(), info


@pytest.mark.parametrize("case,n,M,p", [("uniform", 20000, 32, 6), ("plummer", 20000, 16, 4),
                                        ("plummer", 12000, 16, 8)])
def test_variants_are_bit_identical(case, n, M, p):
    x, q = G.uniform_charges(n, 21) if case == "uniform" else G.plummer(n, 22)
    x = x.astype(np.float32).astype(np.float64)
    pot0, grad0, info = _run(x, q, p, M, None)
    assert info["n_v"] > 0
    for v in VARIANTS:
        pot, grad, _ = _run(x, q, p, M, v)
        assert np.array_equal(pot, pot0) and np.array_equal(grad, grad0), v


def test_pinning_checks_its_arguments():
    from paper_2512_09478_gb300 import KifmmError, Plan
    plan = Plan(p=6, leaf_cap=32, n_max=1000, precision="mixed_fp16")
    for bad in ((3, 1, 4), (4, 2, 3), (2, 3, 3), (2, 1, 1), (2, 1, 17), (2, 2, 5)):
        with pytest.raises(KifmmError) as e:
            plan.set_m2l_tuning(*bad)
        assert e.value.code == 1, bad
    for prec in ("fp32", "fp64"):
        other = Plan(p=6, leaf_cap=32, n_max=1000, precision=prec,
                     dtype=torch.float64 if prec == "fp64" else torch.float32)
        with pytest.raises(KifmmError):
            other.set_m2l_tuning(2, 1, 4)


def test_bounded_waits_time_out_and_the_plan_recovers():
    """The tensor-core M2L's barrier waits are bounded.  With a bound of one
    poll they run out on purpose: the kernel returns, the device status reads
    KIFMM_ERR_TIMEOUT, and with the default bound restored the same plan's
    next evaluate equals a fresh plan's bit for bit (the context stays
    usable; tensor memory was freed)."""
    from paper_2512_09478_gb300 import KifmmError, Plan
    x, q = G.uniform_charges(20000, 41)
    x = x.astype(np.float32).astype(np.float64)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    mk = lambda: Plan(p=4, leaf_cap=32, max_depth=20, precision="mixed_fp16", n_max=len(x), dtype=torch.float32)
    plan = mk()
    plan.set_sources(xt, qt)
    plan.set_m2l_wait_bound(1)
    plan.evaluate()
    torch.cuda.synchronize()
    assert plan.device_status() == 5          # KIFMM_ERR_TIMEOUT
    plan.set_m2l_wait_bound(0)
    pot, grad, _ = plan.evaluate()
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    fresh = mk()
    fresh.set_sources(xt, qt)
    pf, gf, _ = fresh.evaluate()
    assert torch.equal(pot, pf) and torch.equal(grad, gf)
    with pytest.raises(KifmmError):
        plan.set_m2l_wait_bound(-1)
    with pytest.raises(KifmmError):
        Plan(p=4, leaf_cap=32, n_max=100, precision="fp32").set_m2l_wait_bound(1)
