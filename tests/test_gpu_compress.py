"""Compressed M2L (desc.m2l_eps) on the tensor cores against the oracle's
compressed M2L, through the C ABI.

* Ranks: the plan's left/right ranks equal the oracle's (an integer decision
  taken on each side from its own FP64 spectrum: Jacobi eigenvalues of the
  Gram matrices on the GPU, LAPACK SVD of the stacks in the oracle).
* The effect of the compression: the change it makes to the GPU result
  (compressed minus dense mixed plan) matches the change it makes to the
  oracle's (compressed minus dense FP64 KIFMM), element by element, to 5% of
  the change plus the FP32 floor of two mixed-precision runs.
* The compressed GPU result is as close to the compressed oracle as the dense
  GPU result is to the dense oracle (plus a small FP32 allowance).
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
    torch.cuda.set_device(0)


def _run(x, q, p, M, m2l_eps):
    from paper_2512_09478_gb300 import Plan
    plan = Plan(p=p, leaf_cap=M, max_depth=20, precision="mixed_fp16", n_max=len(x), dtype=torch.float32,
                m2l_eps=m2l_eps)
    plan.set_sources(torch.tensor(x, dtype=torch.float32, device="cuda"),
                     torch.tensor(q, dtype=torch.float32, device="cuda"))
    pot, grad, _ = plan.evaluate()
    assert plan.device_status() == 0
    return pot.double().cpu().numpy(), grad.double().cpu().numpy(), plan.tuning()["m2l_ranks"]


CASES = [
    ("uniform", 4096, 32, 6, 1e-5),
    ("dem", 6000, 32, 6, 1e-5),
    ("uniform", 4096, 32, 4, 1e-2),
    ("uniform", 4096, 64, 8, 1e-5),
]


@pytest.mark.parametrize("kind,n,M,p,eps", CASES)
def test_compressed_m2l_matches_oracle(kind, n, M, p, eps):
    if kind == "uniform":
        x, q = G.uniform_charges(n, 500 + p)
    else:
        x, q, _ = G.dem_coulomb(n, 501)
    # the device receives FP32 inputs: the oracle works on the same rounded values
    x = x.astype(np.float32).astype(np.float64)
    q = q.astype(np.float32).astype(np.float64)
    ops = O.operators(p)
    ops_c, info = O.compress_m2l(ops, eps)
    pot_od, grad_od, _ = O.kifmm(x, q, p=p, leaf_cap=M, ops=ops)
    pot_oc, grad_oc, _ = O.kifmm(x, q, p=p, leaf_cap=M, ops=ops_c)
    pot_d, grad_d, r0 = _run(x, q, p, M, 0.0)
    pot_c, grad_c, rc = _run(x, q, p, M, eps)
    assert r0 == (0, 0)
    assert rc == (info["r_l"], info["r_r"])
    # what compressing changes, on both sides
    dp_o, dg_o = pot_oc - pot_od, grad_oc - grad_od
    dp_g, dg_g = pot_c - pot_d, grad_c - grad_d
    ch_p, ch_g = np.linalg.norm(dp_o) / np.linalg.norm(pot_od), np.linalg.norm(dg_o) / np.linalg.norm(grad_od)
    mis_p = np.linalg.norm(dp_g - dp_o) / np.linalg.norm(pot_od)
    mis_g = np.linalg.norm(dg_g - dg_o) / np.linalg.norm(grad_od)
    print("p=%d eps=%g ranks %s: change pot %.2e grad %.2e | mismatch of the change pot %.2e grad %.2e" % (
        p, eps, rc, ch_p, ch_g, mis_p, mis_g))
    # the change matches to 5% of itself plus the FP32 floor of two mixed runs
    assert mis_p <= 0.05 * ch_p + 1.5e-6
    assert mis_g <= 0.05 * ch_g + 3e-6
    # as close to the compressed oracle as the dense plan is to the dense oracle
    assert O.rel_l2(pot_c, pot_oc) <= O.rel_l2(pot_d, pot_od) + 1e-6
    assert O.rel_l2(grad_c, grad_oc) <= O.rel_l2(grad_d, grad_od) + 1e-6


def test_compressed_m2l_argument_rules():
    from paper_2512_09478_gb300 import Plan, KifmmError
    for prec, eps in (("fp32", 1e-5), ("fp64", 1e-5), ("mixed_fp16", -1e-5), ("mixed_fp16", 1.0),
                      ("mixed_fp16", float("nan"))):
        with pytest.raises(KifmmError) as e:
            Plan(p=6, leaf_cap=32, precision=prec, n_max=100,
                 dtype=torch.float64 if prec == "fp64" else torch.float32, m2l_eps=eps)
        assert e.value.code == 1


def test_compressed_plan_with_systems_refresh_and_backward():
    """The compressed M2L composes with the rest of the plan: two systems,
    a kept tree after a small motion (refresh_sources), and the adjoint (which
    keeps the dense transposed operators, so dq differs from the dense plan's by
    the compression's own size only)."""
    from paper_2512_09478_gb300 import Plan
    x1, q1 = G.uniform_charges(2000, 601)
    x2, q2 = G.uniform_charges(3000, 602)
    x = np.concatenate([x1, x2 + 3.0])
    q = np.concatenate([q1, q2])
    off = [0, 2000, 5000]
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    plans = {}
    for eps in (0.0, 1e-5):
        plan = Plan(p=6, leaf_cap=32, max_depth=20, precision="mixed_fp16", n_max=len(x), n_systems_max=2,
                    dtype=torch.float32, m2l_eps=eps)
        plan.set_sources(dev(x), dev(q), sys_offsets=off)
        assert plan.refresh_sources(dev(x + 1e-9), dev(q)) is True
        pot, grad, energy = plan.evaluate(want_energy=True)
        w = torch.linspace(-1.0, 1.0, len(x), device="cuda", dtype=torch.float32)
        dq, dx = plan.backward(w, grad)
        torch.cuda.synchronize()
        assert plan.device_status() == 0
        plans[eps] = [t.double().cpu().numpy() for t in (pot, grad, energy, dq, dx)]
    # each system against its own direct sum
    pot_c = plans[1e-5][0]
    for k in range(2):
        a, b = off[k], off[k + 1]
        xs = (x[a:b] + 1e-9).astype(np.float32).astype(np.float64)
        pd, _ = O.direct(xs, q[a:b])
        assert O.rel_l2(pot_c[a:b], pd) < 1e-5
    # compressed vs dense: within the compression's effect at eps = 1e-5
    for i, name in enumerate(("pot", "grad", "energy", "dq", "dx")):
        assert O.rel_l2(plans[1e-5][i], plans[0.0][i]) < 1e-4, name
