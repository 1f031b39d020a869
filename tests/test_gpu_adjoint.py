"""Adjoint (kifmm_backward) against the oracle, through the C ABI.

* dq = A^T w with A the oracle's own KIFMM operator, assembled column by
  column from unit charges (same tree, lists and operators): rel-L2 <= 1e-11.
* dx against central finite differences of the oracle's L = sum_i w_i pot_i
  with the tree frozen (h = 1e-6 of the box side).
* Energy gradients through the torch.autograd.Function against the
  brute-force gradients dU/dq_i = pot_i, dU/dx_i = q_i grad_i (exact sums),
  within the method's error at that p; FP32 vs FP64 adjoint.
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


def _case(n=160, seed=3):
    x, _ = G.plummer(n, seed)
    rng = np.random.default_rng(seed)
    return x, rng.normal(size=n), rng.normal(size=n)


def _gpu(x, q, M, p, precision="fp64", dtype=torch.float64):
    from paper_2512_09478_gb300 import Plan
    plan = Plan(p=p, leaf_cap=M, precision=precision, n_max=len(x), dtype=dtype)
    xt = torch.tensor(x, dtype=dtype, device="cuda")
    qt = torch.tensor(q, dtype=dtype, device="cuda")
    plan.set_sources(xt, qt)
    pot, grad, _ = plan.evaluate()
    return plan, xt, qt, pot, grad


@pytest.mark.parametrize("M,p", [(4, 4), (8, 6)])
def test_dq_is_oracle_transpose(M, p):
    x, q, w = _case()
    tree = O.sort_and_tree(x, M, 20)
    lst = O.lists(tree)
    ops = O.operators(p)
    assert lst["W"][1].size > 0
    n = len(x)
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = O.kifmm(x, e, p=p, tree=tree, lst=lst, ops=ops)[0]
    plan, xt, qt, pot, grad = _gpu(x, q, M, p)
    dq, dx = plan.backward(torch.tensor(w, device="cuda"), grad)
    assert O.rel_l2(dq.cpu().numpy(), A.T @ w) <= 1e-11
    assert O.rel_l2(pot.cpu().numpy(), A @ q) <= 1e-11


def test_dx_matches_oracle_finite_differences():
    x, q, w = _case(140, 5)
    M, p = 4, 4
    tree = O.sort_and_tree(x, M, 20)
    lst = O.lists(tree)
    ops = O.operators(p)
    plan, xt, qt, pot, grad = _gpu(x, q, M, p)
    _, dx = plan.backward(torch.tensor(w, device="cuda"), grad)
    dx = dx.cpu().numpy()
    h = 1e-6 * tree["side"]
    rng = np.random.default_rng(0)
    for k in rng.choice(len(x), 12, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, d] += h
            xm[k, d] -= h
            Lp = w @ O.kifmm(xp, q, p=p, tree=tree, lst=lst, ops=ops)[0]
            Lm = w @ O.kifmm(xm, q, p=p, tree=tree, lst=lst, ops=ops)[0]
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - dx[k, d]) <= 1e-6 * np.abs(dx).max(), (k, d, fd, dx[k, d])


def test_frozen_tree_finite_differences_on_gpu():
    """update_sources keeps the tree: central differences of the GPU energy
    match the adjoint (FP64)."""
    from paper_2512_09478_gb300.kifmm import energy
    x, q, _ = _case(400, 7)
    plan, xt, qt, pot, grad = _gpu(x, q, 8, 6)
    xg = xt.clone().requires_grad_(True)
    qg = qt.clone().requires_grad_(True)
    U = energy(xg, qg, plan, rebuild=False)
    U.backward()
    side = float((xt.max(0).values - xt.min(0).values).max())
    h = 1e-6 * side
    for k, d in [(3, 0), (77, 1), (250, 2), (399, 0)]:
        xp, xm = xt.clone(), xt.clone()
        xp[k, d] += h
        xm[k, d] -= h
        plan.update_sources(xp, qt)
        Up = 0.5 * torch.dot(qt, plan.evaluate()[0]).item()
        plan.update_sources(xm, qt)
        Um = 0.5 * torch.dot(qt, plan.evaluate()[0]).item()
        fd = (Up - Um) / (2 * h)
        assert abs(fd - xg.grad[k, d].item()) <= 1e-6 * xg.grad.abs().max().item()
    for k in (0, 123):
        qp, qm = qt.clone(), qt.clone()
        qp[k] += 1e-6
        qm[k] -= 1e-6
        plan.update_sources(xt, qp)
        Up = 0.5 * torch.dot(qp, plan.evaluate()[0]).item()
        plan.update_sources(xt, qm)
        Um = 0.5 * torch.dot(qm, plan.evaluate()[0]).item()
        assert abs((Up - Um) / 2e-6 - qg.grad[k].item()) <= 1e-7 * qg.grad.abs().max().item()


@pytest.mark.parametrize("precision,dtype", [("fp64", torch.float64), ("fp32", torch.float32)])
def test_energy_gradient_vs_brute_force(precision, dtype):
    from paper_2512_09478_gb300 import Plan
    from paper_2512_09478_gb300.kifmm import energy
    x, q = G.uniform_charges(3000, 17)
    pd, gd = O.direct(x, q)
    plan = Plan(p=6, leaf_cap=32, precision=precision, n_max=len(x), dtype=dtype)
    xg = torch.tensor(x, dtype=dtype, device="cuda", requires_grad=True)
    qg = torch.tensor(q, dtype=dtype, device="cuda", requires_grad=True)
    U = energy(xg, qg, plan)
    U.backward()
    pot_f, grad_f, _ = O.kifmm(x, q, p=6, leaf_cap=32)
    err_p, err_g = O.rel_l2(pot_f, pd), O.rel_l2(grad_f, gd)
    assert U.item() == pytest.approx(O.energy(q, pd), rel=10 * err_p + 1e-6)
    assert O.rel_l2(qg.grad.double().cpu().numpy(), pd) <= 10 * err_p + 1e-6
    assert O.rel_l2(xg.grad.double().cpu().numpy(), q[:, None] * gd) <= 10 * err_g + 1e-6
