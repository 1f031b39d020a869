"""Adjoint (kifmm_backward) against the oracle, through the C ABI.

* dq = A^T w with A the oracle's own KIFMM operator, assembled column by
  column from unit charges (same tree, lists and operators): rel-L2 <= 1e-11.
* dx against central finite differences of the oracle's L = sum_i w_i pot_i
  with the tree frozen (h = 1e-6 of the box side).
* Energy gradients through the torch.autograd.Function against the
  brute-force gradients dU/dq_i = pot_i, dU/dx_i = q_i grad_i (exact sums),
  within the method's error at that p; FP32 vs FP64 adjoint.
* Losses on the gradient (forces): dq = G^T g against the oracle's assembled
  gradient operator (1e-11), dx against central differences of the oracle's
  loss with the tree frozen, both against the closed forms with exact sums
  (Hessian term and dipole field), and a force loss through autograd.
* The energy's backward is the library's: dU/dq = (pot + A^T q) / 2 against
  the oracle's assembled A, per system; calls out of order are refused.
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


# ---------------------------------------------------------------------------
# Losses on the gradient (forces) and on the energy, through kifmm_backward
# ---------------------------------------------------------------------------
def _kernel_terms(x, q, g):
    """Closed forms with the exact (direct) sums, K = 1/(4 pi r):
    L = sum_i g_i . grad_i  ->  dL/dq_j = sum_i g_i . grad_1 K(x_i, x_j),
    dL/dx_k = H_k g_k + q_k grad_k psi,  psi(y) = sum_i g_i . grad_1 K(x_i, y).
    O(n^2) numpy, pairs at zero distance excluded."""
    d = x[:, None, :] - x[None, :, :]                 # d[k, j] = x_k - x_j
    r2 = np.sum(d * d, axis=-1)
    np.fill_diagonal(r2, np.inf)
    ri = 1.0 / np.sqrt(r2)
    ri3, ri5 = ri ** 3, ri ** 5
    c = 1.0 / (4 * np.pi)
    # dq_j = sum_i g_i . (x_j - x_i) / r^3
    dq = c * np.einsum("jik,ik,ji->j", d, g, ri3)
    # Hessian term: H_k g_k = sum_j q_j (3 (d.g_k) d - r^2 g_k) / r^5
    dg = np.einsum("kjd,kd->kj", d, g)
    hg = c * (3 * np.einsum("kj,kj,kjd->kd", q[None, :] * ri5, dg, d) - np.einsum("kj,kd->kd", q[None, :] * ri3, g))
    # psi at x_k from dipoles g_i at x_i: g_i . (x_k - x_i) / r^3; its gradient
    gi_d = np.einsum("kid,id->ki", d, g)
    gpsi = c * (np.einsum("ki,id->kd", ri3, g) - 3 * np.einsum("ki,ki,kid->kd", ri5, gi_d, d))
    return dq, hg + q[:, None] * gpsi


@pytest.mark.parametrize("M,p", [(4, 4), (8, 6)])
def test_grad_loss_dq_is_oracle_transpose(M, p):
    """dL/dq for L = sum g . grad is G^T g, G the oracle's gradient operator
    assembled column by column (same tree, lists, operators), W lists present."""
    x, q, _ = _case()
    g = np.random.default_rng(11).normal(size=x.shape)
    tree = O.sort_and_tree(x, M, 20)
    lst = O.lists(tree)
    ops = O.operators(p)
    assert lst["W"][1].size > 0
    n = len(x)
    Gt_g = np.empty(n)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Gt_g[j] = np.sum(g * O.kifmm(x, e, p=p, tree=tree, lst=lst, ops=ops)[1])
    plan, xt, qt, pot, grad = _gpu(x, q, M, p)
    dq, dx = plan.backward(None, None, dL_dgrad=torch.tensor(g, device="cuda"))
    assert O.rel_l2(dq.cpu().numpy(), Gt_g) <= 1e-11


@pytest.mark.parametrize("with_w", [False, True])
def test_grad_loss_dx_matches_oracle_finite_differences(with_w):
    """dL/dx for L = sum g . grad (+ sum w pot) against central differences of
    the oracle's L with the tree frozen (h = 1e-6 of the box side)."""
    x, q, w = _case(140, 5)
    g = np.random.default_rng(12).normal(size=x.shape)
    if not with_w:
        w = np.zeros_like(w)
    M, p = 4, 4
    tree = O.sort_and_tree(x, M, 20)
    lst = O.lists(tree)
    ops = O.operators(p)
    plan, xt, qt, pot, grad = _gpu(x, q, M, p)
    wt = torch.tensor(w, device="cuda") if with_w else None
    dq, dx = plan.backward(wt, grad, dL_dgrad=torch.tensor(g, device="cuda"))
    dx = dx.cpu().numpy()
    h = 1e-6 * tree["side"]

    def L(xx):
        po, go, _ = O.kifmm(xx, q, p=p, tree=tree, lst=lst, ops=ops)
        return w @ po + np.sum(g * go)

    rng = np.random.default_rng(1)
    for k in rng.choice(len(x), 12, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, d] += h
            xm[k, d] -= h
            fd = (L(xp) - L(xm)) / (2 * h)
            assert abs(fd - dx[k, d]) <= 1e-6 * np.abs(dx).max(), (k, d, fd, dx[k, d])


@pytest.mark.parametrize("precision,dtype", [("fp64", torch.float64), ("fp32", torch.float32)])
def test_force_loss_gradient_vs_brute_force(precision, dtype):
    """L = sum g . grad on 2000 uniform charges: dq and dx against the closed
    forms with exact sums, within 10x the FMM's own error at p = 6 (+ the FP32
    floor in FP32)."""
    from paper_2512_09478_gb300 import Plan
    x, q = G.uniform_charges(2000, 21)
    g = np.random.default_rng(22).normal(size=x.shape)
    dq_e, dx_e = _kernel_terms(x, q, g)
    pot_f, grad_f, _ = O.kifmm(x, q, p=6, leaf_cap=32)
    pd, gd = O.direct(x, q)
    err = O.rel_l2(grad_f, gd)
    plan = Plan(p=6, leaf_cap=32, precision=precision, n_max=len(x), dtype=dtype)
    xt = torch.tensor(x, dtype=dtype, device="cuda")
    qt = torch.tensor(q, dtype=dtype, device="cuda")
    plan.set_sources(xt, qt)
    plan.evaluate()
    dq, dx = plan.backward(None, None, dL_dgrad=torch.tensor(g, dtype=dtype, device="cuda"))
    floor = 1e-6 if dtype == torch.float64 else 3e-5
    e_q = O.rel_l2(dq.double().cpu().numpy(), dq_e)
    e_x = O.rel_l2(dx.double().cpu().numpy(), dx_e)
    print("%s grad-loss adjoint vs exact: dq %.2e dx %.2e (forward grad error %.2e)" % (precision, e_q, e_x, err))
    assert e_q <= 10 * err + floor and e_x <= 30 * err + floor


def test_force_loss_through_autograd_fd_on_gpu():
    """A loss on the forces F = -q grad through field(): autograd adds the
    explicit q-dependence, the adjoint the rest; central differences of the
    GPU's own loss with the tree frozen (FP64)."""
    from paper_2512_09478_gb300.kifmm import field
    x, q, _ = _case(400, 7)
    c = torch.tensor(np.random.default_rng(8).normal(size=x.shape), device="cuda")
    plan, xt, qt, pot, grad = _gpu(x, q, 8, 6)

    def loss(xx, qq, rebuild):
        po, gr = field(xx, qq, plan, rebuild=rebuild)
        return torch.sum(c * (-qq[:, None] * gr)) + 0.1 * torch.sum(po * po)

    xg = xt.clone().requires_grad_(True)
    qg = qt.clone().requires_grad_(True)
    Lv = loss(xg, qg, False)
    Lv.backward()
    side = float((xt.max(0).values - xt.min(0).values).max())
    h = 1e-6 * side
    with torch.no_grad():
        for k, d in [(3, 0), (77, 1), (250, 2), (399, 0)]:
            xp, xm = xt.clone(), xt.clone()
            xp[k, d] += h
            xm[k, d] -= h
            fd = (loss(xp, qt, False).item() - loss(xm, qt, False).item()) / (2 * h)
            assert abs(fd - xg.grad[k, d].item()) <= 1e-6 * xg.grad.abs().max().item(), (k, d)
        for k in (0, 123):
            qp, qm = qt.clone(), qt.clone()
            qp[k] += 1e-6
            qm[k] -= 1e-6
            fd = (loss(xt, qp, False).item() - loss(xt, qm, False).item()) / 2e-6
            assert abs(fd - qg.grad[k].item()) <= 1e-6 * qg.grad.abs().max().item(), k


def test_energy_backward_is_library_terms():
    """KifmmEnergy: U_s from the library, dU/dq = (pot + A^T q) / 2 with A the
    oracle's assembled operator (1e-11), two systems with separate weights."""
    from paper_2512_09478_gb300 import Plan, KifmmEnergy
    x1, q1, _ = _case(120, 3)
    x2, q2, _ = _case(90, 4)
    X, Q = np.concatenate([x1, x2 + 40.0]), np.concatenate([q1, q2])
    off = [0, 120, 210]
    plan = Plan(p=4, leaf_cap=4, precision="fp64", n_max=210, n_systems_max=2, dtype=torch.float64)
    xg = torch.tensor(X, device="cuda", requires_grad=True)
    qg = torch.tensor(Q, device="cuda", requires_grad=True)
    plan.set_sources(xg.detach(), qg.detach(), sys_offsets=off)
    U = KifmmEnergy.apply(xg, qg, plan, False)
    (2.0 * U[0] + 3.0 * U[1]).backward()
    for s, (xs, qs, wgt) in enumerate(((x1, q1, 2.0), (x2, q2, 3.0))):
        tree = O.sort_and_tree(xs, 4, 20)
        lst = O.lists(tree)
        ops = O.operators(4)
        n = len(xs)
        A = np.empty((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            A[:, j] = O.kifmm(xs, e, p=4, tree=tree, lst=lst, ops=ops)[0]
        sl = slice(off[s], off[s + 1])
        assert U[s].item() == pytest.approx(0.5 * qs @ A @ qs, rel=1e-11)
        want = wgt * 0.5 * (A @ qs + A.T @ qs)
        assert O.rel_l2(qg.grad[sl].cpu().numpy(), want) <= 1e-11


def test_backward_state_errors():
    from paper_2512_09478_gb300 import KifmmError
    x, q, w = _case(100, 9)
    plan, xt, qt, pot, grad = _gpu(x, q, 8, 4)
    g = torch.ones(len(x), 3, dtype=torch.float64, device="cuda")
    plan.backward(None, None, dL_dgrad=g)
    plan.backward(None, None, dL_dgrad=g)   # the densities survive a backward
    with pytest.raises(KifmmError) as e:     # the energy term needs the evaluate's potentials
        plan.backward(None, grad, dL_denergy=torch.ones(1, dtype=torch.float64, device="cuda"))
    assert e.value.code == 6
    plan.update_sources(xt, qt)             # new sources, no evaluate yet
    with pytest.raises(KifmmError) as e:
        plan.backward(None, None, dL_dgrad=g)
    assert e.value.code == 6
    with pytest.raises(KifmmError) as e:
        plan.backward(None, None)
    assert e.value.code == 1


def test_stale_forward_is_refused_by_autograd():
    """Two forwards on one plan, then the first backward: refused (the plan no
    longer holds the first forward's sources)."""
    from paper_2512_09478_gb300.kifmm import potential
    x, q, _ = _case(100, 9)
    plan, xt, qt, pot, grad = _gpu(x, q, 8, 4)
    xa = xt.clone().requires_grad_(True)
    pa = potential(xa, qt, plan)
    potential(xt + 0.01, qt, plan)
    with pytest.raises(RuntimeError):
        pa.sum().backward()
