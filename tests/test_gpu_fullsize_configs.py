"""Full-size parity of the benchmark's other configurations, in the launch
configuration it times (mixed precision, FP32 inputs, the autotuner on):
sampled outputs against the FP64 direct sum over the same FP32-rounded
inputs, which the oracle computes one target at a time.

* 200k rigid clumps x 4 charges (p = 6, leaf cap 128): potential and gradient
  at the charges of 256 sampled clumps, and those clumps' force and torque.
* 4M-body Plummer sphere, positive masses (p = 8, leaf cap 128, depth 12):
  512 sampled targets.
* 64 independent systems, 10k..200k particles each, 4.2M in all (p = 6,
  leaf cap 64): 8 targets in every system against that system's own sum.

Bars: 1e-5 on potentials, 2e-5 on gradients, forces and torques (the errors
measured by the benchmark on these configurations are 2e-6 to 5e-6).
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
    G.build()
    O.build()
    torch.cuda.set_device(0)


def _f32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def _plan_eval(x, q, p, M, D, offsets=None):
    from paper_2512_09478_gb300 import Plan
    ns = 1 if offsets is None else len(offsets) - 1
    plan = Plan(p=p, leaf_cap=M, max_depth=D, precision="mixed_fp16", n_max=len(x), n_systems_max=ns,
                dtype=torch.float32, autotune=True)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    plan.set_sources(xt, qt, sys_offsets=offsets)
    plan.evaluate()                      # the first evaluate tunes the tiles
    pot, grad, _ = plan.evaluate()
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return plan, xt, qt, pot, grad


def test_clumps_200k_x4():
    x, q, off, centres = G.clumps(200_000, 1002)
    x32, q32 = _f32(x), _f32(q)
    plan, xt, qt, pot, grad = _plan_eval(x32, q32, 6, 128, 20)
    F, T = plan.clump_reduce(torch.tensor(off, device="cuda"), xt, qt, grad,
                             torch.tensor(centres, dtype=torch.float32, device="cuda"))
    pot, grad = pot.double().cpu().numpy(), grad.double().cpu().numpy()
    F, T = F.double().cpu().numpy(), T.double().cpu().numpy()
    cl = np.sort(np.random.default_rng(7).choice(len(off) - 1, size=256, replace=False))
    idx = np.concatenate([np.arange(off[c], off[c + 1]) for c in cl])
    pd, gd = O.direct(x32, q32, x32[idx])
    assert O.rel_l2(pot[idx], pd) < 1e-5
    assert O.rel_l2(grad[idx], gd) < 2e-5
    sub_off = np.concatenate([[0], np.cumsum([off[c + 1] - off[c] for c in cl])])
    Fo, To = O.clump_reduce(x32[idx], q32[idx], gd, sub_off, _f32(centres)[cl])
    assert O.rel_l2(F[cl], Fo) < 2e-5
    assert O.rel_l2(T[cl], To) < 2e-5


def test_plummer_gravity_4m():
    x, q = G.plummer(4_000_000, 1003)
    x32, q32 = _f32(x), _f32(q)
    _, _, _, pot, grad = _plan_eval(x32, q32, 8, 128, 12)
    idx = np.sort(np.random.default_rng(8).choice(len(x), size=512, replace=False))
    pd, gd = O.direct(x32, q32, x32[idx])
    assert O.rel_l2(pot.double().cpu().numpy()[idx], pd) < 1e-5
    assert O.rel_l2(grad.double().cpu().numpy()[idx], gd) < 2e-5


def test_batched_64_systems():
    x, q, off = G.batched(64, 1004)
    x32, q32 = _f32(x), _f32(q)
    _, _, _, pot, grad = _plan_eval(x32, q32, 6, 64, 20, offsets=[int(v) for v in off])
    pot, grad = pot.double().cpu().numpy(), grad.double().cpu().numpy()
    rng = np.random.default_rng(9)
    got_p, got_g, ref_p, ref_g = [], [], [], []
    for s in range(64):
        a, b = int(off[s]), int(off[s + 1])
        t = np.sort(rng.choice(np.arange(a, b), size=8, replace=False))
        pd, gd = O.direct(x32[a:b], q32[a:b], x32[t])
        got_p.append(pot[t]); got_g.append(grad[t]); ref_p.append(pd); ref_g.append(gd)
    assert O.rel_l2(np.concatenate(got_p), np.concatenate(ref_p)) < 1e-5
    assert O.rel_l2(np.concatenate(got_g), np.concatenate(ref_g)) < 2e-5
