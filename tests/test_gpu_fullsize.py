"""Full-size parity: the 1M-sphere DEM Coulomb packing (p = 6, leaf cap 128,
mixed precision with the autotuner on), i.e. the workload and launch
configuration the benchmark times.  The oracle cannot run the KIFMM at this
size in a test, so the check is on sampled outputs it computes one by one
(the FP64 direct sum over the FP32 inputs at 512 seeded targets) and on a
property that holds at any size (Newton's third law for the full set).

Budget (the method's error at p = 6, not the precision's, dominates the
gradient on this packing): potential rel-L2 < 1e-5; gradient within 1.1x
the error of the GPU FP64 path on the same targets, plus 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from workloads import generators as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_09478_gb300 import build as B
    B.build()
    G.build()
    O.build()
    torch.cuda.set_device(0)
    x, q, _ = G.dem_coulomb(1_000_000, 1001)
    return x, q


def _evaluate(x, q, precision, dtype, autotune):
    from paper_2512_09478_gb300 import Plan
    plan = Plan(p=6, leaf_cap=128, max_depth=20, precision=precision, n_max=len(x), dtype=dtype,
                autotune=autotune)
    xt = torch.tensor(x, dtype=dtype, device="cuda")
    qt = torch.tensor(q, dtype=dtype, device="cuda")
    plan.set_sources(xt, qt)
    plan.evaluate()                      # the first evaluate tunes the tiles
    pot, grad, _ = plan.evaluate()
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return pot.double().cpu().numpy(), grad.double().cpu().numpy()


def test_dem_1m_mixed_sampled_vs_direct_sum(dem):
    x, q = dem
    # the device receives FP32 data: the reference sums over the same rounded values
    x32 = x.astype(np.float32).astype(np.float64)
    q32 = q.astype(np.float32).astype(np.float64)
    pot_m, grad_m = _evaluate(x, q, "mixed_fp16", torch.float32, True)
    pot_d, grad_d = _evaluate(x32, q32, "fp64", torch.float64, False)
    idx = np.sort(np.random.default_rng(2024).choice(len(x), size=512, replace=False))
    pd, gd = O.direct(x32, q32, x32[idx])
    e_pot_m, e_grad_m = O.rel_l2(pot_m[idx], pd), O.rel_l2(grad_m[idx], gd)
    e_pot_d, e_grad_d = O.rel_l2(pot_d[idx], pd), O.rel_l2(grad_d[idx], gd)
    assert e_pot_m < 1e-5, (e_pot_m, e_pot_d)
    assert e_grad_m <= 1.1 * e_grad_d + 1e-6, (e_grad_m, e_grad_d)
    # FP64 GPU path: the method's own error at p = 6 on this packing
    assert e_pot_d < 1e-5 and e_grad_d < 1e-4, (e_pot_d, e_grad_d)
    # Newton's third law over all 1M particles (pairwise forces cancel up to
    # the FMM error): |sum q grad| small against sum |q grad|
    f = q32[:, None] * grad_m
    resid = np.linalg.norm(f.sum(axis=0)) / np.linalg.norm(f, axis=1).sum()
    assert resid < 1e-5, resid
