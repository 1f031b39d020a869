"""Leaf-relative particle records in FP32 (the FP32-based modes): offsets are
taken from the leaf centre in the caller's coordinates, so a domain far from
the origin loses no more than an ulp of the caller's coordinates.  The FP32
path's error against the FP64 oracle (the same FP32 inputs, the same method)
on a cloud shifted by 1000 box sides stays within twice its error on the
same cloud at the origin."""
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


@pytest.mark.parametrize("precision", ["fp32", "mixed_fp16"])
def test_far_from_origin_records(precision):
    from paper_2512_09478_gb300 import Plan
    x, q = G.uniform_charges(4000, 31)
    errs = []
    for shift in (0.0, 1000.0):
        x32 = (x + shift).astype(np.float32).astype(np.float64)
        q32 = q.astype(np.float32).astype(np.float64)
        po, go, _ = O.kifmm(x32, q32, p=6, leaf_cap=32, eps=1e-9)
        plan = Plan(p=6, leaf_cap=32, max_depth=20, precision=precision, n_max=len(x), dtype=torch.float32)
        plan.set_sources(torch.tensor(x32, dtype=torch.float32, device="cuda"),
                         torch.tensor(q32, dtype=torch.float32, device="cuda"))
        pot, grad, _ = plan.evaluate()
        assert plan.device_status() == 0
        errs.append((O.rel_l2(pot.double().cpu().numpy(), po), O.rel_l2(grad.double().cpu().numpy(), go)))
    print("%s records: origin pot %.2e grad %.2e | shifted pot %.2e grad %.2e" % (precision, *errs[0], *errs[1]))
    assert errs[1][0] <= 2 * errs[0][0] + 1e-7
    assert errs[1][1] <= 2 * errs[0][1] + 1e-7
