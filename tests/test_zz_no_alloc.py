"""kifmm_energy_noalloc: the energy reduction for callers that cannot allocate
device memory (graph capture, foreign memory pools, time-critical loops).

It must agree with the energy output of kifmm_evaluate (the same reduction
with plan workspace) on two consecutive calls, the second on a different
system, and reject sizes beyond its fixed scratch without launching work.
This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
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


def _energy_via_evaluate(x, q):
    from paper_2512_09478_gb300 import Plan
    plan = Plan(p=4, leaf_cap=32, precision="fp64", n_max=len(x), dtype=torch.float64)
    xt = torch.tensor(x, device="cuda")
    qt = torch.tensor(q, device="cuda")
    plan.set_sources(xt, qt)
    pot, _, energy = plan.evaluate(want_grad=False, want_energy=True)
    return qt, pot, energy


def test_noalloc_energy_matches_evaluate_twice():
    from paper_2512_09478_gb300.kifmm import energy_noalloc
    x1, q1 = G.uniform_charges(9000, 81)   # 3 chunks, ragged tail
    x2, q2 = G.uniform_charges(2500, 82)   # 1 chunk
    qa, pa, ea = _energy_via_evaluate(x1, q1)
    qb, pb, eb = _energy_via_evaluate(x2, q2)
    first = energy_noalloc(qa, pa).item()
    second = energy_noalloc(qb, pb).item()
    torch.cuda.synchronize()
    assert first == pytest.approx(ea.item(), rel=1e-12)
    assert second == pytest.approx(eb.item(), rel=1e-12)
    # the shared scratch holds the second call's partials; the first input gives the same answer again
    assert energy_noalloc(qa, pa).item() == first


def test_noalloc_fp32_matches_evaluate_within_rounding():
    """FP32 q and pot: the call sums the FP32 pot it is given, evaluate sums its
    FP64 internal potentials, so the two agree to FP32 rounding of pot (2^-24
    relative per term; the bound below is that times sum |q pot| / |sum q pot|)."""
    from paper_2512_09478_gb300 import Plan
    from paper_2512_09478_gb300.kifmm import energy_noalloc
    x, q = G.uniform_charges(9000, 83)
    plan = Plan(p=4, leaf_cap=32, precision="fp32", n_max=len(x), dtype=torch.float32)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    plan.set_sources(xt, qt)
    pot, _, energy = plan.evaluate(want_grad=False, want_energy=True)
    for _ in range(2):
        got = energy_noalloc(qt, pot).item()
        e = energy.item()
        terms = 0.5 * torch.sum(torch.abs(qt.double() * pot.double())).item()
        assert abs(got - e) <= 2.0 ** -23 * terms + 1e-12 * abs(e)


def test_noalloc_rejects_bad_dtype_on_the_host():
    from paper_2512_09478_gb300.kifmm import energy_noalloc
    q = torch.zeros(8, dtype=torch.float16, device="cuda")
    with pytest.raises(TypeError):
        energy_noalloc(q, q)


def test_noalloc_rejects_oversize_without_work():
    from paper_2512_09478_gb300.kifmm import load
    import ctypes
    lib = load()
    from paper_2512_09478_gb300.kifmm import energy_noalloc  # sets argtypes
    q = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    energy_noalloc(q, q, out)
    out.fill_(12345.0)  # sentinel: a refused call must leave it untouched
    torch.cuda.synchronize()
    code = lib.kifmm_energy_noalloc(16384 * 4096 + 1, 1, ctypes.c_void_p(q.data_ptr()),
                                    ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert code == 2  # KIFMM_ERR_CAPACITY
    assert out.item() == 12345.0
