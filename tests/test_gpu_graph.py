"""Batched independent systems evaluated as one CUDA-graph replay.

The tree of every system is built once (set_sources); update_sources +
evaluate are then captured in one torch.cuda.CUDAGraph, and each replay
re-reads the particles from the same device buffers.  The test moves the
particles in place between replays (the tree stays frozen, as in a DEM loop
that reuses the tree) and checks every system against the oracle run on the
moved particles with that system's frozen tree:

* FP64, 8 systems of 2k..20k particles (uniform and Plummer, as in the
  batched workload): rel-L2 <= 1e-12 per system.
* The benchmark's batched workload itself (64 systems of 10k..200k, p = 6,
  leaf cap 64, FP32 data, 3xFP16 tensor-core M2L): against the oracle with
  the FP32 modes' pseudo-inverse truncation (the same method), within the
  plain FP32 path's own distance to it (the FP32 floor) times 1.5 plus 1e-7.

Two replays with different positions, and the kernel count of one replay
(what the graph launches) is recorded by the library's counter during capture.
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


def _capture(plan, xt, qt, pot, grad, energy):
    """Warm up on a side stream, then capture update_sources + evaluate."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            plan.update_sources(xt, qt)
            plan.evaluate(pot, grad, energy)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    plan.profile_read()   # resets the launch counter (stage timing stays off: no events in the graph)
    with torch.cuda.graph(graph):
        plan.update_sources(xt, qt)
        plan.evaluate(pot, grad, energy)
    launches = plan.profile_read()["launches"]
    return graph, launches


def _moves(off, n, scale, seed):
    """Small in-place displacements (a fraction of each system's extent)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, 3)) * scale


def _graph_run(X, Q, off, precision, dtype, p, M, moves):
    from paper_2512_09478_gb300 import Plan
    n, S = len(X), len(off) - 1
    plan = Plan(p=p, leaf_cap=M, max_depth=20, precision=precision, n_max=n, n_systems_max=S, dtype=dtype)
    xt = torch.tensor(X, dtype=dtype, device="cuda")
    qt = torch.tensor(Q, dtype=dtype, device="cuda")
    plan.set_sources(xt, qt, sys_offsets=off)
    pot = torch.empty(n, dtype=dtype, device="cuda")
    grad = torch.empty(n, 3, dtype=dtype, device="cuda")
    energy = torch.empty(S, dtype=torch.float64, device="cuda")
    graph, launches = _capture(plan, xt, qt, pot, grad, energy)
    outs = []
    for dx in moves:
        xt.copy_(torch.tensor(X + dx, dtype=dtype))   # same buffer, new positions
        graph.replay()
        torch.cuda.synchronize()
        assert plan.device_status() == 0
        outs.append((pot.double().cpu().numpy(), grad.double().cpu().numpy(), energy.cpu().numpy().copy()))
    return outs, launches


def test_graph_replay_fp64_matches_oracle_per_system():
    sizes = G.batch_sizes(8, 11, 2000, 20000)
    X, Q, off = G.batched(8, 11, 2000, 20000)
    assert np.array_equal(np.diff(off), sizes)
    ext = np.array([np.ptp(X[off[s]:off[s + 1]], axis=0).max() for s in range(8)])
    scale = np.repeat(1e-5 * ext, np.diff(off))[:, None]
    moves = [_moves(off, len(X), scale, 5), _moves(off, len(X), scale, 6)]
    outs, launches = _graph_run(X, Q, off, "fp64", torch.float64, 4, 32, moves)
    print("fp64 batched graph: %d kernels per replay" % launches)
    assert launches > 0
    for (pot, grad, energy), dx in zip(outs, moves):
        for s in range(8):
            sl = slice(off[s], off[s + 1])
            t = O.sort_and_tree(X[sl], 32, 20)       # the frozen tree
            lst = O.lists(t)
            xs = X[sl] + dx[sl]
            po, go, _ = O.kifmm(xs, Q[sl], p=4, leaf_cap=32, tree=t, lst=lst)
            assert O.rel_l2(pot[sl], po) <= 1e-12, s
            assert O.rel_l2(grad[sl], go) <= 1e-12, s
            # |U - U_o| <= 1/2 |q| |pot - pot_o| (Cauchy-Schwarz), with the pot bound above
            assert abs(energy[s] - O.energy(Q[sl], po)) <= 0.5 * np.linalg.norm(Q[sl]) * 1e-12 * np.linalg.norm(po)


def test_graph_replay_mixed_batched_workload():
    X, Q, off = G.batched(64, 1004)
    X32 = X.astype(np.float32).astype(np.float64)
    Q32 = Q.astype(np.float32).astype(np.float64)
    ext = np.array([np.ptp(X32[off[s]:off[s + 1]], axis=0).max() for s in range(64)])
    scale = np.repeat(1e-6 * ext, np.diff(off))[:, None]
    dx = _moves(off, len(X), scale, 9)
    Xm = (X32 + dx).astype(np.float32).astype(np.float64)   # what the device holds after the move
    outs = {}
    for prec in ("mixed_fp16", "fp32"):
        res, launches = _graph_run(X32, Q32, off, prec, torch.float32, 6, 64, [np.zeros_like(X32), Xm - X32])
        outs[prec] = res
        print("%s batched graph: %d kernels per replay, %d particles" % (prec, launches, len(X)))
    worst = {"mixed_fp16": [0.0, 0.0], "fp32": [0.0, 0.0]}
    rng = np.random.default_rng(3)
    for s in sorted(rng.choice(64, size=12, replace=False)):   # a dozen systems, both shapes
        sl = slice(off[s], off[s + 1])
        t = O.sort_and_tree(X32[sl], 64, 20)
        lst = O.lists(t)
        for r, xs in enumerate((X32[sl], Xm[sl])):
            po, go, _ = O.kifmm(xs, Q32[sl], p=6, leaf_cap=64, tree=t, lst=lst, eps=1e-9)
            for prec in outs:
                pot, grad, _ = outs[prec][r]
                worst[prec][0] = max(worst[prec][0], O.rel_l2(pot[sl], po))
                worst[prec][1] = max(worst[prec][1], O.rel_l2(grad[sl], go))
    print("worst system vs oracle: mixed pot %.2e grad %.2e | fp32 pot %.2e grad %.2e"
          % (*worst["mixed_fp16"], *worst["fp32"]))
    assert worst["mixed_fp16"][0] <= 1.5 * worst["fp32"][0] + 1e-7
    assert worst["mixed_fp16"][1] <= 1.5 * worst["fp32"][1] + 1e-7
    assert worst["fp32"][0] < 5e-6 and worst["fp32"][1] < 2e-5
