"""Sharding of independent systems over ranks (one GPU per rank).

A single system is never split: the KIFMM of one particle set runs on one
GPU.  A batch of independent systems (uneven sizes) is divided by whole
systems, largest first onto the least-loaded rank, so no collective is needed
on the data path; results meet on rank 0 only when the caller asks for them.
This is host logic (no device work) and runs the same under ``gloo``.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence

import numpy as np


def assign_largest_first(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Greedy longest-processing-time assignment: systems in decreasing size
    (ties by index) each go to the rank with the smallest load so far (ties
    by rank).  Returns, per rank, its system indices in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(v) for v in out]


def local_batch(x: np.ndarray, q: np.ndarray, offsets: Sequence[int], systems: Sequence[int]):
    """The rank's particles: its systems concatenated in the given order, with
    their own offsets (n_local_systems + 1)."""
    off = np.asarray(offsets, dtype=np.int64)
    if len(systems) == 0:
        return x[:0], q[:0], [0]
    xs = np.concatenate([x[off[s]:off[s + 1]] for s in systems])
    qs = np.concatenate([q[off[s]:off[s + 1]] for s in systems])
    loc = np.concatenate([[0], np.cumsum([off[s + 1] - off[s] for s in systems])]).astype(np.int64)
    return xs, qs, [int(v) for v in loc]


def scatter_back(parts, assignment, offsets, n_total: int, width: int = 1):
    """Reassemble per-rank outputs (each in its local system order) into the
    caller's global order.  ``parts[r]`` has shape [n_local_r] or
    [n_local_r, width]."""
    off = np.asarray(offsets, dtype=np.int64)
    shape = (n_total,) if width == 1 else (n_total, width)
    out = None
    for r, systems in enumerate(assignment):
        a = np.asarray(parts[r])
        if out is None:
            out = np.empty(shape, dtype=a.dtype)
        pos = 0
        for s in systems:
            m = int(off[s + 1] - off[s])
            out[off[s]:off[s + 1]] = a[pos:pos + m]
            pos += m
    return out


def gather_to_rank0(local: np.ndarray, assignment, offsets, n_total: int, group=None):
    """Collect every rank's output on rank 0 (global order there, None on the
    other ranks).  Uses torch.distributed object gather: off the hot path,
    works with gloo and nccl."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    parts = [None] * world if rank == 0 else None
    dist.gather_object(np.asarray(local), parts, dst=0, group=group)
    if rank != 0:
        return None
    width = 1 if np.asarray(local).ndim == 1 else np.asarray(local).shape[1]
    return scatter_back(parts, assignment, offsets, n_total, width)
