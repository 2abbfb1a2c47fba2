"""Multi-process rotation sweeps: one process per GPU, rotations sharded.

Rotations are independent, so each rank sweeps a contiguous block of them with
no exchange on the data path; the only collective is the final gather of the
per-rotation peaks (k floats and k ints), after which every rank holds the
full result and the best rotation (largest peak, lowest rotation index on
ties, as on one GPU).  Timing across ranks takes the maximum.
"""
from __future__ import annotations

import numpy as np


def shard_range(k: int, rank: int, world: int):
    """Contiguous, balanced block [start, stop) of k items for `rank` of `world`."""
    base, extra = divmod(k, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_peaks(peak_local, arg_local, k: int, group=None):
    """All ranks' (peak, argmax) blocks -> full arrays on every rank (gloo or NCCL)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    start, stop = shard_range(k, rank, world)
    assert len(peak_local) == stop - start
    width = -(-k // world)  # ceil: pad every block to the same length for all_gather
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    p = torch.full((width,), float("nan"), dtype=torch.float32, device=dev)
    a = torch.full((width,), -1, dtype=torch.int64, device=dev)
    p[: stop - start] = torch.as_tensor(np.asarray(peak_local, np.float32), device=dev)
    a[: stop - start] = torch.as_tensor(np.asarray(arg_local, np.int64), device=dev)
    ps = [torch.empty_like(p) for _ in range(world)]
    as_ = [torch.empty_like(a) for _ in range(world)]
    dist.all_gather(ps, p, group=group)
    dist.all_gather(as_, a, group=group)
    peak = np.empty(k, np.float32)
    arg = np.empty(k, np.int64)
    for r in range(world):
        s0, s1 = shard_range(k, r, world)
        peak[s0:s1] = ps[r][: s1 - s0].cpu().numpy()
        arg[s0:s1] = as_[r][: s1 - s0].cpu().numpy()
    return peak, arg


def best_rotation(peak):
    """Index of the largest peak, lowest index among equal peaks."""
    return int(np.argmax(np.asarray(peak)))


def max_over_ranks(value: float, group=None) -> float:
    import torch
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def distributed_sweep(sweeper, quats, group=None):
    """Sweep of all rotations across the ranks of `group`.

    `sweeper(quats_block) -> (peak, argmax)` runs the local block (on the GPU:
    `lambda q: [t.cpu().numpy() for t in ctx.sweep(A, B, q)]`).  Returns the full
    (peak, argmax) arrays and the best rotation index on every rank."""
    import torch.distributed as dist

    k = len(quats)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    s0, s1 = shard_range(k, rank, world)
    if s1 > s0:
        pl, al = sweeper(np.asarray(quats)[s0:s1])
    else:
        pl, al = np.empty(0, np.float32), np.empty(0, np.int64)
    peak, arg = gather_peaks(pl, al, k, group)
    return peak, arg, best_rotation(peak)
