"""Sharding of independent scans across ranks (one process per GPU).

The scan's units are independent: separate sequences, and separate (sequence, automaton)
pairs of a batch. Ranks therefore split the units and exchange nothing on the data
path; the results are assembled once at the end. This module holds that host logic:
which rank takes which sequences, and how the per-rank count matrices and timings are
combined. It works with any torch.distributed backend (NCCL for CUDA tensors, gloo for
CPU tensors).
"""
from __future__ import annotations

import heapq


def shard_by_bytes(lens, world: int) -> list[list[int]]:
    """Assigns sequence indices to 'world' ranks, balancing bytes: the longest sequence
    goes to the least-loaded rank (ties by rank), repeatedly. Deterministic; every index
    appears in exactly one shard; each shard is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    shards: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(lens)), key=lambda j: (-int(lens[j]), j)):
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + int(lens[i]), r))
    return [sorted(s) for s in shards]


def gather_counts(local_idx, local_counts, n_seqs: int, n_dfas: int, device=None):
    """Assembles the full [n_seqs, n_dfas] int64 count matrix on every rank from each
    rank's rows (local_counts[k] is the row of sequence local_idx[k]): the rows are
    placed in a zero matrix and summed across ranks (one all-reduce)."""
    import torch
    import torch.distributed as dist
    full = torch.zeros((n_seqs, n_dfas), dtype=torch.int64, device=device)
    if len(local_idx):
        idx = torch.as_tensor(list(local_idx), dtype=torch.int64, device=full.device)
        full[idx] = torch.as_tensor(local_counts, dtype=torch.int64).to(full.device)
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(full, op=dist.ReduceOp.SUM)
    return full


def max_over_ranks(x: float, device=None) -> float:
    """The largest of each rank's value (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
