"""Sharding of scans across ranks (one process per GPU).

Independent units (separate sequences, and separate (sequence, automaton) pairs of a
batch) are split across ranks with nothing exchanged on the data path; the results are
assembled once at the end (shard_by_bytes, gather_counts).

One sequence split across ranks (Sec. III-A's input partitioning, one piece per rank)
has a real exchange step: the join of Sec. III-B.4, which needs each piece's true start
state, the end state of the piece before it. scan_sharded speculates each piece's start
(q0, or the state reached from q0 over the bytes just before the piece), scans, and
exchanges one (start, last state, count) summary per rank; a rank whose start differs
from its left neighbour's last state rescans from that state, and the exchange repeats
until every start agrees. After round k the first k + 1 pieces are exact, so at most
'world' rounds are taken; with a converging automaton and a prefix of at least its
definite depth, the first round is already exact.

It works with any torch.distributed backend (NCCL for CUDA tensors, gloo for CPU
tensors).
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


def _all_gather_i64(vals, group=None):
    """Each rank's list of int64 values, gathered on every rank: [world][len(vals)]."""
    import torch
    import torch.distributed as dist
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return [list(vals)]
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor(list(vals), dtype=torch.int64, device=dev)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return [[int(x) for x in o.tolist()] for o in out]


def join_step(summaries):
    """One step of the cross-rank join. 'summaries' is [world] of (start, last, count).
    Returns (starts each rank must scan from, whether every start already agrees):
    piece 0 keeps its start; piece r > 0 must start in the last state of piece r - 1."""
    starts = [summaries[0][0]] + [summaries[r - 1][1] for r in range(1, len(summaries))]
    agreed = all(summaries[r][0] == starts[r] for r in range(len(summaries)))
    return starts, agreed


def library_piece_scanner(dfa, piece, positions=False, capacity=None, stream=None):
    """The scan of one piece through the library (dna_scan_from): a function of the start
    state returning (count, last state, positions tensor or None, counted from the piece's
    first byte). The outputs are allocated once and reused by every rescan."""
    import torch
    from . import scan_from
    dev = piece.device
    count = torch.empty(1, dtype=torch.int64, device=dev)
    last = torch.empty(1, dtype=torch.int32, device=dev)
    pos = None
    if positions:
        cap = int(capacity if capacity is not None else max(1024, piece.numel() // 256))
        pos = torch.empty(cap, dtype=torch.int64, device=dev)

    def scan(start: int):
        scan_from(dfa, piece, start, positions=positions, stream=stream, out=(count, last, pos))
        if stream is not None:
            stream.synchronize()
        else:
            torch.cuda.current_stream(dev).synchronize()
        c = int(count.item())
        return c, int(last.item()), (pos[:min(c, pos.numel())] if positions else None)

    return scan


def library_prefix_state(dfa, prefix, stream=None) -> int:
    """The state reached from q0 over 'prefix' (a CUDA uint8 tensor), through the library."""
    from . import scan_from
    _, last, _ = scan_from(dfa, prefix, 0, stream=stream)
    return int(last.item())


def scan_sharded(scan_piece, offset: int = 0, guess: int = 0, group=None, max_rounds=None):
    """The scan of one sequence split across ranks: this rank holds the piece that starts
    at byte 'offset' and scans it with scan_piece(start) -> (count, last, positions);
    'guess' is its speculated start state (ignored on rank 0, which starts in q0).
    Returns a dict: count (the whole sequence's, on every rank), local_count, positions
    (this piece's, offset to sequence positions; None without positions), start and last
    (this piece's exact start and end states), rounds (exchanges taken), rescans (this
    rank's scans after its first)."""
    import torch.distributed as dist
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    start = 0 if rank == 0 else int(guess)
    count, last, pos = scan_piece(start)
    rounds, rescans = 0, 0
    limit = world if max_rounds is None else max_rounds
    while True:
        summaries = _all_gather_i64([start, last, count], group)
        rounds += 1
        starts, agreed = join_step(summaries)
        if agreed:
            break
        if rounds >= limit:
            raise RuntimeError(f"scan_sharded: starts still disagree after {rounds} rounds")
        if starts[rank] != start:
            start = starts[rank]
            count, last, pos = scan_piece(start)
            rescans += 1
    total = sum(s[2] for s in summaries)
    return {
        "count": total, "local_count": count,
        "positions": None if pos is None else pos + offset,
        "start": start, "last": last, "rounds": rounds, "rescans": rescans,
    }
