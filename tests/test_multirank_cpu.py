"""The N > 1 path on CPU: two gloo ranks shard a batch of independent scans, each
computes its rows with the oracle, and the assembled count matrix equals the
single-process result; timings combine as the slowest rank's. No GPU involved."""
import os
import socket

import numpy as np
import pytest

from paper_1509_01506_gb300 import shard


def test_shard_by_bytes_is_a_balanced_partition():
    lens = [5, 100, 7, 60, 60, 1, 0, 33, 90, 12]
    for world in (1, 2, 3, 4):
        parts = shard.shard_by_bytes(lens, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(lens)))
        loads = [sum(lens[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(lens)
    assert shard.shard_by_bytes(lens, 2) == shard.shard_by_bytes(lens, 2)
    with pytest.raises(ValueError):
        shard.shard_by_bytes(lens, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    import synth
    lens = synth.log_uniform_lengths(31, 10, 200, 20000).tolist()
    seqs = [synth.markov2(310 + i, n) for i, n in enumerate(lens)]
    pats = synth.random_regexes(32, 3) + [synth.CONFIG2_REGEX]
    return seqs, pats


def _oracle_rows(seqs, pats, idx):
    import oracle
    tabs = [oracle.compile_regex(p) for p in pats]
    return [[oracle.run(t, a, seqs[i], positions=False)[0] for t, a in tabs] for i in idx]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seqs, pats = _batch()
        parts = shard.shard_by_bytes([s.size for s in seqs], world)
        mine = parts[rank]
        rows = _oracle_rows(seqs, pats, mine)
        full = shard.gather_counts(mine, rows, len(seqs), len(pats))
        slowest = shard.max_over_ranks(1.0 + rank)
        total = shard.sum_over_ranks(sum(seqs[i].size for i in mine))
        if rank == 0:
            np.save(out_path, full.numpy())
            with open(out_path + ".txt", "w") as f:
                f.write(f"{slowest} {total}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_assemble_the_single_process_result(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    seqs, pats = _batch()
    want = np.array(_oracle_rows(seqs, pats, range(len(seqs))), np.int64)
    assert np.array_equal(np.load(out), want)
    slowest, total = open(out + ".txt").read().split()
    assert float(slowest) == 2.0
    assert int(float(total)) == sum(s.size for s in seqs)


# ------------------------------------------- one sequence split across ranks (the join)


def test_join_step_chains_each_start_to_the_left_neighbours_last_state():
    starts, agreed = shard.join_step([(0, 3, 5), (3, 1, 2), (4, 2, 7)])
    assert starts == [0, 3, 1] and not agreed
    starts, agreed = shard.join_step([(0, 3, 5), (3, 1, 2), (1, 2, 7)])
    assert starts == [0, 3, 1] and agreed
    assert shard.join_step([(0, 9, 1)]) == ([0], True)


def _counter_table(m=5):
    """A non-converging automaton: the number of A's mod m (every symbol permutes the
    states, so no window fixes the start state and speculation from q0 is usually wrong)."""
    t = np.array([[(q + 1) % m, q, q, q] for q in range(m)], dtype=np.int32)
    a = np.zeros(m, dtype=np.uint8)
    a[0] = 1
    return t, a


def _split_case(kind):
    import oracle
    import synth
    seq = synth.markov2(77, 60_000)
    if kind == "kmer":
        t, a = oracle.compile_kmers(["ACGTA", "TTGCA", "GATTACA"])
    else:
        t, a = _counter_table()
    return seq, t, a


def _join_worker(rank, world, port, out_path, kind, use_prefix):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seq, t, a = _split_case(kind)
        cuts = [seq.size * r // world for r in range(world + 1)]
        lo, hi = cuts[rank], cuts[rank + 1]
        piece = seq[lo:hi]

        def scan_piece(q):
            c, last, pos = oracle.run_piece(t, a, q, piece)
            return c, last, pos

        guess = 0
        if use_prefix and rank > 0:
            guess = oracle.run_piece(t, a, 0, seq[max(0, lo - 64):lo])[1]
        r = shard.scan_sharded(scan_piece, offset=lo, guess=guess)
        np.save(f"{out_path}.{rank}.npy", r["positions"])
        with open(f"{out_path}.{rank}.txt", "w") as f:
            f.write(f"{r['count']} {r['local_count']} {r['start']} {r['last']} {r['rounds']} {r['rescans']}\n")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,kind,use_prefix", [(2, "kmer", True), (3, "kmer", False), (3, "counter", False),
                                                   (2, "counter", True)])
def test_gloo_ranks_join_one_sequence_split_across_them(tmp_path, world, kind, use_prefix):
    """Each rank scans its piece from a speculated start; the exchanged summaries repair
    every wrong start, and the joined result equals the whole sequence's run."""
    import oracle
    import torch.multiprocessing as mp
    out = str(tmp_path / "join")
    mp.start_processes(_join_worker, args=(world, _free_port(), out, kind, use_prefix), nprocs=world,
                       join=True, start_method="spawn")
    seq, t, a = _split_case(kind)
    want_c, want_pos = oracle.run(t, a, seq)
    pos = np.concatenate([np.load(f"{out}.{r}.npy") for r in range(world)])
    rows = [open(f"{out}.{r}.txt").read().split() for r in range(world)]
    assert all(int(x[0]) == want_c for x in rows)
    assert sum(int(x[1]) for x in rows) == want_c
    assert np.array_equal(pos, want_pos)
    cuts = [seq.size * r // world for r in range(world + 1)]
    for r in range(world):
        true_start = oracle.run_from(t, a, 0, seq[:cuts[r]])[1]
        assert int(rows[r][2]) == true_start
        assert int(rows[r][3]) == oracle.run_from(t, a, 0, seq[:cuts[r + 1]])[1]
    rounds = {int(x[4]) for x in rows}
    assert len(rounds) == 1 and rounds.pop() <= world
    if kind == "kmer" and use_prefix:
        # a 64-byte prefix exceeds the definite depth: the speculation is exact
        assert all(int(x[4]) == 1 and int(x[5]) == 0 for x in rows)
    if kind == "counter":
        assert any(int(x[5]) > 0 for x in rows)   # some start was wrong and repaired


def _tiny_join_worker(rank, world, port, out_path, n):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, a = _counter_table(3)
        seq = np.frombuffer(b"AACANAAGTAA"[:n], dtype=np.uint8)
        cuts = [n * r // world for r in range(world + 1)]
        lo, hi = cuts[rank], cuts[rank + 1]

        def scan_piece(q):
            return oracle.run_piece(t, a, q, seq[lo:hi])

        r = shard.scan_sharded(scan_piece, offset=lo, guess=(rank * 2) % 3)
        with open(f"{out_path}.{rank}.txt", "w") as f:
            f.write(f"{r['count']} {r['start']} {r['last']} {' '.join(str(x) for x in r['positions'])}\n")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(4, 3), (4, 5), (3, 0)])
def test_gloo_join_with_empty_pieces(tmp_path, world, n):
    """Pieces may be empty (more ranks than bytes, or an empty sequence): an empty piece
    ends where it starts, and the join still gives the whole run's count, positions and
    every piece's true start."""
    import oracle
    import torch.multiprocessing as mp
    out = str(tmp_path / "tiny")
    mp.start_processes(_tiny_join_worker, args=(world, _free_port(), out, n), nprocs=world, join=True,
                       start_method="spawn")
    t, a = _counter_table(3)
    seq = np.frombuffer(b"AACANAAGTAA"[:n], dtype=np.uint8)
    want_c, want_p = oracle.run(t, a, seq)
    rows = [open(f"{out}.{r}.txt").read().split() for r in range(world)]
    assert all(int(x[0]) == want_c for x in rows)
    assert [int(v) for x in rows for v in x[3:]] == list(want_p)
    cuts = [n * r // world for r in range(world + 1)]
    for r in range(world):
        assert int(rows[r][1]) == oracle.run_from(t, a, 0, seq[:cuts[r]])[1]
        assert int(rows[r][2]) == oracle.run_from(t, a, 0, seq[:cuts[r + 1]])[1]


def _flaky_worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    calls = [0]

    def scan_piece(q):
        # a scanner whose last state changes on every call
        calls[0] += 1
        return 0, calls[0] * 7 + rank, None

    try:
        r = shard.scan_sharded(scan_piece, guess=1)
        try:
            shard.scan_sharded(lambda q: (0, 5, None), guess=1, max_rounds=1)
            msg = "no error"
        except RuntimeError as e:
            msg = str(e)
        with open(f"{out_path}.{rank}.txt", "w") as f:
            f.write(f"{r['rounds']}|{msg}")
    finally:
        dist.destroy_process_group()


def test_join_rounds_are_bounded_and_a_round_limit_raises(tmp_path):
    """Piece 0's start is fixed and a piece stops rescanning once its start is its left
    neighbour's last state, so the starts settle within 'world' rounds whatever the
    scanner returns; a round limit below what the starts need raises on every rank."""
    import torch.multiprocessing as mp
    out = str(tmp_path / "flaky")
    mp.start_processes(_flaky_worker, args=(3, _free_port(), out), nprocs=3, join=True, start_method="spawn")
    rows = [open(f"{out}.{r}.txt").read().split("|") for r in range(3)]
    assert all(int(x[0]) <= 3 for x in rows), rows
    assert all("disagree after 1 rounds" in x[1] for x in rows), rows
