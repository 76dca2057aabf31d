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
