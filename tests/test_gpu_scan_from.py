"""GPU parity for the scan of one piece of a longer sequence (dna_scan_from) against the
oracle's piece run: the count, the state after the piece and the positions, from every
kind of start state, for each table placement and the chunk-map path; and the join of
pieces across processes (one sequence split across ranks, Sec. III-A), with the
library's own piece summaries exchanged over gloo."""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_1509_01506_gb300 as dna
import synth
from paper_1509_01506_gb300 import shard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


def _perm_automaton(Q, seed):
    rng = np.random.default_rng(seed)
    table = np.stack([rng.permutation(Q) for _ in range(4)], axis=1).astype(np.uint32)
    acc = (rng.random(Q) < 0.3).astype(np.uint8)
    acc[int(rng.integers(0, Q))] = 1
    return table, acc


def _automaton(kind):
    """(library handle, oracle table, oracle accept) for each path of the scan."""
    if kind == "regex":
        t, a = oracle.compile_regex("ACG[AT]{2,6}C(G|T)T")
        return dna.Dfa.from_regex("ACG[AT]{2,6}C(G|T)T"), t, a
    if kind == "ac1000":
        kmers = synth.random_kmers(6, 1000, 12)
        t, a = oracle.compile_kmers(kmers, minimise=True)
        return dna.Dfa.from_kmers(kmers), t, a
    Q = int(kind[4:])
    table, acc = _perm_automaton(Q, 500 + Q)
    return dna.Dfa(table, dna.pack_accept(acc)), table.astype(np.int32), acc


def _seq(seed, n):
    s = synth.markov2(seed, n)
    if n > 1000:
        synth.overlay_runs(s, seed, 0.1, 300.0, "lower")
        synth.overlay_runs(s, seed + 1, 0.01, 200.0, "N")
    return s


def _to_device(seq, offset):
    buf = torch.empty(seq.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + seq.size]
    view.copy_(torch.from_numpy(seq))
    return view


@pytest.mark.parametrize("kind", ["regex", "ac1000", "perm8", "perm64", "perm150", "perm300"])
@pytest.mark.parametrize("n,offset", [(0, 0), (1, 3), (4097, 5), (100003, 1), (3 * MiB + 777, 7)])
def test_piece_from_any_start_state(kind, n, offset):
    dfa, t, a = _automaton(kind)
    Q = t.shape[0]
    seq = _seq(40 + n % 89, n)
    dseq = _to_device(seq, offset)
    rng = np.random.default_rng(n + Q)
    for start in sorted({0, Q - 1, int(rng.integers(0, Q)), int(rng.integers(0, Q))}):
        want_c, want_last, want_p = oracle.run_piece(t, a, start, seq)
        c, last, p = dna.scan_from(dfa, dseq, start, positions=True, capacity=want_c + 3)
        torch.cuda.synchronize()
        assert int(c.item()) == want_c, (kind, start)
        assert int(last.item()) == want_last, (kind, start)
        assert np.array_equal(p[:want_c].cpu().numpy(), want_p), (kind, start)
        c2, last2, _ = dna.scan_from(dfa, dseq, start)
        torch.cuda.synchronize()
        assert int(c2.item()) == want_c and int(last2.item()) == want_last


@pytest.mark.parametrize("kind", ["regex", "ac1000", "perm8", "perm150", "perm300"])
def test_pieces_chained_through_the_library_equal_the_whole_run(kind):
    """Scanning the pieces in order, each from the last state the library reported for
    the one before, gives the whole sequence's count and positions."""
    dfa, t, a = _automaton(kind)
    seq = _seq(91, 2 * MiB + 333)
    want_c, want_p = oracle.run(t, a, seq)
    rng = np.random.default_rng(92)
    cuts = [0] + sorted(rng.integers(0, seq.size, size=6).tolist()) + [seq.size]
    q, total, pos = 0, 0, []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        c, last, p = dna.scan_from(dfa, _to_device(seq[lo:hi], lo % 16), q, positions=True,
                                   capacity=max(16, hi - lo))
        torch.cuda.synchronize()
        k = int(c.item())
        total += k
        pos.append(p[:k].cpu().numpy() + lo)
        q = int(last.item())
    assert total == want_c
    assert np.array_equal(np.concatenate(pos), want_p)
    assert q == oracle.run_from(t, a, 0, seq)[1]


def test_piece_start_state_is_checked():
    dfa = dna.Dfa.from_regex("ACGT")
    Q = dfa.info().n_states
    with pytest.raises(dna.DnaError):
        dna.scan_from(dfa, _to_device(synth.uniform(1, 100), 0), Q)


# -------------------------------------------------- the join across processes (gloo)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _join_seq():
    return _seq(123, 8 * MiB + 4099)


def _gpu_join_worker(rank, world, port, out_path, kind, use_prefix):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seq = _join_seq()
        dfa, _, _ = _automaton(kind)
        cuts = [seq.size * r // world for r in range(world + 1)]
        lo, hi = cuts[rank], cuts[rank + 1]
        piece = _to_device(seq[lo:hi], rank)
        guess = 0
        if use_prefix and rank > 0:
            guess = shard.library_prefix_state(dfa, _to_device(seq[max(0, lo - 64):lo], 0))
        scan_piece = shard.library_piece_scanner(dfa, piece, positions=True, capacity=hi - lo)
        r = shard.scan_sharded(scan_piece, offset=lo, guess=guess)
        np.save(f"{out_path}.{rank}.npy", r["positions"].cpu().numpy())
        with open(f"{out_path}.{rank}.txt", "w") as f:
            f.write(f"{r['count']} {r['local_count']} {r['start']} {r['last']} {r['rounds']} {r['rescans']}\n")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,kind,use_prefix", [(2, "ac1000", True), (3, "regex", False), (2, "perm150", False)])
def test_processes_join_one_sequence_from_library_summaries(tmp_path, world, kind, use_prefix):
    """'world' processes on this GPU each scan one piece with dna_scan_from and exchange
    (start, last state, count) over gloo until every start is its left neighbour's last
    state; the joined count, the pieces' positions and every piece's start and end state
    equal the oracle's run of the whole sequence. (The processes' kernels never wait on
    one another: the exchange is on the host.)"""
    import torch.multiprocessing as mp
    out = str(tmp_path / "join")
    mp.start_processes(_gpu_join_worker, args=(world, _free_port(), out, kind, use_prefix), nprocs=world,
                       join=True, start_method="spawn")
    seq = _join_seq()
    _, t, a = _automaton(kind)
    want_c, want_p = oracle.run(t, a, seq)
    rows = [open(f"{out}.{r}.txt").read().split() for r in range(world)]
    assert all(int(x[0]) == want_c for x in rows)
    assert np.array_equal(np.concatenate([np.load(f"{out}.{r}.npy") for r in range(world)]), want_p)
    cuts = [seq.size * r // world for r in range(world + 1)]
    for r in range(world):
        assert int(rows[r][2]) == oracle.run_from(t, a, 0, seq[:cuts[r]])[1]
        assert int(rows[r][3]) == oracle.run_from(t, a, 0, seq[:cuts[r + 1]])[1]
    if use_prefix:
        assert all(int(x[4]) == 1 and int(x[5]) == 0 for x in rows)
    if kind.startswith("perm"):
        assert any(int(x[5]) > 0 for x in rows)
