"""GPU parity of the batched path (dna_batch_* / dna_scan_batch) against the CPU oracle:
every (sequence, automaton) count bit-exact, for batches that mix lengths (empty, shorter
than one 16-byte word, ragged tails), unaligned starts, reset bytes and soft-masked
runs, automata that take the persistent kernel and automata that fall back to the
single-sequence path; independent of the plan (chunk length, warps, graph replay)."""
import numpy as np
import pytest

import oracle
import paper_1509_01506_gb300 as dna
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20


def mixed_sequences(seed, n, lo=1 * KiB, hi=300 * KiB):
    lens = synth.log_uniform_lengths(seed, n, lo, hi).tolist()
    lens[:6] = [0, 1, 15, 16, 511, 513]
    seqs = []
    for i, n_i in enumerate(lens):
        s = synth.markov2(seed * 1000 + i, n_i) if n_i else np.zeros(0, np.uint8)
        if n_i > 2000:
            synth.overlay_runs(s, seed * 1000 + i, 0.05, 300.0, "lower")
            synth.overlay_runs(s, seed * 1000 + i + 1, 0.01, 150.0, "N")
        seqs.append(s)
    return seqs


def to_device_list(seqs, unaligned_every=3):
    """One allocation per sequence; every third starts 1..15 bytes past 16-byte alignment."""
    out, keep = [], []
    for i, s in enumerate(seqs):
        off = (i % 15) + 1 if i % unaligned_every == 1 else 0
        buf = torch.empty(s.size + off + 16, dtype=torch.uint8, device="cuda")
        v = buf[off:off + s.size]
        if s.size:
            v.copy_(torch.from_numpy(s))
        out.append(v)
        keep.append(buf)
    return out, keep


def automata():
    """(kind, pattern) list: motif regexes and k-mer sets for the persistent kernel, one
    non-definite regex and one large Aho-Corasick set for the fallback path."""
    pats = [("regex", p) for p in synth.random_regexes(11, 5)]
    pats += [("regex", synth.CONFIG2_REGEX), ("regex", "TATAAA"),
             ("kmers", synth.random_kmers(12, 6, 6, 8)),       # <= 49 states
             ("regex", "A(CG)*T"),                             # not definite: fallback
             ("kmers", synth.random_kmers(13, 300, 12))]       # ~3k states: fallback
    return pats


def oracle_counts(pats, seqs):
    want = np.zeros((len(seqs), len(pats)), np.int64)
    for k, (kind, pat) in enumerate(pats):
        t, a = oracle.compile_regex(pat) if kind == "regex" else oracle.compile_kmers(pat, minimise=True)
        for s, seq in enumerate(seqs):
            want[s, k] = oracle.run(t, a, seq, positions=False)[0]
    return want


def lib_dfas(pats):
    return [dna.Dfa.from_regex(p) if kind == "regex" else dna.Dfa.from_kmers(p) for kind, p in pats]


@pytest.fixture(scope="module")
def mixed():
    pats = automata()
    seqs = mixed_sequences(5, 48)
    dseqs, keep = to_device_list(seqs)
    return pats, seqs, dseqs, keep, oracle_counts(pats, seqs), lib_dfas(pats)


def test_batch_default_plan_matches_oracle(mixed):
    pats, seqs, dseqs, _, want, dfas = mixed
    b = dna.Batch(dfas, dseqs)
    info = b.info()
    assert info.n_fast == 8 and info.n_slow == 2
    got = b.run()
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    b.free()


@pytest.mark.parametrize("chunk,warps", [(512, 8), (2048, 16), (4096, 24), (16384, 16), (131072, 8)])
def test_batch_results_do_not_depend_on_the_plan(mixed, chunk, warps):
    pats, seqs, dseqs, _, want, dfas = mixed
    b = dna.Batch(dfas, dseqs, chunk_bases=chunk, warps_per_cta=warps)
    assert b.info().chunk_bases == chunk and b.info().warps_per_cta == warps
    got = b.run()
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)


def test_batch_one_shot_entry_point(mixed):
    pats, seqs, dseqs, _, want, dfas = mixed
    got = dna.scan_batch(dfas, dseqs)
    assert np.array_equal(got.cpu().numpy(), want)


def test_batch_graph_replay_sees_new_contents_and_autotune(mixed):
    """A graph-captured plan re-reads (re-ingests) the sequences on every run: changing
    a sequence's bytes between runs changes its counts to the oracle's for the new bytes."""
    pats, seqs, dseqs, keep, want, dfas = mixed
    b = dna.Batch(dfas, dseqs, use_graph=True, autotune=True)
    out = torch.empty((len(seqs), len(pats)), dtype=torch.int64, device="cuda")
    b.run(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    i = max(range(len(seqs)), key=lambda j: seqs[j].size)
    new = synth.uniform(77, seqs[i].size)
    dseqs[i].copy_(torch.from_numpy(new))
    b.run(out)
    torch.cuda.synchronize()
    want2 = want.copy()
    want2[i] = oracle_counts(pats, [new])[0]
    assert np.array_equal(out.cpu().numpy(), want2)
    dseqs[i].copy_(torch.from_numpy(seqs[i]))
    torch.cuda.synchronize()


def test_batch_invalid_arguments():
    dfa = dna.Dfa.from_regex("ACGT")
    s = torch.zeros(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(dna.DnaError):
        dna.Batch([dfa], [s], chunk_bases=1000)
    with pytest.raises(dna.DnaError):
        dna.Batch([dfa], [s], warps_per_cta=12)
    with pytest.raises(dna.DnaError):
        dna.Batch([], [s])
    with pytest.raises(dna.DnaError):
        dna.Batch([dfa], [0], lens=[10])


def test_batch_full_size_sampled():
    """The batched workload at full size (4,096 sequences, lengths log-uniform 1 KiB to
    16 MiB, i.i.d. A/C/G/T, 64 motif regexes) with autotuning: a sample of pairs against
    the oracle and every pair's total against one dna_scan per pair for 8 sequences."""
    buf, offs, regexes = synth.batched()
    n_s = offs.size - 1
    dbuf = torch.empty(int(offs[-1]) + 256 * n_s, dtype=torch.uint8, device="cuda")
    starts, lens = [], []
    pos = 0
    hbuf = torch.from_numpy(buf)
    for s in range(n_s):
        n = int(offs[s + 1] - offs[s])
        dbuf[pos:pos + n].copy_(hbuf[int(offs[s]):int(offs[s + 1])], non_blocking=True)
        starts.append(dbuf.data_ptr() + pos)
        lens.append(n)
        pos += (n + 255) // 256 * 256
    torch.cuda.synchronize()
    dfas = [dna.Dfa.from_regex(r) for r in regexes]
    b = dna.Batch(dfas, starts, lens=lens, autotune=True)
    got = b.run()
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    rng = np.random.default_rng(9)
    small = [s for s in range(n_s) if lens[s] < 256 * KiB]
    for s, k in zip(rng.choice(small, 48), rng.integers(0, len(regexes), 48)):
        t, a = oracle.compile_regex(regexes[k])
        seq = buf[int(offs[s]):int(offs[s + 1])]
        assert got[s, k] == oracle.run(t, a, seq, positions=False)[0], (s, k)
    big = sorted(range(n_s), key=lambda s: -lens[s])[:2]
    for s in big:
        k = int(rng.integers(0, len(regexes)))
        t, a = oracle.compile_regex(regexes[k])
        seq = buf[int(offs[s]):int(offs[s + 1])]
        assert got[s, k] == oracle.run(t, a, seq, positions=False)[0], (s, k)
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    for s in rng.choice(n_s, 8, replace=False):
        for k in range(len(regexes)):
            dna.scan_ptr(dfas[k], starts[s], lens[s], out.data_ptr(), int(torch.cuda.current_stream().cuda_stream))
            torch.cuda.synchronize()
            assert int(out.item()) == got[s, k]


def test_fasta_records_scanned_as_a_batch():
    """FASTA ingest: records parsed on the host, copied once, scanned as one batch (a
    pointer per record); each record's counts equal the oracle's on that record alone."""
    rng = np.random.default_rng(12)
    parts, recs = [], []
    for r in range(5):
        s = synth.markov2(500 + r, int(rng.integers(10_000, 300_000)))
        recs.append(s)
        lines = [bytes(s[i:i + 60]) for i in range(0, s.size, 60)]
        parts.append(b">rec%d sample\n" % r + b"\n".join(lines) + b"\n")
    seq, off, hdr = dna.fasta_parse(b"".join(parts))
    assert hdr == ["rec%d sample" % r for r in range(5)]
    d = torch.from_numpy(seq).cuda()
    ptrs = [d.data_ptr() + int(off[r]) for r in range(5)]
    lens = [int(off[r + 1] - off[r]) for r in range(5)]
    pats = [("regex", synth.CONFIG2_REGEX), ("regex", "TATAAA")]
    got = dna.Batch(lib_dfas(pats), ptrs, lens=lens).run()
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle_counts(pats, recs))


def test_regex_dna_per_expression_counts():
    """The paper's regex-dna output: one count per expression of Table V (E1..E9, each a
    pattern | its reverse complement) for each input, from one batch of 9 automata."""
    seqs = [synth.markov2(600 + i, n) for i, n in enumerate((1_000_003, 250_000, 4096))]
    for s in seqs:
        synth.overlay_runs(s, 7, 0.05, 400.0, "lower")
    dseqs, keep = to_device_list(seqs)
    pats = [("regex", e) for e in synth.REGEX_DNA_TABLE_V]
    got = dna.Batch(lib_dfas(pats), dseqs).run()
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle_counts(pats, seqs))


def test_batch_with_a_chunk_map_automaton(mixed):
    """A never-converging automaton in a batch goes to the single-sequence path, which
    uses chunk maps; its column equals the oracle's."""
    pats, seqs, dseqs, _, want, dfas = mixed
    rng = np.random.default_rng(92)
    table = np.stack([rng.permutation(9) for _ in range(4)], axis=1).astype(np.uint32)
    acc = (np.arange(9) % 4 == 1).astype(np.uint8)
    perm = dna.Dfa(table, dna.pack_accept(acc))
    assert perm.info().chunk_maps
    b = dna.Batch(dfas + [perm], dseqs)
    assert b.info().n_slow == 3
    got = b.run()
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    b.free()
    assert np.array_equal(got[:, :-1], want)
    col = [oracle.run(table.astype(np.int32), acc, s, positions=False)[0] for s in seqs]
    assert got[:, -1].tolist() == col
