"""GPU parity of per-pattern results from one automaton (dna_scan_labels): the paper
scans the nine regex-dna expressions of Table V with one DFA and keeps a counter per
accepting state (Alg. 1). Per-label counts, positions and each position's label mask
must equal the oracle's labelled run, bit for bit."""
import numpy as np
import pytest

import oracle
import paper_1509_01506_gb300 as dna
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


def noisy_markov(seed, n, n_frac=0.01, lower_frac=0.1):
    s = synth.markov2(seed, n)
    synth.overlay_runs(s, seed, lower_frac, 300.0, "lower")
    synth.overlay_runs(s, seed + 1, n_frac, 200.0, "N")
    return s


def to_device(seq, offset=0):
    buf = torch.empty(seq.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + seq.size]
    view.copy_(torch.from_numpy(seq))
    return view


def planted(seed, n, words):
    """Markov sequence with the given words planted at random places (so that every
    expression of the set has matches)."""
    s = noisy_markov(seed, n)
    rng = np.random.default_rng(seed)
    for k in range(max(1, n // 4096)):
        w = words[k % len(words)].encode()
        if n > len(w):
            at = int(rng.integers(0, n - len(w)))
            s[at:at + len(w)] = np.frombuffer(w, dtype=np.uint8)
    return s


TABLE_V_WORDS = ["AGGGTAAA", "TTTACCCT", "CGGGTAAA", "TTTACCCA", "ACGGTAAA", "TTTACCAT", "AGAGTAAA",
                 "TTTACTCT", "AGGATAAA", "TTTAGCCT", "AGGGCAAA", "TTTCCCCT", "AGGGTCAA", "TTGACCCT",
                 "AGGGTACA", "TCTACCCT", "AGGGTAAC", "GTTACCCT"]


def check(dfa, t, lab, n_labels, seq, offset=0, capacity=None):
    want_c, want_per, want_p, want_m = oracle.run_labels(t, lab, n_labels, seq)
    d = to_device(seq, offset)
    cap = want_c + 3 if capacity is None else capacity
    c, per, p, m = dna.scan_labels(dfa, d, positions=True, capacity=cap)
    torch.cuda.synchronize()
    assert int(c.item()) == want_c
    assert per.cpu().numpy().tolist() == want_per.tolist()
    k = min(want_c, cap)
    assert np.array_equal(p[:k].cpu().numpy(), want_p[:k])
    assert np.array_equal(m[:k].cpu().numpy().astype(np.uint32), want_m[:k])
    c2, per2, _, _ = dna.scan_labels(dfa, d)
    torch.cuda.synchronize()
    assert int(c2.item()) == want_c and per2.cpu().numpy().tolist() == want_per.tolist()
    return want_c


def test_table_v_as_one_automaton_at_64MiB():
    """The nine Table V expressions as one labelled automaton on a 64 MiB noisy Markov
    sequence with planted words: per-expression counts, positions and masks equal the
    oracle's; the plain dna_scan count of the same handle is the labelled total."""
    pats = synth.REGEX_DNA_TABLE_V
    t, lab = oracle.compile_regex_set(pats)
    dfa = dna.Dfa.from_regex_set(pats)
    assert dfa.info().n_labels == 9 and dfa.info().n_states == t.shape[0]
    seq = planted(81, 64 * MiB, TABLE_V_WORDS)
    total = check(dfa, t, lab, 9, seq, offset=3)
    c, _ = dna.scan(dfa, to_device(seq))
    torch.cuda.synchronize()
    assert int(c.item()) == total


@pytest.mark.parametrize("n,offset", [(1, 0), (17, 1), (4095, 3), (100003, 7), (3 * MiB + 777, 1)])
@pytest.mark.parametrize("which", ["table_v", "small_set"])
def test_lengths_offsets_and_table_placements(which, n, offset):
    """Ragged lengths and unaligned starts; Table V (147 states, one-symbol table) and a
    small set whose automaton takes the two-symbol table."""
    pats = synth.REGEX_DNA_TABLE_V if which == "table_v" else ["TATAAA", "ACG[AT]{2,6}C(G|T)T", "A(C|G)*T"]
    t, lab = oracle.compile_regex_set(pats)
    dfa = dna.Dfa.from_regex_set(pats)
    seq = planted(82 + n % 13, n, TABLE_V_WORDS + ["TATAAA", "ACGATCGT", "ACGT"])
    check(dfa, t, lab, len(pats), seq, offset=offset)


def test_capacity_below_the_count_keeps_label_counts_exact():
    pats = ["A", "AA", "TATAAA"]
    t, lab = oracle.compile_regex_set(pats)
    dfa = dna.Dfa.from_regex_set(pats)
    seq = noisy_markov(83, 2 * MiB + 5)
    check(dfa, t, lab, 3, seq, capacity=1000)


def test_labelled_chunk_map_automaton():
    """Labels on an automaton whose runs never meet (chunk maps, then the positions pass
    from the exact sub-chunk starts)."""
    rng = np.random.default_rng(84)
    Q = 12
    table = np.stack([rng.permutation(Q) for _ in range(4)], axis=1).astype(np.uint32)
    lab = (rng.integers(0, 8, Q) * (rng.random(Q) < 0.4)).astype(np.uint32)
    lab[3] = 5
    dfa = dna.Dfa(table, labels=lab, n_labels=3)
    assert dfa.info().chunk_maps and dfa.info().n_labels == 3
    seq = noisy_markov(85, 5 * MiB + 11)
    check(dfa, table.astype(np.int32), lab, 3, seq, offset=2)


def test_empty_sequence_and_unlabelled_handle():
    dfa = dna.Dfa.from_regex_set(["TATAAA", "AC"])
    c, per, _, _ = dna.scan_labels(dfa, torch.empty(0, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    assert int(c.item()) == 0 and per.cpu().tolist() == [0, 0]
    plain = dna.Dfa.from_regex("TATAAA")
    with pytest.raises(dna.DnaError):
        dna.scan_labels(plain, torch.zeros(16, dtype=torch.uint8, device="cuda"))
