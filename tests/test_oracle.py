"""Pins for the CPU oracle (no GPU): each check ties the oracle to something other
than itself -- hand-worked examples, brute-force substring and regex enumeration,
closed forms and invariants of the method (Memeti & Pllana, Sec. II and III)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.tsv")
BASES = np.frombuffer(b"ACGT", dtype=np.uint8)


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        kind, pats, seq, exp, cite = line.rstrip("\n").split("\t")
        rows.append((kind, pats, seq, [] if exp == "-" else [int(x) for x in exp.split(",")], cite))
    return rows


def _compile(kind, pats, minimise=True):
    if kind == "regex":
        return oracle.compile_regex(pats, minimise=minimise)
    return oracle.compile_kmers(pats.split(","), minimise=minimise)


# --------------------------------------------------------------- brute force


def naive_kmer_positions(seq: bytes, patterns):
    """Brute force: j is reported iff some pattern equals seq[j-k+1..j] (case-folded)."""
    s = seq.upper()
    pats = [p.upper().encode() for p in patterns]
    out = []
    for j in range(len(s)):
        for p in pats:
            k = len(p)
            if j - k + 1 >= 0 and s[j - k + 1:j + 1] == p:
                out.append(j)
                break
    return out


def re_window_positions(seq: bytes, pattern: str):
    """Brute force with Python's re: j is reported iff some window seq[i..j] made only of
    bases fully matches the pattern ('.' means any base)."""
    rx = re.compile(pattern.replace(".", "[ACGT]"), re.IGNORECASE)
    s = seq.decode("latin-1")
    out = []
    for j in range(len(s)):
        i = j
        while i >= 0 and s[i] in "ACGTacgt":
            if rx.fullmatch(s, i, j + 1):
                out.append(j)
                break
            i -= 1
    return out


def random_seq(rng, n, p_reset=0.03, p_lower=0.2):
    s = BASES[rng.integers(0, 4, size=n)].copy()
    low = rng.random(n) < p_lower
    s[low] += 32
    s[rng.random(n) < p_reset] = ord("N")
    return s.tobytes()


# ------------------------------------------------------------------- pins


def test_symbol_mapping_all_bytes():
    """Exactly A/a, C/c, G/g, T/t are bases; every other byte resets (the reading of
    non-base bytes the oracle takes)."""
    want = {ord("A"): 0, ord("a"): 0, ord("C"): 1, ord("c"): 1,
            ord("G"): 2, ord("g"): 2, ord("T"): 3, ord("t"): 3}
    for b in range(256):
        assert oracle.symbol_of_byte(b) == want.get(b, 4)


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: f"{r[1]}:{r[2]}")
def test_hand_worked_examples(row):
    kind, pats, seq, expected, _ = row
    t, a = _compile(kind, pats)
    count, pos = oracle.run(t, a, seq.encode())
    assert list(pos) == expected and count == len(expected)
    t2, a2 = _compile(kind, pats, minimise=False)
    assert list(oracle.run(t2, a2, seq.encode())[1]) == expected


def test_fig2_failure_free_transitions():
    """Sec. III-B.1 / Fig. 2: in the failure-free AC DFA for {acg, cat, cta, tta},
    reading a, c, t after "ac" leads to three distinct states -- those of "ca", "c"
    and "ct" (the longest pattern prefix that is a suffix) -- and g completes acg."""
    t, a = oracle.compile_kmers(["acg", "cat", "cta", "tta"], minimise=False)
    assert t.shape[0] == 12   # root + a, ac, acg, c, ca, cat, ct, cta, t, tt, tta

    def walk(w, q=0):
        for ch in w:
            q = int(t[q, "ACGT".index(ch)])
        return q
    q_ac = walk("AC")
    nxt = {ch: walk(ch, q_ac) for ch in "ACT"}
    assert nxt["A"] == walk("CA") and nxt["C"] == walk("C") and nxt["T"] == walk("CT")
    assert len(set(nxt.values())) == 3
    assert a[walk("G", q_ac)] == 1 and a[q_ac] == 0


def test_literal_minimal_state_count_closed_form():
    """Closed form: the minimal DFA of Sigma*.w for a literal w of length k has k+1
    states (the prefixes of w are pairwise distinguishable)."""
    rng = np.random.default_rng(11)
    for k in range(1, 13):
        for _ in range(4):
            w = "".join("ACGT"[i] for i in rng.integers(0, 4, size=k))
            t, a = oracle.compile_regex(w)
            assert t.shape[0] == k + 1, w
            assert a.sum() == 1


def test_kmer_sets_against_naive_search():
    rng = np.random.default_rng(1)
    for trial in range(300):
        k_lo = int(rng.integers(1, 5))
        pats = synth.random_kmers(int(rng.integers(1 << 30)), int(rng.integers(1, 8)), k_lo, k_lo + 3)
        seq = random_seq(rng, int(rng.integers(0, 300)))
        want = naive_kmer_positions(seq, pats)
        for minimise in (False, True):
            t, a = oracle.compile_kmers(pats, minimise=minimise)
            c, pos = oracle.run(t, a, seq)
            assert list(pos) == want and c == len(want), (pats, seq)


REGEXES = [
    "TATAAA", "ACG[AT]{2,6}C(G|T)T", "A(C|G)*T", "(AC)+G", "A.{2}T", "[AG]C?T",
    "G{2,}A", "(A|CG|TTA)T", "T(A|C){1,3}(G|T)", "AAA", "A[CG]*T[AT]?G",
]


@pytest.mark.parametrize("pattern", REGEXES + synth.random_regexes(5, 12))
def test_regex_against_python_re_windows(pattern):
    rng = np.random.default_rng(abs(hash(pattern)) % (1 << 31))
    t, a = oracle.compile_regex(pattern)
    tr, ar = oracle.compile_regex(pattern, minimise=False)
    for trial in range(25):
        seq = random_seq(rng, int(rng.integers(0, 160)), p_reset=0.02)
        want = re_window_positions(seq, pattern)
        assert list(oracle.run(t, a, seq)[1]) == want, (pattern, seq)
        assert list(oracle.run(tr, ar, seq)[1]) == want


def test_aho_corasick_equals_regex_alternation():
    """Two oracle routes to the same language must give the same canonical minimal
    table: the AC builder (Sec. II, III-B.1) and the regex compiler on p1|p2|..."""
    for seed in range(12):
        pats = synth.random_kmers(100 + seed, 1 + seed % 6, 3, 8)
        ta, aa = oracle.compile_kmers(pats, minimise=True)
        tr, ar = oracle.compile_regex("|".join(pats))
        assert ta.shape == tr.shape and (ta == tr).all() and (aa == ar).all()


def test_regex_dna_table_v_reverse_complement_invariant():
    """Table V: each expression is a form | its reverse complement, so the union is
    closed under reverse complement; all words have length 8, so distinct end
    positions correspond one to one with distinct start positions, and the count of
    a sequence equals the count of its reverse complement."""
    t, a = oracle.compile_regex("|".join(synth.REGEX_DNA_TABLE_V))
    comp = bytes.maketrans(b"ACGTacgt", b"TGCAtgca")
    rng = np.random.default_rng(7)
    for _ in range(20):
        # enrich the sequence with E1-like words so the count is non-trivial
        parts = [random_seq(rng, 40, p_reset=0.01) for _ in range(10)]
        seq = b"AGGGTAAA".join(parts[:5]) + b"TTTACCCT".join(parts[5:])
        rc = seq.translate(comp)[::-1]
        c1 = oracle.run(t, a, seq, positions=False)[0]
        c2 = oracle.run(t, a, rc, positions=False)[0]
        assert c1 == c2 and c1 >= 8   # 4 + 4 inserted words


def test_definite_depth_closed_form():
    """Closed form: for a finite language whose longest word has length m, the DFA of
    Sigma*.L reaches the same state from every start state after any m symbols (the
    state depends only on the last m symbols) -- the property that makes a lookback
    window of m symbols an exact start state for a chunk (Sec. III-A, converging point)."""
    rng = np.random.default_rng(3)
    cases = [("TATAAA", "TATAAA"), ("ACG[AT]{2,6}C(G|T)T", "ACGATATATCGT"),
             ("A.{2}T", "AGCT"), ("T(A|C){1,3}(G|T)", "TACAG")]
    for pat, longest in cases:
        m = len(longest)
        t, a = oracle.compile_regex(pat)
        Q = t.shape[0]

        def run(q, w):
            for s in w:
                q = int(t[q, s])
            return q
        for _ in range(200):
            w = rng.integers(0, 4, size=m)
            assert len({run(q, w) for q in range(Q)}) == 1
        # m-1 symbols are not enough: the longest word minus its first symbol ends in
        # an accepting state from the state reached by that first symbol, not from q0.
        w = ["ACGT".index(ch) for ch in longest]
        q1 = run(0, w[:1])
        assert a[run(q1, w[1:])] == 1 and run(q1, w[1:]) != run(0, w[1:])


def test_chunked_join_reproduces_sequential_run():
    """The join of Sec. III-A: running chunk k from the last state of chunk k-1 and
    summing the counts reproduces the single sequential run, for any split."""
    rng = np.random.default_rng(5)
    t, a = oracle.compile_regex("ACG[AT]{2,6}C(G|T)T")
    seq = synth.markov2(9, 20000)
    seq[rng.random(seq.size) < 0.002] = ord("N")
    total, _ = oracle.run(t, a, seq, positions=False)
    for _ in range(20):
        cuts = np.sort(rng.integers(0, seq.size, size=int(rng.integers(1, 30))))
        bounds = [0] + cuts.tolist() + [seq.size]
        q, acc = 0, 0
        for lo, hi in zip(bounds[:-1], bounds[1:]):
            c, q = oracle.run_from(t, a, q, seq[lo:hi])
            acc += c
        assert acc == total


def test_piece_run_from_reached_state_matches_brute_force():
    """A piece run from the state reached over a prefix w reports exactly the brute-force
    matches of w + piece that end inside the piece, counted from the piece's start, and
    ends where the run over w + piece ends (Sec. III-B: a chunk scanned from its true
    start state)."""
    rng = np.random.default_rng(21)
    for trial in range(40):
        k = int(rng.integers(3, 7))
        pats = ["".join("ACGT"[x] for x in rng.integers(0, 4, size=k)) for _ in range(int(rng.integers(1, 6)))]
        t, a = oracle.compile_kmers(pats)
        w = random_seq(rng, int(rng.integers(0, 40)))
        piece = random_seq(rng, int(rng.integers(0, 200)))
        _, q, _ = oracle.run_piece(t, a, 0, w)
        c, q_end, pos = oracle.run_piece(t, a, q, piece)
        want = [j - len(w) for j in naive_kmer_positions(w + piece, pats) if j >= len(w)]
        assert c == len(want) and list(pos) == want
        assert q_end == oracle.run_from(t, a, 0, w + piece)[1]
        if not w:
            assert q == 0


def test_reset_byte_splits_the_result():
    """A reset byte returns every run to q0, so the result on s1 N s2 is
    the result on s1 followed by the result on s2 shifted by len(s1) + 1."""
    rng = np.random.default_rng(8)
    t, a = oracle.compile_regex("A(C|G)*T")
    for _ in range(50):
        s1 = random_seq(rng, int(rng.integers(0, 80)), p_reset=0)
        s2 = random_seq(rng, int(rng.integers(0, 80)), p_reset=0)
        _, p1 = oracle.run(t, a, s1)
        _, p2 = oracle.run(t, a, s2)
        _, p = oracle.run(t, a, s1 + b"N" + s2)
        assert list(p) == list(p1) + [x + len(s1) + 1 for x in p2]


def test_count_positions_consistency_and_statistics():
    """count == len(positions), positions strictly increasing; on 1 MiB of i.i.d.
    uniform bases the non-self-overlapping 6-mer TATAAA occurs (n-5)/4^6 times in
    expectation (about 256); the oracle's count must lie within 5 sigma."""
    seq, motif = synth.plain_small()
    t, a = oracle.compile_regex(motif)
    c, pos = oracle.run(t, a, seq)
    assert c == len(pos) and (np.diff(pos) > 0).all()
    mean = (seq.size - 5) / 4096
    assert abs(c - mean) < 5 * np.sqrt(mean)
    for p in pos[:50]:
        assert seq[p - 5:p + 1].tobytes() == b"TATAAA"


def test_minimised_and_raw_tables_agree():
    rng = np.random.default_rng(12)
    for pat in REGEXES:
        t, a = oracle.compile_regex(pat)
        tr, ar = oracle.compile_regex(pat, minimise=False)
        tm, am = oracle.minimise_table(tr, ar)
        assert (tm == t).all() and (am == a).all()
        seq = random_seq(rng, 3000)
        assert oracle.run(t, a, seq, positions=False)[0] == oracle.run(tr, ar, seq, positions=False)[0]


def test_raw_table_with_accepting_start_state():
    """For a raw table, the definition is the table's own run: with state 0 in F every
    reset byte (which goes to state 0) is reported."""
    t = np.array([[1, 0, 0, 0], [1, 1, 0, 0]], dtype=np.int32)
    a = np.array([1, 0], dtype=np.uint8)
    c, pos = oracle.run(t, a, b"ANAC")
    # A->1 (no), N->0 (yes), A->1 (no), C->1 (no)
    assert list(pos) == [1]


@pytest.mark.parametrize("bad", ["", "A|", "(AC", "[AX]", "A{3,1}", "[]", "AN"])
def test_syntax_errors(bad):
    with pytest.raises(oracle.OracleError):
        oracle.compile_regex(bad)


@pytest.mark.parametrize("empty", ["A*", "(AC)?", "A{0,3}", "A|C*"])
def test_empty_word_patterns_rejected(empty):
    with pytest.raises(oracle.OracleError, match="empty word"):
        oracle.compile_regex(empty)


def test_markov_generator_gc_fraction():
    """Input recipe check: the order-2 Markov stand-in has 41.0 +- 0.2% GC."""
    seq = synth.markov2(1, 1 << 22)
    gc = np.isin(seq, np.frombuffer(b"CG", np.uint8)).mean()
    assert abs(gc - 0.41) < 0.002


# ------------------------------------------------------- pattern labels (f3)

LABEL_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "label_examples.tsv")


def _label_rows():
    rows = []
    for line in open(LABEL_GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        pats, seq, pos, masks, counts, cite = line.rstrip("\n").split("\t")
        rows.append((pats.split(";"), seq, [int(x) for x in pos.split(",")],
                     [int(x) for x in masks.split(",")], [int(x) for x in counts.split(",")], cite))
    return rows


@pytest.mark.parametrize("row", _label_rows(), ids=lambda r: ";".join(r[0]) + ":" + r[1])
def test_labelled_hand_worked_examples(row):
    """Hand-worked positions, label masks and per-pattern counts (Alg. 1's counter per
    accepting state), from the minimised and the raw labelled automaton."""
    pats, seq, pos, masks, counts, _ = row
    for minimise in (True, False):
        t, lab = oracle.compile_regex_set(pats, minimise=minimise)
        c, per, p, m = oracle.run_labels(t, lab, len(pats), seq.encode())
        assert c == len(pos) and list(p) == pos and list(m) == masks and list(per) == counts


def test_labelled_run_equals_separate_runs_and_brute_force():
    """One automaton for the nine Table V expressions reports, for every expression, the
    positions of that expression's own automaton run alone, and those of Python's re over
    every window; a step counts once in the total however many expressions end there."""
    pats = synth.REGEX_DNA_TABLE_V
    t, lab = oracle.compile_regex_set(pats)
    rng = np.random.default_rng(61)
    for trial in range(3):
        # a short random sequence with planted occurrences of Table V words
        seq = bytearray(random_seq(rng, 3000))
        for w in (b"AGGGTAAA", b"TTTACCCT", b"CGGGTAAA", b"AGGGTAAT", b"GTTACCCT", b"AAGGTAAA"):
            at = int(rng.integers(0, len(seq) - len(w)))
            seq[at:at + len(w)] = w
        seq = bytes(seq)
        c, per, pos, masks = oracle.run_labels(t, lab, len(pats), seq)
        union = set()
        for i, p in enumerate(pats):
            alone = list(oracle.run(*oracle.compile_regex(p), seq)[1])
            assert alone == re_window_positions(seq, p)
            assert per[i] == len(alone)
            assert [int(x) for x, m in zip(pos, masks) if m >> i & 1] == alone
            union |= set(alone)
        assert c == len(union) and list(pos) == sorted(union)
        assert all(m != 0 for m in masks)
    # the union of the labels is the alternation of the expressions compiled as one regex
    seq = synth.markov2(62, 200_000).tobytes()
    ta, aa = oracle.compile_regex("|".join(f"({p})" for p in pats))
    assert oracle.run_labels(t, lab, len(pats), seq, positions=False)[0] == oracle.run(ta, aa, seq, positions=False)[0]


def test_labelled_minimisation_keeps_labels_apart():
    """Minimisation merges only states with equal masks: a set with a repeated pattern
    keeps both counters, and each label's language is that of its own pattern."""
    t, lab = oracle.compile_regex_set(["ACG[AT]{2,6}C(G|T)T", "ACG[AT]{2,6}C(G|T)T", "TATAAA"])
    ts, as_ = oracle.compile_regex("TATAAA")
    seq = synth.markov2(63, 300_000)
    c, per, pos, masks = oracle.run_labels(t, lab, 3, seq)
    assert per[0] == per[1]
    assert per[2] == oracle.run(ts, as_, seq, positions=False)[0]
    raw_t, raw_lab = oracle.compile_regex_set(["ACG[AT]{2,6}C(G|T)T", "ACG[AT]{2,6}C(G|T)T", "TATAAA"],
                                               minimise=False)
    assert raw_t.shape[0] >= t.shape[0]
    c2, per2, pos2, masks2 = oracle.run_labels(raw_t, raw_lab, 3, seq)
    assert c2 == c and list(per2) == list(per) and np.array_equal(pos2, pos) and np.array_equal(masks2, masks)
