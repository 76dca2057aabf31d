"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact for
counts and positions, on seeded synthetic inputs that span many chunks and tiles and
end in a ragged tail, plus the edge cases of the method (resets, unaligned starts,
non-converging automata, capacity limits)."""
import numpy as np
import pytest

import oracle
import paper_1509_01506_gb300 as dna
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


def oracle_tables(kind, pat):
    if kind == "regex":
        return oracle.compile_regex(pat)
    return oracle.compile_kmers(pat, minimise=True)


def lib_dfa(kind, pat):
    return dna.Dfa.from_regex(pat) if kind == "regex" else dna.Dfa.from_kmers(pat)


def to_device(seq: np.ndarray, offset: int = 0):
    """Copies seq to the GPU so that its first byte sits 'offset' bytes past a 256-byte
    aligned allocation (exercises unaligned starts)."""
    buf = torch.empty(seq.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + seq.size]
    view.copy_(torch.from_numpy(seq))
    return view


def gpu_run(dfa, dseq, positions=True, capacity=None, plan=None):
    cnt, pos = dna.scan(dfa, dseq, positions=positions, capacity=capacity, plan=plan)
    torch.cuda.synchronize()
    c = int(cnt.item())
    if not positions:
        return c, None
    k = min(c, pos.numel())
    return c, pos[:k].cpu().numpy()


def check(kind, pat, seq, offset=0, plan=None, positions=True):
    t, a = oracle_tables(kind, pat)
    want_c, want_p = oracle.run(t, a, seq, positions=positions)
    dfa = lib_dfa(kind, pat)
    c, p = gpu_run(dfa, to_device(seq, offset), positions=positions,
                   capacity=max(16, want_c + 5), plan=plan)
    assert c == want_c
    if positions:
        assert np.array_equal(p, want_p)
    return c


def noisy_markov(seed, n, n_frac=0.01, lower_frac=0.1):
    s = synth.markov2(seed, n)
    synth.overlay_runs(s, seed, lower_frac, 300.0, "lower")
    synth.overlay_runs(s, seed + 1, n_frac, 200.0, "N")
    return s


# ------------------------------------------------------------- hand examples

def test_hand_examples_on_gpu():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.tsv")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kind, pats, seq, exp, _ = line.rstrip("\n").split("\t")
        want = [] if exp == "-" else [int(x) for x in exp.split(",")]
        pat = pats if kind == "regex" else pats.split(",")
        dfa = lib_dfa(kind, pat)
        c, p = gpu_run(dfa, to_device(np.frombuffer(seq.encode(), np.uint8)), capacity=64)
        assert c == len(want) and p.tolist() == want, (pats, seq)


# ------------------------------------------------------- workloads, reduced

def test_plain_small_full_size():
    """1 MiB uniform, TATAAA (7 states), count + positions."""
    seq, motif = synth.plain_small()
    check("regex", motif, seq)


def test_plain_markov_reduced():
    seq = synth.markov2(1, 8 * MiB + 77)
    check("regex", synth.CONFIG2_REGEX, seq)


def test_plain_large_reduced_kmers():
    """Markov with soft-masked and N runs; AC automaton of 1,000 random 12-mers."""
    seq = noisy_markov(2, 16 * MiB + 5, n_frac=0.02, lower_frac=0.1)
    kmers = synth.random_kmers(2, 1000, 12)
    check("kmers", kmers, seq, positions=True)


def test_regex_dna_table_v():
    """The nine Table V expressions as one regex: 106 states, too many for per-lane
    two-symbol tables, so per-lane one-symbol tables by default; every placement agrees."""
    seq = noisy_markov(7, 4 * MiB + 3)
    pat = "|".join(synth.REGEX_DNA_TABLE_V)
    assert dna.Dfa.from_regex(pat).info().placement == dna.PLACE_SMEM_ONE
    for plan in (None, dict(placement=2), dict(placement=3), dict(placement=5),
                 dict(placement=6, warps_per_cta=16), dict(placement=6, warps_per_cta=8, chunk_bytes=128)):
        check("regex", pat, seq, plan=plan)


@pytest.mark.parametrize("n_kmers", [14, 30, 48])
def test_per_lane_one_symbol_tables_up_to_their_limit(n_kmers):
    """k-mer automata of about 100 to 350 states take per-lane one-symbol tables (the
    largest with 8 warps); counts and positions equal the oracle's."""
    kmers = synth.random_kmers(90 + n_kmers, n_kmers, 8)
    seq = noisy_markov(91, 2 * MiB + 77)
    check("kmers", kmers, seq, offset=2, plan=dict(placement=6))
    check("kmers", kmers, seq, offset=2, plan=dict(placement=6, warps_per_cta=8))


def test_autotuner_picks_a_measured_placement_and_results_stay_exact():
    """dfa_tune times the placements the automaton fits in and makes the fastest the
    default; the scans after it still equal the oracle's."""
    seq = noisy_markov(92, 8 * MiB + 5)
    for kind, pat in (("regex", synth.CONFIG2_REGEX), ("regex", "|".join(synth.REGEX_DNA_TABLE_V)),
                      ("kmers", synth.random_kmers(93, 300, 10))):
        dfa = dna.Dfa.from_regex(pat) if kind == "regex" else dna.Dfa.from_kmers(pat)
        pl, ms = dfa.tune(to_device(seq))
        assert pl in (1, 2, 3, 5, 6) and ms > 0 and dfa.info().placement == pl
        t, a = oracle_tables(kind, pat)
        want_c, want_p = oracle.run(t, a, seq)
        c, p = gpu_run(dfa, to_device(seq, 1), capacity=want_c + 1)
        assert c == want_c and np.array_equal(p, want_p)


@pytest.mark.parametrize("pattern", synth.random_regexes(3, 12))
def test_random_motif_regexes(pattern):
    seq = synth.uniform(11, 1 * MiB + 13)
    check("regex", pattern, seq)


# ------------------------------------------------------ plan independence

PLANS = [
    dict(chunk_bytes=128, lookback=1, warps_per_cta=32, placement=1),
    dict(chunk_bytes=256, lookback=3, warps_per_cta=8, placement=1),
    dict(chunk_bytes=1152, lookback=12, warps_per_cta=16, placement=1),
    dict(chunk_bytes=8192, lookback=32, warps_per_cta=16, placement=1),
    dict(chunk_bytes=384, lookback=1, warps_per_cta=8, placement=2),
    dict(chunk_bytes=640, lookback=5, warps_per_cta=32, placement=3),
    dict(chunk_bytes=4096, lookback=64, warps_per_cta=16, placement=2),
    dict(chunk_bytes=2048, lookback=1, warps_per_cta=16, placement=5),
    dict(chunk_bytes=256, lookback=7, warps_per_cta=8, placement=5, hot_rows=3),
    dict(chunk_bytes=1280, lookback=1, warps_per_cta=16, placement=5, hot_rows=1),
    dict(chunk_bytes=128, lookback=1, warps_per_cta=24, placement=6),
    dict(chunk_bytes=1024, lookback=9, warps_per_cta=8, placement=6),
]


@pytest.mark.parametrize("plan", PLANS, ids=lambda p: "-".join(str(v) for v in p.values()))
@pytest.mark.parametrize("offset", [0, 5])
def test_results_do_not_depend_on_the_plan(plan, offset):
    """Any chunking, lookback (1 = the paper's one-symbol possible starting states),
    CTA shape or table placement gives the sequential result (Sec. III-A join)."""
    seq = noisy_markov(5, 3 * MiB + 1001)
    check("regex", synth.CONFIG2_REGEX, seq, offset=offset, plan=plan)


# --------------------------------------------------------------- edge cases

@pytest.mark.parametrize("n", [0, 1, 2, 15, 16, 17, 127, 128, 129, 4095, 4097, 100003])
@pytest.mark.parametrize("offset", [0, 1, 7, 15])
def test_lengths_and_alignment(n, offset):
    rng = np.random.default_rng(n * 31 + offset)
    seq = np.frombuffer(b"ACGTN", np.uint8)[rng.integers(0, 5, size=n)].copy() if n else \
        np.zeros(0, np.uint8)
    check("regex", "A[CG]T", seq, offset=offset)


def test_all_reset_bytes_and_all_byte_values():
    check("regex", "TATAAA", np.full(50000, ord("N"), np.uint8))
    rng = np.random.default_rng(1)
    seq = rng.integers(0, 256, size=300000).astype(np.uint8)
    bases = np.frombuffer(b"ACGTacgt", np.uint8)
    pick = rng.random(seq.size) < 0.6
    seq[pick] = bases[rng.integers(0, 8, size=int(pick.sum()))]
    check("regex", "A[CG]T", seq)
    lower = synth.uniform(3, 200000)
    lower += 32
    check("regex", "TATA", lower)


@pytest.mark.parametrize("placement", [2, 3, 5, (5, 2), 6])
def test_one_symbol_rows_with_every_byte_value(placement):
    """The one-symbol loops take a reset byte's entry without branching: every byte value
    (bases of both cases, N, IUPAC codes, control and high bytes) mixed into rows of
    bases, rows of N only and rows of lowercase bases, counts and positions."""
    rng = np.random.default_rng(41)
    seq = rng.integers(0, 256, size=1 * MiB + 37).astype(np.uint8)
    bases = np.frombuffer(b"ACGTacgt", np.uint8)
    pick = rng.random(seq.size) < 0.97
    seq[pick] = bases[rng.integers(0, 8, size=int(pick.sum()))]
    seq[200000:260000] = ord("N")
    seq[300000:400000] = np.frombuffer(b"acgt", np.uint8)[rng.integers(0, 4, size=100000)]
    extra = {}
    if isinstance(placement, tuple):   # the hot-state rows with very few two-symbol rows
        placement, extra = placement[0], dict(hot_rows=placement[1])
    # per-lane one-symbol copies hold at most a few hundred states: a smaller k-mer set
    kmers = synth.random_kmers(41, 40 if placement == 6 else 200, 6, 9)
    for kind, pat in (("regex", "A[CG]T"), ("kmers", kmers)):
        for chunk in (128, 2048):
            check(kind, pat, seq, offset=3, plan=dict(chunk_bytes=chunk, placement=placement, **extra))
    check("regex", "TATA", np.full(70000, ord("N"), np.uint8), plan=dict(placement=placement, **extra))


def test_accepting_start_state_raw_table():
    """Raw table with state 0 in F: every reset byte is reported."""
    table = np.array([[1, 0, 0, 0], [1, 1, 0, 0]], dtype=np.uint32)
    acc = np.array([1, 0], dtype=np.uint8)
    rng = np.random.default_rng(2)
    seq = np.frombuffer(b"ACGTN", np.uint8)[rng.integers(0, 5, size=70001)].copy()
    want_c, want_p = oracle.run(table.astype(np.int32), acc, seq)
    dfa = dna.Dfa(table, dna.pack_accept(acc))
    assert dfa.info().accept_start
    for plan in (None, dict(chunk_bytes=128, placement=2), dict(chunk_bytes=256, placement=3),
                 dict(chunk_bytes=384, placement=5), dict(chunk_bytes=384, placement=5, hot_rows=1),
                 dict(chunk_bytes=256, placement=6)):
        c, p = gpu_run(dfa, to_device(seq, 3), capacity=want_c + 1, plan=plan)
        assert c == want_c and np.array_equal(p, want_p)


def test_single_state_automata():
    seq = noisy_markov(3, 500000)
    for acc in (0, 1):
        table = np.zeros((1, 4), dtype=np.uint32)
        a = np.array([acc], np.uint8)
        want_c, _ = oracle.run(table.astype(np.int32), a, seq, positions=False)
        dfa = dna.Dfa(table, dna.pack_accept(a))
        c, _ = gpu_run(dfa, to_device(seq), positions=False)
        assert c == want_c == (seq.size if acc else 0)


def test_non_definite_automaton_repair_and_cascade():
    """A(C|G)*T never converges on runs of C/G: chunks whose speculated start is wrong
    must be repaired at the converging point or, when the runs never meet, cascaded."""
    rng = np.random.default_rng(9)
    parts = []
    for _ in range(400):
        parts.append(np.frombuffer(b"CG", np.uint8)[rng.integers(0, 2, size=int(rng.integers(50, 3000)))])
        parts.append(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, size=int(rng.integers(1, 30)))])
    seq = np.concatenate(parts)
    for plan in (dict(chunk_bytes=128, lookback=1), dict(chunk_bytes=256, lookback=4, placement=2),
                 dict(chunk_bytes=128, lookback=1, placement=3), None,
                 dict(chunk_bytes=256, placement=5, hot_rows=2), dict(chunk_bytes=128, placement=6)):
        check("regex", "A(C|G)*T", seq, plan=plan)


def test_random_permutation_like_tables():
    """Random tables are mostly not definite: speculation fails often and the repair /
    cascade path carries the result."""
    rng = np.random.default_rng(21)
    for trial in range(12):
        Q = int(rng.integers(2, 40))
        table = rng.integers(0, Q, size=(Q, 4)).astype(np.uint32)
        if trial % 2 == 0:  # permutations never converge
            table = np.stack([rng.permutation(Q) for _ in range(4)], axis=1).astype(np.uint32)
        acc = (rng.random(Q) < 0.3).astype(np.uint8)
        seq = synth.uniform(100 + trial, 200000 + trial * 17)
        want_c, want_p = oracle.run(table.astype(np.int32), acc, seq)
        dfa = dna.Dfa(table, dna.pack_accept(acc))
        for plan in (None, dict(chunk_bytes=128, lookback=2, placement=1),
                     dict(chunk_bytes=512, lookback=1, placement=3),
                     dict(chunk_bytes=256, placement=5, hot_rows=int(rng.integers(1, Q + 1))),
                     dict(chunk_bytes=384, placement=6)):
            c, p = gpu_run(dfa, to_device(seq, trial % 16), capacity=want_c + 3, plan=plan)
            assert c == want_c and np.array_equal(p, want_p), (trial, plan)


def _permutation_automaton(Q, seed):
    rng = np.random.default_rng(seed)
    table = np.stack([rng.permutation(Q) for _ in range(4)], axis=1).astype(np.uint32)
    acc = (rng.random(Q) < 0.3).astype(np.uint8)
    acc[int(rng.integers(0, Q))] = 1
    return table, acc


@pytest.mark.parametrize("Q", [2, 5, 8, 12, 17, 32, 33, 64, 90, 91, 130, 256])
@pytest.mark.parametrize("n,offset", [(1, 0), (4095, 3), (100003, 7), (3 * MiB + 777, 1)])
def test_chunk_maps_for_automata_that_never_converge(Q, n, offset):
    """Permutation automata: runs from different states never meet, so dfa_load picks
    chunk maps (every chunk run from every state, maps composed in order); counts and
    positions equal the oracle's, across resets and ragged ends."""
    table, acc = _permutation_automaton(Q, 300 + Q)
    seq = noisy_markov(400 + n % 97, n) if n > 1000 else synth.uniform(401, n)
    want_c, want_p = oracle.run(table.astype(np.int32), acc, seq)
    dfa = dna.Dfa(table, dna.pack_accept(acc))
    assert dfa.info().chunk_maps
    c, p = gpu_run(dfa, to_device(seq, offset), capacity=want_c + 3)
    assert c == want_c and np.array_equal(p, want_p)
    c2, _ = gpu_run(dfa, to_device(seq, offset), positions=False)
    assert c2 == want_c


@pytest.mark.parametrize("Q", [33, 64, 256])
def test_chunk_maps_of_more_than_32_states_at_64MiB(Q):
    """Automata of more than 32 states whose runs never meet: every chunk is run from
    every state by ceil(Q / 32) warps (two-symbol tables up to about 90 states, one-symbol
    tables above), the wide maps are composed by the join; counts and positions of a
    64 MiB noisy Markov sequence equal the oracle's."""
    table, acc = _permutation_automaton(Q, 900 + Q)
    seq = noisy_markov(901 + Q, 64 * MiB)
    want_c, want_p = oracle.run(table.astype(np.int32), acc, seq)
    dfa = dna.Dfa(table, dna.pack_accept(acc))
    assert dfa.info().chunk_maps
    c, p = gpu_run(dfa, to_device(seq, 5), capacity=want_c + 3)
    assert c == want_c and np.array_equal(p, want_p)
    c2, _ = gpu_run(dfa, to_device(seq, 5), positions=False)
    assert c2 == want_c


def test_non_converging_automaton_above_the_map_limit_is_exact():
    """A 300-state permutation automaton is above the chunk-map limit (256 states): it is
    scanned with speculation and repair, which walks the chunk boundaries in order and is
    exact."""
    table, acc = _permutation_automaton(300, 77)
    seq = noisy_markov(78, 256 * 1024 + 9)
    want_c, want_p = oracle.run(table.astype(np.int32), acc, seq)
    dfa = dna.Dfa(table, dna.pack_accept(acc))
    assert not dfa.info().chunk_maps
    c, p = gpu_run(dfa, to_device(seq, 2), capacity=want_c + 3)
    assert c == want_c and np.array_equal(p, want_p)


def test_chunk_maps_forced_on_a_converging_regex():
    """The chunk-map path requested through the plan gives the same result as the
    speculative path on an automaton that does converge."""
    seq = noisy_markov(31, 5 * MiB + 333)
    dfa = dna.Dfa.from_regex(synth.CONFIG2_REGEX)
    assert not dfa.info().chunk_maps
    check("regex", synth.CONFIG2_REGEX, seq, offset=9, plan=dict(placement=4))
    check("regex", synth.CONFIG2_REGEX, seq, offset=0, plan=dict(placement=4), positions=False)


def _reset_heavy(seed, n, frac):
    """Noisy Markov bases with short N runs covering about 'frac' of the bytes, so that
    most 128-byte rows hold a reset byte."""
    s = synth.markov2(seed, n)
    synth.overlay_runs(s, seed, 0.1, 40.0, "lower")
    synth.overlay_runs(s, seed + 1, frac, 6.0, "N")
    return s


@pytest.mark.parametrize("Q", [2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 15, 16])
@pytest.mark.parametrize("n,offset", [(1, 3), (127, 0), (129, 5), (32 * 4096 - 1, 7), (32 * 4096 + 1, 1),
                                      (1 * MiB + 5, 11), (9 * MiB + 77, 2)])
def test_nibble_chunk_maps_every_state_count(Q, n, offset):
    """Automata of at most 16 states whose runs never meet keep every run of a part in
    4-bit fields of one register (8 states) or two (16 states, where each lookup picks
    between the rows of states 0..7 and 8..15). Every state count, an accepting start
    state, lengths at part and row edges and unaligned starts: counts and positions
    equal the oracle's."""
    rng = np.random.default_rng(700 + Q)
    table = np.stack([rng.permutation(Q) for _ in range(4)], axis=1).astype(np.uint32)
    acc = (rng.random(Q) < 0.4).astype(np.uint8)
    acc[0] = 1
    seq = noisy_markov(701 + n % 89, n) if n > 1000 else synth.uniform(702, n)
    want_c, want_p = oracle.run(table.astype(np.int32), acc, seq)
    dfa = dna.Dfa(table, dna.pack_accept(acc))
    assert dfa.info().chunk_maps
    c, p = gpu_run(dfa, to_device(seq, offset), capacity=want_c + 3)
    assert c == want_c and np.array_equal(p, want_p)
    c2, _ = gpu_run(dfa, to_device(seq, offset), positions=False)
    assert c2 == want_c


@pytest.mark.parametrize("Q", [8, 16])
@pytest.mark.parametrize("frac", [0.3, 0.6, 1.0])
def test_nibble_chunk_maps_with_reset_bytes_in_most_rows(frac, Q):
    """Rows with a reset byte take the one-symbol steps of the nibble kernel (every run
    back to q0, counted when q0 accepts); an all-N sequence resets every byte."""
    table, acc = _permutation_automaton(Q, 711)
    acc[0] = 1
    n = 3 * MiB + 1234
    seq = np.full(n, ord("N"), dtype=np.uint8) if frac == 1.0 else _reset_heavy(712, n, frac)
    want_c, want_p = oracle.run(table.astype(np.int32), acc, seq)
    dfa = dna.Dfa(table, dna.pack_accept(acc))
    c, p = gpu_run(dfa, to_device(seq, 3), capacity=want_c + 3)
    assert c == want_c and np.array_equal(p, want_p)


def test_nibble_chunk_maps_on_a_counter_and_on_forced_small_regexes():
    """A counter automaton (the number of A's mod 8: one symbol permutes, the others
    keep the state), and small regexes whose runs do converge scanned through the
    nibble chunk maps by request: results equal the oracle's."""
    t = np.array([[(q + 1) % 8, q, q, q] for q in range(8)], dtype=np.uint32)
    a = np.zeros(8, dtype=np.uint8)
    a[0] = 1
    seq = noisy_markov(720, 5 * MiB + 17)
    want_c, want_p = oracle.run(t.astype(np.int32), a, seq)
    dfa = dna.Dfa(t, dna.pack_accept(a))
    assert dfa.info().chunk_maps
    c, p = gpu_run(dfa, to_device(seq, 6), capacity=want_c + 3)
    assert c == want_c and np.array_equal(p, want_p)
    for pat in ("ACGT", "A(C|G)T", "TATAAA"):
        assert dna.Dfa.from_regex(pat).info().n_states <= 8
        check("regex", pat, seq, offset=1, plan=dict(placement=4))
        check("regex", pat, seq, offset=0, plan=dict(placement=4), positions=False)


def test_chunk_maps_full_size():
    """64 MiB against an 8-state permutation automaton (never converging)."""
    table, acc = _permutation_automaton(8, 77)
    seq = noisy_markov(78, 64 * MiB)
    want_c, want_p = oracle.run(table.astype(np.int32), acc, seq)
    dfa = dna.Dfa(table, dna.pack_accept(acc))
    c, p = gpu_run(dfa, to_device(seq), capacity=want_c + 3)
    assert c == want_c and np.array_equal(p, want_p)


def test_positions_capacity_smaller_than_count():
    seq = synth.uniform(5, 2 * MiB)
    t, a = oracle.compile_regex("AC")
    want_c, want_p = oracle.run(t, a, seq)
    dfa = dna.Dfa.from_regex("AC")
    for cap in (1, 1000, want_c - 1):
        c, p = gpu_run(dfa, to_device(seq), capacity=cap)
        assert c == want_c and np.array_equal(p, want_p[:cap])


def test_dense_matches_overflow_stash():
    """'A' matches about a quarter of all positions: every chunk overflows its stash
    and is rescanned by the extraction pass."""
    seq = noisy_markov(4, 1 * MiB + 9)
    check("regex", "A", seq)
    check("regex", "[ACGT]", seq)


def test_large_aho_corasick_placements():
    seq = noisy_markov(6, 4 * MiB + 1)
    kmers = synth.random_kmers(6, 1000, 12)
    for plan in (None, dict(placement=2), dict(placement=3), dict(placement=3, lookback=1),
                 dict(placement=5), dict(placement=5, hot_rows=64), dict(placement=5, hot_rows=1000),
                 dict(placement=5, warps_per_cta=8), dict(placement=5, chunk_bytes=128)):
        check("kmers", kmers, seq, plan=plan, positions=True)


def test_hot_state_rows_on_the_large_aho_corasick_automaton():
    """Hot-state rows on the 1,000 12-mers of the 3.2 GiB workload (7,366 states, about
    3,000 two-symbol rows, many lanes taking the one-symbol redo), on soft-masked
    sequence with N runs: results equal the oracle's, counts and positions."""
    kmers = synth.random_kmers(2, 1000, 12)
    seq = noisy_markov(16, 16 * MiB + 3, n_frac=0.02, lower_frac=0.1)
    for plan in (dict(placement=5), dict(placement=5, warps_per_cta=8)):
        check("kmers", kmers, seq, offset=1, plan=plan)


def test_invalid_arguments_are_rejected():
    dfa = dna.Dfa.from_regex("ACGT")
    seq = to_device(synth.uniform(1, 1000))
    with pytest.raises(dna.DnaError):
        dna.scan(dfa, seq, plan=dict(chunk_bytes=100))
    with pytest.raises(dna.DnaError):
        dna.scan(dfa, seq, plan=dict(lookback=65))
    with pytest.raises(dna.DnaError):
        dna.scan(dfa, seq, plan=dict(warps_per_cta=3))
    with pytest.raises(dna.DnaError):
        dna.Dfa(np.array([[0, 0, 0, 2]], np.uint32), np.array([0], np.uint8))
    big = dna.Dfa.from_kmers(synth.random_kmers(1, 400, 12))
    with pytest.raises(dna.DnaError) as ei:
        dna.scan(big, seq, plan=dict(placement=1))
    assert ei.value.code == -3


def test_host_buffer_entry_point():
    """dna_scan_host: host sequence in, host count and positions out, same results as
    the oracle; a capacity below the count reports DNA_ERR_CAPACITY with the true count
    and the smallest positions."""
    pat = synth.CONFIG2_REGEX
    seq = noisy_markov(21, 3 * MiB + 101)
    t, a = oracle.compile_regex(pat)
    want_c, want_p = oracle.run(t, a, seq)
    dfa = dna.Dfa.from_regex(pat)
    c, p = dna.scan_host(dfa, seq, positions=True, capacity=want_c + 3)
    assert c == want_c and np.array_equal(p.astype(np.int64), want_p)
    pinned = torch.from_numpy(seq).pin_memory()
    c2, _ = dna.scan_host(dfa, pinned)
    assert c2 == want_c
    out_c = np.zeros(1, np.uint64)
    out_p = np.zeros(7, np.uint64)
    with pytest.raises(dna.DnaError) as ei:
        dna.scan_host(dfa, seq, positions=True, out_count=out_c, out_positions=out_p)
    assert ei.value.code == -3
    assert int(out_c[0]) == want_c and np.array_equal(out_p.astype(np.int64), want_p[:7])
    c0, p0 = dna.scan_host(dfa, np.zeros(0, np.uint8), positions=True, capacity=4)
    assert c0 == 0 and p0.size == 0


# ------------------------------------------------------ full-size workloads

def test_plain_markov_full_size_launch_config():
    """256 MiB order-2 Markov, ACG[AT]{2,6}C(G|T)T, count + positions, automatic plan
    (the launch configuration the bench times)."""
    seq, pat = synth.plain_markov()
    c = check("regex", pat, seq)
    assert c > 1000


def test_plain_large_full_size_count():
    """3.2 GiB with soft-masked and N runs, AC of 1,000 random 12-mers, count only."""
    seq, kmers = synth.plain_large()
    t, a = oracle.compile_kmers(kmers, minimise=True)
    want_c, _ = oracle.run(t, a, seq, positions=False)
    dfa = dna.Dfa.from_kmers(kmers)
    dseq = torch.from_numpy(seq).cuda()
    del seq
    c, _ = gpu_run(dfa, dseq, positions=False)
    assert c == want_c


def test_back_to_back_scans_on_two_streams_share_nothing_stale():
    """Scans queued back to back on one stream reuse the stream's control words (left
    zero by each scan); interleaving automata of every kind, with and without positions,
    and a second stream gives each scan the oracle's result."""
    seq = noisy_markov(95, 6 * MiB + 13)
    table, acc = _permutation_automaton(6, 96)
    auts = [("regex", synth.CONFIG2_REGEX, dna.Dfa.from_regex(synth.CONFIG2_REGEX)),
            ("kmers", synth.random_kmers(97, 400, 11), None),
            ("perm", None, dna.Dfa(table, dna.pack_accept(acc)))]
    auts[1] = ("kmers", auts[1][1], dna.Dfa.from_kmers(auts[1][1]))
    want = []
    for kind, pat, _ in auts:
        t, a = (table.astype(np.int32), acc) if kind == "perm" else oracle_tables(kind, pat)
        want.append(oracle.run(t, a, seq))
    d = to_device(seq, 4)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for r in range(3):
        for k, (_, _, dfa) in enumerate(auts):
            st = s1 if (r + k) % 2 == 0 else s2
            c, p = dna.scan(dfa, d, positions=(r != 1), capacity=want[k][0] + 1, stream=st)
            outs.append((k, r != 1, c, p))
    torch.cuda.synchronize()
    for k, pos, c, p in outs:
        assert int(c.item()) == want[k][0]
        if pos:
            assert np.array_equal(p[:want[k][0]].cpu().numpy(), want[k][1])


def test_lookup_peak_microbenchmark():
    """dna_lookup_peak measures the lookup rates the rooflines divide by: lanes in their
    own banks beat lanes at random banks, and both beat random L2 gathers."""
    p0, p1, p2 = dna.lookup_peak(0), dna.lookup_peak(1), dna.lookup_peak(2)
    assert p0 > p1 > 0 and p0 > p2 > 0
    with pytest.raises(dna.DnaError):
        dna.lookup_peak(3)


@pytest.mark.parametrize("plan", [None, dict(chunk_bytes=128), dict(chunk_bytes=256, lookback=12),
                                  dict(chunk_bytes=384, warps_per_cta=8), dict(chunk_bytes=4096, lookback=1),
                                  dict(warps_per_cta=16, lookback=30)], ids=str)
def test_count_only_one_symbol_scans(plan):
    """Count-only scans with the shared one-symbol table (the placement of the 3.2 GiB
    workload's automaton): counts equal the oracle's across lengths, offsets, lookback
    windows, resets, every byte value, automata that never meet, and the 7,366-state
    Aho-Corasick automaton."""
    plan = dict(plan or {}, placement=2)
    rng = np.random.default_rng(61)
    for n, off in ((1, 0), (130, 3), (4097, 1), (100003, 7), (2 * MiB + 77, 5)):
        seq = noisy_markov(62 + n % 7, n) if n > 200 else synth.uniform(63, n)
        check("regex", "|".join(synth.REGEX_DNA_TABLE_V), seq, offset=off, plan=plan, positions=False)
    seq = rng.integers(0, 256, size=MiB + 3).astype(np.uint8)
    bases = np.frombuffer(b"ACGTacgt", np.uint8)
    pick = rng.random(seq.size) < 0.97
    seq[pick] = bases[rng.integers(0, 8, size=int(pick.sum()))]
    seq[200000:260000] = ord("N")
    check("kmers", synth.random_kmers(64, 300, 6, 9), seq, offset=2, plan=plan, positions=False)
    check("regex", "A(C|G)*T", noisy_markov(65, MiB + 9), plan=plan, positions=False)
    table = rng.integers(0, 120, size=(120, 4)).astype(np.uint32)
    acc = (rng.random(120) < 0.3).astype(np.uint8)
    useq = synth.uniform(66, 300001)
    want_c, _ = oracle.run(table.astype(np.int32), acc, useq, positions=False)
    c, _ = gpu_run(dna.Dfa(table, dna.pack_accept(acc)), to_device(useq, 3), positions=False, plan=plan)
    assert c == want_c
    check("kmers", synth.random_kmers(6, 1000, 12), noisy_markov(67, 8 * MiB + 1, n_frac=0.02),
          offset=1, plan=plan, positions=False)
