"""CPU-only checks of the library: it loads without a GPU, exports every symbol the
header declares, its host compiler agrees with the oracle's independent compiler, and
its automaton analysis agrees with brute force."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import paper_1509_01506_gb300 as dna
import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "dna_dfa.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|u?int64_t)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_loads_and_exports_header_symbols():
    lib = ctypes.CDLL(dna.build())
    names = header_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(dna.EXPORTED) <= set(names)


def test_status_strings():
    for code in range(-8, 1):
        assert dna.status_string(code) not in ("", "unknown status")
    assert dna.status_string(-99) == "unknown status"


def _oracle_accept(mask, n):
    return np.unpackbits(mask, bitorder="little")[:n]


PATTERNS = [
    "TATAAA", "ACG[AT]{2,6}C(G|T)T", "A(C|G)*T", "(AC)+G", "A.{2}T", "[AG]C?T", "G{2,}A",
    "(A|CG|TTA)T", "T(A|C){1,3}(G|T)", "AAA", "A[CG]*T[AT]?G", "|".join(synth.REGEX_DNA_TABLE_V),
] + synth.random_regexes(3, 40)


@pytest.mark.parametrize("pattern", PATTERNS)
def test_host_compiler_matches_oracle_compiler(pattern):
    """Library (Glushkov + Hopcroft) and oracle (Thompson + Moore) minimal DFAs, both in
    canonical breadth-first numbering, must be identical tables."""
    t, m = dna.compile_regex(pattern)
    to, ao = oracle.compile_regex(pattern)
    assert t.shape == to.shape
    assert (t == to).all()
    assert (_oracle_accept(m, t.shape[0]) == ao).all()


@pytest.mark.parametrize("patterns", [
    synth.REGEX_DNA_TABLE_V, ["TA", "AT"], ["CA", "A"], ["A{2}", "AA", "A"],
    ["ACG[AT]{2,6}C(G|T)T", "TATAAA", "A(C|G)*T"], synth.random_regexes(71, 12), synth.random_regexes(72, 32)])
def test_pattern_set_compiler_matches_oracle(patterns):
    """One labelled automaton for several patterns: the library's (Glushkov positions of
    the union, a mask per state from each pattern's last positions, Hopcroft from the
    partition by mask) and the oracle's (Thompson NFA with an exit per pattern, subset
    construction, Moore from the partition by mask) are identical in canonical numbering."""
    t, lab = dna.compile_regex_set(patterns)
    to, lo = oracle.compile_regex_set(patterns)
    assert t.shape == to.shape and (t == to).all()
    assert (lab == lo).all()


def test_pattern_set_compiler_errors():
    with pytest.raises(dna.DnaError):
        dna.compile_regex_set(["A", "A*"])
    with pytest.raises(dna.DnaError):
        dna.compile_regex_set(["A("])
    with pytest.raises(dna.DnaError):
        dna.compile_regex_set(["A"] * 33)


def test_kmer_compiler_matches_oracle():
    for seed in range(20):
        kmers = synth.random_kmers(seed, 1 + seed * 3, 4, 12)
        t, m = dna.compile_kmers(kmers)
        to, ao = oracle.compile_kmers(kmers, minimise=True)
        assert (t == to).all() and (_oracle_accept(m, t.shape[0]) == ao).all()


@pytest.mark.parametrize("bad,code", [("A|", -6), ("(AC", -6), ("[AX]", -6), ("A{3,1}", -6),
                                      ("A*", -7), ("(AC)?", -7), ("", -6), ("A{0}", -6)])
def test_compiler_errors(bad, code):
    with pytest.raises(dna.DnaError) as ei:
        dna.compile_regex(bad)
    assert ei.value.code == code


def brute_definite_depth(table, cap=10):
    """Smallest m <= cap such that every word of length m maps all states to one."""
    Q = table.shape[0]
    sets = [frozenset(range(Q))]
    for m in range(0, cap + 1):
        if all(len(s) == 1 for s in sets):
            return m
        nxt = set()
        for s in sets:
            for c in range(4):
                nxt.add(frozenset(int(table[q, c]) for q in s))
        sets = list(nxt)
    return -1


def test_definite_depth_against_brute_force():
    rng = np.random.default_rng(4)
    tables = [dna.compile_regex(p)[0] for p in PATTERNS[:11]]
    for _ in range(60):  # random small tables (many are not definite)
        Q = int(rng.integers(1, 7))
        t = rng.integers(0, Q, size=(Q, 4)).astype(np.uint32)
        tables.append(t)
    for t in tables:
        got = dna.definite_depth(t)
        want = brute_definite_depth(t, cap=10)
        if want >= 0:
            assert got == want
        else:
            assert got == -1 or got > 10


def test_definite_depth_closed_form_for_kmers():
    """An Aho-Corasick automaton of k-mers is k-definite (its state is the longest
    suffix of the input that is a pattern prefix, a function of the last k symbols)."""
    for k in (3, 6, 9):
        t, _ = dna.compile_kmers(synth.random_kmers(k, 30, k))
        assert dna.definite_depth(t) == k


def test_pack_accept_layout():
    a = np.zeros(19, dtype=np.uint8)
    a[[0, 9, 18]] = 1
    m = dna.pack_accept(a)
    assert m.tolist() == [1, 2, 4]


# ------------------------------------------------------------------ FASTA ingest

def _fasta_reference(text: bytes):
    """Plain reading of FASTA: records start at '>' lines; sequence lines are joined with
    line breaks, spaces and tabs removed; text before the first header is a record."""
    recs, hdrs, cur = [], [], None
    for line in re.split(rb"\r\n|\n|\r", text):
        if line.startswith(b">"):
            cur = bytearray()
            recs.append(cur)
            hdrs.append(line[1:].decode())
            continue
        body = line.replace(b" ", b"").replace(b"\t", b"")
        if body and cur is None:
            cur = bytearray()
            recs.append(cur)
            hdrs.append("")
        if cur is not None:
            cur.extend(body)
    return recs, hdrs


def test_fasta_parse_against_a_plain_reading():
    text = (b"ACGTN\n"                                        # unnamed first record
            b">chr1 test record\r\nACGTacgtNNNN\r\nTTTA CCC\r\n\r\n"
            b">chr2\nGATTACA\n\n>empty\n>chr3\rACGT\rAC\tGT\n>x\nA>C\n")
    seq, off, hdr = dna.fasta_parse(text)
    recs, want_hdr = _fasta_reference(text)
    assert hdr == want_hdr
    assert len(off) == len(recs) + 1
    for r, rec in enumerate(recs):
        assert bytes(seq[off[r]:off[r + 1]]) == bytes(rec), r
    assert int(off[-1]) == seq.size == sum(len(r) for r in recs)


def test_fasta_parse_capacity_and_sizing():
    lib = dna.lib()
    text = b">a\nACGT\n>b\nGG\n"
    n_out, n_rec = ctypes.c_uint64(), ctypes.c_uint32()
    assert lib.dna_fasta_parse(text, len(text), None, 0, ctypes.byref(n_out), None, None, 0,
                               ctypes.byref(n_rec)) == 0
    assert (n_out.value, n_rec.value) == (6, 2)
    small = (ctypes.c_uint8 * 3)()
    off = (ctypes.c_uint64 * 3)()
    assert lib.dna_fasta_parse(text, len(text), small, 3, ctypes.byref(n_out), off, None, 3,
                               ctypes.byref(n_rec)) == -3
    assert n_out.value == 6
    off2 = (ctypes.c_uint64 * 2)()
    big = (ctypes.c_uint8 * 8)()
    assert lib.dna_fasta_parse(text, len(text), big, 8, ctypes.byref(n_out), off2, None, 2,
                               ctypes.byref(n_rec)) == -3


def test_argument_errors_are_reported_before_any_device_work():
    """Invalid arguments return DNA_ERR_INVALID_ARG synchronously, from checks that run
    before any CUDA call, so they hold with or without a GPU: an entry that names no
    state, zero or too many states, null pointers, an empty batch or request loop."""
    L = dna.lib()
    p = ctypes.c_void_p
    out = p()
    good = np.array([[0, 1, 0, 0], [0, 1, 0, 0]], np.uint32)   # next state = f(symbol)
    bad = good.copy()
    bad[1, 2] = 2                      # names state 2 of a 2-state table
    acc = np.array([2], np.uint8)
    cases = [
        L.dfa_load(bad.ctypes.data, 2, acc.ctypes.data, ctypes.byref(out)),
        L.dfa_load(good.ctypes.data, 0, acc.ctypes.data, ctypes.byref(out)),
        L.dfa_load(good.ctypes.data, (1 << 24) + 1, acc.ctypes.data, ctypes.byref(out)),
        L.dfa_load(None, 2, acc.ctypes.data, ctypes.byref(out)),
        L.dfa_load(good.ctypes.data, 2, None, ctypes.byref(out)),
        L.dfa_load(good.ctypes.data, 2, acc.ctypes.data, None),
    ]
    depth = ctypes.c_int32()
    cases += [
        L.dfa_analyze(bad.ctypes.data, 2, ctypes.byref(depth)),
        L.dfa_analyze(good.ctypes.data, 0, ctypes.byref(depth)),
        L.dfa_info(None, None),
    ]
    cnt = np.zeros(1, np.uint64)
    seq = np.frombuffer(b"ACGT", np.uint8)
    cases += [
        L.dna_scan(None, seq.ctypes.data, 4, None, cnt.ctypes.data, None, 0),
        L.dna_scan_host(None, seq.ctypes.data, 4, None, cnt.ctypes.data, None, 0),
        L.dna_scan_count_static(None, seq.ctypes.data, 4, None, cnt.ctypes.data),
        L.dna_batch_create(None, 1, None, None, 1, None, None, ctypes.byref(out)),
        L.dna_scan_batch(None, 0, None, None, 0, None, None),
        L.dna_server_create(None, 1, None, ctypes.byref(out)),
    ]
    DNA_ERR_INVALID_ARG = -1   # include/dna_dfa.h
    assert cases == [DNA_ERR_INVALID_ARG] * len(cases)
    assert not out.value
    # the analysis itself needs no device: every symbol sends both states to one state,
    # so the table is 1-definite; with A as the identity it is not definite at all
    assert L.dfa_analyze(good.ctypes.data, 2, ctypes.byref(depth)) == 0 and depth.value == 1
    ident = np.array([[0, 1, 0, 0], [1, 1, 0, 0]], np.uint32)
    assert L.dfa_analyze(ident.ctypes.data, 2, ctypes.byref(depth)) == 0 and depth.value == -1
