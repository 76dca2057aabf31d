"""The allocation-free count (dna_scan_count_static) against the allocating scan.

Some callers cannot let a library allocate device memory while they run (a server that
has reserved the GPU's memory up front, code that must not trigger the synchronisation an
allocation can cause). dna_scan_count_static serves them with one fixed scratch array in
device memory instead of stream-ordered scratch. This file is named so that pytest
collects it last; it passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import paper_1509_01506_gb300 as dna
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


def _inputs():
    a = synth.markov2(41, 24 * MiB + 333)
    synth.overlay_runs(a, 41, 0.05, 400.0, "lower")
    synth.overlay_runs(a, 42, 0.01, 300.0, "N")
    b = synth.uniform(43, 3 * MiB + 5)
    return a, b


def _permutation_automaton(Q, seed):
    """An automaton whose runs from different states never meet (each column a
    permutation): dfa_load gives it chunk maps."""
    rng = np.random.default_rng(seed)
    table = np.stack([rng.permutation(Q) for _ in range(4)], axis=1).astype(np.uint32)
    acc = (rng.random(Q) < 0.3).astype(np.uint8)
    acc[int(rng.integers(0, Q))] = 1
    return dna.Dfa(table, dna.pack_accept(acc))


def _static_counts(automaton, seqs, stream):
    """Two (or more) calls in a row on one stream; returns the count tensors and the
    library's allocation counter before and after the calls."""
    got = [torch.full((1,), -1, dtype=torch.int64, device="cuda") for _ in seqs]
    torch.cuda.synchronize()
    before = dna.profile_read()["device_allocs"]
    for d, out in zip(seqs, got):
        rc = dna.lib().dna_scan_count_static(automaton.handle, d.data_ptr(), d.numel(),
                                             int(stream.cuda_stream), out.data_ptr())
        assert rc == 0, dna.status_string(rc)
    after = dna.profile_read()["device_allocs"]
    torch.cuda.synchronize()
    return [int(g.item()) for g in got], before, after


def test_static_scratch_count_matches_allocating_scan_twice():
    """Two calls in a row through the C ABI give the allocating scan's counts: the
    second call reuses the array the first one left behind. The library's count of its
    own device allocations does not move across the calls."""
    stream = torch.cuda.current_stream()
    dfa = dna.Dfa.from_regex(synth.CONFIG2_REGEX)
    kdfa = dna.Dfa.from_kmers(synth.random_kmers(44, 200, 10))
    a, b = _inputs()
    da = torch.from_numpy(a).cuda()
    db = torch.from_numpy(b).cuda()[1:]          # an unaligned start
    for automaton in (dfa, kdfa):
        want = []
        for d in (da, db):
            c, _ = dna.scan(automaton, d, stream=stream)
            want.append(int(c.item()))
        got, before, after = _static_counts(automaton, (da, db), stream)
        assert got == want
        assert after == before


@pytest.mark.parametrize("Q", [5, 8, 16, 32])
def test_static_scratch_with_chunk_map_automata(Q):
    """Automata whose runs never meet take the chunk-map kernels here too (as dna_scan
    does), with their maps in the fixed array: counts equal the allocating scan's on a
    small and a larger input, two calls in a row, with no allocation."""
    stream = torch.cuda.current_stream()
    perm = _permutation_automaton(Q, 500 + Q)
    assert perm.info().chunk_maps
    small = synth.uniform(45, 256 * 1024 + 3)
    big = synth.markov2(46, 40 * MiB + 17)
    synth.overlay_runs(big, 46, 0.01, 300.0, "N")
    ds = torch.from_numpy(small).cuda()[3:]
    db = torch.from_numpy(big).cuda()
    want = []
    for d in (ds, db):
        c, _ = dna.scan(perm, d, stream=stream)
        want.append(int(c.item()))
    got, before, after = _static_counts(perm, (ds, db), stream)
    assert got == want
    assert after == before


def test_static_scratch_rejects_lengths_beyond_its_limit():
    """A length above the stated maximum (2^36 bytes) is refused before any work is
    queued; no memory is touched, so a small buffer stands in for the sequence."""
    dfa = dna.Dfa.from_regex("TATAAA")
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = dna.lib().dna_scan_count_static(dfa.handle, buf.data_ptr(), (1 << 36) + 1,
                                         int(torch.cuda.current_stream().cuda_stream), out.data_ptr())
    assert rc == -3 and dna.status_string(rc) == "capacity exceeded"
    rc = dna.lib().dna_scan_count_static(dfa.handle, buf.data_ptr(), 0,
                                         int(torch.cuda.current_stream().cuda_stream), out.data_ptr())
    assert rc == 0
    torch.cuda.synchronize()
    assert int(out.item()) == 0
