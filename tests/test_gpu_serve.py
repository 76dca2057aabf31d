"""GPU tests of the request loop (dna_server_*): every request's count equals the
oracle's, both when the requests run alone (one slot, one at a time) and when they run
mixed (many slots, memory-capped admission, requests overlapping on the device); the
admission cap and the open-loop arrival schedule are honoured."""
import numpy as np
import pytest

import oracle
import paper_1509_01506_gb300 as dna
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20


def request_bytes(n):
    # the server's charge per request: the sequence rounded up to 4 KiB plus 1 MiB
    return ((n + 4095) // 4096) * 4096 + MiB


@pytest.fixture(scope="module")
def workload():
    pats = [("regex", p) for p in synth.random_regexes(21, 4)]
    pats += [("kmers", synth.random_kmers(22 + i, 12, 8, 16)) for i in range(4)]
    payload = synth.markov2(23, 48 * MiB)
    synth.overlay_runs(payload, 23, 0.05, 500.0, "lower")
    synth.overlay_runs(payload, 24, 0.01, 5000.0, "N")
    pinned = torch.from_numpy(payload).pin_memory()
    rng = np.random.default_rng(25)
    n_req = 120
    lens = synth.log_uniform_lengths(26, n_req, 4 * KiB, 4 * MiB)
    offs = [int(rng.integers(0, payload.size - n)) for n in lens]
    dfa_idx = rng.integers(0, len(pats), n_req).tolist()
    tables = [oracle.compile_regex(p) if k == "regex" else oracle.compile_kmers(p, minimise=True)
              for k, p in pats]
    want = [oracle.run(*tables[d], payload[o:o + int(n)], positions=False)[0]
            for o, n, d in zip(offs, lens, dfa_idx)]
    dfas = [dna.Dfa.from_regex(p) if k == "regex" else dna.Dfa.from_kmers(p) for k, p in pats]
    return pinned, lens, offs, dfa_idx, want, dfas


def run_server(workload, slots, cap, arrivals=None):
    pinned, lens, offs, dfa_idx, _, dfas = workload
    srv = dna.Server(dfas, slots=slots, mem_cap_bytes=cap)
    base = pinned.data_ptr()
    out = {}
    for i, (o, n, d) in enumerate(zip(offs, lens, dfa_idx)):
        rid = srv.submit((base + o, int(n)), d, 0 if arrivals is None else arrivals[i])
        out[rid] = i
        if slots == 1 and arrivals is None:
            srv.drain()     # alone: the next request is submitted after this one finished
    srv.drain()
    comps = srv.poll(max_items=len(lens) + 8)
    assert len(comps) == len(lens)
    srv.free()
    res = [None] * len(lens)
    for c in comps:
        res[out[c["id"]]] = c
    return res


def test_results_alone_and_in_the_mix_equal_the_oracle(workload):
    _, lens, _, _, want, _ = workload
    alone = run_server(workload, slots=1, cap=1 << 30)
    cap = 24 * MiB
    mix = run_server(workload, slots=8, cap=cap)
    assert [c["status"] for c in alone] == [0] * len(lens)
    assert [c["status"] for c in mix] == [0] * len(lens)
    assert [c["count"] for c in alone] == want
    assert [c["count"] for c in mix] == want
    # the mix overlapped requests on the device, and never admitted more than the cap
    ev = sorted([(c["admit_ns"], request_bytes(c["len"])) for c in mix] +
                [(c["done_ns"], -request_bytes(c["len"])) for c in mix], key=lambda x: (x[0], x[1]))
    in_use = peak = conc = max_conc = 0
    for _, b in ev:
        in_use += b
        conc += 1 if b > 0 else -1
        peak = max(peak, in_use)
        max_conc = max(max_conc, conc)
    assert peak <= cap
    assert max_conc >= 2


def test_open_loop_arrivals_are_honoured(workload):
    _, lens, _, _, want, _ = workload
    rng = np.random.default_rng(27)
    t0 = dna.Server.now_ns() + 20_000_000
    arrivals = (t0 + np.cumsum(rng.exponential(1e9 / 2000.0, len(lens)))).astype(np.int64).tolist()
    res = run_server(workload, slots=4, cap=1 << 30, arrivals=arrivals)
    assert [c["count"] for c in res] == want
    assert all(c["admit_ns"] >= c["arrival_ns"] for c in res)
    assert all(c["done_ns"] >= c["admit_ns"] for c in res)


def test_request_larger_than_the_cap_fails_alone(workload):
    pinned, _, _, _, _, dfas = workload
    srv = dna.Server(dfas[:1], slots=2, mem_cap_bytes=4 * MiB)
    big = srv.submit((pinned.data_ptr(), 8 * MiB), 0)
    small = srv.submit((pinned.data_ptr(), 64 * KiB), 0)
    srv.drain(timeout_ms=20000)
    comps = {c["id"]: c for c in srv.poll(16)}
    assert comps[big]["status"] == -3
    assert comps[small]["status"] == 0
    payload = pinned[:64 * KiB].numpy()
    t, a = oracle.compile_regex(synth.random_regexes(21, 1)[0])
    assert comps[small]["count"] == oracle.run(t, a, payload, positions=False)[0]
    srv.free()
    with pytest.raises(dna.DnaError):
        s2 = dna.Server(dfas[:1])
        try:
            s2.submit((pinned.data_ptr(), 100), 5)
        finally:
            s2.free()


def test_request_loop_with_a_chunk_map_automaton(workload):
    """A never-converging automaton (chunk maps) served among ordinary ones."""
    pinned, lens, offs, dfa_idx, want, dfas = workload
    rng = np.random.default_rng(91)
    table = np.stack([rng.permutation(6) for _ in range(4)], axis=1).astype(np.uint32)
    acc = np.array([0, 1, 0, 0, 1, 0], np.uint8)
    perm = dna.Dfa(table, dna.pack_accept(acc))
    assert perm.info().chunk_maps
    srv = dna.Server(dfas + [perm], slots=4)
    base = pinned.data_ptr()
    payload = pinned.numpy()
    ids = {}
    for i in range(30):
        o, n = int(offs[i]), int(lens[i])
        ids[srv.submit((base + o, n), len(dfas))] = (o, n)
    srv.drain()
    comps = srv.poll(64)
    srv.free()
    assert len(comps) == 30
    for c in comps:
        o, n = ids[c["id"]]
        assert c["status"] == 0
        assert c["count"] == oracle.run(table.astype(np.int32), acc, payload[o:o + n], positions=False)[0]


def test_drain_with_a_short_limit_times_out_and_a_later_drain_completes(workload):
    """dna_server_drain's limit: with a 40 MiB request on the device and a second one
    not due for another 300 ms, a 1 ms drain returns DNA_ERR_TIMEOUT (the server keeps
    running); a drain without a limit then finishes both, with the oracle's counts."""
    pinned, _, _, _, _, dfas = workload
    payload = pinned.numpy()
    n = 40 * MiB
    srv = dna.Server(dfas[:1], slots=2)
    base = pinned.data_ptr()
    first = srv.submit((base, n), 0)
    second = srv.submit((base + 4096, n), 0, dna.Server.now_ns() + 300_000_000)
    with pytest.raises(dna.DnaError) as err:
        srv.drain(timeout_ms=1)
    assert err.value.code == -4 and dna.status_string(-4) == "device wait timed out"
    st = srv.stats()
    assert st["submitted"] == 2 and st["completed"] < 2
    srv.drain()
    comps = {c["id"]: c for c in srv.poll(8)}
    srv.free()
    assert set(comps) == {first, second}
    t, a = oracle.compile_regex(synth.random_regexes(21, 1)[0])
    for rid, off in ((first, 0), (second, 4096)):
        assert comps[rid]["status"] == 0
        assert comps[rid]["count"] == oracle.run(t, a, payload[off:off + n], positions=False)[0]
    assert comps[second]["admit_ns"] >= comps[second]["arrival_ns"]


def test_bench_serving_sample_equals_the_oracle():
    """A seeded sample of 64 requests of the bench's serving workload (the 16 resident
    automata, the 256 MiB soft-masked payload with N runs, the largest requests near
    64 MiB included), served through the request loop, gives the oracle's counts."""
    w = synth.serving(n_states=lambda km: dna.compile_kmers(km)[0].shape[0])
    lens, offs, didx = w["lens"], w["offs"], w["didx"]
    rng = np.random.default_rng(77)
    pick = set(np.argsort(lens)[-8:].tolist())                 # the largest requests
    for k in range(16):                                         # one of every automaton
        pick.add(int(np.flatnonzero(didx == k)[0]))
    while len(pick) < 64:
        pick.add(int(rng.integers(0, len(lens))))
    pick = sorted(pick)
    assert max(lens[i] for i in pick) > 60 * MiB
    pinned = torch.from_numpy(w["payload"]).pin_memory()
    dfas, tables = [], []
    for kind, pat in w["patterns"]:
        if kind == "kmers":
            dfas.append(dna.Dfa.from_kmers(pat))
            tables.append(oracle.compile_kmers(pat, minimise=True))
        else:
            dfas.append(dna.Dfa.from_regex(pat))
            tables.append(oracle.compile_regex(pat))
    srv = dna.Server(dfas, slots=8)
    ids = {}
    for i in pick:
        ids[srv.submit((pinned.data_ptr() + int(offs[i]), int(lens[i])), int(didx[i]))] = i
    srv.drain()
    comps = srv.poll(256)
    srv.free()
    assert len(comps) == len(pick)
    payload = w["payload"]
    for c in comps:
        i = ids[c["id"]]
        assert c["status"] == 0
        want = oracle.run(*tables[int(didx[i])], payload[int(offs[i]):int(offs[i]) + int(lens[i])], positions=False)[0]
        assert c["count"] == want, (i, int(lens[i]), int(didx[i]))
