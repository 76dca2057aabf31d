"""Benchmark of the GB300 DNA automaton scan (one JSON line on rank 0).

Workload (default): the plain scan of a 256 MiB order-2 Markov A/C/G/T sequence
(41% GC, seed 1) with the minimal DFA of ACG[AT]{2,6}C(G|T)T, returning the exact count
and all match positions. A step is one dna_scan call over the whole sequence: ingest,
speculation, chunk scan, join/repair and position extraction. The input (256 MiB) is
larger than L2 (129 MB), so consecutive steps do not hit a warm cache.

Arms:
  default            the library (CUDA kernels through the C ABI);
  --impl reference   the CPU oracle (plain single-threaded C) on a bounded sample of
                     the same workload, timed on the host cores.
Under torchrun (N > 1) every rank scans its own sequence (independent problems, no
collective): weak scaling, value = all ranks' bytes / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MiB = 1 << 20
SPACER_CYCLES = 400_000   # about 0.2 ms at 2 GHz
PLACEMENTS = ["auto", "smem pair", "smem one-symbol", "global one-symbol", "chunk maps", "smem hot-state rows",
              "smem one-symbol per lane"]
METRIC = "sequence GB/s scanned (count + positions)"
WORKLOAD = ("plain scan: 256 MiB order-2 Markov A/C/G/T (41% GC, seed 1), minimal DFA of "
            "ACG[AT]{2,6}C(G|T)T, exact count + all match positions")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bytes", type=int, default=256 * MiB)
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-runs", type=int, default=10)
    ap.add_argument("--batch-seqs", type=int, default=4096)
    ap.add_argument("--batch-dfas", type=int, default=64)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-percall", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-plain-configs", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=4000)
    ap.add_argument("--profile-case", default=None,
                    choices=["large_ac_512MiB", "map_perm8_256MiB", "map_perm64_64MiB", "batched_256x16"],
                    help="run one case a few times for a profiler capture and exit (no JSON line)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the scan kernel's source: its template and join (scan_kernel.cuh) and the
    device helpers it uses (dna_device.cuh). Host code does not change its traffic."""
    h = hashlib.sha256()
    for f in ("scan_kernel.cuh", "dna_device.cuh"):
        with open(os.path.join(ROOT, "paper_1509_01506_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the scan kernel from the committed ncu summary, or None
    when the kernel source changed since that capture."""
    path = os.path.join(ROOT, "profiles", "scan_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("kernel_source_sha256_16") != kernel_source_hash():
            return None
        return float(rec["dram_bytes_per_launch_full"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None,
                "reasons": sorted(reasons), "samples": len(sms)}


def host_cpu() -> dict:
    """The host's logical CPU count and CPU model (lscpu 'Model name', else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"host_cores": os.cpu_count(), "cpu_model": model or "unknown"}


def cpu_oracle_rate(seq: np.ndarray, pattern: str, seconds: float):
    """The oracle (single-threaded C) on consecutive 32 MiB slices of the workload until
    'seconds' have elapsed; returns (GB/s, bytes scanned)."""
    import oracle
    t, a = oracle.compile_regex(pattern)
    slice_bytes = 32 * MiB
    done, t0 = 0, time.perf_counter()
    i = 0
    while True:
        lo = (i * slice_bytes) % seq.size
        part = seq[lo:lo + slice_bytes]
        oracle.run(t, a, part, positions=True, cap=1 << 16)
        done += part.size
        i += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return done / el / 1e9, done


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    # a bounded sample per step, so that the whole run stays near half a minute of oracle
    # work (about 12 GB at the oracle's 0.3-0.5 GB/s) whatever --steps is
    n = int(min(args.bytes, 64 * MiB, max(256 * 1024, 12e9 // max(1, args.steps))))
    seq, pattern = synth.plain_markov(args.bytes)
    seq = seq[:n]
    import oracle
    t, a = oracle.compile_regex(pattern)
    for _ in range(args.warmup):
        oracle.run(t, a, seq[:MiB], positions=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(t, a, seq, positions=True, cap=1 << 16)
    el = time.perf_counter() - t0
    gbs = n * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": WORKLOAD, "bytes_per_step": n,
                                        "sample": f"first {n} bytes of the workload per step"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n} bytes of the 256 MiB sequence per step", **host_cpu()},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


BATCH_WORKLOAD = ("batched: 4,096 i.i.d. A/C/G/T sequences, lengths log-uniform 1 KiB..16 MiB (seed 3), "
                  "x 64 minimised motif regexes of 5-60 states; per-(sequence, automaton) exact counts")


def lds_lookup_peak(sms: int, mhz: float) -> float:
    """Shared-memory lookups per second the SMs can issue: one 32-lane LDS wavefront per
    SM per clock (bank-conflict free)."""
    return sms * 32 * mhz * 1e6


def cpu_batched_rate(buf, offs, regexes, seconds: float):
    """The oracle (unchanged, single-threaded C) over independent (sequence, automaton)
    pairs of the batched workload, one pair per task on every host core (ctypes releases
    the GIL during each run). Sequences are taken in a seeded random order, each against
    all automata, until 'seconds' have elapsed. Returns the (sequence x automaton) GB/s,
    the threads used and the sample."""
    import concurrent.futures as cf
    import oracle
    tables = [oracle.compile_regex(r) for r in regexes]
    order = np.random.Generator(np.random.PCG64(3)).permutation(offs.size - 1)
    threads = os.cpu_count() or 1
    done_bytes, pairs, seqs = 0, 0, 0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        for si in order:
            part = buf[int(offs[si]):int(offs[si + 1])]
            futs = [ex.submit(oracle.run, t, a, part, False) for t, a in tables]
            for f in futs:
                f.result()
            done_bytes += part.size * len(tables)
            pairs += len(tables)
            seqs += 1
            if time.perf_counter() - t0 >= seconds:
                break
    el = time.perf_counter() - t0
    return {"value": done_bytes / el / 1e9, "unit": "GB/s (sequence x automaton)", "cores": threads,
            "kind": "oracle", "sample": f"{seqs} sequences x {len(tables)} automata ({pairs} pairs, "
                                        f"{done_bytes / 1e9:.2f} GB of sequence x automaton) in a seeded random "
                                        f"order, one pair per task on {threads} threads", **host_cpu()}


def bench_batched(args, dna, torch, stream, clocks_mhz):
    """The batched configuration: one plan (autotuned, graph-captured), K timed runs;
    then the same pairs through one dna_scan call each."""
    import synth
    buf, offs, regexes = synth.batched(n_seqs=args.batch_seqs, n_dfas=args.batch_dfas,
                                       n_states=lambda r: dna.compile_regex(r)[0].shape[0])
    n_s = offs.size - 1
    lens = [int(offs[i + 1] - offs[i]) for i in range(n_s)]
    total = int(offs[-1])
    dbuf = torch.empty(total + 256 * n_s, dtype=torch.uint8, device="cuda")
    hbuf = torch.from_numpy(buf)
    starts, pos = [], 0
    for i in range(n_s):
        dbuf[pos:pos + lens[i]].copy_(hbuf[int(offs[i]):int(offs[i + 1])])
        starts.append(dbuf.data_ptr() + pos)
        pos += (lens[i] + 255) // 256 * 256
    del hbuf
    cpu_batched = None
    if not args.no_cpu_baseline:
        cpu_batched = cpu_batched_rate(buf, offs, regexes, args.cpu_seconds)
    del buf
    dfas = [dna.Dfa.from_regex(r) for r in regexes]
    states = [d.info().n_states for d in dfas]
    t0 = time.perf_counter()
    plan = dna.Batch(dfas, starts, lens=lens, autotune=True, use_graph=True, stream=stream)
    tune_s = time.perf_counter() - t0
    info = plan.info()
    out = torch.empty((n_s, len(dfas)), dtype=torch.int64, device="cuda")
    for _ in range(3):
        plan.run(out, stream=stream)
    torch.cuda.synchronize()
    dna.profile_read(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batch_runs):
        plan.run(out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = dna.profile_read(reset=True)["kernel_launches"]
    ms = e0.elapsed_time(e1) / args.batch_runs
    # kernel times from a separate pass with events around each launch (a graph replay
    # records no per-launch events, so this pass uses the same plan without a graph)
    plain = dna.Batch(dfas, starts, lens=lens, chunk_bases=info.chunk_bases,
                      warps_per_cta=info.warps_per_cta, stream=stream)
    plain.run(out, stream=stream)
    torch.cuda.synchronize()
    dna.profile_read(reset=True)
    dna.profile_enable(True)
    for _ in range(3):
        plain.run(out, stream=stream)
    torch.cuda.synchronize()
    dna.profile_enable(False)
    prof = dna.profile_read(reset=True)
    plain.free()
    k_ms = prof["batch_kernel_ms"] / max(1, prof["batch_kernel_calls"])
    i_ms = prof["ingest_kernel_ms"] / max(1, prof["ingest_kernel_calls"])
    counts = out.cpu().numpy()
    res = {
        "workload": BATCH_WORKLOAD, "n_seqs": n_s, "n_dfas": len(dfas), "bytes": total,
        "states_min": min(states), "states_max": max(states),
        "plan": {"chunk_bases": info.chunk_bases, "warps_per_cta": info.warps_per_cta, "grid": info.grid,
                 "groups_per_task": info.groups_per_task, "n_fast": info.n_fast, "n_slow": info.n_slow,
                 "autotune_s": tune_s, "graph": True},
        "runs": args.batch_runs, "ms_per_run": ms, "gpu_launches_per_run": launches / args.batch_runs,
        "unique_gbs": total / (ms * 1e-3) / 1e9,
        "seq_x_dfa_gbs": total * len(dfas) / (ms * 1e-3) / 1e9,
        "ingest_ms": i_ms, "batch_kernel_ms": k_ms,
        "total_matches": int(counts.sum()),
        "cpu_baseline": cpu_batched,
    }
    # the method's unit: one transition per base per automaton; the kernel takes them two at
    # a time (one two-symbol lookup per 2 bases per automaton, each lane in its own bank),
    # so its peak is twice the measured conflict-free lookup rate
    peak_lk = dna.lookup_peak(0, stream=stream)
    transitions = total * info.n_fast
    res["roofline"] = {"bound": "alu", "unit": "transitions/s", "achieved": transitions / (k_ms * 1e-3),
                       "peak": 2 * peak_lk, "frac": transitions / (k_ms * 1e-3) / (2 * peak_lk),
                       "lookups_per_s": transitions * 0.5 / (k_ms * 1e-3), "lookup_peak": peak_lk,
                       "peak_source": "dna_lookup_peak mode 0 (measured: shared-memory lookups with no bank "
                                      "conflict, 8 chains per thread, one full block per SM) x 2 transitions "
                                      "per two-symbol lookup",
                       "derived_peak_for_context": lds_lookup_peak(
                           torch.cuda.get_device_properties(0).multi_processor_count, clocks_mhz or 2070.0)}
    if not args.no_percall:
        # the same pairs, one dna_scan (count only) per (sequence, automaton)
        cnt = torch.empty((n_s, len(dfas)), dtype=torch.int64, device="cuda")
        sh = int(stream.cuda_stream)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        c0.record(stream)
        base = cnt.data_ptr()
        for si in range(n_s):
            for k, d in enumerate(dfas):
                dna.scan_ptr(d, starts[si], lens[si], base + 8 * (si * len(dfas) + k), sh)
        c1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        pc_ms = c0.elapsed_time(c1)
        same = bool(torch.equal(cnt, out))
        res["per_call"] = {"calls": n_s * len(dfas), "ms": pc_ms, "wall_s": wall,
                           "seq_x_dfa_gbs": total * len(dfas) / (pc_ms * 1e-3) / 1e9,
                           "identical_counts": same}
        res["batched_over_per_call"] = pc_ms / ms
    plan.free()
    del dbuf
    torch.cuda.empty_cache()
    return res



SERVE_WORKLOAD = ("serving: Poisson arrivals at 2,000 req/s (seed 4), lengths log-uniform 4 KiB..64 MiB, "
                  "slices of a 256 MiB order-2 Markov sequence with soft-masked and N runs in pinned host "
                  "memory; 16 resident automata (8 Aho-Corasick sets of 8-16-mers <= 500 states, 8 motif "
                  "regexes); 8 slots, 40 GiB admission cap")


def serve_automata(dna, patterns):
    """The 16 resident automata of the serving workload (synth.serving's pattern sets)."""
    dfas, kinds = [], []
    for kind, pat in patterns:
        d = dna.Dfa.from_kmers(pat) if kind == "kmers" else dna.Dfa.from_regex(pat)
        dfas.append(d)
        kinds.append((kind, len(pat) if kind == "kmers" else pat, d.info().n_states))
    return dfas, kinds


def run_served(dna, dfas, base, lens, offs, didx, arrivals, slots=8):
    """Submits every request (host slices of the pinned payload at 'base') with its
    arrival time and drains; returns the completions in request order."""
    n_req = len(lens)
    srv = dna.Server(dfas, slots=slots, mem_cap_bytes=40 << 30)
    for i in range(16):   # first-call set-up of each kernel variant on the slots
        srv.submit((base, 1 << 20), i % len(dfas))
    srv.drain()
    srv.poll(64)
    ids = {}
    for i in range(n_req):
        ids[srv.submit((base + int(offs[i]), int(lens[i])), int(didx[i]), int(arrivals[i]))] = i
    srv.drain()
    comps = srv.poll(max_items=n_req + 16)
    srv.free()
    assert len(comps) == n_req
    res = [None] * n_req
    for c in comps:
        res[ids[c["id"]]] = c
    return res


def serve_stats(res, lens):
    lat = np.array([(c["done_ns"] - c["arrival_ns"]) / 1e6 for c in res])
    lat_noh2d = np.array([(c["done_ns"] - c["arrival_ns"]) / 1e6 - c["h2d_us"] / 1e3 for c in res])
    dev = np.array([c["device_us"] / 1e3 for c in res])
    span_s = (max(c["done_ns"] for c in res) - min(c["arrival_ns"] for c in res)) / 1e9
    ev = sorted([(c["admit_ns"], 1) for c in res] + [(c["done_ns"], -1) for c in res])
    conc = peak = 0
    for _, d in ev:
        conc += d
        peak = max(peak, conc)
    return {"gbs": int(lens.sum()) / span_s / 1e9, "span_s": span_s,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p50_ms_without_h2d": float(np.percentile(lat_noh2d, 50)),
            "p99_ms_without_h2d": float(np.percentile(lat_noh2d, 99)),
            "device_p50_ms": float(np.percentile(dev, 50)), "device_p99_ms": float(np.percentile(dev, 99)),
            "max_concurrent": peak, "all_ok": all(c["status"] == 0 for c in res)}


def bench_serve(args, dna, torch):
    """The serving workload at its Poisson rate (2,000 req/s), then overloaded (every
    request queued at once: the loop's capacity), then the same requests one at a time
    through dna_scan_host (the per-call path); counts must agree across all three and
    with one dna_scan of each slice. (A seeded sample of these requests, 64 MiB ones and
    every automaton included, is checked against the oracle by
    tests/test_gpu_serve.py::test_bench_serving_sample_equals_the_oracle.)"""
    import synth
    w = synth.serving(n_req=args.serve_requests, n_states=lambda km: dna.compile_kmers(km)[0].shape[0])
    pinned = torch.from_numpy(w["payload"]).pin_memory()
    dfas, kinds = serve_automata(dna, w["patterns"])
    lens, offs, didx, gaps = w["lens"], w["offs"], w["didx"], w["gaps_ns"]
    n_req = len(lens)
    total = int(lens.sum())
    base = pinned.data_ptr()
    t0 = dna.Server.now_ns() + 50_000_000
    poisson = run_served(dna, dfas, base, lens, offs, didx, (t0 + np.cumsum(gaps)).astype(np.int64))
    t1 = dna.Server.now_ns() + 20_000_000
    overload = run_served(dna, dfas, base, lens, offs, didx, np.full(n_req, t1, np.int64))
    # the per-call path: the same requests one after another through dna_scan_host
    stream = torch.cuda.current_stream()
    cnt = np.zeros(1, np.uint64)
    payload = w["payload"]
    for i in range(8):
        dna.scan_host(dfas[int(didx[i])], pinned[int(offs[i]):int(offs[i]) + int(lens[i])], stream=stream,
                      out_count=cnt)
    serial_counts = np.empty(n_req, np.int64)
    s0 = time.perf_counter()
    for i in range(n_req):
        c, _ = dna.scan_host(dfas[int(didx[i])], pinned[int(offs[i]):int(offs[i]) + int(lens[i])],
                             stream=stream, out_count=cnt)
        serial_counts[i] = c
    serial_s = time.perf_counter() - s0
    # every count against one dna_scan of the same slice on the device
    dpay = pinned.cuda()
    out = torch.empty(n_req, dtype=torch.int64, device="cuda")
    sh = int(stream.cuda_stream)
    for i in range(n_req):
        dna.scan_ptr(dfas[int(didx[i])], dpay.data_ptr() + int(offs[i]), int(lens[i]), out.data_ptr() + 8 * i, sh)
    torch.cuda.synchronize()
    single = out.cpu().numpy()
    del dpay, payload
    pc = np.array([c["count"] for c in poisson], np.int64)
    oc = np.array([c["count"] for c in overload], np.int64)
    p_stats, o_stats = serve_stats(poisson, lens), serve_stats(overload, lens)
    res = {"workload": SERVE_WORKLOAD, "requests": n_req, "bytes": total,
           "offered_gbs": total / (float(gaps.sum()) / 1e9) / 1e9}
    res.update(p_stats)
    res["capacity"] = {"gbs": o_stats["gbs"], "span_s": o_stats["span_s"], "all_ok": o_stats["all_ok"],
                       "max_concurrent": o_stats["max_concurrent"],
                       "p50_ms": o_stats["p50_ms"], "p99_ms": o_stats["p99_ms"],
                       "note": "every request queued at once; latencies include the queueing"}
    res["serial"] = {"gbs": total / serial_s / 1e9, "s": serial_s,
                     "api": "dna_scan_host, one request after another (pinned host slices)"}
    res["served_over_serial"] = o_stats["gbs"] / (total / serial_s / 1e9)
    res["identical_to_single_calls"] = bool(np.array_equal(pc, single) and np.array_equal(oc, single)
                                            and np.array_equal(serial_counts, single))
    res["automata_states"] = [k[2] for k in kinds]
    res["oracle_checked_by"] = "tests/test_gpu_serve.py::test_bench_serving_sample_equals_the_oracle"
    return res



def bench_plain_configs(dna, torch, stream, peak):
    """The other plain workloads: 1 MiB i.i.d. with TATAAA (count + positions; launch-bound
    at this size) and 3.2 GiB with soft-masked and N runs against the Aho-Corasick
    automaton of 1,000 random 12-mers (count only)."""
    import synth
    out = {}

    def timed(fn, steps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def kernel_ms(fn, steps):
        dna.profile_read(reset=True)
        dna.profile_enable(True)
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        dna.profile_enable(False)
        pr = dna.profile_read(reset=True)
        return pr["scan_kernel_ms"] / max(1, pr["scan_kernel_calls"])

    seq, motif = synth.plain_small()
    dfa = dna.Dfa.from_regex(motif)
    d = torch.from_numpy(seq).cuda()
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    pos = torch.empty(1 << 12, dtype=torch.int64, device="cuda")
    fn = lambda: dna.scan(dfa, d, positions=True, stream=stream, out_count=cnt, out_positions=pos)
    ms = timed(fn, 2000)
    out["small_1MiB_TATAAA"] = {"bytes": int(seq.size), "ms_per_step": ms, "gbs": seq.size / (ms * 1e-3) / 1e9,
                                "matches": int(cnt.item()), "output": "count + positions",
                                "note": "launch-bound: two kernels of about 10 us each"}
    del d
    # an automaton whose runs never meet (an 8-state permutation table): chunk maps
    full, _ = synth.plain_markov(256 * MiB)
    rng = np.random.Generator(np.random.PCG64(8))
    table = np.stack([rng.permutation(8) for _ in range(4)], axis=1).astype(np.uint32)
    acc = (rng.random(8) < 0.25).astype(np.uint8)
    acc[0] = 0
    acc[int(rng.integers(1, 8))] = 1
    dfa = dna.Dfa(table, dna.pack_accept(acc))
    d = torch.from_numpy(full).cuda()
    fn = lambda: dna.scan(dfa, d, stream=stream, out_count=cnt)
    ms = timed(fn, 10)
    out["nonconverging_256MiB_perm8"] = {
        "bytes": int(full.size), "ms_per_step": ms, "gbs": full.size / (ms * 1e-3) / 1e9,
        "matches": int(cnt.item()), "chunk_maps": bool(dfa.info().chunk_maps), "output": "count",
        "note": "runs from different states never meet: every chunk is run from all 8 states, "
                "held as 4-bit fields of one register per lane and moved by byte permutes"}
    # 16 states whose runs never meet: every run as a 4-bit field of two registers per lane
    rng = np.random.Generator(np.random.PCG64(16))
    table = np.stack([rng.permutation(16) for _ in range(4)], axis=1).astype(np.uint32)
    acc = (rng.random(16) < 0.25).astype(np.uint8)
    acc[0] = 0
    acc[int(rng.integers(1, 16))] = 1
    dfa16 = dna.Dfa(table, dna.pack_accept(acc))
    fn = lambda: dna.scan(dfa16, d, stream=stream, out_count=cnt)
    ms = timed(fn, 10)
    out["nonconverging_256MiB_perm16"] = {
        "bytes": int(full.size), "ms_per_step": ms, "gbs": full.size / (ms * 1e-3) / 1e9,
        "matches": int(cnt.item()), "chunk_maps": bool(dfa16.info().chunk_maps), "output": "count",
        "note": "16 states whose runs never meet: every run a 4-bit field of two registers per lane; "
                "each lookup picks between the rows of states 0-7 and 8-15"}
    # 64 states whose runs never meet: two warps per chunk, one per block of 32 start states
    rng = np.random.Generator(np.random.PCG64(64))
    table = np.stack([rng.permutation(64) for _ in range(4)], axis=1).astype(np.uint32)
    acc = (rng.random(64) < 0.25).astype(np.uint8)
    acc[0] = 0
    acc[int(rng.integers(1, 64))] = 1
    dfa64 = dna.Dfa(table, dna.pack_accept(acc))
    fn = lambda: dna.scan(dfa64, d, stream=stream, out_count=cnt)
    ms = timed(fn, 5)
    out["nonconverging_256MiB_perm64"] = {
        "bytes": int(full.size), "ms_per_step": ms, "gbs": full.size / (ms * 1e-3) / 1e9,
        "matches": int(cnt.item()), "chunk_maps": bool(dfa64.info().chunk_maps), "output": "count",
        "note": "64 states whose runs never meet: every chunk is run from all 64 states by two warps"}
    # the nine Table V expressions as one labelled automaton: a count per expression from
    # one scan (the extraction pass walks every row with a match and adds its labels)
    lab_dfa = dna.Dfa.from_regex_set(synth.REGEX_DNA_TABLE_V)
    lab_counts = torch.empty(9, dtype=torch.int64, device="cuda")
    lh = int(stream.cuda_stream)

    def lab_step():
        rc = dna.lib().dna_scan_labels(lab_dfa.handle, d.data_ptr(), d.numel(), lh, cnt.data_ptr(),
                                       lab_counts.data_ptr(), None, None, 0)
        assert rc == 0
    ms = timed(lab_step, 10)
    sep = [dna.Dfa.from_regex(p) for p in synth.REGEX_DNA_TABLE_V]
    sep_cnt = torch.empty(9, dtype=torch.int64, device="cuda")

    def sep_step():
        for k, sd in enumerate(sep):
            dna.scan_ptr(sd, d.data_ptr(), d.numel(), sep_cnt.data_ptr() + 8 * k, lh)
    ms_sep = timed(sep_step, 10)
    per = lab_counts.cpu().tolist()
    out["regex_dna_table_v_labels_256MiB"] = {
        "bytes": int(full.size), "ms_per_step": ms, "gbs": full.size / (ms * 1e-3) / 1e9,
        "matches": int(cnt.item()), "per_expression": per, "n_states": lab_dfa.info().n_states,
        "output": "count per expression (9 labels) from one scan",
        "nine_separate_scans_ms": ms_sep, "identical_to_separate_scans": per == sep_cnt.cpu().tolist()}
    del d, full
    seq, kmers = synth.plain_large()
    dfa = dna.Dfa.from_kmers(kmers)
    info = dfa.info()
    d = torch.from_numpy(seq).cuda()
    n = seq.size
    del seq
    fn = lambda: dna.scan(dfa, d, stream=stream, out_count=cnt)
    ms = timed(fn, 10)
    kms = kernel_ms(fn, 5)
    # the same scan with the one-symbol table in L2 (the placement of automata too large for
    # shared memory), and the measured lookup peaks each placement is bound by
    fn_g = lambda: dna.scan(dfa, d, stream=stream, out_count=cnt, plan=dict(placement=3))
    kms_g = kernel_ms(fn_g, 3)
    lk_smem, lk_l2 = dna.lookup_peak(1, stream=stream), dna.lookup_peak(2, stream=stream)
    out["large_3_2GiB_AC1000"] = {
        "bytes": n, "ms_per_step": ms, "gbs": n / (ms * 1e-3) / 1e9, "matches": int(cnt.item()),
        "n_states": info.n_states, "placement": PLACEMENTS[info.placement],
        "kernel_ms": kms, "hbm_frac": n / (kms * 1e-3) / 1e9 / peak, "output": "count",
        "lookup_roofline": {"unit": "lookups/s", "achieved": n / (kms * 1e-3), "peak": lk_smem,
                            "frac": n / (kms * 1e-3) / lk_smem,
                            "peak_source": "dna_lookup_peak mode 1 (measured: shared-memory lookups at random "
                                           "banks)"},
        "global_placement": {"kernel_ms": kms_g, "gbs": n / (kms_g * 1e-3) / 1e9,
                             "lookups_per_s": n / (kms_g * 1e-3), "gather_peak": lk_l2,
                             "frac_of_gather_peak": n / (kms_g * 1e-3) / lk_l2,
                             "peak_source": "dna_lookup_peak mode 2 (measured: random 4-byte gathers from a "
                                            "128 KiB global table through L1/L2)"}}
    del d
    torch.cuda.empty_cache()
    return out



def profile_case(name):
    """One workload, a few launches, for an ncu capture (the profiles' commands)."""
    import torch
    import paper_1509_01506_gb300 as dna
    import synth
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    if name == "large_ac_512MiB":
        seq, kmers = synth.plain_large(n=512 * MiB)
        dfa = dna.Dfa.from_kmers(kmers)
        d = torch.from_numpy(seq).cuda()
        runs = [lambda: dna.scan(dfa, d, out_count=cnt, plan=dict(placement=2))] * 5
    elif name.startswith("map_perm"):
        q, n = (8, 256 * MiB) if name == "map_perm8_256MiB" else (64, 64 * MiB)
        rng = np.random.Generator(np.random.PCG64(q))
        table = np.stack([rng.permutation(q) for _ in range(4)], axis=1).astype(np.uint32)
        acc = (rng.random(q) < 0.25).astype(np.uint8)
        acc[0] = 0
        acc[int(rng.integers(1, q))] = 1
        dfa = dna.Dfa(table, dna.pack_accept(acc))
        d = torch.from_numpy(synth.plain_markov(n)[0]).cuda()
        runs = [lambda: dna.scan(dfa, d, out_count=cnt)] * 5
    else:   # batched_256x16: 256 sequences x 16 automata of the batched workload's recipe
        buf, offs, regexes = synth.batched(n_seqs=256, n_dfas=16,
                                           n_states=lambda r: dna.compile_regex(r)[0].shape[0])
        dbuf = torch.from_numpy(buf).cuda()
        lens = [int(offs[i + 1] - offs[i]) for i in range(offs.size - 1)]
        starts = [dbuf.data_ptr() + int(offs[i]) for i in range(offs.size - 1)]
        dfas = [dna.Dfa.from_regex(r) for r in regexes]
        plan = dna.Batch(dfas, starts, lens=lens, autotune=False)
        out = torch.empty((len(lens), len(dfas)), dtype=torch.int64, device="cuda")
        runs = [lambda: plan.run(out)] * 5
    for r in runs:
        r()
    torch.cuda.synchronize()
    print(f"{name}: done", flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_1509_01506_gb300 as dna
    from paper_1509_01506_gb300 import shard
    import synth

    seq_np, pattern = synth.plain_markov(args.bytes)
    n = seq_np.size
    dfa = dna.Dfa.from_regex(pattern)
    dseq = torch.from_numpy(seq_np).cuda()
    cap = 1 << 20
    out_count = torch.empty(1, dtype=torch.int64, device="cuda")
    out_pos = torch.empty(cap, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        dna.scan(dfa, dseq, positions=True, stream=stream, out_count=out_count,
                 out_positions=out_pos, capacity=cap)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n_matches = int(out_count.item())

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    sampler.start()
    time.sleep(0.3)
    dna.profile_enable(False)
    dna.profile_read(reset=True)          # zeroes the launch counter
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # a short device-side spacer before the start event: while it runs the host queues
    # the first steps, so the timed region holds the K steps back to back rather than the
    # first step waiting for its own launch from an idle host (the spacer is not timed)
    torch.cuda._sleep(SPACER_CYCLES)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    launches = dna.profile_read(reset=True)["kernel_launches"]
    clocks = sampler.stop()
    ms_total = ev0.elapsed_time(ev1)
    ms_total = shard.max_over_ranks(ms_total, device="cuda")   # the slowest rank
    ms_step = ms_total / args.steps
    value = n * world / (ms_step * 1e-3) / 1e9

    # ---- where a short run's time goes: the same number of steps (at most 50) after the
    # same idle pause, with an event pair around every step
    n_diag = max(1, min(args.steps, 50))
    torch.cuda.synchronize()
    time.sleep(0.3)
    dev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_diag)]
    for a, b in dev:
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    per_step_us = [a.elapsed_time(b) * 1e3 for a, b in dev]
    step_times = {"steps": n_diag, "first_us": per_step_us[0],
                  "median_us": statistics.median(per_step_us),
                  "max_us": max(per_step_us), "min_us": min(per_step_us),
                  "note": "device time of each step (events around it) after a 0.3 s idle pause"}

    # ---- the scan kernel's own time: a separate pass with per-launch events (the timed
    # region above runs without them)
    prof_steps = max(1, min(args.steps, 2000))
    dna.profile_enable(True)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    dna.profile_enable(False)
    prof = dna.profile_read(reset=True)
    emit_ms = prof["emit_kernel_ms"] / max(1, prof["emit_kernel_calls"])
    step_times["scan_kernel_us"] = prof["scan_kernel_ms"] / max(1, prof["scan_kernel_calls"]) * 1e3
    step_times["emit_kernel_us"] = emit_ms * 1e3
    ns = max(1, prof["conv_scans"])
    chunks = prof["conv_chunks"] / ns
    speculation = {
        "chunks_per_scan": chunks,
        "wrong_start_repaired_in_block": prof["conv_inblock"] / ns,
        "block_first_wrong_start": prof["conv_blockfirst"] / ns,
        "repaired_by_last_block": prof["conv_pending"] / ns,
        "last_state_changed": prof["conv_diverged"] / ns,
        "cascade_walks": prof["conv_cascade"] / ns,
        "wrong_start_fraction": (prof["conv_inblock"] + prof["conv_blockfirst"] + prof["conv_pending"]) / ns / max(1.0, chunks),
        "note": "q0 speculation; a wrong start is repaired where the runs meet (converging point)"}

    # ---- end to end through dna_scan_host: pinned host sequence in, count and positions
    # back in pinned host memory, every step (the call returns when they are on the host)
    host_in = torch.from_numpy(seq_np).pin_memory()
    host_count = torch.zeros(1, dtype=torch.int64).pin_memory()
    host_pos = torch.empty(cap, dtype=torch.int64).pin_memory()
    e2e_steps = max(1, args.e2e_steps)

    def e2e_step():
        return dna.scan_host(dfa, host_in, positions=True, stream=stream, out_count=host_count,
                             out_positions=host_pos)

    for _ in range(3):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c_host, _ = e2e_step()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    barrier()
    assert c_host == n_matches
    e2e_ms = shard.max_over_ranks(e2e_ms, device="cuda")
    e2e_value = n * world / (e2e_ms * 1e-3) / 1e9
    # the bound of the end-to-end number: the host link, timed as a plain copy of the same
    # pinned sequence into device memory (copy engine, CUDA events on the same stream)
    link_dst = torch.empty(n, dtype=torch.uint8, device="cuda")
    l0 = torch.cuda.Event(enable_timing=True)
    l1 = torch.cuda.Event(enable_timing=True)
    link_ms = []
    for r in range(6):
        l0.record(stream)
        link_dst.copy_(host_in, non_blocking=True)
        l1.record(stream)
        l1.synchronize()
        if r:
            link_ms.append(l0.elapsed_time(l1))
    del link_dst
    link_gbs = n / (statistics.median(link_ms) * 1e-3) / 1e9

    # ---- roofline of the dominant kernel (the chunk scan), timed live with events
    peak, peak_kind = load_peaks()
    kms = prof["scan_kernel_ms"] / max(1, prof["scan_kernel_calls"])
    achieved = n / (kms * 1e-3) / 1e9
    traffic = recorded_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": n, "kernel_ms": kms}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, done = cpu_oracle_rate(seq_np, pattern, args.cpu_seconds)
        cpu = {"value": rate, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{done / MiB:.0f} MiB scanned as 32 MiB slices of the 256 MiB workload "
                         f"(count + positions), single thread", **host_cpu()}

    plain_configs = None
    if world == 1 and not args.no_plain_configs:
        plain_configs = bench_plain_configs(dna, torch, stream, load_peaks()[0])

    batched = None
    if world == 1 and not args.no_batched:
        batched = bench_batched(args, dna, torch, stream, clocks.get("sm_mhz"))

    serve = None
    if world == 1 and not args.no_serve:
        serve = bench_serve(args, dna, torch)

    info = dfa.info()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "bytes_per_gpu": n, "n_states": info.n_states,
                       "definite_depth": info.definite_depth, "lookback": info.lookback,
                       "placement": info.placement, "matches": n_matches,
                       "l2": "inputs larger than L2 (256 MiB > 129 MB), no flush",
                       "timing": "CUDA events on the launching stream around the K steps; a 0.2 ms device "
                                 "spacer (torch.cuda._sleep) is queued before the start event so the first "
                                 "step does not wait untimed-but-counted for its host launch",
                       "parallelism": f"independent sequences on {world} GPU(s)",
                       "e2e_steps": e2e_steps},
            "roofline": roofline,
            "speculation": speculation,
            "step_times": step_times,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": n,
                    "d2h_bytes_per_step": 8 + 8 * n_matches, "ms_per_step": e2e_ms,
                    "api": "dna_scan_host (pinned host buffers, synchronous)",
                    "host_link_gbs": link_gbs, "frac_of_host_link": e2e_value / world / link_gbs,
                    "host_link_source": "cudaMemcpyAsync of the same pinned 256 MiB to the device, median of 5"},
            "gpu_launches": launches,
            "plain_configs": plain_configs,
            "batched": batched,
            "serve": serve,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
