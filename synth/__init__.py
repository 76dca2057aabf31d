"""Seeded synthetic DNA workloads, shared by the tests, the bench and the oracle leg.

This module produces input bytes and pattern strings only; it holds no automaton or
scan arithmetic. Sequences come from the C generators in ``gen.c`` (xoshiro256**),
pattern sets from numpy's PCG64 with fixed seeds. The recipes stand in for the
paper's GenBank genomes (Table IV: 0.19-3.25 GB) and regex-dna patterns (Table V),
which are not available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libsynth.so")
_lock = threading.Lock()
_lib = None

MiB = 1 << 20
GiB = 1 << 30


def build(force: bool = False) -> str:
    """Compiles gen.c into synth/_lib/libsynth.so (host code, portable C)."""
    src = os.path.join(_HERE, "gen.c")
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(src)):
        return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, dbl, p = ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.syn_uniform.argtypes = [u64, p, u64]
            lib.syn_uniform.restype = None
            lib.syn_markov2.argtypes = [u64, dbl, p, u64]
            lib.syn_markov2.restype = None
            lib.syn_markov2_params.argtypes = [u64, dbl, p]
            lib.syn_markov2_params.restype = None
            lib.syn_overlay_runs.argtypes = [u64, p, u64, dbl, dbl, ctypes.c_int]
            lib.syn_overlay_runs.restype = u64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def uniform(seed: int, n: int) -> np.ndarray:
    """i.i.d. uniform A/C/G/T bytes."""
    out = np.empty(n, dtype=np.uint8)
    if n:
        _load().syn_uniform(seed, _ptr(out), n)
    return out


def markov2(seed: int, n: int, gc: float = 0.41) -> np.ndarray:
    """Order-2 Markov A/C/G/T bytes with stationary GC fraction ``gc``."""
    out = np.empty(n, dtype=np.uint8)
    if n:
        _load().syn_markov2(seed, gc, _ptr(out), n)
    return out


def markov2_params(seed: int, gc: float = 0.41) -> np.ndarray:
    p = np.empty((16, 4), dtype=np.float64)
    _load().syn_markov2_params(seed, gc, _ptr(p))
    return p


def overlay_runs(seq: np.ndarray, seed: int, coverage: float, run_mean: float,
                 mode: str) -> int:
    """Paints runs in place: mode 'lower' soft-masks, mode 'N' writes N bytes."""
    assert seq.dtype == np.uint8 and seq.flags.c_contiguous
    m = {"lower": 0, "N": 1}[mode]
    return int(_load().syn_overlay_runs(seed, _ptr(seq), seq.size, coverage, run_mean, m))


# ----------------------------------------------------------------- pattern sets

_BASES = "ACGT"


def random_kmers(seed: int, count: int, k_lo: int, k_hi: int | None = None) -> list[str]:
    """``count`` distinct random k-mers with k uniform in [k_lo, k_hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k_hi = k_lo if k_hi is None else k_hi
    out, seen = [], set()
    while len(out) < count:
        k = int(rng.integers(k_lo, k_hi + 1))
        s = "".join(_BASES[i] for i in rng.integers(0, 4, size=k))
        if s not in seen:
            seen.add(s)
            out.append(s)
    return out


def random_motif_regex(rng: np.random.Generator) -> str:
    """A motif of 6-14 positions, each a literal base or a 2-3 base class, with up to
    two single-position bounded repeats {a,b} (b <= 4)."""
    k = int(rng.integers(6, 15))
    parts = []
    for _ in range(k):
        if rng.random() < 0.7:
            parts.append(_BASES[int(rng.integers(0, 4))])
        else:
            size = int(rng.integers(2, 4))
            cls = sorted(rng.choice(4, size=size, replace=False).tolist())
            parts.append("[" + "".join(_BASES[i] for i in cls) + "]")
    n_rep = int(rng.integers(0, 3))
    for pos in rng.choice(k, size=n_rep, replace=False).tolist():
        a = int(rng.integers(1, 3))
        b = int(rng.integers(a, 5))
        parts[pos] = parts[pos] + ("{%d}" % a if a == b else "{%d,%d}" % (a, b))
    return "".join(parts)


def random_regexes(seed: int, count: int) -> list[str]:
    rng = np.random.Generator(np.random.PCG64(seed))
    return [random_motif_regex(rng) for _ in range(count)]


def log_uniform_lengths(seed: int, count: int, lo: int, hi: int, align: int = 1) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    lens = np.maximum(lo, np.floor(x).astype(np.int64))
    if align > 1:
        lens = (lens // align) * align
    return lens


# --------------------------------------------------------------- the workloads

# Paper, Table V (regex-dna patterns E1..E9, each a forward form | its reverse
# complement), restated in this library's regex syntax.
REGEX_DNA_TABLE_V = [
    "AGGGTAAA|TTTACCCT",
    "[CGT]GGGTAAA|TTTACCC[ACG]",
    "A[ACT]GGTAAA|TTTACC[AGT]T",
    "AG[ACT]GTAAA|TTTAC[AGT]CT",
    "AGG[ACT]TAAA|TTTA[AGT]CCT",
    "AGGG[ACG]AAA|TTT[CGT]CCCT",
    "AGGGT[CGT]AA|TT[ACG]ACCCT",
    "AGGGTA[CGT]A|T[ACG]TACCCT",
    "AGGGTAA[CGT]|[ACG]TTACCCT",
]

CONFIG2_REGEX = "ACG[AT]{2,6}C(G|T)T"
CONFIG1_MOTIF = "TATAAA"


def plain_small(n: int = 1 * MiB) -> tuple[np.ndarray, str]:
    """1 MiB i.i.d. uniform (seed 0) and the literal motif TATAAA."""
    return uniform(0, n), CONFIG1_MOTIF


def plain_markov(n: int = 256 * MiB) -> tuple[np.ndarray, str]:
    """Order-2 Markov, 41% GC (seed 1), and the regex ACG[AT]{2,6}C(G|T)T."""
    return markov2(1, n, 0.41), CONFIG2_REGEX


def plain_large(n: int = 3435973837, kmers: int = 1000) -> tuple[np.ndarray, list[str]]:
    """Order-2 Markov (seed 2) with 10% soft-masked lowercase runs (mean 1 kb) and N runs
    covering 2% (mean 50 kb), and 1,000 random 12-mers (seed 2)."""
    seq = markov2(2, n, 0.41)
    overlay_runs(seq, 2, 0.10, 1000.0, "lower")
    overlay_runs(seq, 2, 0.02, 50000.0, "N")
    return seq, random_kmers(2, kmers, 12)


def batched(n_seqs: int = 4096, n_dfas: int = 64, lo: int = 1024, hi: int = 16 * MiB,
            seed: int = 3, n_states=None, state_range: tuple[int, int] = (5, 60)
            ) -> tuple[np.ndarray, np.ndarray, list[str]]:
    """Sequences with log-uniform lengths in [lo, hi] (i.i.d. ACGT, one contiguous
    buffer) and random motif regexes. Returns (buffer, offsets[n_seqs+1], regexes).
    With 'n_states' (a callable giving a pattern's minimal state count, supplied by the
    caller), motifs are drawn until n_dfas fall inside state_range; without it the
    first n_dfas motifs are returned."""
    lens = log_uniform_lengths(seed, n_seqs, lo, hi)
    offs = np.zeros(n_seqs + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    buf = uniform(seed, int(offs[-1]))
    if n_states is None:
        return buf, offs, random_regexes(seed, n_dfas)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n_dfas:
        r = random_motif_regex(rng)
        if state_range[0] <= n_states(r) <= state_range[1]:
            out.append(r)
    return buf, offs, out


def serving(n_req: int = 4000, rate: float = 2000.0, n_states=None, payload_bytes: int = 256 * MiB):
    """The serving workload: a 256 MiB order-2 Markov payload (seed 4) with 10% soft-masked
    and 2% N runs; n_req requests with lengths log-uniform on [4 KiB, 64 MiB], offsets into
    the payload, automaton indices and Poisson inter-arrival gaps (ns) at 'rate' per second
    (seed 4); and 16 pattern sets: 8 sets of random 8..16-mers and 8 motif regexes. With
    'n_states' (a callable giving a k-mer set's state count, supplied by the caller) each
    k-mer set is shrunk by 4 until its automaton has at most 500 states.
    Returns dict(payload, lens, offs, didx, gaps_ns, patterns=[("kmers", list) | ("regex", str)])."""
    payload = markov2(4, payload_bytes)
    overlay_runs(payload, 4, 0.10, 1000.0, "lower")
    overlay_runs(payload, 5, 0.02, 50000.0, "N")
    pats = []
    for i in range(8):
        n = 40
        while True:
            km = random_kmers(400 + i, n, 8, 16)
            if n_states is None or n_states(km) <= 500 or n <= 4:
                break
            n -= 4
        pats.append(("kmers", km))
    for r in random_regexes(4, 8):
        pats.append(("regex", r))
    rng = np.random.Generator(np.random.PCG64(4))
    lens = log_uniform_lengths(4, n_req, 4 * 1024, 64 * MiB)
    offs = np.array([int(rng.integers(0, payload_bytes - n + 1)) for n in lens], np.int64)
    didx = rng.integers(0, len(pats), n_req)
    gaps = rng.exponential(1e9 / rate, n_req)
    return dict(payload=payload, lens=lens, offs=offs, didx=didx, gaps_ns=gaps, patterns=pats)
