"""CPU oracle for the DNA DFA scan -- TEST INFRASTRUCTURE.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline / reference leg
may import this package. It wraps ``oracle.c`` (plain single-threaded C: its own regex
parser, Thompson NFA, subset construction, Moore minimisation, Aho-Corasick builder,
and the sequential run that defines the result) and shares no code with the CUDA
library in ``paper_1509_01506_gb300``.

Tables here are int32 [n_states, 4] with columns A, C, G, T; accept is uint8
[n_states] (0/1); state 0 is the start state and the target of the reset symbol.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {-1: "syntax error", -2: "capacity exceeded", -3: "pattern matches the empty word",
          -4: "out of memory", -5: "invalid argument"}


class OracleError(ValueError):
    pass


def build(force: bool = False) -> str:
    """Compiles oracle.c (plain C, gcc, no CUDA) into oracle/_lib/liboracle.so."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(src)):
        return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p, i32, i64, cp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_char_p
            lib.or_run.argtypes = [p, p, i32, p, i64, p, i64]
            lib.or_run.restype = i64
            lib.or_run_from.argtypes = [p, p, i32, i32, p, i64, p]
            lib.or_run_from.restype = i64
            lib.or_run_piece.argtypes = [p, p, i32, i32, p, i64, p, p, i64]
            lib.or_run_piece.restype = i64
            lib.or_compile_regex.argtypes = [cp, ctypes.c_int, p, p, i32]
            lib.or_compile_regex.restype = i32
            lib.or_compile_kmers.argtypes = [cp, ctypes.c_int, p, p, i32]
            lib.or_compile_kmers.restype = i32
            lib.or_minimise_table.argtypes = [p, p, i32, p, p, i32]
            lib.or_minimise_table.restype = i32
            lib.or_compile_regex_set.argtypes = [cp, ctypes.c_int, p, p, i32]
            lib.or_compile_regex_set.restype = i32
            lib.or_run_labels.argtypes = [p, p, i32, p, i64, p, i32, p, p, i64]
            lib.or_run_labels.restype = i64
            lib.or_symbol_of_byte.argtypes = [ctypes.c_int]
            lib.or_symbol_of_byte.restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(rc: int) -> int:
    if rc < 0:
        raise OracleError(ERRORS.get(rc, f"error {rc}"))
    return rc


def _compile(fn, arg: bytes, minimise: bool, cap: int):
    while True:
        table = np.empty((cap, 4), dtype=np.int32)
        acc = np.empty(cap, dtype=np.uint8)
        rc = fn(arg, int(minimise), table.ctypes.data, acc.ctypes.data, cap)
        if rc == -2 and cap < (1 << 24):
            cap *= 4
            continue
        n = _check(rc)
        return table[:n].copy(), acc[:n].copy()


def compile_regex(pattern: str, minimise: bool = True, cap: int = 4096):
    """DFA of Sigma*.L(pattern): (table int32 [Q,4], accept uint8 [Q])."""
    return _compile(_load().or_compile_regex, pattern.encode(), minimise, cap)


def compile_kmers(patterns, minimise: bool = False, cap: int = 4096):
    """Failure-free Aho-Corasick DFA for a set of base strings."""
    if not isinstance(patterns, str):
        patterns = ",".join(patterns)
    return _compile(_load().or_compile_kmers, patterns.encode(), minimise,
                    max(cap, len(patterns) + 2))


def minimise_table(table: np.ndarray, accept: np.ndarray):
    table = np.ascontiguousarray(table, dtype=np.int32)
    accept = np.ascontiguousarray(accept, dtype=np.uint8)
    n = table.shape[0]
    out_t = np.empty((n, 4), dtype=np.int32)
    out_a = np.empty(n, dtype=np.uint8)
    k = _check(_load().or_minimise_table(table.ctypes.data, accept.ctypes.data, n,
                                         out_t.ctypes.data, out_a.ctypes.data, n))
    return out_t[:k].copy(), out_a[:k].copy()


def _as_bytes(seq) -> np.ndarray:
    if isinstance(seq, (bytes, bytearray)):
        return np.frombuffer(bytes(seq), dtype=np.uint8)
    a = np.ascontiguousarray(seq)
    assert a.dtype == np.uint8
    return a


def run(table: np.ndarray, accept: np.ndarray, seq, positions: bool = True,
        cap: int | None = None):
    """The definition: sequential run from q0. Returns (count, positions int64 or None)."""
    table = np.ascontiguousarray(table, dtype=np.int32)
    accept = np.ascontiguousarray(accept, dtype=np.uint8)
    s = _as_bytes(seq)
    lib = _load()
    if not positions:
        return _check(lib.or_run(table.ctypes.data, accept.ctypes.data, table.shape[0],
                                 s.ctypes.data, s.size, None, 0)), None
    if cap is None:
        cap = 1024
    while True:
        pos = np.empty(cap, dtype=np.int64)
        c = _check(lib.or_run(table.ctypes.data, accept.ctypes.data, table.shape[0],
                              s.ctypes.data, s.size, pos.ctypes.data, cap))
        if c <= cap:
            return c, pos[:c].copy()
        cap = c


def compile_regex_set(patterns, minimise: bool = True, cap: int = 4096):
    """One DFA of Sigma*.(L1|...|Ln) for up to 32 regexes: (table int32 [Q,4], labels
    uint32 [Q]) where bit i of labels[q] means pattern i ends at a step landing in q."""
    arg = "\n".join(patterns).encode()
    while True:
        table = np.empty((cap, 4), dtype=np.int32)
        lab = np.empty(cap, dtype=np.uint32)
        rc = _load().or_compile_regex_set(arg, int(minimise), table.ctypes.data, lab.ctypes.data, cap)
        if rc == -2 and cap < (1 << 24):
            cap *= 4
            continue
        n = _check(rc)
        return table[:n].copy(), lab[:n].copy()


def run_labels(table: np.ndarray, labels: np.ndarray, n_labels: int, seq, positions: bool = True,
               cap: int | None = None):
    """The plain run with pattern labels: (count, per-label counts int64 [n_labels],
    positions int64 or None, position masks uint32 or None)."""
    table = np.ascontiguousarray(table, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.uint32)
    s = _as_bytes(seq)
    lib = _load()
    counts = np.zeros(n_labels, dtype=np.int64)
    if not positions:
        c = _check(lib.or_run_labels(table.ctypes.data, labels.ctypes.data, table.shape[0], s.ctypes.data,
                                     s.size, counts.ctypes.data, n_labels, None, None, 0))
        return c, counts, None, None
    if cap is None:
        cap = 1024
    while True:
        pos = np.empty(cap, dtype=np.int64)
        pl = np.empty(cap, dtype=np.uint32)
        c = _check(lib.or_run_labels(table.ctypes.data, labels.ctypes.data, table.shape[0], s.ctypes.data,
                                     s.size, counts.ctypes.data, n_labels, pos.ctypes.data, pl.ctypes.data,
                                     cap))
        if c <= cap:
            return c, counts, pos[:c].copy(), pl[:c].copy()
        cap = c


def run_from(table, accept, q_start: int, seq):
    """Run from an arbitrary start state; returns (count, end_state)."""
    table = np.ascontiguousarray(table, dtype=np.int32)
    accept = np.ascontiguousarray(accept, dtype=np.uint8)
    s = _as_bytes(seq)
    q_end = ctypes.c_int32(0)
    c = _check(_load().or_run_from(table.ctypes.data, accept.ctypes.data, table.shape[0],
                                   q_start, s.ctypes.data, s.size, ctypes.byref(q_end)))
    return c, q_end.value


def run_piece(table, accept, q_start: int, seq, cap: int | None = None):
    """The run of one piece from 'q_start': (count, end state, positions int64 counted
    from the piece's first byte)."""
    table = np.ascontiguousarray(table, dtype=np.int32)
    accept = np.ascontiguousarray(accept, dtype=np.uint8)
    s = _as_bytes(seq)
    q_end = ctypes.c_int32(0)
    cap = 1024 if cap is None else cap
    while True:
        pos = np.empty(max(1, cap), dtype=np.int64)
        c = _check(_load().or_run_piece(table.ctypes.data, accept.ctypes.data, table.shape[0], q_start,
                                        s.ctypes.data, s.size, ctypes.byref(q_end), pos.ctypes.data, cap))
        if c <= cap:
            return c, q_end.value, pos[:c].copy()
        cap = c


def symbol_of_byte(b: int) -> int:
    return _load().or_symbol_of_byte(b)
