"""Python binding of libdnadfa.so (the C ABI declared in include/dna_dfa.h).

Argument marshalling only: every step of a scan runs in the library's CUDA kernels.
PyTorch provides device memory and streams. There is no CPU fallback: if the shared
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

_lock = threading.Lock()
_lib = None

DNA_OK = 0
PLACE_AUTO, PLACE_SMEM_PAIR, PLACE_SMEM_ONE, PLACE_GLOBAL_ONE, PLACE_MAP, PLACE_SMEM_HOT, PLACE_SMEM_ONE_REP = \
    0, 1, 2, 3, 4, 5, 6

EXPORTED = [
    "dfa_load", "dfa_free", "dfa_info", "dfa_analyze", "dna_scan", "dna_scan_planned", "dna_scan_batch",
    "dna_scan_count_static", "dna_scan_host", "dna_scan_from", "dfa_load_labeled", "dna_scan_labels",
    "dna_compile_regex_set", "dfa_tune", "dna_lookup_peak",
    "dna_batch_create", "dna_batch_run", "dna_batch_info", "dna_batch_free",
    "dna_server_create", "dna_server_submit", "dna_server_poll", "dna_server_drain",
    "dna_server_stats", "dna_server_now_ns", "dna_server_free", "dna_fasta_parse",
    "dna_status_string", "dna_compile_regex", "dna_compile_kmers", "dna_free_host",
    "dna_profile_enable", "dna_profile_read",
]


class DnaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = status_string(code) if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


class _Info(ctypes.Structure):
    _fields_ = [("n_states", ctypes.c_uint32), ("definite_depth", ctypes.c_int32),
                ("lookback", ctypes.c_uint32), ("placement", ctypes.c_uint32),
                ("accept_start", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("chunk_maps", ctypes.c_uint32), ("n_labels", ctypes.c_uint32)]


class _Plan(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_uint32), ("lookback", ctypes.c_uint32),
                ("warps_per_cta", ctypes.c_uint32), ("placement", ctypes.c_uint32),
                ("prefetch_tiles", ctypes.c_uint32), ("hot_rows", ctypes.c_uint32)]


class _Profile(ctypes.Structure):
    _fields_ = [("scan_kernel_ms", ctypes.c_double), ("scan_kernel_calls", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64),
                ("emit_kernel_ms", ctypes.c_double), ("emit_kernel_calls", ctypes.c_uint64),
                ("batch_kernel_ms", ctypes.c_double), ("batch_kernel_calls", ctypes.c_uint64),
                ("ingest_kernel_ms", ctypes.c_double), ("ingest_kernel_calls", ctypes.c_uint64),
                ("conv_scans", ctypes.c_uint64), ("conv_chunks", ctypes.c_uint64),
                ("conv_inblock", ctypes.c_uint64), ("conv_pending", ctypes.c_uint64),
                ("conv_blockfirst", ctypes.c_uint64), ("conv_diverged", ctypes.c_uint64),
                ("conv_cascade", ctypes.c_uint64), ("device_allocs", ctypes.c_uint64)]


class _BatchOpts(ctypes.Structure):
    _fields_ = [("chunk_bases", ctypes.c_uint32), ("warps_per_cta", ctypes.c_uint32),
                ("autotune", ctypes.c_uint32), ("use_graph", ctypes.c_uint32)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("chunk_bases", ctypes.c_uint32), ("warps_per_cta", ctypes.c_uint32),
                ("grid", ctypes.c_uint32), ("groups_per_task", ctypes.c_uint32),
                ("n_fast", ctypes.c_uint32), ("n_slow", ctypes.c_uint32),
                ("n_chunks", ctypes.c_uint64), ("packed_tiles", ctypes.c_uint64),
                ("max_states", ctypes.c_uint32)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("mem_cap_bytes", ctypes.c_uint64)]


class _Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("dfa", ctypes.c_uint32),
                ("count", ctypes.c_uint64), ("len", ctypes.c_uint64), ("arrival_ns", ctypes.c_uint64),
                ("admit_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64),
                ("h2d_us", ctypes.c_float), ("device_us", ctypes.c_float)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("in_flight", ctypes.c_uint32), ("slots", ctypes.c_uint32),
                ("mem_in_use", ctypes.c_uint64), ("mem_cap", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    return _build.build(force=force)


def library_path() -> str:
    return _build.LIBPATH


def lib():
    """Loads libdnadfa.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIBPATH):
            raise RuntimeError(f"libdnadfa.so not found at {_build.LIBPATH}; run build()")
        L = ctypes.CDLL(_build.LIBPATH)
        p, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        L.dfa_load.argtypes = [p, u32, p, ctypes.POINTER(p)]
        L.dfa_load.restype = i32
        L.dfa_free.argtypes = [p]
        L.dfa_free.restype = None
        L.dfa_info.argtypes = [p, ctypes.POINTER(_Info)]
        L.dfa_info.restype = i32
        L.dfa_analyze.argtypes = [p, u32, ctypes.POINTER(ctypes.c_int32)]
        L.dfa_analyze.restype = i32
        L.dna_scan.argtypes = [p, p, u64, p, p, p, u64]
        L.dna_scan.restype = i32
        L.dna_scan_planned.argtypes = [p, p, u64, p, p, p, u64, ctypes.POINTER(_Plan)]
        L.dna_scan_planned.restype = i32
        L.dna_scan_count_static.argtypes = [p, p, u64, p, p]
        L.dna_scan_count_static.restype = i32
        L.dna_scan_host.argtypes = [p, p, u64, p, p, p, u64]
        L.dna_scan_host.restype = i32
        L.dna_scan_from.argtypes = [p, p, u64, u32, p, p, p, p, u64]
        L.dna_scan_from.restype = i32
        L.dfa_load_labeled.argtypes = [p, u32, p, u32, ctypes.POINTER(p)]
        L.dfa_load_labeled.restype = i32
        L.dna_scan_labels.argtypes = [p, p, u64, p, p, p, p, p, u64]
        L.dna_scan_labels.restype = i32
        L.dna_compile_regex_set.argtypes = [p, u32, ctypes.POINTER(p), ctypes.POINTER(p), ctypes.POINTER(u32)]
        L.dna_compile_regex_set.restype = i32
        L.dfa_tune.argtypes = [p, p, u64, p, ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_float)]
        L.dfa_tune.restype = i32
        L.dna_lookup_peak.argtypes = [u32, p, ctypes.POINTER(ctypes.c_double)]
        L.dna_lookup_peak.restype = i32
        L.dna_batch_create.argtypes = [p, u32, p, p, u32, ctypes.POINTER(_BatchOpts), p, ctypes.POINTER(p)]
        L.dna_batch_create.restype = i32
        L.dna_batch_run.argtypes = [p, p, p]
        L.dna_batch_run.restype = i32
        L.dna_batch_info.argtypes = [p, ctypes.POINTER(_BatchInfo)]
        L.dna_batch_info.restype = i32
        L.dna_batch_free.argtypes = [p]
        L.dna_batch_free.restype = None
        L.dna_server_create.argtypes = [p, u32, ctypes.POINTER(_ServerOpts), ctypes.POINTER(p)]
        L.dna_server_create.restype = i32
        L.dna_server_submit.argtypes = [p, p, u64, u32, u64]
        L.dna_server_submit.restype = ctypes.c_int64
        L.dna_server_poll.argtypes = [p, ctypes.POINTER(_Completion), u32, ctypes.c_int32]
        L.dna_server_poll.restype = i32
        L.dna_server_drain.argtypes = [p, ctypes.c_int32]
        L.dna_server_drain.restype = i32
        L.dna_server_stats.argtypes = [p, ctypes.POINTER(_ServerStats)]
        L.dna_server_stats.restype = i32
        L.dna_server_now_ns.argtypes = []
        L.dna_server_now_ns.restype = u64
        L.dna_server_free.argtypes = [p]
        L.dna_server_free.restype = None
        L.dna_fasta_parse.argtypes = [ctypes.c_char_p, u64, p, u64, ctypes.POINTER(u64), p, p, u32,
                                      ctypes.POINTER(u32)]
        L.dna_fasta_parse.restype = i32
        L.dna_scan_batch.argtypes = [p, u32, p, p, u32, p, p]
        L.dna_scan_batch.restype = i32
        L.dna_status_string.argtypes = [i32]
        L.dna_status_string.restype = ctypes.c_char_p
        L.dna_compile_regex.argtypes = [ctypes.c_char_p, ctypes.POINTER(p), ctypes.POINTER(p),
                                        ctypes.POINTER(u32)]
        L.dna_compile_regex.restype = i32
        L.dna_compile_kmers.argtypes = [p, u32, ctypes.POINTER(p), ctypes.POINTER(p),
                                        ctypes.POINTER(u32)]
        L.dna_compile_kmers.restype = i32
        L.dna_free_host.argtypes = [p]
        L.dna_free_host.restype = None
        L.dna_profile_enable.argtypes = [i32]
        L.dna_profile_enable.restype = None
        L.dna_profile_read.argtypes = [ctypes.POINTER(_Profile), i32]
        L.dna_profile_read.restype = i32
        _lib = L
        return L


def status_string(code: int) -> str:
    return lib().dna_status_string(code).decode()


def _check(rc: int, what: str):
    if rc != DNA_OK:
        raise DnaError(rc, what)


# ------------------------------------------------------------------ compilers

def _take_table(tp, ap, n):
    L = lib()
    try:
        table = np.ctypeslib.as_array(ctypes.cast(tp, ctypes.POINTER(ctypes.c_uint32)),
                                      shape=(n, 4)).copy()
        mask = np.ctypeslib.as_array(ctypes.cast(ap, ctypes.POINTER(ctypes.c_uint8)),
                                     shape=((n + 7) // 8,)).copy()
    finally:
        L.dna_free_host(tp)
        L.dna_free_host(ap)
    return table, mask


def compile_regex(pattern: str):
    """Host compiler: (table uint32 [Q,4] columns A,C,G,T; bit-packed accept mask)."""
    tp, ap, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_uint32()
    _check(lib().dna_compile_regex(pattern.encode(), ctypes.byref(tp), ctypes.byref(ap),
                                   ctypes.byref(n)), f"compile_regex({pattern!r})")
    return _take_table(tp, ap, n.value)


def compile_kmers(kmers):
    arr = (ctypes.c_char_p * len(kmers))(*[k.encode() for k in kmers])
    tp, ap, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_uint32()
    _check(lib().dna_compile_kmers(ctypes.cast(arr, ctypes.c_void_p), len(kmers),
                                   ctypes.byref(tp), ctypes.byref(ap), ctypes.byref(n)),
           "compile_kmers")
    return _take_table(tp, ap, n.value)


def compile_regex_set(patterns):
    """Host compiler for several patterns at once: (table uint32 [Q,4], labels uint32 [Q])
    where bit i of labels[q] means pattern i ends at a step landing in q."""
    arr = (ctypes.c_char_p * len(patterns))(*[p.encode() for p in patterns])
    tp, lp, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_uint32()
    L = lib()
    _check(L.dna_compile_regex_set(ctypes.cast(arr, ctypes.c_void_p), len(patterns), ctypes.byref(tp),
                                   ctypes.byref(lp), ctypes.byref(n)), "compile_regex_set")
    try:
        table = np.ctypeslib.as_array(ctypes.cast(tp, ctypes.POINTER(ctypes.c_uint32)),
                                      shape=(n.value, 4)).copy()
        labels = np.ctypeslib.as_array(ctypes.cast(lp, ctypes.POINTER(ctypes.c_uint32)),
                                       shape=(n.value,)).copy()
    finally:
        L.dna_free_host(tp)
        L.dna_free_host(lp)
    return table, labels


def fasta_parse(text: bytes):
    """dna_fasta_parse: (sequence bytes as a uint8 array, record offsets [n+1], headers).
    Record r is seq[offsets[r]:offsets[r+1]]."""
    L = lib()
    n_out, n_rec = ctypes.c_uint64(), ctypes.c_uint32()
    _check(L.dna_fasta_parse(text, len(text), None, 0, ctypes.byref(n_out), None, None, 0,
                             ctypes.byref(n_rec)), "dna_fasta_parse")
    seq = np.empty(n_out.value, dtype=np.uint8)
    off = np.empty(n_rec.value + 1, dtype=np.uint64)
    hdr = np.empty(2 * (n_rec.value + 1), dtype=np.uint64)
    _check(L.dna_fasta_parse(text, len(text), seq.ctypes.data, seq.size, ctypes.byref(n_out),
                             off.ctypes.data, hdr.ctypes.data, off.size, ctypes.byref(n_rec)),
           "dna_fasta_parse")
    headers = [text[int(hdr[2 * r]):int(hdr[2 * r + 1])].decode(errors="replace") for r in range(n_rec.value)]
    return seq, off.astype(np.int64), headers


def definite_depth(table) -> int:
    """Host-only analysis (dfa_analyze): definite depth, or -1."""
    t = np.ascontiguousarray(table, dtype=np.uint32)
    m = ctypes.c_int32()
    _check(lib().dfa_analyze(t.ctypes.data, t.shape[0], ctypes.byref(m)), "dfa_analyze")
    return m.value


def pack_accept(accept) -> np.ndarray:
    """0/1 per state -> the bit-packed mask dfa_load takes."""
    a = np.asarray(accept).astype(bool)
    return np.packbits(a, bitorder="little")


# ----------------------------------------------------------------- automata

@dataclass
class DfaInfo:
    n_states: int
    definite_depth: int
    lookback: int
    placement: int
    accept_start: bool
    device: int
    chunk_maps: bool
    n_labels: int = 0


class Dfa:
    """A device-resident automaton (dfa_load / dfa_free; dfa_load_labeled when 'labels'
    is given: uint32 [n_states] pattern masks over n_labels patterns)."""

    def __init__(self, table, accept_mask=None, labels=None, n_labels: int = 0):
        table = np.ascontiguousarray(table, dtype=np.uint32)
        if table.ndim != 2 or table.shape[1] != 4:
            raise ValueError("table must be [n_states, 4]")
        n = table.shape[0]
        h = ctypes.c_void_p()
        if labels is not None:
            lab = np.ascontiguousarray(labels, dtype=np.uint32)
            if lab.size != n:
                raise ValueError("labels must have one mask per state")
            if not n_labels:
                n_labels = max(1, int(lab.max()).bit_length())
            _check(lib().dfa_load_labeled(table.ctypes.data, n, lab.ctypes.data, n_labels, ctypes.byref(h)),
                   "dfa_load_labeled")
            mask = pack_accept(lab != 0)
            self.labels = lab
        else:
            mask = np.ascontiguousarray(accept_mask, dtype=np.uint8)
            if mask.size < (n + 7) // 8:
                raise ValueError("accept mask too short")
            _check(lib().dfa_load(table.ctypes.data, n, mask.ctypes.data, ctypes.byref(h)), "dfa_load")
            self.labels = None
        self._h = h
        self.table = table
        self.accept_mask = mask

    @classmethod
    def from_regex_set(cls, patterns) -> "Dfa":
        """One automaton for several regexes, each step labelled with the patterns ending there."""
        table, labels = compile_regex_set(list(patterns))
        return cls(table, labels=labels, n_labels=len(patterns))

    @classmethod
    def from_regex(cls, pattern: str) -> "Dfa":
        return cls(*compile_regex(pattern))

    @classmethod
    def from_kmers(cls, kmers) -> "Dfa":
        return cls(*compile_kmers(list(kmers)))

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("automaton was freed")
        return self._h.value

    def info(self) -> DfaInfo:
        i = _Info()
        _check(lib().dfa_info(self.handle, ctypes.byref(i)), "dfa_info")
        return DfaInfo(i.n_states, i.definite_depth, i.lookback, i.placement,
                       bool(i.accept_start), i.device, bool(i.chunk_maps), i.n_labels)

    def tune(self, seq, stream=None) -> tuple[int, float]:
        """dfa_tune: times every table placement the automaton fits in on 'seq' (a CUDA
        uint8 tensor) and makes the fastest the default. Returns (placement, ms)."""
        pl, ms = ctypes.c_uint32(), ctypes.c_float()
        _check(lib().dfa_tune(self.handle, seq.data_ptr(), seq.numel(), _stream_handle(stream),
                              ctypes.byref(pl), ctypes.byref(ms)), "dfa_tune")
        return pl.value, ms.value

    def free(self):
        if self._h:
            lib().dfa_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ------------------------------------------------------------------- scans

def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def scan(dfa: Dfa, seq, positions: bool = False, capacity: int | None = None,
         stream=None, plan: dict | None = None, out_count=None, out_positions=None):
    """dna_scan on a CUDA uint8 tensor. Returns (count tensor [1] uint64-as-int64,
    positions tensor or None). Results are ready when the stream completes."""
    import torch
    if not (isinstance(seq, torch.Tensor) and seq.is_cuda and seq.dtype == torch.uint8):
        raise TypeError("seq must be a CUDA uint8 tensor")
    if not seq.is_contiguous():
        raise ValueError("seq must be contiguous")
    dev = seq.device
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=dev)
    pos_ptr, cap = None, 0
    if positions:
        if out_positions is None:
            cap = int(capacity if capacity is not None else max(1024, seq.numel() // 256))
            out_positions = torch.empty(cap, dtype=torch.int64, device=dev)
        else:
            cap = out_positions.numel() if capacity is None else int(capacity)
        pos_ptr = out_positions.data_ptr()
    sh = _stream_handle(stream)
    L = lib()
    if plan:
        pl = _Plan(plan.get("chunk_bytes", 0), plan.get("lookback", 0),
                   plan.get("warps_per_cta", 0), plan.get("placement", 0),
                   plan.get("prefetch_tiles", 0), plan.get("hot_rows", 0))
        rc = L.dna_scan_planned(dfa.handle, seq.data_ptr(), seq.numel(), sh,
                                out_count.data_ptr(), pos_ptr, cap, ctypes.byref(pl))
    else:
        rc = L.dna_scan(dfa.handle, seq.data_ptr(), seq.numel(), sh, out_count.data_ptr(),
                        pos_ptr, cap)
    _check(rc, "dna_scan")
    return out_count, (out_positions if positions else None)


def scan_from(dfa: Dfa, seq, start_state: int = 0, positions: bool = False,
              capacity: int | None = None, stream=None, out=None):
    """dna_scan_from on a CUDA uint8 tensor: the scan of one piece of a longer sequence,
    starting in 'start_state'. Returns (count [1] int64, last state [1] int32, positions
    counted from the piece's first byte, or None). 'out' (or None) supplies the three
    output tensors (count, last, positions) to write into. Results are ready when the
    stream completes."""
    import torch
    if not (isinstance(seq, torch.Tensor) and seq.is_cuda and seq.dtype == torch.uint8):
        raise TypeError("seq must be a CUDA uint8 tensor")
    if not seq.is_contiguous():
        raise ValueError("seq must be contiguous")
    dev = seq.device
    if out is not None:
        count, last, pos = out
        cap = pos.numel() if (positions and pos is not None) else 0
    else:
        count = torch.empty(1, dtype=torch.int64, device=dev)
        last = torch.empty(1, dtype=torch.int32, device=dev)
        pos, cap = None, 0
        if positions:
            cap = int(capacity if capacity is not None else max(1024, seq.numel() // 256))
            pos = torch.empty(cap, dtype=torch.int64, device=dev)
    _check(lib().dna_scan_from(dfa.handle, seq.data_ptr(), seq.numel(), int(start_state),
                               _stream_handle(stream), count.data_ptr(), last.data_ptr(),
                               pos.data_ptr() if positions else None, cap), "dna_scan_from")
    return count, last, (pos if positions else None)


def scan_labels(dfa: Dfa, seq, positions: bool = False, capacity: int | None = None, stream=None):
    """dna_scan_labels on a CUDA uint8 tensor (automaton from dfa_load_labeled). Returns
    (count [1], per-label counts [n_labels] int64, positions or None, position label masks
    (int32) or None). Results are ready when the stream completes."""
    import torch
    if not (isinstance(seq, torch.Tensor) and seq.is_cuda and seq.dtype == torch.uint8):
        raise TypeError("seq must be a CUDA uint8 tensor")
    if not seq.is_contiguous():
        raise ValueError("seq must be contiguous")
    dev = seq.device
    n_labels = dfa.info().n_labels
    count = torch.empty(1, dtype=torch.int64, device=dev)
    lab = torch.empty(max(1, n_labels), dtype=torch.int64, device=dev)
    pos = pos_lab = None
    cap = 0
    if positions:
        cap = int(capacity if capacity is not None else max(1024, seq.numel() // 256))
        pos = torch.empty(cap, dtype=torch.int64, device=dev)
        pos_lab = torch.empty(cap, dtype=torch.int32, device=dev)
    _check(lib().dna_scan_labels(dfa.handle, seq.data_ptr(), seq.numel(), _stream_handle(stream),
                                 count.data_ptr(), lab.data_ptr(),
                                 pos.data_ptr() if positions else None,
                                 pos_lab.data_ptr() if positions else None, cap), "dna_scan_labels")
    return count, lab[:n_labels], pos, pos_lab


def scan_ptr(dfa: Dfa, ptr: int, length: int, out_count_ptr: int, stream_handle: int,
             positions_ptr: int | None = None, capacity: int = 0) -> None:
    """Raw-pointer form of dna_scan (device or host-mapped pointers)."""
    _check(lib().dna_scan(dfa.handle, ptr, length, stream_handle, out_count_ptr,
                          positions_ptr, capacity), "dna_scan")


def scan_count_static(dfa: Dfa, seq, stream=None, out_count=None):
    """dna_scan_count_static: the count of dna_scan without any device allocation (the
    library's fixed scratch array is used; see include/dna_dfa.h for its limits)."""
    import torch
    if not (isinstance(seq, torch.Tensor) and seq.is_cuda and seq.dtype == torch.uint8):
        raise TypeError("seq must be a CUDA uint8 tensor")
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=seq.device)
    _check(lib().dna_scan_count_static(dfa.handle, seq.data_ptr(), seq.numel(),
                                       _stream_handle(stream), out_count.data_ptr()),
           "dna_scan_count_static")
    return out_count


def scan_host(dfa: Dfa, seq, positions: bool = False, capacity: int | None = None,
              stream=None, out_count=None, out_positions=None):
    """dna_scan_host: scans a host uint8 array (a numpy array or a CPU tensor, pinned for
    the fastest copy); returns (count, positions array or None) in host memory. The call
    is synchronous. A count above the capacity raises DnaError (DNA_ERR_CAPACITY)."""
    import torch
    if isinstance(seq, np.ndarray):
        if seq.dtype != np.uint8 or not seq.flags.c_contiguous:
            raise TypeError("seq must be a contiguous uint8 array")
        ptr, n = seq.ctypes.data, seq.size
    elif isinstance(seq, torch.Tensor) and not seq.is_cuda and seq.dtype == torch.uint8:
        if not seq.is_contiguous():
            raise ValueError("seq must be contiguous")
        ptr, n = seq.data_ptr(), seq.numel()
    else:
        raise TypeError("seq must be a host uint8 array or CPU tensor")
    if out_count is None:
        out_count = np.zeros(1, dtype=np.uint64)
    cptr = out_count.ctypes.data if isinstance(out_count, np.ndarray) else out_count.data_ptr()
    pos_ptr, cap = None, 0
    if positions:
        if out_positions is None:
            cap = int(capacity if capacity is not None else max(1024, n // 256))
            out_positions = np.empty(cap, dtype=np.uint64)
        else:
            cap = (out_positions.size if isinstance(out_positions, np.ndarray)
                   else out_positions.numel()) if capacity is None else int(capacity)
        pos_ptr = (out_positions.ctypes.data if isinstance(out_positions, np.ndarray)
                   else out_positions.data_ptr())
    _check(lib().dna_scan_host(dfa.handle, ptr, n, _stream_handle(stream), cptr, pos_ptr, cap),
           "dna_scan_host")
    c = int(out_count[0])
    return c, (out_positions[:c] if positions else None)


def _batch_arrays(dfas, seqs, lens=None):
    """ctypes arrays of handles, device pointers and lengths. 'seqs' holds CUDA uint8
    tensors, or raw device pointers when 'lens' is given."""
    n_d, n_s = len(dfas), len(seqs)
    hs = (ctypes.c_void_p * n_d)(*[d.handle for d in dfas])
    if lens is None:
        ptrs = (ctypes.c_void_p * n_s)(*[t.data_ptr() for t in seqs])
        ls = (ctypes.c_uint64 * n_s)(*[t.numel() for t in seqs])
    else:
        ptrs = (ctypes.c_void_p * n_s)(*[int(x) for x in seqs])
        ls = (ctypes.c_uint64 * n_s)(*[int(x) for x in lens])
    return hs, ptrs, ls


def scan_batch(dfas, seqs, stream=None, out=None, lens=None):
    """dna_scan_batch: counts [n_seqs, n_dfas] (int64 tensor) of CUDA uint8 tensors (or
    raw device pointers with 'lens'). Synchronous (one-shot plan)."""
    import torch
    n_d, n_s = len(dfas), len(seqs)
    hs, ptrs, ls = _batch_arrays(dfas, seqs, lens)
    if out is None:
        out = torch.empty((n_s, n_d), dtype=torch.int64, device="cuda")
    _check(lib().dna_scan_batch(ctypes.cast(hs, ctypes.c_void_p), n_d,
                                ctypes.cast(ptrs, ctypes.c_void_p), ctypes.cast(ls, ctypes.c_void_p),
                                n_s, _stream_handle(stream), out.data_ptr()), "dna_scan_batch")
    return out


@dataclass
class BatchInfo:
    chunk_bases: int
    warps_per_cta: int
    grid: int
    groups_per_task: int
    n_fast: int
    n_slow: int
    n_chunks: int
    packed_tiles: int
    max_states: int


class Batch:
    """A reusable batched-scan plan (dna_batch_create / dna_batch_run / dna_batch_free).
    The sequences (CUDA uint8 tensors, or device pointers with 'lens') must stay
    allocated while the plan exists; the automata must outlive it too."""

    def __init__(self, dfas, seqs, lens=None, chunk_bases: int = 0, warps_per_cta: int = 0,
                 autotune: bool = False, use_graph: bool = False, stream=None):
        self._dfas = list(dfas)
        self._seqs = list(seqs)
        self.n_dfas, self.n_seqs = len(self._dfas), len(self._seqs)
        hs, ptrs, ls = _batch_arrays(self._dfas, self._seqs, lens)
        opts = _BatchOpts(chunk_bases, warps_per_cta, 1 if autotune else 0, 1 if use_graph else 0)
        h = ctypes.c_void_p()
        _check(lib().dna_batch_create(ctypes.cast(hs, ctypes.c_void_p), self.n_dfas,
                                      ctypes.cast(ptrs, ctypes.c_void_p), ctypes.cast(ls, ctypes.c_void_p),
                                      self.n_seqs, ctypes.byref(opts), _stream_handle(stream),
                                      ctypes.byref(h)), "dna_batch_create")
        self._h = h

    def run(self, out=None, stream=None):
        """Queues the batch; returns the [n_seqs, n_dfas] int64 counts tensor."""
        import torch
        if not self._h:
            raise ValueError("batch was freed")
        if out is None:
            out = torch.empty((self.n_seqs, self.n_dfas), dtype=torch.int64, device="cuda")
        _check(lib().dna_batch_run(self._h, _stream_handle(stream), out.data_ptr()), "dna_batch_run")
        return out

    def info(self) -> BatchInfo:
        i = _BatchInfo()
        _check(lib().dna_batch_info(self._h, ctypes.byref(i)), "dna_batch_info")
        return BatchInfo(i.chunk_bases, i.warps_per_cta, i.grid, i.groups_per_task, i.n_fast,
                         i.n_slow, i.n_chunks, i.packed_tiles, i.max_states)

    def free(self):
        if self._h:
            lib().dna_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """The request loop (dna_server_*): scans of host sequences against resident automata,
    admitted continuously into 'slots' device streams under a device-memory cap."""

    def __init__(self, dfas, slots: int = 8, mem_cap_bytes: int = 40 << 30):
        self._dfas = list(dfas)
        hs = (ctypes.c_void_p * len(self._dfas))(*[d.handle for d in self._dfas])
        opts = _ServerOpts(slots, mem_cap_bytes)
        h = ctypes.c_void_p()
        _check(lib().dna_server_create(ctypes.cast(hs, ctypes.c_void_p), len(self._dfas), ctypes.byref(opts),
                                       ctypes.byref(h)), "dna_server_create")
        self._h = h
        self._keep = {}

    @staticmethod
    def now_ns() -> int:
        return int(lib().dna_server_now_ns())

    def submit(self, seq, dfa: int, arrival_ns: int = 0, keep=None) -> int:
        """Queues a scan of a host uint8 buffer (numpy array or pinned CPU tensor, or a raw
        (pointer, length) pair). 'keep' holds a reference until the request finishes."""
        import torch
        if isinstance(seq, tuple):
            ptr, n = seq
        elif isinstance(seq, np.ndarray):
            ptr, n = seq.ctypes.data, seq.size
        elif isinstance(seq, torch.Tensor) and not seq.is_cuda:
            ptr, n = seq.data_ptr(), seq.numel()
        else:
            raise TypeError("seq must be host memory")
        rid = int(lib().dna_server_submit(self._h, ptr, n, dfa, arrival_ns))
        if rid < 0:
            raise DnaError(rid, "dna_server_submit")
        if keep is not None:
            self._keep[rid] = keep
        return rid

    def poll(self, max_items: int = 1024, timeout_ms: int = 0) -> list[dict]:
        buf = (_Completion * max_items)()
        n = lib().dna_server_poll(self._h, buf, max_items, timeout_ms)
        if n < 0:
            raise DnaError(n, "dna_server_poll")
        out = []
        for i in range(n):
            c = buf[i]
            self._keep.pop(c.id, None)
            out.append({k: getattr(c, k) for k, _ in _Completion._fields_})
        return out

    def drain(self, timeout_ms: int = -1):
        _check(lib().dna_server_drain(self._h, timeout_ms), "dna_server_drain")

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().dna_server_stats(self._h, ctypes.byref(st)), "dna_server_stats")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def free(self):
        if self._h:
            lib().dna_server_free(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def lookup_peak(mode: int, stream=None) -> float:
    """dna_lookup_peak: measured lookups per second (0: shared memory without bank
    conflicts, 1: shared memory at random banks, 2: random L2 gathers)."""
    v = ctypes.c_double()
    _check(lib().dna_lookup_peak(mode, _stream_handle(stream), ctypes.byref(v)), "dna_lookup_peak")
    return v.value


def profile_enable(on: bool = True):
    lib().dna_profile_enable(1 if on else 0)


def profile_read(reset: bool = False) -> dict:
    pr = _Profile()
    _check(lib().dna_profile_read(ctypes.byref(pr), 1 if reset else 0), "dna_profile_read")
    return {k: getattr(pr, k) for k, _ in _Profile._fields_}
