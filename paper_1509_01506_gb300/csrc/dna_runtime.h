// dna_runtime.h -- host-side internals shared by the library's CUDA translation units
// (dna_scan.cu and dna_batch.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/dna_dfa.h"

// A loaded automaton: its tables on the device it was loaded on, plus the host-side
// analysis that the scans plan with.
struct dna_dfa {
    uint32_t n_states = 0;
    int device = 0;
    int definite_depth = -1;
    uint32_t lookback = 0;
    uint32_t placement = DNA_PLACE_AUTO;
    uint32_t accept0 = 0;
    uint32_t reset_entry = 0;
    uint32_t *d_one = nullptr;    // [n_states][4] one-symbol entries, code order A, C, T, G
    uint32_t *d_pair = nullptr;   // [n_states][16] compact pair entries (small automata)
    bool map_mode = false;        // scans use chunk maps (runs from different states do not meet)
    uint32_t *d_labels = nullptr; // [n_states] label mask of each state (dfa_load_labeled), or null
    uint32_t n_labels = 0;
    // hot-state tables (automata too large for per-lane two-symbol tables): u16 two-symbol
    // rows [n_states][16] and one-symbol rows [n_states][4]; the device numbering puts the
    // states a random walk visits most first, perm[q] = device number of the caller's q
    uint16_t *d_hot2 = nullptr;
    uint16_t *d_hot1 = nullptr;
    std::vector<uint32_t> perm;
    uint32_t *d_perm_inv = nullptr;   // [n_states] device -> caller numbering (when renumbered)
    double hot_cover = 0;         // visit share of the hot rows that fit (random walk)
    // resident blocks per SM of each scan kernel variant with this automaton's shared
    // memory footprint ([mode][warp option][positions]; 0 = not yet queried)
    std::atomic<int> per_sm[5][4][2] = {};
};

namespace dnalib {

int cuda_status(cudaError_t e);

struct DeviceProps {
    int sms = 0;
    size_t smem_optin = 0;
};
DeviceProps device_props(int dev);

// Raises a kernel's dynamic shared-memory limit to 'bytes' once per (kernel, device).
int ensure_smem_optin(const void *fn, int device, size_t bytes);

size_t align_up(size_t x, size_t a);

// Counts kernels launched by the library (reported by dna_profile_read).
void record_launch(int n = 1);

// Device memory the library allocates; every allocation is counted (dna_profile_read's
// device_allocs).
// scratch_alloc / scratch_free: stream-ordered scratch from the library's own memory pool
// on device 'dev' (created on first use). The pool keeps up to kScratchKeepBytes
// reserved between calls: the device's default pool hands its memory back at every
// synchronisation, and the next call would then map it again.
constexpr uint64_t kScratchKeepBytes = 1ull << 30;
int scratch_alloc(int dev, size_t bytes, cudaStream_t s, void **out);
int scratch_free(void *p, cudaStream_t s);
// device_alloc: a plain (counted) cudaMalloc for memory that lives as long as a handle.
cudaError_t device_alloc(void **p, size_t bytes);
// pool_alloc: a (counted) stream-ordered allocation from a pool the caller owns.
cudaError_t pool_alloc(void **p, size_t bytes, cudaMemPool_t pool, cudaStream_t s);

// Per-label outputs of a scan (dna_scan_labels): the extraction pass walks every hit row
// and adds each accepting step's label mask into 'counts' (device, zeroed by the caller);
// 'pos_labels' (device or null) receives each written position's mask.
struct LabelOut {
    const uint32_t *labels = nullptr;   // [n_states] device label masks
    unsigned long long *counts = nullptr;
    uint32_t *pos_labels = nullptr;
    uint32_t n_labels = 0;
};

// A scan of a piece of a longer sequence (dna_scan_from): the state the piece starts in
// (device numbering) and where to write the state after it (caller's numbering), or null.
struct ScanFrom {
    uint32_t start = 0;
    uint32_t *out_last = nullptr;
};

// The single-sequence scan behind dna_scan / dna_scan_planned (dispatches to the
// chunk-map path for automata that need it). 'lab' (or null) asks for per-label outputs;
// 'from' (or null: start in q0, no last state) for a piece of a longer sequence.
int scan_impl(const dna_dfa *d, const uint8_t *seq, uint64_t len, cudaStream_t stream,
              uint64_t *out_count, uint64_t *out_positions, uint64_t cap, const dna_plan *ov,
              const LabelOut *lab = nullptr, const ScanFrom *from = nullptr);
// The speculative chunk scan; 'given_start' (per chunk, or null) supplies exact chunk
// start states, in which case nothing is speculated or repaired.
int scan_impl_given(const dna_dfa *d, const uint8_t *seq, uint64_t len, cudaStream_t stream,
                    uint64_t *out_count, uint64_t *out_positions, uint64_t cap, const dna_plan *ov,
                    const uint32_t *given_start, const LabelOut *lab = nullptr,
                    const ScanFrom *from = nullptr);
// The chunk-map scan (dna_map.cu); n_states <= kMaxMapStates. 'ext' (count only, or
// null) is caller-provided scratch of ext_bytes bytes used instead of the library's pool.
constexpr uint32_t kMaxMapStates = 256;
int map_scan_impl(const dna_dfa *d, const uint8_t *seq, uint64_t len, cudaStream_t stream,
                  uint64_t *out_count, uint64_t *out_positions, uint64_t cap,
                  uint8_t *ext = nullptr, size_t ext_bytes = 0, const LabelOut *lab = nullptr,
                  const ScanFrom *from = nullptr);

// Kernel timing: prof_begin records an event on the stream when profiling is enabled
// (otherwise returns an empty token); prof_end records the closing event.
enum ProfKernel { PROF_SCAN = 0, PROF_EMIT = 1, PROF_BATCH = 2, PROF_INGEST = 3, PROF_N = 4 };
struct ProfToken {
    cudaEvent_t a = nullptr, b = nullptr;
};
ProfToken prof_begin(cudaStream_t s);
void prof_end(ProfToken t, cudaStream_t s, int which);
// Convergence counters of one scan (control words 1..5 of its scratch), copied to the
// host and summed when profiling is enabled.
void prof_conv(cudaStream_t s, const uint32_t *dev_ctrl, uint64_t nseg);
void profile_set(int on);
bool profiling();
void profile_collect(dna_profile_t *out, int reset);

}  // namespace dnalib

#define DNA_CUDA(call)                                           \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return dnalib::cuda_status(_e);   \
    } while (0)
