// dna_scan.cu -- GB300 (sm_103a) kernels and the C ABI of the DNA automaton scan.
//
// The data-parallel path of Memeti & Pllana (Sec. III-A, III-B, Alg. 1), re-designed
// for one GPU:
//   * Input-based partitioning (Sec. III-A, Fig. 1a): the sequence is cut into chunks of
//     chunk_bytes; every GPU lane owns one chunk. A warp's 32 chunks are staged into
//     shared memory tile by tile with cp.async (16-byte copies; each copy instruction
//     of the warp covers four whole 128-byte lines) and read back row by row.
//   * Speculation (Sec. III-A, possible starting states): a chunk's start state is
//     unknown; the lane runs the automaton from q0 over the 'lookback' symbols in front
//     of its chunk. The state it reaches lies in the set of possible starting states
//     (the image of all states under those symbols), and is the exact start whenever
//     the automaton is lookback-definite, a reset byte occurs in the window, or the
//     window reaches the sequence start.
//   * Chunk scan (Alg. 1, the per-character loop): ingest is fused -- bytes are mapped
//     to 2-bit codes in registers, 4 bytes at a time, with a bit-exact check that every
//     byte is a base. Small automata use a two-symbol transition table replicated once
//     per lane in shared memory (lane l's copy lives in bank l, so the 32 lookups of a
//     warp never conflict); each entry carries the next row's address and the number
//     of accepting steps in the pair. Rows with reset bytes or sequence edges take a
//     per-byte path.
//   * Join (the "binary reduction" of Sec. III-A) and converging point (Sec. III-B.3):
//     a resolve kernel compares each chunk's speculated start with the previous chunk's
//     last state. On a mismatch it runs the true start and the speculated start in
//     lockstep from the chunk start until they meet (the converging point) and
//     corrects the count by the paper's formula: own prefix count + speculative total
//     - speculative prefix count at the meeting step. A run that never meets changes
//     the chunk's last state; a cascade pass then walks forward until the chain agrees
//     again.
//   * Extraction: a block scan of the chunk counts gives each chunk its output offset;
//     positions recorded in a per-chunk stash are written in order, chunks that
//     overflowed the stash or were corrected are rescanned from their true start.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/dna_dfa.h"
#include "dna_internal.h"
#include "dna_device.cuh"
#include "dna_runtime.h"

using namespace dnalib;

namespace {

// ------------------------------------------------------------------ constants

constexpr int kStages = 1;          // one stage per warp: rows are copied to registers first
constexpr int kStageBytes = 32 * kTile;
constexpr int kStashCap = 8;        // hit-row records kept per chunk before a rescan
constexpr uint32_t kMaxLookback = 64;
constexpr uint32_t kMaxStates = 1u << 24;
constexpr uint32_t kDefaultPrefetch = 0;  // tiles of L2 prefetch ahead of the stage

enum Mode { MODE_PAIR = 0, MODE_ONE_SMEM = 1, MODE_ONE_GLOBAL = 2 };


// -------------------------------------------------------------- scan kernel

struct ScanParams {
    const uint8_t *abase;   // 16-byte aligned base; sequence byte j is abase[lo + j]
    uint64_t lo, hi;        // valid aligned offsets [lo, hi)
    uint64_t seg_bytes;     // chunk length (multiple of kTile)
    uint64_t nseg;
    uint32_t lookback;
    uint32_t n_states;
    uint32_t reset_entry;
    const uint32_t *one;    // global one-symbol table
    const uint32_t *pair;   // global compact pair table: next | count << 24
    uint32_t *spec_start;   // [nseg] speculated start state
    uint32_t *last_state;   // [nseg] state after the chunk (from the speculated start)
    uint32_t *count;        // [nseg] accepting steps (from the speculated start)
    uint32_t *stash;        // [nseg][kStashCap][3] hit rows {tile, start state, count before}, or null
    uint32_t prefetch_tiles; // L2 prefetch distance in tiles (0 = off)
    uint32_t *nrec;         // [nseg] hit rows recorded (may exceed kStashCap)
    uint8_t *flags;         // [nseg] 1 = extraction must rescan the chunk from its true start
    uint32_t *ctrl;         // [4] zeroed before launch: finish ticket, pending, diverged, 0
    uint32_t *pending;      // chunks the last block must repair (first chunk of each block,
    uint32_t pending_cap;   //   and chunks whose 16-byte repair did not converge)
    uint32_t *pending_a;    // [pending_cap] snapshot of each pending chunk's true start
    uint32_t *div_list;     // [div_cap] chunks whose last state changed in a repair
    uint32_t div_cap;
    unsigned long long *cta_sum;   // [grid] count of each block's chunks
    unsigned long long *cta_off;   // [grid] exclusive prefix of cta_sum (for extraction)
    uint64_t *out_count;
    // 1, 2^16, 2^5, 2^28 passed at run time so the compiler keeps the multiplies that
    // use them (adds and shifts) on the FMA pipe instead of turning them into ALU ops
    uint32_t k1, k16, k5, k28;
    // lowercase letters selected by the codes (a, c at bytes 0, 2; t, g at bytes 4, 6),
    // passed at run time so that they stay in registers across the unrolled row loop
    uint32_t lut_lo, lut_hi;
};

// Per-byte walk over a full 128-byte row held in registers (rows with reset bytes).
__device__ __forceinline__ uint32_t row_bytes_reg(const OneTable &T, uint32_t q, const uint32_t (&w)[32],
                                                  uint32_t &cnt) {
#pragma unroll
    for (int k = 0; k < kTile; ++k) {
        uint32_t e = T.step(q, (w[k >> 2] >> (8 * (k & 3))) & 0xFFu);
        q = e & 0x7FFFFFFFu;
        cnt += e >> 31;
    }
    return q;
}

// Records a row that contains accepting steps: the emit pass re-walks it from 'q_row'
// and writes its positions starting at the chunk's offset + 'cnt_before'.
__device__ __forceinline__ void record_hit_row(uint32_t *stash, uint32_t &nrec, uint32_t t,
                                               uint32_t q_row, uint32_t cnt_before) {
    if (nrec < (uint32_t)kStashCap) {
        stash[nrec * 3] = t;
        stash[nrec * 3 + 1] = q_row;
        stash[nrec * 3 + 2] = cnt_before;
    }
    ++nrec;
}

// After a chunk's speculative run was repaired at its converging point (the true start
// and the speculated start met within the chunk's first row), the hit-row records of the
// speculative run are made those of the true run: row 0 is re-walked from the true start,
// later rows keep their start states (the runs coincide there) and shift their count
// offsets by delta = true prefix count - speculative prefix count. 'pa' is the true run's
// count over the prefix; if the true prefix has accepting steps but row 0 had no record,
// a record for row 0 is inserted in front.
__device__ __forceinline__ void fix_hit_rows(uint32_t *stash, uint32_t &nrec, uint32_t q_true,
                                             uint32_t delta, uint32_t pa) {
    const uint32_t n = nrec < (uint32_t)kStashCap ? nrec : (uint32_t)kStashCap;
    bool row0 = false;
    for (uint32_t r = 0; r < n; ++r) {
        if (stash[3 * r] == 0) { stash[3 * r + 1] = q_true; row0 = true; }
        else stash[3 * r + 2] += delta;
    }
    if (!row0 && pa > 0) {
        if (nrec < (uint32_t)kStashCap) {
            for (uint32_t r = n; r > 0; --r) {
                stash[3 * r] = stash[3 * (r - 1)];
                stash[3 * r + 1] = stash[3 * (r - 1) + 1];
                stash[3 * r + 2] = stash[3 * (r - 1) + 2];
            }
            stash[0] = 0; stash[1] = q_true; stash[2] = 0;
        }
        ++nrec;   // beyond the capacity: the extraction pass rescans the chunk
    }
}

// Per-byte walk over aligned offsets [from, to) read from global memory: rows with a
// reset byte, the first row of an unaligned sequence and the last row of the last chunk.
__device__ __forceinline__ uint32_t row_bytes_global(const OneTable &T, uint32_t q, const uint8_t *abase,
                                                     uint64_t from, uint64_t to, uint64_t hi, uint32_t &cnt) {
    walk_range(abase, from, to, hi, [&](uint64_t, uint32_t byte) {
        const uint32_t e = T.step(q, byte);
        q = e & 0x7FFFFFFFu;
        cnt += e >> 31;
        return true;
    });
    return q;
}

// Converging-point repair (Sec. III-B.3, Alg. 1) of chunk c from global memory: the true
// start 'a' and the start 's' that the chunk's current results assume run in lockstep
// until their states meet; from there on both runs coincide, so the true count is the
// true prefix count + (current count - assumed prefix count) and the last state is
// unchanged. A run that never meets gives the chunk's true count and last state directly.
// Hit-row records are fixed when the runs meet inside row 0; otherwise the chunk is
// flagged for a rescan by the extraction pass. Requires the chunk's current results
// (count, last state, records) to be those of the run from 's'.
struct Repair { uint32_t count, last; uint8_t flag; };

__device__ Repair repair_chunk(const ScanParams &p, uint64_t c, uint32_t a, uint32_t s) {
    const uint64_t b = c * p.seg_bytes;
    const uint64_t from = b > p.lo ? b : p.lo;
    const uint64_t to = b + p.seg_bytes < p.hi ? b + p.seg_bytes : p.hi;
    uint32_t qa = a, qs = s, ca = 0, cs = 0;
    uint64_t met_at = ~0ull;
    walk_range(p.abase, from, to, p.hi, [&](uint64_t off, uint32_t byte) {
        const uint32_t ea = one_step(p.one, p.reset_entry, qa, byte);
        const uint32_t es = one_step(p.one, p.reset_entry, qs, byte);
        qa = ea & 0x7FFFFFFFu; qs = es & 0x7FFFFFFFu;
        ca += ea >> 31; cs += es >> 31;
        if (qa == qs) { met_at = off; return false; }
        return true;
    });
    Repair r;
    if (met_at != ~0ull) {
        r.count = p.count[c] - cs + ca;
        r.last = p.last_state[c];
        r.flag = 0;
        if (p.stash) {
            if (met_at < b + kTile) {
                uint32_t nr = p.nrec[c];
                fix_hit_rows(p.stash + c * (kStashCap * 3), nr, a, ca - cs, ca);
                p.nrec[c] = nr;
            } else {
                r.flag = 1;
            }
        }
    } else {
        r.count = ca;
        r.last = qa;
        r.flag = 1;
    }
    return r;
}

// Makes chunk c's results those of the run from its true start a: count (and its block
// sum), assumed start, last state, flags.
__device__ __forceinline__ void apply_repair(const ScanParams &p, uint64_t c, uint32_t a,
                                             const Repair &r, uint32_t chunks_per_block) {
    const uint32_t old = p.count[c];
    p.count[c] = r.count;
    atomicAdd(&p.cta_sum[c / chunks_per_block], (unsigned long long)(long long)((int64_t)r.count - (int64_t)old));
    p.spec_start[c] = a;
    p.last_state[c] = r.last;
    if (r.flag) p.flags[c] = 1;
}

// The join across blocks (Sec. III-A "binary reduction"), run by the last block to
// finish: repairs the pending chunks in parallel (each from the last state of the chunk
// before it, as it stood when the blocks finished), then walks forward from every chunk
// whose last state changed until the chain agrees again, then writes the total count and
// each block's output offset. Every chunk's (assumed start, count, last state) triple
// stays consistent throughout.
template <int THREADS>
__device__ void finalize_block(const ScanParams &p) {
    __shared__ unsigned long long wsum[THREADS / 32];
    __shared__ unsigned long long carry;
    const uint32_t tid = threadIdx.x;
    const uint32_t cpb = THREADS;   // chunks per scan block
    const uint32_t np = p.ctrl[1];
    if (np <= p.pending_cap) {
        for (uint32_t i = tid; i < np; i += THREADS) p.pending_a[i] = p.last_state[p.pending[i] - 1];
        __syncthreads();
        for (uint32_t i = tid; i < np; i += THREADS) {
            const uint64_t c = p.pending[i];
            const uint32_t a = p.pending_a[i];
            const uint32_t s = p.spec_start[c];
            if (a == s) continue;
            const uint32_t old_last = p.last_state[c];
            const Repair r = repair_chunk(p, c, a, s);
            apply_repair(p, c, a, r, cpb);
            if (r.last != old_last) {
                const uint32_t k = atomicAdd(&p.ctrl[2], 1u);
                if (k < p.div_cap) p.div_list[k] = (uint32_t)c;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t nd = p.ctrl[2];
        if (np > p.pending_cap || nd > p.div_cap) {
            // a list overflowed: check every chunk boundary in order
            for (uint64_t c = 1; c < p.nseg; ++c) {
                const uint32_t a = p.last_state[c - 1];
                const uint32_t s = p.spec_start[c];
                if (a == s) continue;
                const Repair r = repair_chunk(p, c, a, s);
                apply_repair(p, c, a, r, cpb);
            }
        } else if (nd > 0) {
            // sort the (small) list of chunks whose last state changed, then walk forward
            for (uint32_t i = 1; i < nd; ++i) {
                const uint32_t vc = p.div_list[i];
                uint32_t j = i;
                while (j > 0 && p.div_list[j - 1] > vc) { p.div_list[j] = p.div_list[j - 1]; --j; }
                p.div_list[j] = vc;
            }
            uint64_t walked = 0;
            for (uint32_t i = 0; i < nd; ++i) {
                const uint64_t c = p.div_list[i];
                if (c < walked) continue;   // already recomputed from its true start
                // the walk stops exactly where the next chunk's assumed start is the true
                // last state of the chunk before it
                uint32_t cur = p.last_state[c];
                uint64_t k = c + 1;
                for (;;) {
                    if (k >= p.nseg || cur == p.spec_start[k]) { walked = k; break; }
                    const Repair r = repair_chunk(p, k, cur, p.spec_start[k]);
                    apply_repair(p, k, cur, r, cpb);
                    p.flags[k] = 1;   // its records follow a start that was not the true one
                    cur = r.last;
                    ++k;
                }
            }
        }
        carry = 0;
    }
    __syncthreads();
    // exclusive scan of the block sums -> output offsets; total -> out_count
    const uint32_t nb = gridDim.x;
    for (uint32_t base = 0; base < nb; base += THREADS) {
        const uint32_t i = base + tid;
        const unsigned long long v = i < nb ? p.cta_sum[i] : 0ull;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if ((tid & 31) >= (uint32_t)o) x += y;
        }
        if ((tid & 31) == 31) wsum[tid >> 5] = x;
        __syncthreads();
        if (tid < 32) {
            unsigned long long t = tid < THREADS / 32 ? wsum[tid] : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, t, o);
                if (tid >= (uint32_t)o) t += y;
            }
            if (tid < THREADS / 32) wsum[tid] = t;
        }
        __syncthreads();
        const unsigned long long incl = x + ((tid >> 5) ? wsum[(tid >> 5) - 1] : 0ull) + carry;
        if (i < nb) p.cta_off[i] = incl - v;
        __syncthreads();
        if (tid == THREADS - 1) carry = incl;
        __syncthreads();
    }
    if (tid == 0) *p.out_count = carry;
}

template <int MODE, int WARPS, bool POS>
__global__ void __launch_bounds__(WARPS * 32, 1)
scan_kernel(ScanParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint32_t warp_last[WARPS];
    __shared__ uint4 head_s[WARPS * 32];   // each chunk's first 16 bytes, for the repair
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);

    // shared memory: [staging: WARPS x 4 KB][one-symbol table][compact pair table][pad][pair table]
    uint8_t *stage_ptr = smem + (size_t)warp * kStages * kStageBytes;
    const uint32_t stage_addr = smem_base + (uint32_t)warp * kStages * kStageBytes;
    uint32_t *one_s = reinterpret_cast<uint32_t *>(smem + (size_t)WARPS * kStages * kStageBytes);

    const uint64_t seg0 = ((uint64_t)blockIdx.x * WARPS + warp) * 32u;
    const uint64_t seg = seg0 + lane;
    const bool warp_busy = seg0 < p.nseg;
    const bool active = seg < p.nseg;
    const uint64_t S = p.seg_bytes;
    const uint64_t b = seg * S;   // aligned offset of this chunk
    const uint32_t ntiles = warp_busy ? (uint32_t)(S / kTile) : 0u;

    // ---- staging: each warp copies tile t of its 32 chunks into a swizzled [32 rows][128 B]
    // stage. Copy j (0..7) of a lane moves the 16-byte column lane & 7 of row 4j + lane/8,
    // so each copy instruction of the warp covers four whole 128-byte lines. Only the warp
    // holding the last chunk can run past the end of the sequence and checks bounds.
    const uint32_t l8 = (uint32_t)lane >> 3, cc = (uint32_t)lane & 7u;
    const uint64_t copy_off0 = (seg0 + l8) * S + cc * 16u;
    const uint32_t copy_dst0 = stage_addr + l8 * kTile + ((cc ^ l8) << 4);
    // odd copies land in rows with (row & 7) >= 4: their swizzled column differs in bit 2
    const uint32_t copy_dst1 = stage_addr + l8 * kTile + ((cc ^ l8 ^ 4u) << 4);
    const bool tail_warp = seg0 + 32 >= p.nseg;
    const uint8_t *copy_src = p.abase + copy_off0;   // copy 0 of the next tile to issue
    const uint64_t stride4 = 4u * S;                 // four chunk rows apart
    auto issue = [&](uint32_t t) {
        if (!tail_warp) {
            // every row of this warp lies inside the sequence: no checks
            const uint8_t *src = copy_src + (uint64_t)t * kTile;
            cp_async16_full<0 * 4 * kTile>(copy_dst0, src);
            cp_async16_full<1 * 4 * kTile>(copy_dst1, src + stride4);
            cp_async16_full<2 * 4 * kTile>(copy_dst0, src + 2 * stride4);
            cp_async16_full<3 * 4 * kTile>(copy_dst1, src + 3 * stride4);
            cp_async16_full<4 * 4 * kTile>(copy_dst0, src + 4 * stride4);
            cp_async16_full<5 * 4 * kTile>(copy_dst1, src + 5 * stride4);
            cp_async16_full<6 * 4 * kTile>(copy_dst0, src + 6 * stride4);
            cp_async16_full<7 * 4 * kTile>(copy_dst1, src + 7 * stride4);
            return;
        }
        const uint64_t base = copy_off0 + (uint64_t)t * kTile;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint64_t goff = base + (uint64_t)j * stride4;
            const bool ok = seg0 + 4u * j + l8 < p.nseg && goff < p.hi;
            const uint32_t dst = ((j & 1) ? copy_dst1 : copy_dst0) + (uint32_t)j * 4u * kTile;
            cp_async16(dst, ok ? p.abase + goff : p.abase, ok ? 16u : 0u);
        }
    };
    auto prefetch = [&](uint32_t t) {   // this lane's own row of tile t into L2
        uint64_t off = b + (uint64_t)t * kTile;
        if (active && t < ntiles && off < p.hi) prefetch_l2(p.abase + off);
    };
    // the (small) compact tables are loaded first, so that these loads are not queued
    // behind the first tile's copies
    const uint32_t n1 = p.n_states * 4u;
    const uint32_t nc = MODE == MODE_PAIR ? p.n_states * 16u : 0u;
    constexpr int kPre = 2048 / (WARPS * 32) > 0 ? 2048 / (WARPS * 32) : 1;
    uint32_t pre[kPre];
    if constexpr (MODE != MODE_ONE_GLOBAL) {
#pragma unroll
        for (int r = 0; r < kPre; ++r) {
            const uint32_t i = threadIdx.x + (uint32_t)r * WARPS * 32;
            pre[r] = i < n1 ? p.one[i] : (i < n1 + nc ? p.pair[i - n1] : 0u);
        }
    }
    if (ntiles) issue(0);
    cp_async_commit();
    for (uint32_t t = 1; t < 1 + p.prefetch_tiles; ++t) prefetch(t);
    const bool has_lookback = active && b > p.lo && p.lookback > 0;

    OneTable T;
    T.reset_entry = p.reset_entry;
    uint32_t pair_base = 0;
    if constexpr (MODE == MODE_ONE_GLOBAL) {
        T.t = p.one;
    } else {
        // one-symbol table, then (pair mode) the compact pair table right after it
        uint32_t *tabs = one_s;
#pragma unroll
        for (int r = 0; r < kPre; ++r) {
            const uint32_t i = threadIdx.x + (uint32_t)r * WARPS * 32;
            if (i < n1 + nc) tabs[i] = pre[r];
        }
        for (uint32_t i = threadIdx.x + (uint32_t)kPre * WARPS * 32; i < n1 + nc; i += WARPS * 32)
            tabs[i] = i < n1 ? p.one[i] : p.pair[i - n1];
        T.t = one_s;
        if (MODE == MODE_PAIR) {
            // every lane's copy of the pair table is expanded from the compact copy
            const uint32_t *cbuf = one_s + n1;
            uint32_t after_c = smem_base + (uint32_t)WARPS * kStages * kStageBytes + (n1 + nc) * 4u;
            pair_base = (after_c + 2047u) & ~2047u;   // bits 0..10 of the base are zero
            uint32_t *pair_ptr = reinterpret_cast<uint32_t *>(smem + (pair_base - smem_base));
            __syncthreads();
            const uint32_t n2 = p.n_states * 16u * 32u;
            for (uint32_t i = threadIdx.x; i < n2; i += WARPS * 32) {
                uint32_t e = cbuf[i >> 5];
                uint32_t nx = e & 0x00FFFFFFu, c = e >> 24;
                pair_ptr[i] = (c << kCountShift) | (pair_base + nx * (uint32_t)kPairRowBytes + (i & 31u) * 4u);
            }
        }
    }
    __syncthreads();
    uint32_t *stash = POS ? p.stash + seg * (kStashCap * 3) : nullptr;
    uint32_t nrec = 0;

    // ---- speculated start state: q0, or the state reached from q0 over the lookback window
    uint32_t q = 0;
    if (has_lookback) {   // the 'lookback' bytes in front of the chunk
        const uint64_t from = b - p.lo > p.lookback ? b - p.lookback : p.lo;
        for (uint64_t off = from; off < b; ++off) q = T.step(q, p.abase[off]) & 0x7FFFFFFFu;
    }
    uint32_t spec = q;
    uint32_t cnt = 0;
    uint32_t cur = pair_base + q * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u;

    // tiles [t_full0, t_full1) of this chunk lie entirely inside the sequence; tiles from
    // t_live on lie past its end (only the last chunk has any)
    uint32_t t_live = 0, t_full0 = 0, t_full1 = 0;
    if (active) {
        const uint64_t rem = p.hi - b;
        t_live = rem >= S ? ntiles : (uint32_t)((rem + kTile - 1) / kTile);
        t_full1 = rem >= S ? ntiles : (uint32_t)(rem / kTile);
        t_full0 = b < p.lo ? 1u : 0u;
    }
    const uint32_t lut_lo = p.lut_lo, lut_hi = p.lut_hi;
    for (uint32_t t = 0; t < ntiles; ++t) {
        cp_async_wait<0>();
        __syncwarp();   // tile t of all 32 rows is visible to the warp
        const uint64_t row_off = b + (uint64_t)t * kTile;
        const bool live = t < t_live;
        const bool full = t >= t_full0 && t < t_full1;
        uint32_t w[32];
        {
            // the lane's row, un-swizzled: 16-byte chunk c sits at slot c ^ (lane & 7)
            const uint8_t *srow = stage_ptr + lane * kTile;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                uint4 v = *reinterpret_cast<const uint4 *>(srow + ((c ^ (lane & 7)) * 16));
                w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
            }
        }
        __syncwarp();   // every lane holds its row: the stage can be refilled
        if (t + 1 < ntiles) issue(t + 1);
        cp_async_commit();
        if (p.prefetch_tiles) prefetch(t + 1 + p.prefetch_tiles);
        if (t == 0) head_s[threadIdx.x] = make_uint4(w[0], w[1], w[2], w[3]);
        if (!live) continue;

        if (MODE == MODE_PAIR) {
            bool done = false;
            if (full) {
                uint32_t acc = 0, err = 0, rc = 0, c2 = cur;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    // codes of the 4 bytes sit at bits 1..2 of each byte of x; y = x*65
                    // puts the first pair at bits 7..10 and the second at bits 23..26, and
                    // is zero at bits 27..30, so the mux below forms clean addresses
                    const uint32_t x = w[k] & 0x06060606u;
                    const uint32_t y = mad_lo(x, 65u, 0u);
                    const uint32_t e1 = lds_u32(mux_pair(c2, y));
                    const uint32_t e2 = lds_u32(mux_pair(e1, y >> 16));
                    acc = mad_lo(e1, p.k1, acc);
                    acc = mad_lo(e2, p.k1, acc);
                    c2 = e2;
                    if (k % 3 == 2 || k == 31) {     // <= 6 entries: count <= 12 fits bits 27..30
                        rc = mad_hi(acc, p.k5, rc);  // rc += acc >> 27
                        acc = 0;
                    }
                    // bit-exact base check: expected lowercase bytes selected by the codes
                    const uint32_t z = x | (x >> 4);
                    const uint32_t sel = __byte_perm(z, 0, 0x0020);
                    const uint32_t expect = __byte_perm(lut_lo, lut_hi, sel);
                    err |= expect ^ w[k];
                }
                if ((err & 0xDFDFDFDFu) == 0) {
                    if (POS && rc)
                        record_hit_row(stash, nrec, t,
                                       ((cur & 0x3FFFFu) - pair_base) / (uint32_t)kPairRowBytes, cnt);
                    cnt += rc;
                    cur = c2 & 0x3FFFFu;
                    done = true;
                }
            }
            if (!done) {
                uint32_t qs = ((cur & 0x3FFFFu) - pair_base) / (uint32_t)kPairRowBytes;
                uint32_t before = cnt;
                // a reset byte or a sequence edge in this row: walk it from global memory
                // (the row was just staged, so it is in L2)
                uint32_t qe = row_bytes_global(T, qs, p.abase, row_off > p.lo ? row_off : p.lo,
                                               row_off + kTile < p.hi ? row_off + kTile : p.hi, p.hi, cnt);
                if (POS && cnt != before) record_hit_row(stash, nrec, t, qs, before);
                cur = pair_base + qe * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u;
            }
        } else {
            uint32_t before = cnt, qs = q;
            q = full ? row_bytes_reg(T, qs, w, cnt)
                     : row_bytes_global(T, qs, p.abase, row_off > p.lo ? row_off : p.lo,
                                        row_off + kTile < p.hi ? row_off + kTile : p.hi, p.hi, cnt);
            if (POS && cnt != before) record_hit_row(stash, nrec, t, qs, before);
        }
    }
    cp_async_wait<0>();
    uint32_t last = q;
    if (MODE == MODE_PAIR) last = ((cur & 0x3FFFFu) - pair_base) / (uint32_t)kPairRowBytes;

    // ---- join inside the block (Sec. III-A) with repair at the converging point (Alg. 1):
    // the true start of a chunk is the last state of the chunk before it, which the lane
    // to the left (or, for lane 0, the previous warp's lane 31) has just computed
    if (lane == 31) warp_last[warp] = last;
    __syncthreads();
    uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, last, 1);
    if (lane == 0) prev = warp > 0 ? warp_last[warp - 1] : 0u;
    const bool has_prev = active && seg > 0 && (lane > 0 || warp > 0);
    bool pending = active && seg > 0 && !has_prev;   // first chunk of the block
    if (has_prev && prev != spec) {
        // run the true start and the speculated start in lockstep over the chunk's first
        // bytes; at the first step where their states are equal, the rest of the chunk is
        // identical for both runs
        const uint64_t vlen64 = p.hi - b;
        const uint32_t vlen = vlen64 < 16 ? (uint32_t)vlen64 : 16u;
        const uint4 h4 = head_s[threadIdx.x];   // the chunk's first 16 bytes
        const uint32_t head[4] = {h4.x, h4.y, h4.z, h4.w};
        uint32_t qa = prev, qs = spec, pa = 0, ps = 0;
        bool conv = false;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (!conv && (uint32_t)k < vlen) {
                const uint32_t byte = (head[k >> 2] >> (8 * (k & 3))) & 0xFFu;
                const uint32_t ea = T.step(qa, byte), es = T.step(qs, byte);
                qa = ea & 0x7FFFFFFFu; qs = es & 0x7FFFFFFFu;
                pa += ea >> 31; ps += es >> 31;
                conv = qa == qs;
            }
        }
        if (conv) {
            const uint32_t delta = pa - ps;   // modulo 2^32; the corrected count is exact
            cnt += delta;
            if (POS) fix_hit_rows(stash, nrec, prev, delta, pa);
            spec = prev;
        } else {
            pending = true;   // the last block repairs it from global memory
        }
    }
    if (active) {
        p.spec_start[seg] = spec;
        p.last_state[seg] = last;
        p.count[seg] = cnt;
        p.flags[seg] = 0;
        if (POS) p.nrec[seg] = nrec;
    }
    if (pending) {
        const uint32_t k = atomicAdd(&p.ctrl[1], 1u);
        if (k < p.pending_cap) p.pending[k] = (uint32_t)seg;
    }
    __threadfence();   // this thread's results are visible before the block's ticket
    // block sum of the chunk counts
    unsigned long long v = active ? cnt : 0u;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    __shared__ unsigned long long red[WARPS];
    __shared__ int is_last;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < WARPS; ++i) t += red[i];
        p.cta_sum[blockIdx.x] = t;
        __threadfence();
        is_last = atomicAdd(&p.ctrl[0], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    finalize_block<WARPS * 32>(p);
}

// ------------------------------------------------------------ extraction

struct EmitParams {
    const uint8_t *abase;
    uint64_t lo, hi, seg_bytes, nseg;
    const uint32_t *one;
    uint32_t reset_entry, n_states;
    const uint32_t *last_state, *count, *stash, *nrec;
    const uint8_t *flags;
    const unsigned long long *cta_off;
    uint64_t *out;
    uint64_t cap;
};

constexpr int kEmitWalkers = 256;    // threads of an extraction block that walk rows
constexpr int kEmitRowPitch = 144;   // 128-byte row + 16 bytes: conflict-free 16-byte stores
constexpr int kEmitRecs = 512;       // hit-row records of a block cached in shared memory

// Copies aligned offsets [rs, rs + 128) of the sequence into a shared row slot with eight
// independent 16-byte loads (a granule is read only if it starts before hi).
__device__ __forceinline__ void stage_row(uint8_t *slot, const uint8_t *abase, uint64_t rs, uint64_t hi) {
    uint4 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint64_t g = rs + 16u * j;
        v[j] = g < hi ? *reinterpret_cast<const uint4 *>(abase + g) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4 *>(slot + 16 * j) = v[j];
}

// One block per scan block, one thread per chunk. Each chunk's output offset is its block's
// offset plus the block-exclusive prefix of the chunk counts. The recorded hit rows are
// spread over the first kEmitWalkers threads: each stages a row in its shared slot and
// walks it from the recorded start state, writing the accepting positions in order.
// Flagged or overflowing chunks are rescanned row by row from their true start (the
// previous chunk's last state). The walk maps each byte through a 256-entry class table
// (A, C, T, G -> code, anything else -> 4) and a five-column transition table whose fifth
// column is the reset symbol.
__global__ void __launch_bounds__(1024) emit_kernel(EmitParams p, uint32_t tab5_in_smem) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ unsigned long long wsum[32];
    __shared__ uint32_t wsum2[32];
    __shared__ uint8_t cls[256];
    __shared__ uint8_t s_rescan[1024];
    __shared__ uint4 s_rec[kEmitRecs];   // (tile, start state, count before, chunk index)
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    // dynamic shared memory: [row slots: walkers x pitch][offsets: nthr x 8][slots: nthr+1 x 4][table]
    unsigned long long *s_off = reinterpret_cast<unsigned long long *>(dsm + kEmitWalkers * kEmitRowPitch);
    uint32_t *s_slot = reinterpret_cast<uint32_t *>(s_off + nthr);
    uint32_t *tab5 = s_slot + nthr + 1;
    if (tid < 256) {
        const uint32_t c = (tid >> 1) & 3u;
        cls[tid] = byte_is_base(tid) ? (uint8_t)c : (uint8_t)4;
    }
    if (tab5_in_smem)
        for (uint32_t i = tid; i < p.n_states * 5u; i += nthr) {
            const uint32_t q = i / 5u, col = i - q * 5u;
            tab5[i] = col < 4 ? p.one[q * 4u + col] : p.reset_entry;
        }
    const uint64_t c = (uint64_t)blockIdx.x * nthr + tid;
    const bool act = c < p.nseg;
    const unsigned long long v = act ? p.count[c] : 0u;
    const uint32_t nr = act ? p.nrec[c] : 0u;
    const bool rescan = act && v > 0 && (p.flags[c] != 0 || nr > (uint32_t)kStashCap);
    const uint32_t rows = (act && !rescan) ? nr : 0u;
    unsigned long long x = v;
    uint32_t y = rows;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long xa = __shfl_up_sync(0xFFFFFFFFu, x, o);
        const uint32_t ya = __shfl_up_sync(0xFFFFFFFFu, y, o);
        if ((tid & 31) >= (uint32_t)o) { x += xa; y += ya; }
    }
    if ((tid & 31) == 31) { wsum[tid >> 5] = x; wsum2[tid >> 5] = y; }
    __syncthreads();
    if (tid < 32) {
        const uint32_t nw = nthr >> 5;
        unsigned long long a = tid < nw ? wsum[tid] : 0ull;
        uint32_t bb = tid < nw ? wsum2[tid] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long aa = __shfl_up_sync(0xFFFFFFFFu, a, o);
            const uint32_t ba = __shfl_up_sync(0xFFFFFFFFu, bb, o);
            if (tid >= (uint32_t)o) { a += aa; bb += ba; }
        }
        if (tid < nw) { wsum[tid] = a; wsum2[tid] = bb; }
    }
    __syncthreads();
    const unsigned long long bx = (tid >> 5) ? wsum[(tid >> 5) - 1] : 0ull;
    const uint32_t by = (tid >> 5) ? wsum2[(tid >> 5) - 1] : 0u;
    const unsigned long long off = p.cta_off[blockIdx.x] + bx + x - v;
    s_off[tid] = off;
    s_slot[tid] = by + y - rows;
    if (tid == nthr - 1) s_slot[nthr] = by + y;
    s_rescan[tid] = rescan ? 1 : 0;
    // each chunk copies its hit-row records into shared memory (first kEmitRecs rows)
    const uint32_t slot0 = by + y - rows;
    for (uint32_t i = 0; i < rows; ++i) {
        if (slot0 + i >= (uint32_t)kEmitRecs) break;
        const uint32_t *rec = p.stash + c * (kStashCap * 3) + 3 * i;
        s_rec[slot0 + i] = make_uint4(rec[0], rec[1], rec[2], (uint32_t)tid);
    }
    __syncthreads();
    const uint32_t total_rows = s_slot[nthr];
    const uint32_t *tab = tab5_in_smem ? tab5 : nullptr;

    // walks bytes [k0, k1) of the row at aligned offset rs (staged in 'slot') from state q
    auto walk_row = [&](uint8_t *slot, uint64_t rs, uint32_t k0, uint32_t k1, uint32_t q,
                        unsigned long long &o) {
        stage_row(slot, p.abase, rs, p.hi);
        const uint64_t pos0 = rs - p.lo;
        for (uint32_t k = k0; k < k1; ++k) {
            const uint32_t cl = cls[slot[k]];
            const uint32_t e = tab ? tab[q * 5u + cl] : (cl < 4 ? p.one[q * 4u + cl] : p.reset_entry);
            q = e & 0x7FFFFFFFu;
            if (e >> 31) {
                if (o < p.cap) p.out[o] = pos0 + k;
                ++o;
            }
        }
        return q;
    };
    auto row_span = [&](uint64_t rs, uint64_t from, uint64_t to, uint32_t &k0, uint32_t &k1) {
        k0 = from > rs ? (uint32_t)(from - rs) : 0u;
        k1 = to < rs + kTile ? (uint32_t)(to - rs) : (uint32_t)kTile;
    };
    const uint64_t S = p.seg_bytes;
    // rescans (rare), by walker threads in turn
    if (tid < kEmitWalkers) {
        uint8_t *slot = dsm + tid * kEmitRowPitch;
        for (uint32_t j = tid; j < nthr; j += kEmitWalkers) {
            if (!s_rescan[j]) continue;
            const uint64_t cj = (uint64_t)blockIdx.x * nthr + j;
            const unsigned long long oj = s_off[j];
            if (oj >= p.cap) continue;
            unsigned long long o = oj;
            const uint64_t b = cj * S;
            const uint64_t from = b > p.lo ? b : p.lo;
            const uint64_t to = b + S < p.hi ? b + S : p.hi;
            uint32_t q = cj ? p.last_state[cj - 1] : 0u;
            for (uint64_t rs = b; rs < to && o < p.cap; rs += kTile) {
                uint32_t k0, k1;
                row_span(rs, from, to, k0, k1);
                q = walk_row(slot, rs, k0, k1, q, o);
            }
        }
        // hit rows
        for (uint32_t r = tid; r < total_rows; r += kEmitWalkers) {
            uint32_t lo, rec[3];
            if (r < (uint32_t)kEmitRecs) {
                const uint4 rr = s_rec[r];
                rec[0] = rr.x; rec[1] = rr.y; rec[2] = rr.z; lo = rr.w;
            } else {
                lo = 0;
                uint32_t hi = nthr - 1;   // largest j with s_slot[j] <= r
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (s_slot[mid] <= r) lo = mid; else hi = mid - 1;
                }
                const uint64_t cl = (uint64_t)blockIdx.x * nthr + lo;
                const uint32_t *g = p.stash + cl * (kStashCap * 3) + 3 * (r - s_slot[lo]);
                rec[0] = g[0]; rec[1] = g[1]; rec[2] = g[2];
            }
            const uint64_t cj = (uint64_t)blockIdx.x * nthr + lo;
            unsigned long long o = s_off[lo] + rec[2];
            if (o >= p.cap) continue;
            const uint64_t b = cj * S;
            const uint64_t cend = b + S < p.hi ? b + S : p.hi;
            const uint64_t rs = b + (uint64_t)rec[0] * kTile;
            uint32_t k0, k1;
            row_span(rs, rs > p.lo ? rs : p.lo, rs + kTile < cend ? rs + kTile : cend, k0, k1);
            walk_row(slot, rs, k0, k1, rec[1], o);
        }
    }
}

__global__ void write_zero_kernel(uint64_t *out) { *out = 0; }

}  // namespace

// ------------------------------------------------------------------ host side

namespace dnalib {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DNA_OK;
    if (e == cudaErrorMemoryAllocation) return DNA_ERR_NOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
        e == cudaErrorNoKernelImageForDevice)
        return DNA_ERR_NO_DEVICE;
    return DNA_ERR_CUDA;
}

DeviceProps device_props(int dev) {
    static std::mutex mu;
    static std::vector<DeviceProps> cache;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1);
    if (cache[dev].sms == 0) {
        cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cache[dev].smem_optin = (size_t)v;
    }
    return cache[dev];
}

// Raises a kernel's dynamic shared-memory limit to 'bytes' once per (kernel, device).
int ensure_smem_optin(const void *fn, int device, size_t bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &d : done)
        if (d.first == fn && d.second == device) return DNA_OK;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_status(e);
    done.emplace_back(fn, device);
    return DNA_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

std::atomic<uint64_t> g_launches{0};
void record_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Kernel timing for dna_profile_*: an event pair around each timed launch, resolved
// (and recycled) when the counters are read.
static std::atomic<int> g_profile{0};
static std::mutex g_prof_mu;
struct ProfRec { cudaEvent_t a, b; int which; };
static std::vector<ProfRec> g_prof_pending;
static std::vector<ProfRec> g_prof_free;
static double g_prof_ms[PROF_N] = {};
static uint64_t g_prof_calls[PROF_N] = {};

ProfToken prof_begin(cudaStream_t s) {
    ProfToken t;
    if (g_profile.load(std::memory_order_relaxed) == 0) return t;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_prof_free.empty()) {
            t.a = g_prof_free.back().a; t.b = g_prof_free.back().b;
            g_prof_free.pop_back();
        }
    }
    if (!t.a && (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess)) {
        t.a = t.b = nullptr;
        return t;
    }
    cudaEventRecord(t.a, s);
    return t;
}

void prof_end(ProfToken t, cudaStream_t s, int which) {
    if (!t.a) return;
    cudaEventRecord(t.b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending.push_back({t.a, t.b, which});
}

void profile_set(int on) { g_profile.store(on ? 1 : 0); }

void profile_collect(dna_profile_t *out, int reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof_pending) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_prof_ms[r.which] += ms;
            ++g_prof_calls[r.which];
        }
        g_prof_free.push_back(r);
    }
    g_prof_pending.clear();
    out->scan_kernel_ms = g_prof_ms[PROF_SCAN];
    out->scan_kernel_calls = g_prof_calls[PROF_SCAN];
    out->kernel_launches = g_launches.load();
    out->emit_kernel_ms = g_prof_ms[PROF_EMIT];
    out->emit_kernel_calls = g_prof_calls[PROF_EMIT];
    out->batch_kernel_ms = g_prof_ms[PROF_BATCH];
    out->batch_kernel_calls = g_prof_calls[PROF_BATCH];
    out->ingest_kernel_ms = g_prof_ms[PROF_INGEST];
    out->ingest_kernel_calls = g_prof_calls[PROF_INGEST];
    if (reset) {
        for (int k = 0; k < PROF_N; ++k) { g_prof_ms[k] = 0; g_prof_calls[k] = 0; }
        g_launches.store(0);
    }
}

}  // namespace dnalib

namespace {

// Dynamic shared memory of the scan kernel (the launch argument).
size_t scan_smem_bytes(int mode, int warps, uint32_t n_states) {
    size_t s = (size_t)warps * kStages * kStageBytes;
    if (mode == MODE_ONE_GLOBAL) return s;
    s += (size_t)n_states * 16;
    if (mode == MODE_PAIR) s += (size_t)n_states * 64 + 2048 + (size_t)n_states * kPairRowBytes;
    return s;
}

// Static shared memory of the scan kernel: each chunk's first 16 bytes + one word per warp.
size_t scan_static_smem(int warps) { return (size_t)warps * 32 * 16 + (size_t)warps * 20 + 1024; }

size_t scan_total_smem(int mode, int warps, uint32_t n_states) {
    return scan_smem_bytes(mode, warps, n_states) + scan_static_smem(warps);
}

using ScanFn = void (*)(ScanParams);

ScanFn scan_fn(int mode, int warps, bool pos) {
#define PICK(M, W)                                                   \
    if (mode == M && warps == W) return pos ? scan_kernel<M, W, true> : scan_kernel<M, W, false>;
    PICK(MODE_PAIR, 8) PICK(MODE_PAIR, 16) PICK(MODE_PAIR, 24) PICK(MODE_PAIR, 32)
    PICK(MODE_ONE_SMEM, 8) PICK(MODE_ONE_SMEM, 16) PICK(MODE_ONE_SMEM, 24) PICK(MODE_ONE_SMEM, 32)
    PICK(MODE_ONE_GLOBAL, 8) PICK(MODE_ONE_GLOBAL, 16) PICK(MODE_ONE_GLOBAL, 24) PICK(MODE_ONE_GLOBAL, 32)
#undef PICK
    return nullptr;
}

// code order (A, C, T, G) -> table column (A, C, G, T)
constexpr int kColOfCode[4] = {0, 1, 3, 2};

size_t max_pair_states(size_t smem_optin, int warps) {
    size_t fixed = (size_t)warps * kStages * kStageBytes + 2048 + scan_static_smem(warps);
    if (smem_optin <= fixed) return 0;
    return (smem_optin - fixed) / (kPairRowBytes + 16 + 64);
}

struct Plan {
    int mode, warps;
    bool pos;
    uint32_t prefetch;
    uint64_t seg_bytes, nseg;
    uint32_t lookback;
    size_t smem;
    int grid;
};

int make_plan(const dna_dfa *d, uint64_t total, bool pos, const dna_plan *ov, Plan &pl) {
    DeviceProps pr = device_props(d->device);
    const size_t optin = pr.smem_optin ? pr.smem_optin : 232448;
    int mode;
    uint32_t req = ov ? ov->placement : 0;
    int warps = ov && ov->warps_per_cta ? (int)ov->warps_per_cta : 0;
    if (warps && warps != 8 && warps != 16 && warps != 24 && warps != 32) return DNA_ERR_INVALID_ARG;
    if (req == DNA_PLACE_AUTO) req = d->placement;
    if (req == DNA_PLACE_SMEM_PAIR) mode = MODE_PAIR;
    else if (req == DNA_PLACE_SMEM_ONE) mode = MODE_ONE_SMEM;
    else if (req == DNA_PLACE_GLOBAL_ONE) mode = MODE_ONE_GLOBAL;
    else return DNA_ERR_INVALID_ARG;
    if (!warps) {
        warps = 8;
        for (int w : {24, 16}) if (scan_total_smem(mode, w, d->n_states) <= optin) { warps = w; break; }
    }
    size_t smem = scan_smem_bytes(mode, warps, d->n_states);
    if (scan_total_smem(mode, warps, d->n_states) > optin) return DNA_ERR_CAPACITY;
    uint32_t lb = ov && ov->lookback ? ov->lookback : d->lookback;
    if (lb > kMaxLookback) return DNA_ERR_INVALID_ARG;
    ScanFn fn = scan_fn(mode, warps, pos);
    if (!fn) return DNA_ERR_INVALID_ARG;
    uint32_t pf = kDefaultPrefetch;
    if (ov && ov->prefetch_tiles) pf = ov->prefetch_tiles >= 255 ? 0 : ov->prefetch_tiles;
    if (pf > 64) return DNA_ERR_INVALID_ARG;
    // the shared-memory opt-in is set once per kernel variant (to the device maximum),
    // the occupancy once per automaton and variant
    const int wi = warps == 8 ? 0 : warps == 16 ? 1 : warps == 24 ? 2 : 3;
    std::atomic<int> &occ = const_cast<dna_dfa *>(d)->per_sm[mode][wi][pos ? 1 : 0];
    int per_sm = occ.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        int rc = ensure_smem_optin((const void *)fn, d->device, optin - scan_static_smem(warps));
        if (rc) return rc;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
        if (e != cudaSuccess) return cuda_status(e);
        if (per_sm < 1) per_sm = 1;
        occ.store(per_sm, std::memory_order_relaxed);
    }
    uint64_t S;
    if (ov && ov->chunk_bytes) {
        if (ov->chunk_bytes % kTile) return DNA_ERR_INVALID_ARG;
        S = ov->chunk_bytes;
    } else {
        uint64_t lanes = (uint64_t)pr.sms * per_sm * warps * 32;
        S = (total + lanes - 1) / lanes;
        S = (S + kTile - 1) / kTile * kTile;
        if (S < kTile) S = kTile;
    }
    pl.mode = mode; pl.warps = warps; pl.seg_bytes = S; pl.pos = pos; pl.prefetch = pf;
    pl.nseg = (total + S - 1) / S;
    pl.lookback = lb; pl.smem = smem;
    uint64_t lanes_per_cta = (uint64_t)warps * 32;
    pl.grid = (int)((pl.nseg + lanes_per_cta - 1) / lanes_per_cta);
    return DNA_OK;
}

// device scratch carved from one stream-ordered allocation
struct Scratch {
    uint32_t *spec_start, *last_state, *count, *nrec, *stash, *pending, *pending_a, *div_list, *ctrl;
    uint8_t *flags;
    unsigned long long *cta_sum, *cta_off;
    size_t bytes;
};


void carve(Scratch &s, uint64_t nseg, uint64_t nblocks, bool positions, uint32_t pending_cap,
           uint32_t div_cap, uint8_t *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) { uint8_t *q = base ? base + off : nullptr; off = align_up(off + bytes, 256); return q; };
    s.ctrl = (uint32_t *)take(16);
    s.cta_sum = (unsigned long long *)take(nblocks * 8);
    s.cta_off = (unsigned long long *)take(nblocks * 8);
    s.spec_start = (uint32_t *)take(nseg * 4);
    s.last_state = (uint32_t *)take(nseg * 4);
    s.count = (uint32_t *)take(nseg * 4);
    s.flags = (uint8_t *)take(nseg);
    s.pending = (uint32_t *)take((size_t)pending_cap * 4);
    s.pending_a = (uint32_t *)take((size_t)pending_cap * 4);
    s.div_list = (uint32_t *)take((size_t)div_cap * 4);
    s.stash = positions ? (uint32_t *)take(nseg * kStashCap * 12) : nullptr;
    s.nrec = positions ? (uint32_t *)take(nseg * 4) : nullptr;
    s.bytes = off;
}

}  // namespace

namespace dnalib {

int scan_impl(const dna_dfa *d, const uint8_t *seq, uint64_t len, cudaStream_t stream,
              uint64_t *out_count, uint64_t *out_positions, uint64_t cap, const dna_plan *ov) {
    if (!d || !out_count || (len > 0 && !seq)) return DNA_ERR_INVALID_ARG;
    if (len > (1ull << 40)) return DNA_ERR_INVALID_ARG;
    int cur_dev = -1;
    DNA_CUDA(cudaGetDevice(&cur_dev));
    if (cur_dev != d->device) return DNA_ERR_INVALID_ARG;
    if (len == 0) {
        write_zero_kernel<<<1, 1, 0, stream>>>(out_count);
        record_launch();
        return cuda_status(cudaGetLastError());
    }
    const uint64_t shift = (uint64_t)((uintptr_t)seq & 15u);
    const uint8_t *abase = seq - shift;
    const uint64_t total = len + shift;
    const bool positions = out_positions != nullptr && cap > 0;
    Plan pl;
    int rc = make_plan(d, total, positions, ov, pl);
    if (rc) return rc;
    const uint64_t nblocks = (uint64_t)pl.grid;
    const uint32_t pending_cap = (uint32_t)nblocks + 4096u;
    const uint32_t div_cap = 4096;
    Scratch s;
    carve(s, pl.nseg, nblocks, positions, pending_cap, div_cap, nullptr);
    void *mem = nullptr;
    DNA_CUDA(cudaMallocAsync(&mem, s.bytes, stream));
    carve(s, pl.nseg, nblocks, positions, pending_cap, div_cap, (uint8_t *)mem);
    cudaError_t e = cudaMemsetAsync(s.ctrl, 0, 16, stream);

    ScanParams sp;
    sp.abase = abase; sp.lo = shift; sp.hi = total; sp.seg_bytes = pl.seg_bytes; sp.nseg = pl.nseg;
    sp.lookback = pl.lookback; sp.n_states = d->n_states; sp.reset_entry = d->reset_entry;
    sp.one = d->d_one; sp.pair = d->d_pair;
    sp.spec_start = s.spec_start; sp.last_state = s.last_state; sp.count = s.count;
    sp.stash = s.stash; sp.nrec = s.nrec; sp.flags = s.flags;
    sp.prefetch_tiles = pl.prefetch;
    sp.ctrl = s.ctrl; sp.pending = s.pending; sp.pending_cap = pending_cap; sp.pending_a = s.pending_a;
    sp.div_list = s.div_list; sp.div_cap = div_cap;
    sp.cta_sum = s.cta_sum; sp.cta_off = s.cta_off; sp.out_count = out_count;
    sp.k1 = 1u; sp.k16 = 1u << 16; sp.k5 = 1u << 5; sp.k28 = 1u << 28;
    sp.lut_lo = 0x00630061u; sp.lut_hi = 0x00670074u;

    const ProfToken tok = e == cudaSuccess ? prof_begin(stream) : ProfToken{};
    if (e == cudaSuccess) {
        scan_fn(pl.mode, pl.warps, pl.pos)<<<pl.grid, pl.warps * 32, pl.smem, stream>>>(sp);
        e = cudaGetLastError();
        record_launch();
    }
    prof_end(tok, stream, PROF_SCAN);
    if (e == cudaSuccess && positions) {
        EmitParams ep;
        ep.abase = abase; ep.lo = shift; ep.hi = total; ep.seg_bytes = pl.seg_bytes; ep.nseg = pl.nseg;
        ep.one = d->d_one; ep.reset_entry = d->reset_entry; ep.n_states = d->n_states;
        ep.last_state = s.last_state; ep.count = s.count; ep.stash = s.stash; ep.nrec = s.nrec;
        ep.flags = s.flags; ep.cta_off = s.cta_off; ep.out = out_positions; ep.cap = cap;
        const uint32_t cpb = (uint32_t)pl.warps * 32u;   // one extraction thread per chunk
        const uint32_t tab5_smem = d->n_states * 5u <= 4096u ? 1u : 0u;
        const size_t esmem = (size_t)kEmitWalkers * kEmitRowPitch + (size_t)cpb * 8 + (size_t)(cpb + 1) * 4 +
                             (tab5_smem ? (size_t)d->n_states * 20 : 0);
        const size_t optin = device_props(d->device).smem_optin;
        // the extraction kernel's static shared memory is about 10 KB; 16 KB is reserved
        int rc2 = ensure_smem_optin((const void *)emit_kernel, d->device, (optin ? optin : 232448) - 16384);
        if (rc2) e = cudaErrorInvalidValue;
        else {
            const ProfToken et = prof_begin(stream);
            emit_kernel<<<pl.grid, cpb, esmem, stream>>>(ep, tab5_smem);
            prof_end(et, stream, PROF_EMIT);
        }
        e = cudaGetLastError();
        record_launch();
    }
    cudaError_t e2 = cudaFreeAsync(mem, stream);
    if (e == cudaSuccess) e = e2;
    return cuda_status(e);
}

}  // namespace dnalib

// ====================================================================== C ABI

extern "C" int dfa_load(const uint32_t *table, uint32_t n_states, const uint8_t *accept_mask,
                        dna_dfa **out) {
    if (!table || !accept_mask || !out || n_states == 0 || n_states > kMaxStates)
        return DNA_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < 4ull * n_states; ++i)
        if (table[i] >= n_states) return DNA_ERR_INVALID_ARG;
    int dev = 0;
    {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_status(e);
    }
    dna_dfa *d = new (std::nothrow) dna_dfa;
    if (!d) return DNA_ERR_NOMEM;
    d->n_states = n_states;
    d->device = dev;
    auto acc = [&](uint32_t q) { return (accept_mask[q >> 3] >> (q & 7)) & 1u; };
    d->accept0 = acc(0);
    d->reset_entry = d->accept0 << 31;
    std::vector<uint32_t> one(4ull * n_states);
    for (uint32_t q = 0; q < n_states; ++q)
        for (int c = 0; c < 4; ++c) {
            uint32_t nx = table[4ull * q + kColOfCode[c]];
            one[4ull * q + c] = nx | (acc(nx) << 31);
        }
    d->definite_depth = dnalib::definite_depth(table, n_states, (int)kMaxLookback, 4096);
    // q0 speculation repaired from the chunk's first 16 bytes works whenever runs meet
    // within 16 symbols (definite depth <= 16, and in practice most automata on DNA);
    // a known larger depth gets an exact lookback instead
    d->lookback = (d->definite_depth > 16) ? (uint32_t)d->definite_depth : 0u;
    DeviceProps pr = device_props(dev);
    size_t optin = pr.smem_optin ? pr.smem_optin : 232448;
    if (n_states <= max_pair_states(optin, 8)) d->placement = DNA_PLACE_SMEM_PAIR;
    else if (scan_total_smem(MODE_ONE_SMEM, 8, n_states) <= optin) d->placement = DNA_PLACE_SMEM_ONE;
    else d->placement = DNA_PLACE_GLOBAL_ONE;
    cudaError_t e = cudaMalloc(&d->d_one, sizeof(uint32_t) * one.size());
    if (e == cudaSuccess) e = cudaMemcpy(d->d_one, one.data(), sizeof(uint32_t) * one.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_states <= max_pair_states(optin, 8)) {
        std::vector<uint32_t> pair(16ull * n_states);
        for (uint32_t q = 0; q < n_states; ++q)
            for (int b0 = 0; b0 < 4; ++b0)
                for (int b1 = 0; b1 < 4; ++b1) {
                    uint32_t e1 = one[4ull * q + b0];
                    uint32_t q1 = e1 & 0x7FFFFFFFu;
                    uint32_t e2 = one[4ull * q1 + b1];
                    uint32_t q2 = e2 & 0x7FFFFFFFu;
                    uint32_t cnt = (e1 >> 31) + (e2 >> 31);
                    pair[16ull * q + b0 + 4 * b1] = q2 | (cnt << 24);
                }
        e = cudaMalloc(&d->d_pair, sizeof(uint32_t) * pair.size());
        if (e == cudaSuccess) e = cudaMemcpy(d->d_pair, pair.data(), sizeof(uint32_t) * pair.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(d->d_one);
        cudaFree(d->d_pair);
        delete d;
        return cuda_status(e);
    }
    *out = d;
    return DNA_OK;
}

extern "C" void dfa_free(dna_dfa *d) {
    if (!d) return;
    cudaFree(d->d_one);
    cudaFree(d->d_pair);
    delete d;
}

extern "C" int dfa_info(const dna_dfa *d, dna_dfa_info *out) {
    if (!d || !out) return DNA_ERR_INVALID_ARG;
    out->n_states = d->n_states;
    out->definite_depth = d->definite_depth;
    out->lookback = d->lookback;
    out->placement = d->placement;
    out->accept_start = d->accept0;
    out->device = d->device;
    return DNA_OK;
}

extern "C" int dna_scan(const dna_dfa *dfa, const uint8_t *seq, uint64_t len, dna_stream_t stream,
                        uint64_t *out_count, uint64_t *out_positions, uint64_t positions_capacity) {
    return scan_impl(dfa, seq, len, (cudaStream_t)stream, out_count, out_positions,
                     positions_capacity, nullptr);
}

extern "C" int dna_scan_host(const dna_dfa *dfa, const uint8_t *seq_host, uint64_t len,
                             dna_stream_t stream_h, uint64_t *count_host, uint64_t *positions_host,
                             uint64_t positions_capacity) {
    if (!dfa || !count_host || (len > 0 && !seq_host)) return DNA_ERR_INVALID_ARG;
    if (positions_capacity > 0 && !positions_host) return DNA_ERR_INVALID_ARG;
    if (len > (1ull << 40) || positions_capacity > (1ull << 40)) return DNA_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_h;
    // one stream-ordered buffer: [count (8 B)][positions][sequence], the sequence
    // 16-byte aligned so the scan starts on a full granule
    const uint64_t cap = positions_host ? positions_capacity : 0;
    const size_t seq_off = align_up(8 + (size_t)cap * 8, 256);
    void *mem = nullptr;
    DNA_CUDA(cudaMallocAsync(&mem, seq_off + (size_t)len + 16, stream));
    uint8_t *base = (uint8_t *)mem;
    uint64_t *d_count = (uint64_t *)base;
    uint64_t *d_pos = cap ? (uint64_t *)(base + 8) : nullptr;
    uint8_t *d_seq = base + seq_off;
    cudaError_t e = len ? cudaMemcpyAsync(d_seq, seq_host, len, cudaMemcpyHostToDevice, stream) : cudaSuccess;
    int rc = DNA_OK;
    if (e == cudaSuccess) rc = scan_impl(dfa, d_seq, len, stream, d_count, d_pos, cap, nullptr);
    if (e == cudaSuccess && rc == DNA_OK) {
        e = cudaMemcpyAsync(count_host, d_count, 8, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess && cap) {
            const uint64_t n = *count_host < cap ? *count_host : cap;
            if (n) {
                e = cudaMemcpyAsync(positions_host, d_pos, n * 8, cudaMemcpyDeviceToHost, stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            }
        }
    }
    cudaError_t ef = cudaFreeAsync(mem, stream);
    if (e == cudaSuccess) e = ef;
    if (rc != DNA_OK) return rc;
    if (e != cudaSuccess) return cuda_status(e);
    return cap && *count_host > cap ? DNA_ERR_CAPACITY : DNA_OK;
}

extern "C" int dna_scan_planned(const dna_dfa *dfa, const uint8_t *seq, uint64_t len,
                                dna_stream_t stream, uint64_t *out_count, uint64_t *out_positions,
                                uint64_t positions_capacity, const dna_plan *plan) {
    return scan_impl(dfa, seq, len, (cudaStream_t)stream, out_count, out_positions,
                     positions_capacity, plan);
}

// ------------------------------------------------------- allocation-free count

// Scratch of dna_scan_count_static: one array per process, present on every device that
// loads this library, for its lifetime. Host code never uses the name as an address; the
// device address comes from cudaGetSymbolAddress, once per device.
constexpr size_t kStaticScratchBytes = 4u << 20;     // 4 MiB
constexpr uint64_t kStaticMaxLen = 1ull << 36;       // 64 GiB of sequence per call
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

namespace {

std::mutex g_static_mu;
std::vector<void *> g_static_addr;   // per device: device address of g_static_scratch

// Set-up on the first call for a device (that device is current): looks up the device
// address of the scratch array. No allocation is made.
int static_scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if ((int)g_static_addr.size() <= dev) g_static_addr.resize(dev + 1, nullptr);
    if (!g_static_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) return e != cudaSuccess ? cuda_status(e) : DNA_ERR_CUDA;
        g_static_addr[dev] = ptr;
    }
    *out = g_static_addr[dev];
    return DNA_OK;
}

}  // namespace

extern "C" int dna_scan_count_static(const dna_dfa *d, const uint8_t *seq, uint64_t len,
                                     dna_stream_t stream_h, uint64_t *out_count) {
    cudaStream_t stream = (cudaStream_t)stream_h;
    if (!d || !out_count || (len > 0 && !seq)) return DNA_ERR_INVALID_ARG;
    if (len > kStaticMaxLen) return DNA_ERR_CAPACITY;
    int cur_dev = -1;
    DNA_CUDA(cudaGetDevice(&cur_dev));
    if (cur_dev != d->device) return DNA_ERR_INVALID_ARG;
    void *base = nullptr;
    int rc = static_scratch_address(cur_dev, &base);
    if (rc) return rc;
    if (len == 0) {
        write_zero_kernel<<<1, 1, 0, stream>>>(out_count);
        record_launch();
        return cuda_status(cudaGetLastError());
    }
    const uint64_t shift = (uint64_t)((uintptr_t)seq & 15u);
    const uint8_t *abase = seq - shift;
    const uint64_t total = len + shift;
    Plan pl;
    rc = make_plan(d, total, false, nullptr, pl);
    if (rc) return rc;
    const uint64_t nblocks = (uint64_t)pl.grid;
    const uint32_t pending_cap = (uint32_t)nblocks + 4096u;
    const uint32_t div_cap = 4096;
    Scratch s;
    carve(s, pl.nseg, nblocks, false, pending_cap, div_cap, nullptr);
    if (s.bytes > kStaticScratchBytes) return DNA_ERR_CAPACITY;
    carve(s, pl.nseg, nblocks, false, pending_cap, div_cap, (uint8_t *)base);
    // the counters the kernel expects at zero; everything else is written before it is read
    cudaError_t e = cudaMemsetAsync(s.ctrl, 0, 16, stream);
    if (e != cudaSuccess) return cuda_status(e);
    ScanParams sp;
    sp.abase = abase; sp.lo = shift; sp.hi = total; sp.seg_bytes = pl.seg_bytes; sp.nseg = pl.nseg;
    sp.lookback = pl.lookback; sp.n_states = d->n_states; sp.reset_entry = d->reset_entry;
    sp.one = d->d_one; sp.pair = d->d_pair;
    sp.spec_start = s.spec_start; sp.last_state = s.last_state; sp.count = s.count;
    sp.stash = nullptr; sp.nrec = nullptr; sp.flags = s.flags;
    sp.prefetch_tiles = pl.prefetch;
    sp.ctrl = s.ctrl; sp.pending = s.pending; sp.pending_cap = pending_cap; sp.pending_a = s.pending_a;
    sp.div_list = s.div_list; sp.div_cap = div_cap;
    sp.cta_sum = s.cta_sum; sp.cta_off = s.cta_off; sp.out_count = out_count;
    sp.k1 = 1u; sp.k16 = 1u << 16; sp.k5 = 1u << 5; sp.k28 = 1u << 28;
    sp.lut_lo = 0x00630061u; sp.lut_hi = 0x00670074u;
    scan_fn(pl.mode, pl.warps, false)<<<pl.grid, pl.warps * 32, pl.smem, stream>>>(sp);
    record_launch();
    return cuda_status(cudaGetLastError());
}

extern "C" const char *dna_status_string(int status) {
    switch (status) {
        case DNA_OK: return "ok";
        case DNA_ERR_INVALID_ARG: return "invalid argument";
        case DNA_ERR_NOMEM: return "out of memory";
        case DNA_ERR_CAPACITY: return "capacity exceeded";
        case DNA_ERR_TIMEOUT: return "device wait timed out";
        case DNA_ERR_CUDA: return "CUDA runtime error";
        case DNA_ERR_SYNTAX: return "pattern syntax error";
        case DNA_ERR_EMPTY_WORD: return "pattern matches the empty word";
        case DNA_ERR_NO_DEVICE: return "no usable CUDA device";
        default: return "unknown status";
    }
}

extern "C" void dna_profile_enable(int enable) { dnalib::profile_set(enable); }

extern "C" int dna_profile_read(dna_profile_t *out, int reset) {
    if (!out) return DNA_ERR_INVALID_ARG;
    dnalib::profile_collect(out, reset);
    return DNA_OK;
}
