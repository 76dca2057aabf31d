// scan_kernel.cuh -- the single-sequence chunk-scan kernel (template) and the device
// code of its join. Included by the files that instantiate the kernel variants
// (scan_inst_*.cu); the host side (dna_scan.cu) sees only ScanParams and the
// per-variant lookup functions declared at the end. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "dna_device.cuh"

namespace dnalib {

// ------------------------------------------------------------------ constants

constexpr int kStages = 1;          // one stage per warp: rows are copied to registers first
constexpr int kStageBytes = 32 * kTile;
constexpr int kStashCap = 8;        // hit-row records kept per chunk before a rescan
// set in a hit-row record's tile field when the scan saw the whole row and every byte of
// it was a base (the extraction then walks it two symbols at a time without checking)
constexpr uint32_t kRowAllBases = 0x80000000u;
constexpr uint32_t kMaxLookback = 64;
constexpr uint32_t kMaxStates = 1u << 24;
constexpr uint32_t kDefaultPrefetch = 0;  // tiles of L2 prefetch ahead of the stage

enum Mode { MODE_PAIR = 0, MODE_ONE_SMEM = 1, MODE_ONE_GLOBAL = 2, MODE_HOT = 3, MODE_ONE_REP = 4 };

// MODE_ONE_REP: one-symbol table copied once per lane (lane l's copy in bank l). A state's
// row holds [code][lane] entries of 4 bytes, 512 B in all; an entry is the shared address
// of the next state's row for the same lane (bits 2..6 lane, bits 9..17 row; bits 7..8
// take the next code) | next state accepts (bit 0).
constexpr uint32_t kRepRowBytes = 512;
constexpr uint32_t kRepAddrMask = 0x3FE7Cu;

// Hot-state mode: automata of up to kHotMaxStates states (14-bit state numbers in u16
// entries); its kernels run kHotWarps warps per block.
constexpr uint32_t kHotMaxStates = 16383;
constexpr int kHotWarps = 16;


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
    const uint32_t *given_start;   // [nseg] exact start state of each chunk, or null (speculate)
    uint32_t *spec_start;   // [nseg] speculated start state
    uint32_t *last_state;   // [nseg] state after the chunk (from the speculated start)
    uint32_t *count;        // [nseg] accepting steps (from the speculated start)
    uint32_t *stash;        // [nseg][kStashCap][3] hit rows {tile, start state, count before}, or null
    uint32_t prefetch_tiles; // L2 prefetch distance in tiles (0 = off)
    uint32_t *nrec;         // [nseg] hit rows recorded (may exceed kStashCap)
    uint8_t *flags;         // [nseg] kFlag* bits for the extraction pass
    uint32_t *fix_delta;    // [nseg] count offset shift of a kFlagFixed chunk's later rows
    uint32_t *ctrl;         // [8] zero at launch: finish ticket, pending, diverged, then
                            //   counters: chunks repaired in-block at the converging point,
                            //   block-first chunks joined with a wrong start, cascade walks
    uint32_t reset_ctrl;    // 1: the last block zeroes ctrl[0..5] when it is done with them
                            //   (a control block that stays with the stream between scans)
    uint32_t *pending;      // chunks whose 16-byte in-block repair did not converge (the last
    uint32_t pending_cap;   //   block repairs them; it joins every block's first chunk anyway)
    uint32_t *div_list;     // [div_cap] chunks whose last state changed in a repair
    uint32_t div_cap;
    unsigned long long *cta_sum;   // [grid] count of each block's chunks
    unsigned long long *cta_off;   // [grid] exclusive prefix of cta_sum (for extraction)
    uint4 *block_head;             // [grid] first 16 bytes of each block's first chunk
    uint64_t *out_count;
    // 1 and 2^5 passed at run time so the compiler keeps the multiplies that use them
    // (adds and shifts) on the FMA pipe instead of turning them into ALU ops
    uint32_t k1, k5;
    // lowercase letters selected by the codes (a, c at bytes 0, 2; t, g at bytes 4, 6),
    // passed at run time so that they stay in registers across the unrolled row loop
    uint32_t lut_lo, lut_hi;
    // MODE_HOT: u16 two-symbol rows of the first hot_rows states and one-symbol rows of
    // every state (read as 32-bit words)
    const uint32_t *hot2, *hot1;
    uint32_t hot_rows;
    uint32_t start_state;   // the state the first chunk starts in (q0 for a whole sequence)
    uint32_t *out_last;     // null, or receives the state after the last byte
    const uint32_t *perm_inv;   // null, or device -> caller state numbering (for out_last)
};

using ScanFn = void (*)(ScanParams);

// Kernel variant lookup, one function per placement mode (each defined in its own
// translation unit so the variants compile in parallel); nullptr for an unknown warps.
ScanFn scan_fn_pair(int warps, bool pos);
ScanFn scan_fn_one_smem(int warps, bool pos);
ScanFn scan_fn_one_global(int warps, bool pos);
ScanFn scan_fn_hot(int warps, bool pos);
ScanFn scan_fn_one_rep(int warps, bool pos);

}  // namespace dnalib

namespace {

using namespace dnalib;

// -------------------------------------------------------------- scan kernel


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

// Chunk flag bits (ScanParams::flags), read by the extraction pass.
constexpr uint8_t kFlagRescan = 1;    // extract by rescanning the chunk from its true start
constexpr uint8_t kFlagFixed = 2;     // the speculative run met the true run inside row 0:
                                      // row 0 starts from the true start (spec_start) and
                                      // later rows' count offsets move by fix_delta
constexpr uint8_t kFlagRow0Rec = 4;   // the speculative run recorded row 0
constexpr uint8_t kFlagPrefixHit = 8; // the true run accepts before the meeting point

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
struct Repair { uint32_t count, last, old_count, delta; uint8_t flag; };

__device__ Repair repair_chunk(const ScanParams &p, const OneTable &T, uint64_t c, uint32_t a, uint32_t s,
                              const uint4 *head) {
    const uint64_t b = c * p.seg_bytes;
    const uint64_t from = b > p.lo ? b : p.lo;
    const uint64_t to = b + p.seg_bytes < p.hi ? b + p.seg_bytes : p.hi;
    // the chunk's current results, loaded up front so they overlap the walk
    const uint32_t cur_count = p.count[c], cur_last = p.last_state[c];
    const uint8_t cur_flags = p.stash ? p.flags[c] : 0;
    uint32_t qa = a, qs = s, ca = 0, cs = 0;
    uint64_t met_at = ~0ull;
    auto step = [&](uint64_t off, uint32_t byte) {
        const uint32_t ea = T.step(qa, byte);
        const uint32_t es = T.step(qs, byte);
        qa = ea & 0x7FFFFFFFu; qs = es & 0x7FFFFFFFu;
        ca += ea >> 31; cs += es >> 31;
        if (qa == qs) { met_at = off; return false; }
        return true;
    };
    uint64_t resume = from;
    if (head) {
        // the chunk's first 16 bytes, saved by its block: the runs almost always meet here
        const uint32_t hw[4] = {head->x, head->y, head->z, head->w};
        for (int k = 0; k < 16; ++k) {
            const uint64_t off = b + (uint64_t)k;
            if (off < from) continue;
            if (off >= to || !step(off, (hw[k >> 2] >> (8 * (k & 3))) & 0xFFu)) break;
        }
        resume = b + 16;
    }
    if (met_at == ~0ull && resume < to) walk_range(p.abase, resume, to, p.hi, step);
    Repair r;
    r.old_count = cur_count;
    r.delta = 0;
    if (met_at != ~0ull) {
        r.count = cur_count - cs + ca;
        r.last = cur_last;
        r.flag = 0;
        if (p.stash) {
            if (met_at < b + kTile)   // the extraction fixes the records (row 0 and offsets)
                r.flag = (uint8_t)((cur_flags & kFlagRow0Rec) | kFlagFixed | (ca > 0 ? kFlagPrefixHit : 0));
            else
                r.flag = kFlagRescan;
            r.delta = ca - cs;
        }
    } else {
        r.count = ca;
        r.last = qa;
        r.flag = kFlagRescan;
    }
    return r;
}

// Makes chunk c's results those of the run from its true start a: count (and its block
// sum), assumed start, last state, flags.
__device__ __forceinline__ void apply_repair(const ScanParams &p, uint64_t c, uint32_t a,
                                             const Repair &r, uint32_t chunks_per_block,
                                             unsigned long long *sums) {
    const uint32_t old = r.old_count;
    p.count[c] = r.count;
    atomicAdd(&sums[c / chunks_per_block], (unsigned long long)(long long)((int64_t)r.count - (int64_t)old));
    p.spec_start[c] = a;
    p.last_state[c] = r.last;
    if (r.flag) p.flags[c] = r.flag;
    if (r.flag & kFlagFixed) p.fix_delta[c] = r.delta;
}

// The join across blocks (Sec. III-A "binary reduction"), run by the last block to
// finish. Each chunk's true start is the last state of the chunk before it. The first
// chunk of every block and the chunks whose in-block repair did not meet within 16
// bytes are repaired in parallel (Sec. III-B.3); every repair leaves a consistent
// (assumed start, count, last state) triple, so a chunk whose last state changed is
// followed forward until the next chunk's assumed start equals the true last state
// before it (the cascade). Then the block sums are scanned into output offsets and the
// total is written. 's_sum' is shared memory for the block sums (the staging area, idle
// by now) or null, in which case they are updated in global memory.
template <int THREADS>
__device__ void finalize_block(const ScanParams &p, const OneTable &T, unsigned long long *s_sum) {
    __shared__ unsigned long long wsum[THREADS / 32];
    __shared__ unsigned long long carry;
    const uint32_t tid = threadIdx.x;
    const uint32_t cpb = THREADS;   // chunks per scan block
    const uint32_t nb = gridDim.x;
    unsigned long long *sums = s_sum ? s_sum : p.cta_sum;
    if (s_sum)
        for (uint32_t i = tid; i < nb; i += THREADS) s_sum[i] = p.cta_sum[i];
    const uint32_t np = p.ctrl[1];
    __syncthreads();
    auto repair_one = [&](uint64_t c, const uint4 *head) {
        const uint32_t a = p.last_state[c - 1];
        const uint32_t s = p.spec_start[c];
        if (a == s) return;
        if (head) atomicAdd(&p.ctrl[4], 1u);
        const uint32_t old_last = p.last_state[c];
        const Repair r = repair_chunk(p, T, c, a, s, head);
        apply_repair(p, c, a, r, cpb, sums);
        if (r.last != old_last) {
            const uint32_t k = atomicAdd(&p.ctrl[2], 1u);
            if (k < p.div_cap) p.div_list[k] = (uint32_t)c;
        }
    };
    // the first chunk of every block but the first, with its saved first 16 bytes
    for (uint32_t b = tid + 1; b < nb; b += THREADS) {
        const uint64_t c = (uint64_t)b * cpb;
        if (c < p.nseg) repair_one(c, &p.block_head[b]);
    }
    // chunks whose in-block repair did not converge
    if (np <= p.pending_cap)
        for (uint32_t i = tid; i < np; i += THREADS) repair_one(p.pending[i], nullptr);
    __syncthreads();
    if (tid == 0) {
        const uint32_t nd = p.ctrl[2];
        if (np > p.pending_cap || nd > p.div_cap) {
            // a list overflowed: check every chunk boundary in order
            for (uint64_t c = 1; c < p.nseg; ++c) {
                const uint32_t a = p.last_state[c - 1];
                const uint32_t s = p.spec_start[c];
                if (a == s) continue;
                const Repair r = repair_chunk(p, T, c, a, s, nullptr);
                apply_repair(p, c, a, r, cpb, sums);
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
                    const Repair r = repair_chunk(p, T, k, cur, p.spec_start[k], nullptr);
                    apply_repair(p, k, cur, r, cpb, sums);
                    atomicAdd(&p.ctrl[5], 1u);
                    p.flags[k] = kFlagRescan;   // its records follow a start that was not the true one
                    cur = r.last;
                    ++k;
                }
            }
        }
        carry = 0;
    }
    __syncthreads();
    // exclusive scan of the block sums -> output offsets; total -> out_count
    for (uint32_t base = 0; base < nb; base += THREADS) {
        const uint32_t i = base + tid;
        const unsigned long long v = i < nb ? sums[i] : 0ull;
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
    if (tid == 0) {
        *p.out_count = carry;
        if (p.out_last) {
            const uint32_t l = p.last_state[p.nseg - 1];
            *p.out_last = p.perm_inv ? p.perm_inv[l] : l;
        }
        // every other block took its ticket before this one, after its last use of the
        // control words: leave them zero for the next scan on this stream
        if (p.reset_ctrl)
            for (int i = 0; i < 6; ++i) p.ctrl[i] = 0;
    }
}

template <int MODE, int WARPS, bool POS>
__global__ void __launch_bounds__(WARPS * 32, 1)
scan_kernel(ScanParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint32_t warp_last[WARPS];
    __shared__ uint4 head_s[WARPS * 32];   // each chunk's first 16 bytes, for the repair
    __shared__ uint32_t s_nfix;            // chunks of this block repaired at their converging point
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
    uint32_t rep_base = 0;   // MODE_ONE_REP: shared address of the replicated table
    constexpr int kPre = 2048 / (WARPS * 32) > 0 ? 2048 / (WARPS * 32) : 1;
    uint32_t pre[kPre];
    if constexpr (MODE != MODE_ONE_GLOBAL && MODE != MODE_HOT) {
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
    // MODE_HOT: shared addresses of the two-symbol rows (32 B per hot state) and of the
    // one-symbol rows (8 B per state) that follow them
    const uint32_t hot_p = smem_base + (uint32_t)WARPS * kStages * kStageBytes;
    const uint32_t hot_o = hot_p + (p.hot_rows + 1u) * 32u;
    if constexpr (MODE == MODE_ONE_GLOBAL) {
        T.t = p.one;
    } else if constexpr (MODE == MODE_HOT) {
        // the one-symbol table of the per-byte paths (rows with resets, the join's
        // repairs) stays in global memory, where it is L2 resident
        T.t = p.one;
        // two-symbol rows of the hot states plus the sentinel row: entries next x 4 +
        // accepting steps, a next state without a row replaced by the sentinel; then the
        // one-symbol rows of every state (next | accepts << 14)
        const uint32_t h = p.hot_rows, n2w = (h + 1u) * 8u, n1w = p.n_states * 2u;
        auto conv = [&](uint32_t e) {
            const uint32_t nx = e & 0x3FFFu;
            return (nx < h ? nx : h) * 4u + (e >> 14);
        };
        for (uint32_t i = threadIdx.x; i < n2w; i += WARPS * 32) {
            uint32_t v;
            if (i < h * 8u) {
                const uint32_t e = p.hot2[i];
                v = conv(e & 0xFFFFu) | (conv(e >> 16) << 16);
            } else {
                v = (h * 4u) | ((h * 4u) << 16);
            }
            one_s[i] = v;
        }
        for (uint32_t i = threadIdx.x; i < n1w; i += WARPS * 32) one_s[n2w + i] = p.hot1[i];
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
        if (MODE == MODE_ONE_REP) {
            // every lane's copy of the one-symbol table, expanded from the compact copy
            const uint32_t after = smem_base + (uint32_t)WARPS * kStages * kStageBytes + n1 * 4u;
            rep_base = (after + 2047u) & ~2047u;
            uint32_t *rep_ptr = reinterpret_cast<uint32_t *>(smem + (rep_base - smem_base));
            __syncthreads();
            const uint32_t nr = p.n_states * 128u;
            for (uint32_t i = threadIdx.x; i < nr; i += WARPS * 32) {
                const uint32_t e = one_s[i >> 5];
                rep_ptr[i] = (rep_base + (e & 0x7FFFFFFFu) * kRepRowBytes + (i & 31u) * 4u) | (e >> 31);
            }
        }
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
    // Launched as a programmatic dependent of the kernel before it on the stream, this
    // grid may start while that kernel finishes: everything above reads only the
    // automaton's tables and the sequence. Anything a kernel before it may write or still
    // read (the chunk start states of the chunk-map path, this call's scratch, which the
    // memory pool may hand over from an earlier call, the output) is touched only after
    // the wait. Without a programmatic predecessor the wait returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    uint32_t *stash = POS ? p.stash + seg * (kStashCap * 3) : nullptr;
    uint32_t nrec = 0;
    bool row0rec = false;   // the chunk's row 0 has a hit-row record

    // ---- speculated start state: q0, or the state reached from q0 over the lookback window
    uint32_t q = 0;
    if (p.given_start) {
        // the chunk's exact start is known (computed from per-chunk state maps)
        if (active) q = p.given_start[seg];
    } else if (seg == 0) {
        q = p.start_state;   // the first chunk's start is known
    } else if (has_lookback) {   // the 'lookback' bytes in front of the chunk
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
    // run-time 2 and 16 (from k1 and k5), so the multiplies by them stay multiplies
    const uint32_t k2 = p.k1 << 1, k16 = p.k5 >> 1;
    // shared address of the one-symbol table; when it is 256-aligned its low byte is free
    // for a code's column offset (otherwise every row is walked byte by byte from global
    // memory)
    const uint32_t one_addr = smem_base + (uint32_t)WARPS * kStages * kStageBytes;
    const bool one_fast = (one_addr & 0xFFu) == 0;
    const uint32_t reset_e = p.reset_entry;
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
        if (t == 0) {
            head_s[threadIdx.x] = make_uint4(w[0], w[1], w[2], w[3]);
            if (threadIdx.x == 0) p.block_head[blockIdx.x] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        if (MODE == MODE_HOT) {
            // Two symbols per lookup through the hot states' rows. Their entries hold
            // next state x 4 + accepting steps in the pair; a next state without a row
            // reads as the sentinel row hot_rows, whose entries point to itself. A lane
            // whose word (4 symbols) met the sentinel redoes it exactly with four
            // one-symbol lookups, in a branch the warp enters only when some lane needs it.
            // The whole warp runs the loop (lanes without a full row of this chunk follow
            // along and discard the result), so that the vote sees every lane. The row is
            // walked as two halves of 16 words through the same code.
            const bool go = live && full;
            const uint32_t qs = q;
            uint32_t err = 0, rc = 0, qq = q, base_seen = 0;
            const uint32_t k32 = p.k5, k8 = p.k5 >> 2;
            const uint32_t sentinel = p.hot_rows;
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const uint32_t x = w[k] & 0x06060606u;
                    const uint32_t y = mad_lo(x, 65u, 0u);   // pair codes at bits 7..10 and 23..26
                    const uint32_t b1 = hot_p + ((y >> 6) & 30u), b2 = hot_p + ((y >> 22) & 30u);
                    const uint32_t e1 = lds_u16(mad_lo(min(qq, sentinel), k32, b1));
                    const uint32_t e2 = lds_u16(mad_lo(e1 & 0xFFFCu, k8, b2));
                    uint32_t nq = e2 >> 2, nrc = rc + (e1 & 3u) + (e2 & 3u);
                    const uint32_t z = x | (x >> 4);
                    const uint32_t bad = (__byte_perm(lut_lo, lut_hi, __byte_perm(z, 0, 0x0020)) ^ w[k]) & 0xDFDFDFDFu;
                    err |= bad;
                    // a zero byte of 'bad' is a base: rows without any (N runs) take no walk
                    base_seen |= (bad - 0x01010101u) & ~bad & 0x80808080u;
                    // only a lane whose row is still all bases needs the exact redo (the
                    // others discard this row's walk and take the per-byte path)
                    const bool cold = go && nq == sentinel && err == 0;
                    if (__any_sync(0xFFFFFFFFu, cold)) {
                        // lanes that need no redo read one shared word (no bank conflict)
                        uint32_t st = cold ? qq : 0u, c = 0;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t ej = lds_u16(mad_lo(st, k8, hot_o) + (cold ? ((x >> (8 * j)) & 6u) : 0u));
                            st = cold ? (ej & 0x3FFFu) : 0u;
                            c += ej >> 14;
                        }
                        if (cold) { nq = st; nrc = rc + c; }
                    }
                    qq = nq;
                    rc = nrc;
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) w[k] = w[k + 16];
            }
            if (!live) continue;
            if (go && err == 0) {
                if (POS && rc) { row0rec |= t == 0; record_hit_row(stash, nrec, t | kRowAllBases, qs, cnt); }
                cnt += rc;
                q = qq;
            } else if (go && base_seen == 0) {
                // every byte of the row resets: the run ends in q0, and counts each byte
                // when q0 accepts
                const uint32_t add = (reset_e >> 31) * (uint32_t)kTile;
                if (POS && add) { row0rec |= t == 0; record_hit_row(stash, nrec, t, qs, cnt); }
                cnt += add;
                q = 0;
            } else {
                // reset bytes or a sequence edge in this row: byte by byte with the global
                // one-symbol table (a reset byte takes no lookup); the row is in L2
                const uint32_t before = cnt;
                q = row_bytes_global(T, qs, p.abase, row_off > p.lo ? row_off : p.lo,
                                     row_off + kTile < p.hi ? row_off + kTile : p.hi, p.hi, cnt);
                if (POS && cnt != before) { row0rec |= t == 0; record_hit_row(stash, nrec, t, qs, before); }
            }
            continue;
        }
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
                    if (POS && rc) {
                        row0rec |= t == 0;
                        record_hit_row(stash, nrec, t | kRowAllBases,
                                       ((cur & 0x3FFFFu) - pair_base) / (uint32_t)kPairRowBytes, cnt);
                    }
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
                if (POS && cnt != before) { row0rec |= t == 0; record_hit_row(stash, nrec, t, qs, before); }
                cur = pair_base + qe * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u;
            }
        } else {
            uint32_t before = cnt, qs = q;
            bool done = false;
            if (MODE == MODE_ONE_SMEM && full && one_fast) {
                // One lookup per byte. The shared address of the next entry is entry * 16 +
                // table base + code * 4: the product drops the accept bit (bit 31) and
                // leaves the next state's row offset, so a base costs one multiply-add, one
                // load and one multiply-high (count += entry >> 31). A reset byte (its
                // lowercase form is not that of its code's letter) takes the reset entry in
                // place of the loaded one, without a branch.
                uint32_t e = q, rc = 0, err = 0;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const uint32_t x = w[k] & 0x06060606u;
                    const uint32_t v = mad_lo(x, k2, 0u);
                    const uint32_t z = x | (x >> 4);
                    const uint32_t bad = (__byte_perm(lut_lo, lut_hi, __byte_perm(z, 0, 0x0020)) ^ w[k]) & 0xDFDFDFDFu;
                    err |= bad;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t a = lds_u32(mad_lo(e, k16, __byte_perm(v, one_addr, 0x7650u | (uint32_t)j)));
                        e = (bad & (0xFFu << (8 * j))) ? reset_e : a;
                        rc = mad_hi(e, k2, rc);
                    }
                }
                if (POS && rc) { row0rec |= t == 0; record_hit_row(stash, nrec, t | (err ? 0u : kRowAllBases), qs, cnt); }
                cnt += rc;
                q = e & 0x7FFFFFFFu;
                done = true;
            }
            if (MODE == MODE_ONE_REP && full) {
                // One lookup per byte in the lane's own copy (no bank conflict): the entry
                // already is the next row's address; the byte's code enters at bits 7..8.
                // A reset byte takes the lane's row of q0 (with q0's accept bit) instead.
                const uint32_t reset_l = (rep_base + (uint32_t)lane * 4u) | (reset_e >> 31);
                uint32_t e = rep_base + q * kRepRowBytes + (uint32_t)lane * 4u, rc = 0, err = 0;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const uint32_t x = w[k] & 0x06060606u;
                    const uint32_t z = x | (x >> 4);
                    const uint32_t bad = (__byte_perm(lut_lo, lut_hi, __byte_perm(z, 0, 0x0020)) ^ w[k]) & 0xDFDFDFDFu;
                    err |= bad;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t off = (j == 0 ? (x << 6) : (x >> (8 * j - 6))) & 0x180u;
                        const uint32_t a = lds_u32((e & kRepAddrMask) | off);
                        e = (bad & (0xFFu << (8 * j))) ? reset_l : a;
                        rc += e & 1u;
                    }
                }
                if (POS && rc) { row0rec |= t == 0; record_hit_row(stash, nrec, t | (err ? 0u : kRowAllBases), qs, cnt); }
                cnt += rc;
                q = ((e & 0x3FE00u) - rep_base) / kRepRowBytes;
                done = true;
            }
            if (!done) {
                q = (MODE != MODE_ONE_SMEM && MODE != MODE_ONE_REP && full) ? row_bytes_reg(T, qs, w, cnt)
                         : row_bytes_global(T, qs, p.abase, row_off > p.lo ? row_off : p.lo,
                                            row_off + kTile < p.hi ? row_off + kTile : p.hi, p.hi, cnt);
                if (POS && cnt != before) { row0rec |= t == 0; record_hit_row(stash, nrec, t, qs, before); }
            }
        }
    }
    cp_async_wait<0>();
    uint32_t last = q;
    if (MODE == MODE_PAIR) last = ((cur & 0x3FFFFu) - pair_base) / (uint32_t)kPairRowBytes;

    // ---- join inside the block (Sec. III-A) with repair at the converging point (Alg. 1):
    // the true start of a chunk is the last state of the chunk before it, which the lane
    // to the left (or, for lane 0, the previous warp's lane 31) has just computed
    if (lane == 31) warp_last[warp] = last;
    if (threadIdx.x == 0) s_nfix = 0;
    __syncthreads();
    uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, last, 1);
    if (lane == 0) prev = warp > 0 ? warp_last[warp - 1] : 0u;
    const bool has_prev = active && seg > 0 && (lane > 0 || warp > 0);
    bool pending = false;   // a block's first chunk is joined by the last block directly
    bool fixed = false, prefix_hit = false;
    uint32_t fix_delta = 0;
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
            fix_delta = delta;
            fixed = true;
            prefix_hit = pa > 0;
            spec = prev;
        } else {
            pending = true;   // the last block repairs it from global memory
        }
    }
    if (active) {
        p.spec_start[seg] = spec;
        p.last_state[seg] = last;
        p.count[seg] = cnt;
        if (POS) {
            // the records stay those of the speculative run; the flags say how the
            // extraction turns them into the true run's
            p.flags[seg] = (row0rec ? kFlagRow0Rec : 0) |
                           (fixed ? kFlagFixed | (prefix_hit ? kFlagPrefixHit : 0) : 0);
            if (fixed) p.fix_delta[seg] = fix_delta;
            p.nrec[seg] = nrec;
        } else {
            p.flags[seg] = 0;
        }
    }
    if (pending) {
        const uint32_t k = atomicAdd(&p.ctrl[1], 1u);
        if (k < p.pending_cap) p.pending[k] = (uint32_t)seg;
    }
    {   // convergence statistics: chunks whose speculated start was repaired in-block
        // (added up in shared memory; one global add per block before its ticket)
        const uint32_t nfix = __popc(__ballot_sync(0xFFFFFFFFu, fixed));
        if (lane == 0 && nfix) atomicAdd(&s_nfix, nfix);
    }
    __threadfence();   // this thread's results are visible before the block's ticket
    // the extraction kernel (launched as a programmatic dependent) may be scheduled once
    // every block has got here; it still waits for this grid to finish before reading
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
        if (s_nfix) atomicAdd(&p.ctrl[3], s_nfix);
        __threadfence();
        is_last = atomicAdd(&p.ctrl[0], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // the staging area is idle now: it holds the block sums while the last block joins
    unsigned long long *s_sum = gridDim.x * 8u <= (uint32_t)WARPS * kStageBytes
                                    ? reinterpret_cast<unsigned long long *>(smem) : nullptr;
    finalize_block<WARPS * 32>(p, T, s_sum);
}

}  // namespace
