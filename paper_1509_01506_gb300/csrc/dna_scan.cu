// dna_scan.cu -- host side of the single-sequence path (planning, scratch, launches),
// the position-extraction kernel and the C ABI of the automata and scans.
//
// The data-parallel path of Memeti & Pllana (Sec. III-A, III-B, Alg. 1), re-designed
// for one GPU (the chunk-scan kernel itself is in scan_kernel.cuh):
//   * Input-based partitioning (Sec. III-A, Fig. 1a): the sequence is cut into chunks of
//     chunk_bytes; every GPU lane owns one chunk. A warp's 32 chunks are staged into
//     shared memory tile by tile with cp.async (16-byte copies; each copy instruction
//     of the warp covers four whole 128-byte lines) and read back row by row.
//   * Speculation (Sec. III-A, possible starting states): a chunk's start state is
//     unknown. By default the lane starts it in q0; with a lookback window it runs
//     from q0 over the symbols in front of the chunk, which gives the exact start when
//     the automaton is definite within the window.
//   * Chunk scan (Alg. 1, the per-character loop): ingest is fused -- bytes are mapped
//     to 2-bit codes in registers, 4 bytes at a time, with a bit-exact check that every
//     byte is a base. Small automata use a two-symbol transition table replicated once
//     per lane in shared memory (lane l's copy lives in bank l, so the 32 lookups of a
//     warp never conflict); each entry carries the next row's address and the number
//     of accepting steps in the pair. Rows with reset bytes or sequence edges take a
//     per-byte path.
//   * Join (the "binary reduction" of Sec. III-A) and converging point (Sec. III-B.3):
//     inside a block, each chunk's true start is its left neighbour's last state; on a
//     mismatch the lane runs the true and the speculated start in lockstep over the
//     chunk's first 16 bytes, and where they meet corrects the count by the paper's
//     formula (own prefix count + speculative total - speculative prefix count). The
//     block that finishes last joins across blocks and repairs, from global memory,
//     the chunks whose runs did not meet early; a cascade follows a changed last state
//     forward until the chain agrees again.
//   * Extraction: a block scan of the chunk counts gives each chunk its output offset;
//     positions are re-walked from the hit rows recorded during the scan, and chunks
//     that overflowed their records or were corrected late are rescanned from their
//     true start.

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
#include "scan_kernel.cuh"

using namespace dnalib;

namespace {

// ------------------------------------------------------------ extraction

struct EmitParams {
    const uint8_t *abase;
    uint64_t lo, hi, seg_bytes, nseg;
    const uint32_t *one;
    uint32_t reset_entry, n_states;
    const uint32_t *last_state, *count, *stash, *nrec, *spec_start, *fix_delta;
    const uint8_t *flags;
    const unsigned long long *cta_off;
    uint64_t *out;
    uint64_t cap;
    uint32_t lut_lo, lut_hi;   // expected lowercase bytes per code, for the base check
    uint32_t start_state;   // the state the first chunk starts in
    // per-label outputs (null labels: none): every hit row is walked, whatever the
    // capacity, and each accepting step's label mask is added into label_counts
    const uint32_t *labels;
    unsigned long long *label_counts;
    uint32_t *pos_labels;
    uint32_t n_labels;
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
// Walks one whole 128-byte row of bases with the two-symbol table 'ptab' (entry: next
// state | accept after the first symbol << 30 | accept after the second << 31) and
// writes the accepting positions from output index o. The walk itself has no branches:
// the accept bits of the 128 positions collect in a 4-word mask, which is turned into
// positions afterwards. q and o leave as the state after the row and the next output
// index (rescans continue from them). Unless 'checked', the row is first tested for
// non-base bytes; then it returns false (writing nothing, q and o unchanged) and the
// caller walks the row byte by byte.
__device__ __forceinline__ bool walk_row_pairs(const EmitParams &p, const uint32_t *ptab, uint64_t rs,
                                               uint32_t &q, unsigned long long &o, bool checked) {
    const uint4 *src = reinterpret_cast<const uint4 *>(p.abase + rs);
    if (!checked) {
        uint32_t err = 0;
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const uint4 v = src[h];
            const uint32_t ww[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t x = ww[i] & 0x06060606u;
                const uint32_t z = x | (x >> 4);
                err |= __byte_perm(p.lut_lo, p.lut_hi, __byte_perm(z, 0, 0x0020)) ^ ww[i];
            }
        }
        if (err & 0xDFDFDFDFu) return false;
    }
    const uint32_t pbase = (uint32_t)__cvta_generic_to_shared(ptab);
    uint32_t m[4];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        uint4 v[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) v[h] = src[4 * half + h];
#pragma unroll
        for (int mw = 0; mw < 2; ++mw) {          // one mask word: 32 positions = 8 words
            uint32_t bits = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int wi = 8 * mw + i;        // word within this half
                const uint32_t w = wi % 4 == 0 ? v[wi / 4].x : wi % 4 == 1 ? v[wi / 4].y
                                 : wi % 4 == 2 ? v[wi / 4].z : v[wi / 4].w;
                const uint32_t y = (w & 0x06060606u) * 65u;   // pair codes at bits 7..10, 23..26
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t e = lds_u32(pbase + (q * 16u + ((y >> (j ? 23 : 7)) & 15u)) * 4u);
                    q = e & 0x3FFFFFFFu;
                    bits |= (e >> 30) << (4 * i + 2 * j);
                }
            }
            m[2 * half + mw] = bits;
        }
    }
    const uint64_t pos0 = rs - p.lo;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t bits = m[k];
        while (bits) {
            const int b = __ffs(bits) - 1;
            if (o < p.cap) p.out[o] = pos0 + 32u * k + (uint32_t)b;
            ++o;
            bits &= bits - 1;
        }
    }
    return true;
}

// The two-symbol row walk that also follows the state: the same walk over a whole row
// of bases (returns false, writing nothing, when the row holds a non-base byte and is not
// 'checked'), writing positions as it goes. With per-label outputs a pair with an
// accepting step resolves the state of that step (after the pair's second symbol: the
// entry's next state; after its first: one extra one-symbol lookup) and its label mask,
// writes the mask beside the position and adds it into the walker's counters 'wl' (label
// i at wl[i * kEmitWalkers]). 'q' is the state before the row and, after a walk, the
// state after it (rescans continue from it).
__device__ __forceinline__ bool walk_row_pairs_lab(const EmitParams &p, const uint32_t *ptab, uint64_t rs,
                                                   uint32_t &q, unsigned long long &o, bool checked,
                                                   uint32_t *wl) {
    const uint4 *src = reinterpret_cast<const uint4 *>(p.abase + rs);
    if (!checked) {
        uint32_t err = 0;
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const uint4 v = src[h];
            const uint32_t ww[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t x = ww[i] & 0x06060606u;
                const uint32_t z = x | (x >> 4);
                err |= __byte_perm(p.lut_lo, p.lut_hi, __byte_perm(z, 0, 0x0020)) ^ ww[i];
            }
        }
        if (err & 0xDFDFDFDFu) return false;
    }
    const uint32_t pbase = (uint32_t)__cvta_generic_to_shared(ptab);
    const uint64_t pos0 = rs - p.lo;
    auto hit = [&](uint64_t pos, uint32_t m) {   // m: label mask (0 without labels)
        if (o < p.cap) {
            p.out[o] = pos;
            if (p.pos_labels) p.pos_labels[o] = m;
        }
        ++o;
        while (m) {
            wl[(__ffs(m) - 1) * kEmitWalkers] += 1u;
            m &= m - 1;
        }
    };
#pragma unroll 1
    for (int h = 0; h < 8; ++h) {
        const uint4 v = src[h];
        const uint32_t ww[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t y = (ww[i] & 0x06060606u) * 65u;   // pair codes at bits 7..10, 23..26
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint32_t pc = (y >> (j ? 23 : 7)) & 15u;
                const uint32_t e = lds_u32(pbase + (q * 16u + pc) * 4u);
                if (e >> 30) {
                    const uint64_t pos = pos0 + 16u * h + 4u * i + 2u * j;
                    if (e & 0x40000000u)
                        hit(pos, p.labels ? p.labels[p.one[q * 4u + (pc & 3u)] & 0x7FFFFFFFu] : 0u);
                    if (e >> 31) hit(pos + 1, p.labels ? p.labels[e & 0x3FFFFFFFu] : 0u);
                }
                q = e & 0x3FFFFFFFu;
            }
        }
    }
    return true;
}

// Record i of chunk c as the true run's: records are written by the speculative run; a
// chunk repaired at its converging point inside row 0 (kFlagFixed) takes its row-0 start
// from the true start and moves later rows' count offsets by its delta, and when the
// true run accepts before the meeting point but the speculative run recorded no row 0,
// a row-0 record is inserted in front (ins = 1).
__device__ __forceinline__ uint3 chunk_record(const EmitParams &p, uint64_t c, uint32_t i, bool fixed,
                                              uint32_t ins, uint32_t delta, uint32_t row0) {
    if (ins && i == 0) return make_uint3(0u, row0, 0u);
    const uint32_t *g = p.stash + c * (kStashCap * 3) + 3 * (i - ins);
    uint3 r = make_uint3(g[0], g[1], g[2]);
    if (fixed) {
        if ((r.x & ~kRowAllBases) == 0) r.y = row0;
        else r.z += delta;
    }
    return r;
}

__global__ void __launch_bounds__(1024) emit_kernel(EmitParams p, uint32_t tab5_in_smem, uint32_t ptab_in_smem) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ unsigned long long wsum[32];
    __shared__ uint32_t wsum2[32];
    __shared__ uint8_t cls[256];
    __shared__ uint8_t s_rescan[1024];
    __shared__ uint4 s_rec[kEmitRecs];   // (tile, start state, count before, chunk index)
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const bool lab = p.labels != nullptr;
    // dynamic shared memory: [row slots: walkers x pitch][offsets: nthr x 8][fix: nthr x 8]
    //                        [slots: nthr+1 x 4][tables]
    unsigned long long *s_off = reinterpret_cast<unsigned long long *>(dsm + kEmitWalkers * kEmitRowPitch);
    uint2 *s_fix = reinterpret_cast<uint2 *>(s_off + nthr);
    uint32_t *s_slot = reinterpret_cast<uint32_t *>(s_fix + nthr);
    uint32_t *tab5 = s_slot + nthr + 1;
    uint32_t *ptab = tab5 + (tab5_in_smem ? p.n_states * 5u : 0u);
    // per-label outputs: each walker's own counters, [label][walker]
    uint32_t *s_wlab = ptab + (ptab_in_smem ? p.n_states * 16u : 0u);
    if (lab)
        for (uint32_t i = tid; i < 32u * kEmitWalkers; i += nthr) s_wlab[i] = 0;
    if (tid < 256) {
        const uint32_t c = (tid >> 1) & 3u;
        cls[tid] = byte_is_base(tid) ? (uint8_t)c : (uint8_t)4;
    }
    if (tab5_in_smem)
        for (uint32_t i = tid; i < p.n_states * 5u; i += nthr) {
            const uint32_t q = i / 5u, col = i - q * 5u;
            tab5[i] = col < 4 ? p.one[q * 4u + col] : p.reset_entry;
        }
    if (ptab_in_smem)
        for (uint32_t i = tid; i < p.n_states * 16u; i += nthr) {
            // pair index: first code in bits 0..1, second in bits 2..3 (code = (byte >> 1) & 3)
            const uint32_t q = i >> 4;
            const uint32_t e1 = p.one[q * 4u + (i & 3u)];
            const uint32_t e2 = p.one[(e1 & 0x7FFFFFFFu) * 4u + ((i >> 2) & 3u)];
            ptab[i] = (e2 & 0x3FFFFFFFu) | ((e1 >> 31) << 30) | ((e2 >> 31) << 31);
        }
    // everything above reads only the automaton; the scan's results are read below, after
    // the scan grid has completed (a no-op when not launched as a programmatic dependent)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // the next scan on the stream may start its prologue now (it waits for this grid
    // before it touches memory this grid uses)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint64_t c = (uint64_t)blockIdx.x * nthr + tid;
    const bool act = c < p.nseg;
    const unsigned long long v = act ? p.count[c] : 0u;
    const uint32_t nr = act ? p.nrec[c] : 0u;
    const uint8_t fl = act ? p.flags[c] : 0;
    const bool fixed = (fl & kFlagFixed) != 0;
    const uint32_t ins = fixed && !(fl & kFlagRow0Rec) && (fl & kFlagPrefixHit) ? 1u : 0u;
    const bool rescan = act && v > 0 && ((fl & kFlagRescan) != 0 || nr + ins > (uint32_t)kStashCap);
    // a chunk without matches has no rows to walk, whatever its speculative run recorded
    const uint32_t rows = (act && v > 0 && !rescan) ? nr + ins : 0u;
    uint2 fix = make_uint2(0u, 0u);
    if (fixed && rows) fix = make_uint2(p.fix_delta[c], p.spec_start[c]);
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
    s_rescan[tid] = (rescan ? 1 : 0) | (fixed ? 2 : 0) | (ins ? 4 : 0);
    s_fix[tid] = fix;
    // each chunk copies its hit-row records into shared memory (first kEmitRecs rows)
    const uint32_t slot0 = by + y - rows;
    for (uint32_t i = 0; i < rows; ++i) {
        if (slot0 + i >= (uint32_t)kEmitRecs) break;
        const uint3 r = chunk_record(p, c, i, fixed, ins, fix.x, fix.y);
        s_rec[slot0 + i] = make_uint4(r.x, r.y, r.z, (uint32_t)tid);
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
                if (lab) {
                    // the pattern labels of the state this step lands in
                    uint32_t m = p.labels[q];
                    if (o < p.cap && p.pos_labels) p.pos_labels[o] = m;
                    uint32_t *wl = s_wlab + tid;
                    while (m) {
                        wl[(__ffs(m) - 1) * kEmitWalkers] += 1u;
                        m &= m - 1;
                    }
                }
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
            if (!(s_rescan[j] & 1)) continue;
            const uint64_t cj = (uint64_t)blockIdx.x * nthr + j;
            const unsigned long long oj = s_off[j];
            if (oj >= p.cap && !lab) continue;
            unsigned long long o = oj;
            const uint64_t b = cj * S;
            const uint64_t from = b > p.lo ? b : p.lo;
            const uint64_t to = b + S < p.hi ? b + S : p.hi;
            uint32_t q = cj ? p.last_state[cj - 1] : p.start_state;
            for (uint64_t rs = b; rs < to && (o < p.cap || lab); rs += kTile) {
                uint32_t k0, k1;
                row_span(rs, from, to, k0, k1);
                // a whole row of bases: two symbols per lookup (without labels, the
                // branch-free walk that writes the positions from the row's mask)
                if (ptab_in_smem && k0 == 0 && k1 == (uint32_t)kTile &&
                    (lab ? walk_row_pairs_lab(p, ptab, rs, q, o, false, s_wlab + tid)
                         : walk_row_pairs(p, ptab, rs, q, o, false)))
                    continue;
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
                const uint8_t bits = s_rescan[lo];
                const uint3 g = chunk_record(p, cl, r - s_slot[lo], (bits & 2) != 0, (bits >> 2) & 1u,
                                             s_fix[lo].x, s_fix[lo].y);
                rec[0] = g.x; rec[1] = g.y; rec[2] = g.z;
            }
            const uint64_t cj = (uint64_t)blockIdx.x * nthr + lo;
            unsigned long long o = s_off[lo] + rec[2];
            if (o >= p.cap && !lab) continue;
            const uint64_t b = cj * S;
            const uint64_t cend = b + S < p.hi ? b + S : p.hi;
            const bool all_bases = (rec[0] & kRowAllBases) != 0;
            const uint64_t rs = b + (uint64_t)(rec[0] & ~kRowAllBases) * kTile;
            uint32_t k0, k1;
            row_span(rs, rs > p.lo ? rs : p.lo, rs + kTile < cend ? rs + kTile : cend, k0, k1);
            uint32_t q_row = rec[1];
            if (ptab_in_smem && k0 == 0 && k1 == (uint32_t)kTile &&
                (lab ? walk_row_pairs_lab(p, ptab, rs, q_row, o, all_bases, s_wlab + tid)
                     : walk_row_pairs(p, ptab, rs, q_row, o, all_bases)))
                continue;
            walk_row(slot, rs, k0, k1, rec[1], o);
        }
    }
    if (lab) {
        __syncthreads();
        if (tid < p.n_labels) {
            unsigned long long t = 0;
            for (int w = 0; w < kEmitWalkers; ++w) t += s_wlab[tid * kEmitWalkers + w];
            if (t) atomicAdd(&p.label_counts[tid], t);
        }
    }
}

__global__ void write_zero_kernel(uint64_t *out) { *out = 0; }

// An empty sequence (or piece): no match, and the run ends where it started.
__global__ void write_empty_kernel(uint64_t *out, uint32_t *out_last, uint32_t last) {
    *out = 0;
    if (out_last) *out_last = last;
}

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

static std::atomic<uint64_t> g_dev_allocs{0};

cudaError_t device_alloc(void **p, size_t bytes) {
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(p, bytes);
}

cudaError_t pool_alloc(void **p, size_t bytes, cudaMemPool_t pool, cudaStream_t s) {
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// The library's scratch pools, one per device, created on first use and kept for the
// life of the process.
static std::mutex g_pool_mu;
static std::vector<cudaMemPool_t> g_pools;

int scratch_alloc(int dev, size_t bytes, cudaStream_t s, void **out) {
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
        if (!g_pools[dev]) {
            cudaMemPoolProps pp = {};
            pp.allocType = cudaMemAllocationTypePinned;
            pp.handleTypes = cudaMemHandleTypeNone;
            pp.location.type = cudaMemLocationTypeDevice;
            pp.location.id = dev;
            cudaMemPool_t np = nullptr;
            DNA_CUDA(cudaMemPoolCreate(&np, &pp));
            uint64_t keep = kScratchKeepBytes;
            cudaError_t e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(np);
                return cuda_status(e);
            }
            g_pools[dev] = np;
        }
        pool = g_pools[dev];
    }
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    DNA_CUDA(cudaMallocFromPoolAsync(out, bytes, pool, s));
    return DNA_OK;
}

// Control words of the chunk scan that stay with a stream: zeroed once when first used,
// and left zero by every scan's last block, so a scan needs no memset before it. Kept for
// the life of the process (32 bytes per device and stream, at most kStreamCtrlMax).
static std::mutex g_sctrl_mu;
struct StreamCtrl { int dev; cudaStream_t s; uint32_t *ctrl; };
static std::vector<StreamCtrl> g_sctrl;
constexpr size_t kStreamCtrlMax = 1024;

uint32_t *stream_ctrl(int dev, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_sctrl_mu);
    for (const StreamCtrl &c : g_sctrl)
        if (c.dev == dev && c.s == s) return c.ctrl;
    if (g_sctrl.size() >= kStreamCtrlMax) return nullptr;
    // not while the stream is being captured into a graph (no allocation there)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    uint32_t *c = nullptr;
    if (device_alloc((void **)&c, 32) != cudaSuccess) return nullptr;
    if (cudaMemset(c, 0, 32) != cudaSuccess) { cudaFree(c); return nullptr; }
    g_sctrl.push_back({dev, s, c});
    return c;
}

int scratch_free(void *p, cudaStream_t s) {
    if (!p) return DNA_OK;
    return cuda_status(cudaFreeAsync(p, s));
}

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

struct ConvRec { uint32_t *host; cudaEvent_t ev; uint64_t nseg; };
static std::vector<ConvRec> g_conv_pending, g_conv_free;
static uint64_t g_conv[7] = {};   // scans, chunks, in-block, pending, block-first, diverged, cascade

void prof_conv(cudaStream_t s, const uint32_t *dev_ctrl, uint64_t nseg) {
    if (g_profile.load(std::memory_order_relaxed) == 0) return;
    ConvRec r{nullptr, nullptr, nseg};
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_conv_free.empty()) { r.host = g_conv_free.back().host; r.ev = g_conv_free.back().ev; g_conv_free.pop_back(); }
    }
    if (!r.host) {
        if (cudaMallocHost(&r.host, 32) != cudaSuccess) return;
        if (cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess) { cudaFreeHost(r.host); return; }
    }
    if (cudaMemcpyAsync(r.host, dev_ctrl, 32, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaEventRecord(r.ev, s) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_conv_free.push_back(r);
        return;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_conv_pending.push_back(r);
}

void profile_set(int on) { g_profile.store(on ? 1 : 0); }
bool profiling() { return g_profile.load(std::memory_order_relaxed) != 0; }

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
    for (auto &r : g_conv_pending) {
        if (cudaEventSynchronize(r.ev) == cudaSuccess) {
            g_conv[0] += 1;
            g_conv[1] += r.nseg;
            g_conv[2] += r.host[3];   // in-block repairs
            g_conv[3] += r.host[1];   // pending (last block)
            g_conv[4] += r.host[4];   // block-first chunks with a wrong start
            g_conv[5] += r.host[2];   // diverged
            g_conv[6] += r.host[5];   // cascade walks
        }
        g_conv_free.push_back(r);
    }
    g_conv_pending.clear();
    out->conv_scans = g_conv[0];
    out->conv_chunks = g_conv[1];
    out->conv_inblock = g_conv[2];
    out->conv_pending = g_conv[3];
    out->conv_blockfirst = g_conv[4];
    out->conv_diverged = g_conv[5];
    out->conv_cascade = g_conv[6];
    out->device_allocs = g_dev_allocs.load();
    if (reset) {
        for (int k = 0; k < PROF_N; ++k) { g_prof_ms[k] = 0; g_prof_calls[k] = 0; }
        for (int k = 0; k < 7; ++k) g_conv[k] = 0;
        g_launches.store(0);
    }
}

}  // namespace dnalib

namespace {

// Static shared memory of the scan kernel: each chunk's first 16 bytes + one word per warp.
size_t scan_static_smem(int warps) { return (size_t)warps * 32 * 16 + (size_t)warps * 20 + 1024; }

// MODE_HOT: how many states get a two-symbol row (32 B each; one more row is the sentinel)
// beside the one-symbol rows of every state (8 B each) and the staging area, within the
// shared memory of a block.
uint32_t hot_rows_for(size_t optin, int warps, uint32_t n_states) {
    const size_t fixed = (size_t)warps * kStages * kStageBytes + scan_static_smem(warps) + 256 +
                         (size_t)n_states * 8 + 32;
    if (optin <= fixed) return 0;
    const size_t h = (optin - fixed) / 32;
    return (uint32_t)std::min<size_t>(h, n_states);
}

// Dynamic shared memory of the scan kernel (the launch argument).
size_t scan_smem_bytes(int mode, int warps, uint32_t n_states, uint32_t hot_rows = 0) {
    size_t s = (size_t)warps * kStages * kStageBytes;
    if (mode == MODE_ONE_GLOBAL) return s;
    if (mode == MODE_HOT) return s + (size_t)(hot_rows + 1) * 32 + (size_t)n_states * 8;
    s += (size_t)n_states * 16;
    if (mode == MODE_ONE_REP) s += 2048 + (size_t)n_states * kRepRowBytes;
    if (mode == MODE_PAIR) s += (size_t)n_states * 64 + 2048 + (size_t)n_states * kPairRowBytes;
    return s;
}

size_t scan_total_smem(int mode, int warps, uint32_t n_states, uint32_t hot_rows = 0) {
    return scan_smem_bytes(mode, warps, n_states, hot_rows) + scan_static_smem(warps);
}

ScanFn scan_fn(int mode, int warps, bool pos) {
    if (mode == MODE_PAIR) return scan_fn_pair(warps, pos);
    if (mode == MODE_ONE_SMEM) return scan_fn_one_smem(warps, pos);
    if (mode == MODE_ONE_GLOBAL) return scan_fn_one_global(warps, pos);
    if (mode == MODE_HOT) return scan_fn_hot(warps, pos);
    if (mode == MODE_ONE_REP) return scan_fn_one_rep(warps, pos);
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
    uint32_t hot_rows;
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
    else if (req == DNA_PLACE_SMEM_HOT) mode = MODE_HOT;
    else if (req == DNA_PLACE_SMEM_ONE_REP) mode = MODE_ONE_REP;
    else return DNA_ERR_INVALID_ARG;
    if (mode == MODE_ONE_REP && warps == 32) return DNA_ERR_CAPACITY;
    if (mode == MODE_PAIR && !d->d_pair) return DNA_ERR_CAPACITY;
    uint32_t hot_rows = 0;
    if (mode == MODE_HOT) {
        if (!d->d_hot2) return DNA_ERR_CAPACITY;
        if (!warps) warps = kHotWarps;
        if (warps != 8 && warps != 16) return DNA_ERR_CAPACITY;
        hot_rows = hot_rows_for(optin, warps, d->n_states);
        if (ov && ov->hot_rows) hot_rows = std::min(hot_rows, ov->hot_rows);
        else if (hot_rows < std::min<uint32_t>(64, d->n_states)) return DNA_ERR_CAPACITY;
        if (hot_rows == 0) return DNA_ERR_CAPACITY;
    }
    if (!warps) {
        warps = 8;
        for (int w : {24, 16}) if (scan_total_smem(mode, w, d->n_states) <= optin) { warps = w; break; }
    }
    size_t smem = scan_smem_bytes(mode, warps, d->n_states, hot_rows);
    if (scan_total_smem(mode, warps, d->n_states, hot_rows) > optin) return DNA_ERR_CAPACITY;
    uint32_t lb = ov && ov->lookback ? ov->lookback : d->lookback;
    if (lb > kMaxLookback) return DNA_ERR_INVALID_ARG;
    ScanFn fn = scan_fn(mode, warps, pos);
    if (!fn) return DNA_ERR_INVALID_ARG;
    uint32_t pf = kDefaultPrefetch;
    if (ov && ov->prefetch_tiles) pf = ov->prefetch_tiles >= 255 ? 0 : ov->prefetch_tiles;
    if (pf > 64) return DNA_ERR_INVALID_ARG;
    // the shared-memory opt-in is set once per kernel variant (to the device maximum),
    // the occupancy once per automaton and variant
    const int wi = warps == 8 ? 0 : warps == 16 ? 1 : warps == 24 ? 2 : 3;   // per_sm[mode][wi][pos]
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
    pl.hot_rows = hot_rows;
    pl.nseg = (total + S - 1) / S;
    pl.lookback = lb; pl.smem = smem;
    uint64_t lanes_per_cta = (uint64_t)warps * 32;
    pl.grid = (int)((pl.nseg + lanes_per_cta - 1) / lanes_per_cta);
    return DNA_OK;
}

// device scratch carved from one stream-ordered allocation
struct Scratch {
    uint32_t *spec_start, *last_state, *count, *nrec, *stash, *fix_delta, *pending, *div_list, *ctrl;
    uint8_t *flags;
    unsigned long long *cta_sum, *cta_off;
    uint4 *block_head;
    size_t bytes;
};


void carve(Scratch &s, uint64_t nseg, uint64_t nblocks, bool positions, uint32_t pending_cap,
           uint32_t div_cap, uint8_t *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) { uint8_t *q = base ? base + off : nullptr; off = align_up(off + bytes, 256); return q; };
    s.ctrl = (uint32_t *)take(32);
    s.cta_sum = (unsigned long long *)take(nblocks * 8);
    s.cta_off = (unsigned long long *)take(nblocks * 8);
    s.block_head = (uint4 *)take(nblocks * 16);
    s.spec_start = (uint32_t *)take(nseg * 4);
    s.last_state = (uint32_t *)take(nseg * 4);
    s.count = (uint32_t *)take(nseg * 4);
    s.flags = (uint8_t *)take(nseg);
    s.pending = (uint32_t *)take((size_t)pending_cap * 4);
    s.div_list = (uint32_t *)take((size_t)div_cap * 4);
    s.stash = positions ? (uint32_t *)take(nseg * kStashCap * 12) : nullptr;
    s.nrec = positions ? (uint32_t *)take(nseg * 4) : nullptr;
    s.fix_delta = positions ? (uint32_t *)take(nseg * 4) : nullptr;
    s.bytes = off;
}

}  // namespace

namespace dnalib {

// The outputs of an empty scan (the start state in the caller's numbering as the last).
int write_empty(cudaStream_t stream, uint64_t *out_count, const dna_dfa *d, const ScanFrom *from) {
    uint32_t last = 0;
    if (from) {
        last = from->start;
        if (!d->perm.empty())
            for (uint32_t q = 0; q < d->n_states; ++q)
                if (d->perm[q] == from->start) { last = q; break; }
    }
    write_empty_kernel<<<1, 1, 0, stream>>>(out_count, from ? from->out_last : nullptr, last);
    record_launch();
    return cuda_status(cudaGetLastError());
}

int scan_impl(const dna_dfa *d, const uint8_t *seq, uint64_t len, cudaStream_t stream,
              uint64_t *out_count, uint64_t *out_positions, uint64_t cap, const dna_plan *ov,
              const LabelOut *lab, const ScanFrom *from) {
    if (!d || !out_count || (len > 0 && !seq)) return DNA_ERR_INVALID_ARG;
    const uint32_t req = ov ? ov->placement : 0u;
    if (req > DNA_PLACE_SMEM_ONE_REP) return DNA_ERR_INVALID_ARG;
    if (req == DNA_PLACE_MAP || (req == 0 && d->map_mode)) {
        if (d->n_states > kMaxMapStates) return DNA_ERR_CAPACITY;
        if (len > (1ull << 40)) return DNA_ERR_INVALID_ARG;
        int cur_dev = -1;
        DNA_CUDA(cudaGetDevice(&cur_dev));
        if (cur_dev != d->device) return DNA_ERR_INVALID_ARG;
        if (len == 0) return write_empty(stream, out_count, d, from);
        return map_scan_impl(d, seq, len, stream, out_count, out_positions, cap, nullptr, 0, lab, from);
    }
    return scan_impl_given(d, seq, len, stream, out_count, out_positions, cap, ov, nullptr, lab, from);
}

int scan_impl_given(const dna_dfa *d, const uint8_t *seq, uint64_t len, cudaStream_t stream,
                    uint64_t *out_count, uint64_t *out_positions, uint64_t cap, const dna_plan *ov,
                    const uint32_t *given_start, const LabelOut *lab, const ScanFrom *from) {
    if (!d || !out_count || (len > 0 && !seq)) return DNA_ERR_INVALID_ARG;
    if (len > (1ull << 40)) return DNA_ERR_INVALID_ARG;
    int cur_dev = -1;
    DNA_CUDA(cudaGetDevice(&cur_dev));
    if (cur_dev != d->device) return DNA_ERR_INVALID_ARG;
    if (len == 0) return write_empty(stream, out_count, d, from);
    const uint64_t shift = (uint64_t)((uintptr_t)seq & 15u);
    const uint8_t *abase = seq - shift;
    const uint64_t total = len + shift;
    const bool positions = (out_positions != nullptr && cap > 0) || lab != nullptr;
    if (!out_positions) cap = 0;
    Plan pl;
    int rc = make_plan(d, total, positions, ov, pl);
    if (rc) return rc;
    const uint64_t nblocks = (uint64_t)pl.grid;
    // every chunk may be pending (automata that converge slowly): the last block then
    // repairs them all in parallel instead of walking every boundary in order
    const uint32_t pending_cap = (uint32_t)std::min<uint64_t>(pl.nseg + 16u, 1ull << 31);
    const uint32_t div_cap = 4096;
    Scratch s;
    carve(s, pl.nseg, nblocks, positions, pending_cap, div_cap, nullptr);
    void *mem = nullptr;
    rc = scratch_alloc(d->device, s.bytes, stream, &mem);
    if (rc) return rc;
    carve(s, pl.nseg, nblocks, positions, pending_cap, div_cap, (uint8_t *)mem);
    // the stream's own control words (already zero) unless profiling reads them back
    uint32_t *sctrl = profiling() ? nullptr : stream_ctrl(d->device, stream);
    cudaError_t e = cudaSuccess;
    if (sctrl) s.ctrl = sctrl;
    else e = cudaMemsetAsync(s.ctrl, 0, 32, stream);

    ScanParams sp;
    sp.abase = abase; sp.lo = shift; sp.hi = total; sp.seg_bytes = pl.seg_bytes; sp.nseg = pl.nseg;
    sp.lookback = pl.lookback; sp.n_states = d->n_states; sp.reset_entry = d->reset_entry;
    sp.one = d->d_one; sp.pair = d->d_pair; sp.given_start = given_start;
    sp.spec_start = s.spec_start; sp.last_state = s.last_state; sp.count = s.count;
    sp.stash = s.stash; sp.nrec = s.nrec; sp.flags = s.flags; sp.fix_delta = s.fix_delta;
    sp.prefetch_tiles = pl.prefetch;
    sp.ctrl = s.ctrl; sp.pending = s.pending; sp.pending_cap = pending_cap;
    sp.reset_ctrl = sctrl ? 1u : 0u;
    sp.start_state = from ? from->start : 0u;
    sp.out_last = from ? from->out_last : nullptr;
    sp.perm_inv = d->d_perm_inv;
    sp.div_list = s.div_list; sp.div_cap = div_cap;
    sp.cta_sum = s.cta_sum; sp.cta_off = s.cta_off; sp.block_head = s.block_head; sp.out_count = out_count;
    sp.k1 = 1u; sp.k5 = 1u << 5;
    sp.lut_lo = 0x00630061u; sp.lut_hi = 0x00670074u;
    sp.hot2 = reinterpret_cast<const uint32_t *>(d->d_hot2);
    sp.hot1 = reinterpret_cast<const uint32_t *>(d->d_hot1);
    sp.hot_rows = pl.hot_rows;

    const ProfToken tok = e == cudaSuccess ? prof_begin(stream) : ProfToken{};
    if (e == cudaSuccess) {
        // programmatic dependent launch: the scan's prologue (tables into shared memory,
        // the first tile's copies) overlaps the end of the kernel before it on the stream;
        // the kernel waits (griddepcontrol.wait) before touching anything that kernel may
        // write. Profiling serialises it (events sit between the kernels).
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)pl.grid);
        cfg.blockDim = dim3((unsigned)(pl.warps * 32));
        cfg.dynamicSmemBytes = pl.smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = tok.a ? 0 : 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, scan_fn(pl.mode, pl.warps, pl.pos), sp);
        if (e == cudaSuccess) e = cudaGetLastError();
        record_launch();
    }
    prof_end(tok, stream, PROF_SCAN);
    if (e == cudaSuccess) prof_conv(stream, s.ctrl, pl.nseg);
    if (e == cudaSuccess && positions) {
        EmitParams ep;
        ep.abase = abase; ep.lo = shift; ep.hi = total; ep.seg_bytes = pl.seg_bytes; ep.nseg = pl.nseg;
        ep.one = d->d_one; ep.reset_entry = d->reset_entry; ep.n_states = d->n_states;
        ep.last_state = s.last_state; ep.count = s.count; ep.stash = s.stash; ep.nrec = s.nrec;
        ep.spec_start = s.spec_start; ep.fix_delta = s.fix_delta;
        ep.flags = s.flags; ep.cta_off = s.cta_off; ep.out = out_positions; ep.cap = cap;
        ep.lut_lo = 0x00630061u; ep.lut_hi = 0x00670074u;
        ep.start_state = sp.start_state;
        ep.labels = lab ? lab->labels : nullptr;
        ep.label_counts = lab ? lab->counts : nullptr;
        ep.pos_labels = lab ? lab->pos_labels : nullptr;
        ep.n_labels = lab ? lab->n_labels : 0u;
        const uint32_t cpb = (uint32_t)pl.warps * 32u;   // one extraction thread per chunk
        const uint32_t tab5_smem = d->n_states * 5u <= 4096u ? 1u : 0u;
        const uint32_t ptab_smem = d->n_states <= 1024u ? 1u : 0u;   // 64 B per state
        const size_t esmem = (size_t)kEmitWalkers * kEmitRowPitch + (size_t)cpb * 16 + (size_t)(cpb + 1) * 4 +
                             (tab5_smem ? (size_t)d->n_states * 20 : 0) + (ptab_smem ? (size_t)d->n_states * 64 : 0) +
                             (lab ? (size_t)32 * kEmitWalkers * 4 : 0);
        const size_t optin = device_props(d->device).smem_optin;
        // the extraction kernel's static shared memory is about 10 KB; 16 KB is reserved
        int rc2 = ensure_smem_optin((const void *)emit_kernel, d->device, (optin ? optin : 232448) - 16384);
        if (rc2) e = cudaErrorInvalidValue;
        else {
            const ProfToken et = prof_begin(stream);
            // programmatic dependent launch: the extraction grid is scheduled while the
            // scan's last block joins, and waits (griddepcontrol.wait) for its results
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)pl.grid);
            cfg.blockDim = dim3(cpb);
            cfg.dynamicSmemBytes = esmem;
            cfg.stream = stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = et.a ? 0 : 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, emit_kernel, ep, tab5_smem, ptab_smem);
            if (e == cudaSuccess) e = cudaGetLastError();
            prof_end(et, stream, PROF_EMIT);
            record_launch();
        }
    }
    const int rf = scratch_free(mem, stream);
    if (e != cudaSuccess) return cuda_status(e);
    return rf;
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
    DeviceProps pr = device_props(dev);
    size_t optin = pr.smem_optin ? pr.smem_optin : 232448;
    auto acc_in = [&](uint32_t q) { return (accept_mask[q >> 3] >> (q & 7)) & 1u; };
    d->accept0 = acc_in(0);
    d->reset_entry = d->accept0 << 31;
    // Automata too large for per-lane two-symbol tables get a hot-state table (see
    // MODE_HOT): the device tables number the states by how often a walk on random
    // DNA visits them (q0 stays state 0), so the most visited states come first. No
    // state number leaves the library, so the renumbering is internal.
    std::vector<uint32_t> ren;        // renumbered table (columns A, C, G, T), or empty
    std::vector<uint8_t> ren_acc;
    std::vector<double> visit;        // visit share of each (new) state
    const bool hot_ok = n_states > max_pair_states(optin, 8) && n_states <= kHotMaxStates;
    const bool hot_tables = n_states <= kHotMaxStates;   // small automata may request it too
    if (hot_ok) {
        std::vector<uint64_t> hits(n_states, 0);
        uint64_t x = 0x2545F4914F6CDD1Dull;
        uint32_t q = 0;
        const uint64_t steps = 1ull << 22;
        for (uint64_t k = 0; k < steps; ++k) {
            x ^= x << 13; x ^= x >> 7; x ^= x << 17;
            q = table[4ull * q + (uint32_t)(x >> 62)];
            ++hits[q];
        }
        std::vector<uint32_t> order(n_states);
        for (uint32_t i = 0; i < n_states; ++i) order[i] = i;
        std::stable_sort(order.begin() + 1, order.end(),
                         [&](uint32_t a, uint32_t b) { return hits[a] > hits[b]; });
        d->perm.assign(n_states, 0);   // old -> new
        for (uint32_t i = 0; i < n_states; ++i) d->perm[order[i]] = i;
        ren.resize(4ull * n_states);
        ren_acc.resize(n_states);
        visit.resize(n_states);
        for (uint32_t i = 0; i < n_states; ++i) {
            const uint32_t o = order[i];
            for (int c = 0; c < 4; ++c) ren[4ull * i + c] = d->perm[table[4ull * o + c]];
            ren_acc[i] = (uint8_t)acc_in(o);
            visit[i] = (double)hits[o] / (double)steps;
        }
    }
    const uint32_t *tab = hot_ok ? ren.data() : table;
    auto acc = [&](uint32_t q) { return hot_ok ? (uint32_t)ren_acc[q] : acc_in(q); };
    std::vector<uint32_t> one(4ull * n_states);
    for (uint32_t q = 0; q < n_states; ++q)
        for (int c = 0; c < 4; ++c) {
            uint32_t nx = tab[4ull * q + kColOfCode[c]];
            one[4ull * q + c] = nx | (acc(nx) << 31);
        }
    d->definite_depth = dnalib::definite_depth(table, n_states, (int)kMaxLookback, 4096);
    // q0 speculation repaired from the chunk's first 16 bytes works whenever runs meet
    // within 16 symbols (definite depth <= 16, and in practice most automata on DNA);
    // a known larger depth gets an exact lookback instead
    d->lookback = (d->definite_depth > 16) ? (uint32_t)d->definite_depth : 0u;
    // automata that are not definite within 64 symbols: do the runs from all states meet
    // within 16 symbols of typical DNA? Checked on 8 seeded random windows of 256 bases
    // (automata of at most kMaxMapStates states); if not, scans run every chunk from every
    // state (chunk maps)
    if (d->definite_depth < 0 && n_states <= kMaxMapStates) {
        uint64_t x = 0x9E3779B97F4A7C15ull;
        int slow = 0;
        const uint32_t nw = (n_states + 63) / 64;
        std::vector<uint64_t> live(nw), next(nw);
        for (int trial = 0; trial < 8; ++trial) {
            for (uint32_t q = 0; q < n_states; ++q) live[q >> 6] |= 1ull << (q & 63);
            int met = -1;
            for (int k = 0; k < 256 && met < 0; ++k) {
                x ^= x << 13; x ^= x >> 7; x ^= x << 17;
                const uint32_t col = (uint32_t)(x >> 62);
                std::fill(next.begin(), next.end(), 0ull);
                uint32_t n_live = 0;
                for (uint32_t q = 0; q < n_states; ++q)
                    if (live[q >> 6] >> (q & 63) & 1u) {
                        const uint32_t t = table[q * 4u + col];
                        next[t >> 6] |= 1ull << (t & 63);
                    }
                live.swap(next);
                for (uint64_t w : live) n_live += (uint32_t)__builtin_popcountll(w);
                if (n_live <= 1) met = k + 1;
            }
            std::fill(live.begin(), live.end(), 0ull);
            if (met < 0 || met > 16) ++slow;
        }
        d->map_mode = slow > 2;
    }
    // the table placement (measured on GB300): two-symbol copies per lane while they fit,
    // else one shared one-symbol table, else the one-symbol table in L2; the per-lane
    // one-symbol copies and the hot-state rows measured slower than the shared table
    // and are chosen only by dfa_tune or a plan
    if (n_states <= max_pair_states(optin, 8)) d->placement = DNA_PLACE_SMEM_PAIR;
    else if (scan_total_smem(MODE_ONE_SMEM, 8, n_states) <= optin) d->placement = DNA_PLACE_SMEM_ONE;
    else d->placement = DNA_PLACE_GLOBAL_ONE;
    if (hot_ok) {
        // the visit share of the hot rows that fit (reported; the hot-state rows are not
        // the default: measured on GB300 they lose to the one-symbol table even when every
        // state has a row, and dfa_tune picks them only if they win on the caller's data)
        const uint32_t h = hot_rows_for(optin, kHotWarps, n_states);
        double cover = 0;
        for (uint32_t i = 0; i < h && i < n_states; ++i) cover += visit[i];
        d->hot_cover = cover;
    }
    cudaError_t e = device_alloc((void **)&d->d_one, sizeof(uint32_t) * one.size());
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
        e = device_alloc((void **)&d->d_pair, sizeof(uint32_t) * pair.size());
        if (e == cudaSuccess) e = cudaMemcpy(d->d_pair, pair.data(), sizeof(uint32_t) * pair.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && hot_tables) {
        // u16 tables: two-symbol rows (next state | accepting steps in the pair << 14) and
        // one-symbol rows (next state | next state accepts << 14), code order A, C, T, G
        std::vector<uint16_t> h2(16ull * n_states), h1(4ull * n_states);
        for (uint32_t q = 0; q < n_states; ++q)
            for (int b0 = 0; b0 < 4; ++b0) {
                const uint32_t e1 = one[4ull * q + b0];
                const uint32_t q1 = e1 & 0x7FFFFFFFu;
                h1[4ull * q + b0] = (uint16_t)(q1 | ((e1 >> 31) << 14));
                for (int b1 = 0; b1 < 4; ++b1) {
                    const uint32_t e2 = one[4ull * q1 + b1];
                    const uint32_t cnt = (e1 >> 31) + (e2 >> 31);
                    h2[16ull * q + b0 + 4 * b1] = (uint16_t)((e2 & 0x7FFFFFFFu) | (cnt << 14));
                }
            }
        e = device_alloc((void **)&d->d_hot2, sizeof(uint16_t) * h2.size());
        if (e == cudaSuccess) e = cudaMemcpy(d->d_hot2, h2.data(), sizeof(uint16_t) * h2.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = device_alloc((void **)&d->d_hot1, sizeof(uint16_t) * h1.size());
        if (e == cudaSuccess) e = cudaMemcpy(d->d_hot1, h1.data(), sizeof(uint16_t) * h1.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && !d->perm.empty()) {
        // device -> caller numbering, for the last state a piece's scan reports
        std::vector<uint32_t> inv(n_states);
        for (uint32_t q = 0; q < n_states; ++q) inv[d->perm[q]] = q;
        e = device_alloc((void **)&d->d_perm_inv, sizeof(uint32_t) * n_states);
        if (e == cudaSuccess)
            e = cudaMemcpy(d->d_perm_inv, inv.data(), sizeof(uint32_t) * n_states, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(d->d_one);
        cudaFree(d->d_pair);
        cudaFree(d->d_hot2);
        cudaFree(d->d_hot1);
        cudaFree(d->d_perm_inv);
        delete d;
        return cuda_status(e);
    }
    *out = d;
    return DNA_OK;
}

extern "C" int dfa_load_labeled(const uint32_t *table, uint32_t n_states, const uint32_t *labels,
                                uint32_t n_labels, dna_dfa **out) {
    if (!table || !labels || !out || n_states == 0 || n_states > kMaxStates || n_labels == 0 || n_labels > 32)
        return DNA_ERR_INVALID_ARG;
    const uint32_t allowed = n_labels == 32 ? 0xFFFFFFFFu : ((1u << n_labels) - 1u);
    std::vector<uint8_t> mask((n_states + 7) / 8, 0);
    for (uint32_t q = 0; q < n_states; ++q) {
        if (labels[q] & ~allowed) return DNA_ERR_INVALID_ARG;
        if (labels[q]) mask[q >> 3] |= (uint8_t)(1u << (q & 7));
    }
    dna_dfa *d = nullptr;
    int rc = dfa_load(table, n_states, mask.data(), &d);
    if (rc) return rc;
    // the device numbering of the states (see dfa_load)
    std::vector<uint32_t> lab(labels, labels + n_states);
    if (!d->perm.empty())
        for (uint32_t q = 0; q < n_states; ++q) lab[d->perm[q]] = labels[q];
    cudaError_t e = device_alloc((void **)&d->d_labels, sizeof(uint32_t) * n_states);
    if (e == cudaSuccess)
        e = cudaMemcpy(d->d_labels, lab.data(), sizeof(uint32_t) * n_states, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dfa_free(d);
        return cuda_status(e);
    }
    d->n_labels = n_labels;
    *out = d;
    return DNA_OK;
}

extern "C" void dfa_free(dna_dfa *d) {
    if (!d) return;
    cudaFree(d->d_one);
    cudaFree(d->d_pair);
    cudaFree(d->d_hot2);
    cudaFree(d->d_hot1);
    cudaFree(d->d_labels);
    cudaFree(d->d_perm_inv);
    delete d;
}

extern "C" int dna_scan_labels(const dna_dfa *dfa, const uint8_t *seq, uint64_t len, dna_stream_t stream_h,
                               uint64_t *out_count, uint64_t *out_label_counts, uint64_t *out_positions,
                               uint32_t *out_pos_labels, uint64_t positions_capacity) {
    if (!dfa || !out_count || !out_label_counts || (len > 0 && !seq)) return DNA_ERR_INVALID_ARG;
    if (!dfa->d_labels || dfa->n_labels == 0) return DNA_ERR_INVALID_ARG;
    if (out_pos_labels && !out_positions) return DNA_ERR_INVALID_ARG;
    if (len > (1ull << 40)) return DNA_ERR_INVALID_ARG;
    int cur_dev = -1;
    DNA_CUDA(cudaGetDevice(&cur_dev));
    if (cur_dev != dfa->device) return DNA_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_h;
    DNA_CUDA(cudaMemsetAsync(out_label_counts, 0, sizeof(uint64_t) * dfa->n_labels, stream));
    if (len == 0) return scan_impl(dfa, seq, len, stream, out_count, nullptr, 0, nullptr);
    LabelOut lab;
    lab.labels = dfa->d_labels;
    lab.counts = reinterpret_cast<unsigned long long *>(out_label_counts);
    lab.pos_labels = out_positions ? out_pos_labels : nullptr;
    lab.n_labels = dfa->n_labels;
    return scan_impl(dfa, seq, len, stream, out_count, out_positions, out_positions ? positions_capacity : 0,
                     nullptr, &lab);
}

extern "C" int dfa_info(const dna_dfa *d, dna_dfa_info *out) {
    if (!d || !out) return DNA_ERR_INVALID_ARG;
    out->n_states = d->n_states;
    out->definite_depth = d->definite_depth;
    out->lookback = d->lookback;
    out->placement = d->placement;
    out->accept_start = d->accept0;
    out->device = d->device;
    out->chunk_maps = d->map_mode ? 1u : 0u;
    out->n_labels = d->n_labels;
    return DNA_OK;
}

extern "C" int dna_scan(const dna_dfa *dfa, const uint8_t *seq, uint64_t len, dna_stream_t stream,
                        uint64_t *out_count, uint64_t *out_positions, uint64_t positions_capacity) {
    return scan_impl(dfa, seq, len, (cudaStream_t)stream, out_count, out_positions,
                     positions_capacity, nullptr);
}

extern "C" int dna_scan_from(const dna_dfa *dfa, const uint8_t *seq, uint64_t len, uint32_t start_state,
                             dna_stream_t stream, uint64_t *out_count, uint32_t *out_last_state,
                             uint64_t *out_positions, uint64_t positions_capacity) {
    if (!dfa || start_state >= dfa->n_states) return DNA_ERR_INVALID_ARG;
    ScanFrom from;
    from.start = dfa->perm.empty() ? start_state : dfa->perm[start_state];
    from.out_last = out_last_state;
    return scan_impl(dfa, seq, len, (cudaStream_t)stream, out_count, out_positions, positions_capacity,
                     nullptr, nullptr, &from);
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
    {
        const int ra = scratch_alloc(dfa->device, seq_off + (size_t)len + 16, stream, &mem);
        if (ra) return ra;
    }
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
    const int rf = scratch_free(mem, stream);
    if (rc != DNA_OK) return rc;
    if (e == cudaSuccess && rf != DNA_OK) return rf;
    if (e != cudaSuccess) return cuda_status(e);
    return cap && *count_host > cap ? DNA_ERR_CAPACITY : DNA_OK;
}

extern "C" int dfa_tune(dna_dfa *d, const uint8_t *seq, uint64_t len, dna_stream_t stream_h,
                        uint32_t *out_placement, float *out_ms) {
    if (!d || !seq || len == 0 || !out_placement) return DNA_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_h;
    int cur_dev = -1;
    DNA_CUDA(cudaGetDevice(&cur_dev));
    if (cur_dev != d->device) return DNA_ERR_INVALID_ARG;
    if (d->map_mode) {   // chunk maps: no table placement to choose
        *out_placement = DNA_PLACE_MAP;
        return DNA_OK;
    }
    uint64_t *cnt = nullptr;
    int rc = scratch_alloc(d->device, 8, stream, (void **)&cnt);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        scratch_free(cnt, stream);
        return cuda_status(ce);
    }
    const uint32_t cands[] = {DNA_PLACE_SMEM_PAIR, DNA_PLACE_SMEM_ONE, DNA_PLACE_SMEM_ONE_REP,
                              DNA_PLACE_SMEM_HOT, DNA_PLACE_GLOBAL_ONE};
    float best = 3.4e38f;
    uint32_t best_pl = d->placement;
    for (uint32_t pl : cands) {
        dna_plan plan = {};
        plan.placement = pl;
        // a placement the automaton does not fit in is skipped
        if (scan_impl(d, seq, len, stream, cnt, nullptr, 0, &plan) != DNA_OK) continue;
        float ms_sum = 0;
        bool ok = true;
        for (int r = 0; r < 3 && ok; ++r) {
            ok = cudaEventRecord(e0, stream) == cudaSuccess &&
                 scan_impl(d, seq, len, stream, cnt, nullptr, 0, &plan) == DNA_OK &&
                 cudaEventRecord(e1, stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0;
            if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms_sum += ms;
            else ok = false;
        }
        if (ok && ms_sum / 3 < best) { best = ms_sum / 3; best_pl = pl; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    scratch_free(cnt, stream);
    DNA_CUDA(cudaStreamSynchronize(stream));
    d->placement = best_pl;
    *out_placement = best_pl;
    if (out_ms) *out_ms = best;
    return DNA_OK;
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
    if (d->map_mode) {
        // automata whose runs never meet: the chunk-map kernels, as dna_scan runs them,
        // with their per-chunk maps in the fixed array
        return map_scan_impl(d, seq, len, stream, out_count, nullptr, 0, (uint8_t *)base,
                             kStaticScratchBytes);
    }
    const uint64_t shift = (uint64_t)((uintptr_t)seq & 15u);
    const uint8_t *abase = seq - shift;
    const uint64_t total = len + shift;
    Plan pl;
    rc = make_plan(d, total, false, nullptr, pl);
    if (rc) return rc;
    const uint64_t nblocks = (uint64_t)pl.grid;
    // every chunk may be pending (automata that converge slowly): the last block then
    // repairs them all in parallel instead of walking every boundary in order
    const uint32_t pending_cap = (uint32_t)std::min<uint64_t>(pl.nseg + 16u, 1ull << 31);
    const uint32_t div_cap = 4096;
    Scratch s;
    carve(s, pl.nseg, nblocks, false, pending_cap, div_cap, nullptr);
    if (s.bytes > kStaticScratchBytes) return DNA_ERR_CAPACITY;
    carve(s, pl.nseg, nblocks, false, pending_cap, div_cap, (uint8_t *)base);
    // the counters the kernel expects at zero; everything else is written before it is read
    cudaError_t e = cudaMemsetAsync(s.ctrl, 0, 32, stream);
    if (e != cudaSuccess) return cuda_status(e);
    ScanParams sp;
    sp.abase = abase; sp.lo = shift; sp.hi = total; sp.seg_bytes = pl.seg_bytes; sp.nseg = pl.nseg;
    sp.lookback = pl.lookback; sp.n_states = d->n_states; sp.reset_entry = d->reset_entry;
    sp.one = d->d_one; sp.pair = d->d_pair; sp.given_start = nullptr;
    sp.spec_start = s.spec_start; sp.last_state = s.last_state; sp.count = s.count;
    sp.stash = nullptr; sp.nrec = nullptr; sp.flags = s.flags; sp.fix_delta = nullptr;
    sp.prefetch_tiles = pl.prefetch;
    sp.ctrl = s.ctrl; sp.pending = s.pending; sp.pending_cap = pending_cap;
    sp.reset_ctrl = 0u;
    sp.start_state = 0u;
    sp.out_last = nullptr;
    sp.perm_inv = nullptr;
    sp.div_list = s.div_list; sp.div_cap = div_cap;
    sp.cta_sum = s.cta_sum; sp.cta_off = s.cta_off; sp.block_head = s.block_head; sp.out_count = out_count;
    sp.k1 = 1u; sp.k5 = 1u << 5;
    sp.lut_lo = 0x00630061u; sp.lut_hi = 0x00670074u;
    sp.hot2 = reinterpret_cast<const uint32_t *>(d->d_hot2);
    sp.hot1 = reinterpret_cast<const uint32_t *>(d->d_hot1);
    sp.hot_rows = pl.hot_rows;
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
