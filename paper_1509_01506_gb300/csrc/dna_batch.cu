// dna_batch.cu -- the batched path: many sequences x many automata in one persistent
// launch (counts only), plus its plan object and the C ABI around it.
//
// The work of a batch is the set of (sequence, automaton) pairs. Every sequence is cut
// into chunks (input-based partitioning, Sec. III-A, Fig. 1a); a chunk is scanned by one
// lane. Automata whose definite depth m is at most 64 (every word of m symbols sends all
// states to one state; Sec. III-B.3 observes that the runs from all possible starting
// states meet within a few symbols) get their exact chunk start state by running from q0
// over the m symbols in front of the chunk, so no join between chunks is needed and the
// per-chunk counts of a sequence simply add up. The steps on the device:
//   1. ingest: the sequences' bytes are mapped to 2-bit codes (16 per 32-bit word, one
//      128-byte row per 512 bases) with one flag byte per 512-base tile that marks a
//      reset byte (N, IUPAC, any non-base byte) or the sequence end inside the tile;
//   2. scan: a persistent kernel takes tasks from an atomic ticket. A task is a run of
//      chunk groups (one chunk per lane of the block) and one automaton; the block loads
//      that automaton's two-symbol table into shared memory (replicated per lane, as in
//      the single-sequence kernel) and its warps stage their lanes' rows with cp.async.
//      Flagged tiles are walked byte by byte from the original sequence with the
//      one-symbol table. Lane counts are added per sequence inside the warp and then
//      atomically into out[sequence][automaton].
// Tasks are ordered group-major, automaton-minor, so blocks that run at the same time
// read the same rows (from L2) with different automata. Automata that do not qualify
// (no definite depth <= 64, or too many states for the shared-memory table) are scanned
// with the single-sequence path, one call per (sequence, automaton).

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/dna_dfa.h"
#include "dna_device.cuh"
#include "dna_runtime.h"

using namespace dnalib;

namespace {

constexpr int kBasesPerTile = 512;            // one 128-byte row of packed codes
constexpr int kWordsPerTile = 32;             // 16 codes per 32-bit word
constexpr uint32_t kBatchMaxDepth = 64;
constexpr int kIngestTilesPerUnit = 64;       // tiles one ingest warp converts per unit

// ------------------------------------------------------------------- ingest

struct IngestParams {
    const uint8_t *const *seqs;   // [n_seqs] device pointers
    const uint64_t *lens;         // [n_seqs]
    const uint64_t *tile0;        // [n_seqs] first tile of each sequence in 'codes'
    const uint2 *units;           // [n_units] {sequence, first tile of the unit}
    uint32_t n_units;
    uint32_t *codes;              // [total tiles][32]
    uint8_t *tflags;              // [total tiles]
    uint32_t lut_lo, lut_hi;      // lowercase letters selected by the codes (see below)
};

// Four bytes -> four 2-bit codes (code = (byte >> 1) & 3: A 0, C 1, T 2, G 3) packed
// into bits 0..7, code i at bits 2i..2i+1. The codes sit at bits 0..1 of each byte of
// x; the multiply moves code i to bit 24 + 2i (every partial product lands on its own
// pair of bits, so nothing carries) and the packed byte is bits 24..31.
__device__ __forceinline__ uint32_t pack4(uint32_t w) {
    const uint32_t x = (w >> 1) & 0x03030303u;
    return x * 0x01041040u;   // 2^24 + 2^18 + 2^12 + 2^6
}

// Non-zero (outside the case bit) iff some byte of w is not a base: the expected byte
// for each code is read from {lut_lo, lut_hi} with a byte permute.
__device__ __forceinline__ uint32_t base_err(uint32_t w, uint32_t lut_lo, uint32_t lut_hi) {
    const uint32_t x = w & 0x06060606u;
    const uint32_t z = x | (x >> 4);
    const uint32_t sel = __byte_perm(z, 0, 0x0020);
    return (__byte_perm(lut_lo, lut_hi, sel) ^ w) & 0xDFDFDFDFu;
}

__global__ void __launch_bounds__(256) ingest_kernel(IngestParams p) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = blockDim.x >> 5;
    for (uint32_t u = blockIdx.x * warps + (threadIdx.x >> 5); u < p.n_units; u += gridDim.x * warps) {
        const uint2 unit = p.units[u];
        const uint8_t *src = p.seqs[unit.x];
        const uint64_t len = p.lens[unit.x];
        const uint64_t tiles = (len + kBasesPerTile - 1) / kBasesPerTile;
        const uint64_t t_end = unit.y + (uint64_t)kIngestTilesPerUnit < tiles ? unit.y + kIngestTilesPerUnit : tiles;
        const bool aligned = ((uintptr_t)src & 15u) == 0;
        uint32_t *out = p.codes + p.tile0[unit.x] * kWordsPerTile;
        uint8_t *fl = p.tflags + p.tile0[unit.x];
        for (uint64_t t = unit.y; t < t_end; ++t) {
            const uint64_t b = t * kBasesPerTile + (uint64_t)lane * 16u;   // this lane's 16 bases
            uint32_t w[4];
            uint32_t bad = 0;
            if (aligned && b + 16 <= len) {
                const uint4 v = *reinterpret_cast<const uint4 *>(src + b);
                w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
            } else {
                // unaligned sequence or its last 16 bytes: byte loads; bytes past the end
                // read as 'A' and the tile is flagged
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    uint32_t v = 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t o = b + 4u * i + k;
                        const uint32_t byte = o < len ? src[o] : 0x41u;
                        v |= byte << (8 * k);
                    }
                    w[i] = v;
                }
                bad = b + 16 > len;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) bad |= base_err(w[i], p.lut_lo, p.lut_hi);
            const uint32_t word = __byte_perm(__byte_perm(pack4(w[0]), pack4(w[1]), 0x0073),
                                              __byte_perm(pack4(w[2]), pack4(w[3]), 0x0073), 0x5410);
            out[t * kWordsPerTile + lane] = word;
            const bool any_bad = __any_sync(0xFFFFFFFFu, bad != 0);
            if (lane == 0) fl[t] = any_bad ? 1 : 0;
        }
    }
}

// ----------------------------------------------------------------- scan

struct BatchDfa {
    const uint32_t *one;      // [n_states][4] one-symbol entries (next | accept << 31)
    const uint32_t *pair;     // [n_states][16] compact pair entries (next | count << 24)
    uint32_t n_states;
    uint32_t lookback;        // bases run from q0 in front of a chunk (multiple of 16, <= 64)
    uint32_t reset_entry;
    uint32_t col;             // output column
};

struct BatchParams {
    const uint32_t *codes;
    const uint8_t *tflags;
    const uint8_t *const *seqs;
    const uint64_t *lens;
    const uint64_t *tile0;
    const uint2 *chunks;      // [n_chunks] {sequence, chunk index within the sequence}
    uint64_t n_chunks;
    uint32_t chunk_tiles;     // tiles per chunk
    uint32_t groups_per_task;
    uint64_t n_groups;        // ceil(n_chunks / lanes per block)
    uint64_t n_tasks;         // ceil(n_groups / groups_per_task) * n_fast
    const BatchDfa *dfas;
    uint32_t n_fast;
    uint32_t out_stride;
    uint32_t *ticket;         // zeroed before the launch
    unsigned long long *out;  // [n_seqs][out_stride], zeroed before the launch
    uint32_t max_states;      // table capacity of the shared-memory layout
    uint32_t k1, k5;          // 1 and 32 at run time (multiplies stay on the FMA pipe)
};

// shared memory: [staging: WARPS x 32 rows x 128 B][one-symbol table: max_states x 16 B]
//                [pad to a 2048-byte shared address][pair table: max_states x 2048 B]
// The pad is computed from the block's actual shared address; 2048 bytes of slack are
// allocated for it.
__host__ __device__ constexpr uint32_t batch_one_off(int warps) { return (uint32_t)warps * 32u * kTile; }
inline size_t batch_smem_bytes(int warps, uint32_t max_states) {
    return (size_t)batch_one_off(warps) + (size_t)max_states * 16 + 2048 + (size_t)max_states * kPairRowBytes;
}

// One word (16 bases) of a chain through the pair table. Pair k of the word (bits
// 4k..4k+3) must arrive at bits 7..10 of the mux operand with bits 27..30 clear: pairs
// 0..2 come from the word's low 12 bits shifted left 7, 3 and right 1; pairs 3..7 from
// right shifts of 5..21, which leave bits 27..30 zero. The 8 entries are summed as they
// arrive: their address parts add up to less than 2^21 and bits 29..31 are zero, so the
// pair counts (at most 16) land in bits 27..31 of the sum, which moves into cnt once.
__device__ __forceinline__ uint32_t word_pairs(uint32_t cur, uint32_t wd, uint32_t k1, uint32_t k5, uint32_t &cnt) {
    (void)k1;
    const uint32_t lo = wd & 0xFFFu;
    const uint32_t e0 = lds_u32(mux_pair(cur, lo << 7));
    const uint32_t e1 = lds_u32(mux_pair(e0, lo << 3));
    const uint32_t e2 = lds_u32(mux_pair(e1, lo >> 1));
    uint32_t t = e0 + e1 + e2;
    const uint32_t e3 = lds_u32(mux_pair(e2, wd >> 5));
    const uint32_t e4 = lds_u32(mux_pair(e3, wd >> 9));
    t = t + e3 + e4;
    const uint32_t e5 = lds_u32(mux_pair(e4, wd >> 13));
    const uint32_t e6 = lds_u32(mux_pair(e5, wd >> 17));
    t = t + e5 + e6;
    const uint32_t e7 = lds_u32(mux_pair(e6, wd >> 21));
    cnt = mad_hi(t + e7, k5, cnt);      // cnt += sum >> 27
    return e7;
}

// Walks bytes [from, to) of a sequence (offsets from the 16-byte aligned 'abase'; bytes at
// or past 'hi' are never read past their 16-byte granule) with the one-symbol table from
// state q, adding accepting steps to *cnt. Rare (steps with a reset byte or a sequence
// end, lookback windows over them), so it is kept out of line with one load in flight.
__device__ __noinline__ uint32_t walk_bytes(const OneTable &T, const uint8_t *abase, uint64_t from, uint64_t to,
                                            uint64_t hi, uint32_t q, uint32_t *cnt) {
    uint32_t c = 0;
    for (uint64_t g = from & ~(uint64_t)15; g < to; g += 16) {
        const uint4 v = g < hi ? *reinterpret_cast<const uint4 *>(abase + g) : make_uint4(0, 0, 0, 0);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const uint64_t o = g + (uint64_t)i;
            if (o >= from && o < to) {
                const uint32_t e = T.step(q, (w[i >> 2] >> (8 * (i & 3))) & 0xFFu);
                q = e & 0x7FFFFFFFu;
                c += e >> 31;
            }
        }
    }
    if (cnt) *cnt += c;
    return q;
}

constexpr int kStepBases = 256;                // bases per lane per staging step (64 B)
constexpr int kStepWords = 16;
constexpr int kBatchRows = 64;                 // staged rows per warp: two chunks per lane

// Persistent: each block takes tasks from the ticket. A lane walks two chunks (rows lane
// and lane + 32 of its warp's 64) as two independent chains, so the lookups of one
// chain overlap the latency of the other's.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) batch_kernel(BatchParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ unsigned long long row_src[WARPS][kBatchRows];   // word offset of each row's chunk in 'codes'
    __shared__ uint32_t row_steps[WARPS][kBatchRows];
    __shared__ uint32_t task_s;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t stage_addr = smem_base + (uint32_t)warp * kBatchRows * 64u;
    const uint8_t *stage_ptr = smem + (size_t)warp * kBatchRows * 64u;
    uint32_t *one_s = reinterpret_cast<uint32_t *>(smem + batch_one_off(WARPS));
    const uint32_t pair_base = (smem_base + batch_one_off(WARPS) + p.max_states * 16u + 2047u) & ~2047u;
    uint32_t *pair_s = reinterpret_cast<uint32_t *>(smem + (pair_base - smem_base));
    const uint32_t r8 = (uint32_t)lane >> 2, cc = (uint32_t)lane & 3u;
    uint32_t cur_dfa = 0xFFFFFFFFu;

    for (;;) {
        __syncthreads();   // every warp is done with the previous task's table
        if (threadIdx.x == 0) task_s = atomicAdd(p.ticket, 1u);
        __syncthreads();
        const uint64_t task = task_s;
        if (task >= p.n_tasks) break;
        const uint64_t tg = task / p.n_fast;
        const uint32_t k = (uint32_t)(task % p.n_fast);
        const BatchDfa D = p.dfas[k];
        if (k != cur_dfa) {
            for (uint32_t i = threadIdx.x; i < D.n_states * 4u; i += WARPS * 32) one_s[i] = D.one[i];
            const uint32_t n2 = D.n_states * 16u * 32u;
            for (uint32_t i = threadIdx.x; i < n2; i += WARPS * 32) {
                const uint32_t e = D.pair[i >> 5];
                const uint32_t nx = e & 0x00FFFFFFu, c = e >> 24;
                pair_s[i] = (c << kCountShift) | (pair_base + nx * (uint32_t)kPairRowBytes + (i & 31u) * 4u);
            }
            cur_dfa = k;
            __syncthreads();
        }
        OneTable T;
        T.t = one_s;
        T.reset_entry = D.reset_entry;
        const uint64_t g_end = (tg + 1) * p.groups_per_task < p.n_groups ? (tg + 1) * p.groups_per_task : p.n_groups;
        for (uint64_t g = tg * p.groups_per_task; g < g_end; ++g) {
            // the lane's two chunks: rows lane and lane + 32 of the warp's 64
            uint32_t s[2] = {0xFFFFFFFFu, 0xFFFFFFFFu}, steps[2] = {0, 0}, cur[2], cnt[2] = {0, 0};
            uint64_t base0[2] = {0, 0}, len[2] = {0, 0}, ctile[2] = {0, 0};
            bool active[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint64_t ci = (g * WARPS + warp) * kBatchRows + (uint64_t)(32 * h + lane);
                active[h] = ci < p.n_chunks;
                if (active[h]) {
                    const uint2 c = p.chunks[ci];
                    s[h] = c.x;
                    len[h] = p.lens[c.x];
                    base0[h] = (uint64_t)c.y * p.chunk_tiles * kBasesPerTile;
                    const uint64_t rem = len[h] - base0[h];
                    const uint64_t cap = (uint64_t)p.chunk_tiles * kBasesPerTile;
                    steps[h] = (uint32_t)(((rem < cap ? rem : cap) + kStepBases - 1) / kStepBases);
                    ctile[h] = p.tile0[c.x] + (uint64_t)c.y * p.chunk_tiles;
                }
                row_src[warp][32 * h + lane] = ctile[h] * kWordsPerTile;
                row_steps[warp][32 * h + lane] = steps[h];
            }
            __syncwarp();
            const uint32_t nsteps = __reduce_max_sync(0xFFFFFFFFu, steps[0] > steps[1] ? steps[0] : steps[1]);
            // copy j of a lane moves 16-byte column cc of row 8j + lane/4 (rows past their
            // chunk's end are zero-filled and never read); column c of row r sits at slot
            // c ^ ((r >> 1) & 3), so the lanes of each 128-bit read phase hit distinct banks
            auto issue = [&](uint32_t st) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t r = 8u * j + r8;
                    const bool ok = st < row_steps[warp][r];
                    const uint32_t *src = p.codes + row_src[warp][r] + (uint64_t)st * kStepWords + cc * 4u;
                    const uint32_t dst = stage_addr + r * 64u + ((cc ^ ((r >> 1) & 3u)) << 4);
                    cp_async16(dst, ok ? (const void *)src : (const void *)p.codes, ok ? 16u : 0u);
                }
            };
            if (nsteps) issue(0);
            cp_async_commit();

            // exact start states: run from q0 over the 'lookback' bases in front of each
            // chunk (they lie in the previous tile of the same sequence)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                cur[h] = pair_base + (uint32_t)lane * 4u;   // state 0, this lane's copy
                if (active[h] && base0[h] > 0 && D.lookback > 0) {
                    const uint64_t pt = ctile[h] - 1;
                    if (p.tflags[pt] == 0) {
                        const uint32_t nw = D.lookback / 16u;
                        const uint32_t *lw = p.codes + pt * kWordsPerTile + (kWordsPerTile - nw);
                        uint32_t discard = 0;
                        for (uint32_t i = 0; i < nw; ++i) cur[h] = word_pairs(cur[h], lw[i], p.k1, p.k5, discard);
                    } else {
                        const uint8_t *src = p.seqs[s[h]];
                        const uint64_t sh = (uint64_t)((uintptr_t)src & 15u);
                        const uint32_t q = walk_bytes(T, src - sh, sh + base0[h] - D.lookback, sh + base0[h],
                                                      sh + len[h], 0u, nullptr);
                        cur[h] = pair_base + q * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u;
                    }
                }
            }
            for (uint32_t st = 0; st < nsteps; ++st) {
                cp_async_wait<0>();
                __syncwarp();
                uint32_t wa[kStepWords], wb[kStepWords];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t ra = (uint32_t)lane, rb = (uint32_t)lane + 32u;
                    const uint4 va = *reinterpret_cast<const uint4 *>(stage_ptr + ra * 64u + ((c ^ ((ra >> 1) & 3u)) << 4));
                    const uint4 vb = *reinterpret_cast<const uint4 *>(stage_ptr + rb * 64u + ((c ^ ((rb >> 1) & 3u)) << 4));
                    wa[4 * c] = va.x; wa[4 * c + 1] = va.y; wa[4 * c + 2] = va.z; wa[4 * c + 3] = va.w;
                    wb[4 * c] = vb.x; wb[4 * c + 1] = vb.y; wb[4 * c + 2] = vb.z; wb[4 * c + 3] = vb.w;
                }
                __syncwarp();
                if (st + 1 < nsteps) issue(st + 1);
                cp_async_commit();
                // a step is 256 bases, half of an ingest tile; flagged tiles are walked byte by byte
                const bool live_a = st < steps[0], live_b = st < steps[1];
                const bool fast_a = live_a && p.tflags[ctile[0] + (st >> 1)] == 0;
                const bool fast_b = live_b && p.tflags[ctile[1] + (st >> 1)] == 0;
                if (fast_a && fast_b) {
#pragma unroll
                    for (int kk = 0; kk < kStepWords; ++kk) {
                        cur[0] = word_pairs(cur[0], wa[kk], p.k1, p.k5, cnt[0]);
                        cur[1] = word_pairs(cur[1], wb[kk], p.k1, p.k5, cnt[1]);
                    }
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const bool live = h ? live_b : live_a;
                        const bool fast = h ? fast_b : fast_a;
                        if (!live) continue;
                        if (fast) {
#pragma unroll
                            for (int kk = 0; kk < kStepWords; ++kk)
                                cur[h] = word_pairs(cur[h], h ? wb[kk] : wa[kk], p.k1, p.k5, cnt[h]);
                        } else {
                            // a reset byte or the sequence end in this step's 256 bases
                            const uint32_t q0 = ((cur[h] & 0x3FFFFu) - pair_base) / (uint32_t)kPairRowBytes;
                            const uint8_t *src = p.seqs[s[h]];
                            const uint64_t sh = (uint64_t)((uintptr_t)src & 15u);
                            const uint64_t tb = base0[h] + (uint64_t)st * kStepBases;
                            const uint64_t te = tb + kStepBases < len[h] ? tb + kStepBases : len[h];
                            uint32_t c2 = cnt[h];
                            const uint32_t q = walk_bytes(T, src - sh, sh + tb, sh + te, sh + len[h], q0, &c2);
                            cnt[h] = c2;
                            cur[h] = pair_base + q * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u;
                        }
                    }
                }
            }
            cp_async_wait<0>();
            // add the lane counts per sequence (a warp's chunks are ordered by sequence,
            // so usually one or two distinct sequences)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned todo = __ballot_sync(0xFFFFFFFFu, active[h]);
                while (todo) {
                    const int leader = __ffs(todo) - 1;
                    const uint32_t key = __shfl_sync(0xFFFFFFFFu, s[h], leader);
                    const bool mine = active[h] && s[h] == key;
                    uint32_t v = mine ? cnt[h] : 0u;
#pragma unroll
                    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                    if (lane == leader && v)
                        atomicAdd(p.out + (uint64_t)key * p.out_stride + D.col, (unsigned long long)v);
                    todo &= ~__ballot_sync(0xFFFFFFFFu, mine);
                }
            }
            __syncwarp();   // row_src / row_steps are rewritten by the next group
        }
    }
}

using BatchFn = void (*)(BatchParams);
BatchFn batch_fn(int warps) {
    switch (warps) {
        case 8: return batch_kernel<8>;
        case 16: return batch_kernel<16>;
        case 24: return batch_kernel<24>;
        default: return nullptr;
    }
}

// static shared memory of batch_kernel<W> (row_src, row_steps, task_s), as compiled
size_t batch_static_smem(int warps) {
    static std::atomic<size_t> cached[3] = {};
    const int i = warps == 8 ? 0 : warps == 16 ? 1 : 2;
    size_t v = cached[i].load(std::memory_order_relaxed);
    if (v == 0) {
        cudaFuncAttributes a;
        v = cudaFuncGetAttributes(&a, (const void *)batch_fn(warps)) == cudaSuccess && a.sharedSizeBytes
                ? a.sharedSizeBytes : (size_t)warps * kBatchRows * 12 + 1024;
        cached[i].store(v, std::memory_order_relaxed);
    }
    return v;
}

}  // namespace

// ===================================================================== plan object

struct dna_batch {
    int device = 0;
    uint32_t n_dfas = 0, n_seqs = 0;
    std::vector<const dna_dfa *> dfas;
    std::vector<const uint8_t *> seqs;
    std::vector<uint64_t> lens;
    std::vector<uint32_t> fast, slow;       // output columns of each path
    uint32_t max_states = 0;
    uint64_t total_tiles = 0, n_units = 0;
    // device memory (one allocation): [seq ptrs][lens][tile0][units][dfa descs][chunks][ticket][tflags][codes]
    uint8_t *mem = nullptr;
    const uint8_t **d_seqs = nullptr;
    uint64_t *d_lens = nullptr, *d_tile0 = nullptr;
    uint2 *d_units = nullptr, *d_chunks = nullptr;
    BatchDfa *d_dfas = nullptr;
    uint32_t *d_ticket = nullptr, *d_codes = nullptr;
    uint8_t *d_tflags = nullptr;
    size_t chunk_cap = 0;                   // entries of d_chunks
    // the chosen plan
    uint32_t chunk_tiles = 8, warps = 16, groups_per_task = 4;
    uint64_t n_chunks = 0;
    int grid = 0, ingest_grid = 0;
    bool use_graph = false;
    cudaGraphExec_t graph = nullptr;
    int graph_kernels = 0;                  // kernel nodes in the captured graph
    uint64_t *graph_out = nullptr;
    std::mutex mu;
};

namespace {

constexpr uint32_t kLutLo = 0x00630061u, kLutHi = 0x00670074u;

// Chunk list for a chunk length: full chunks first, then the sequences' last (partial)
// chunks by decreasing length, so that the lanes of a warp have similar work.
std::vector<uint2> build_chunks(const dna_batch &b, uint32_t chunk_tiles) {
    const uint64_t C = (uint64_t)chunk_tiles * kBasesPerTile;
    std::vector<uint2> full, part;
    std::vector<uint64_t> part_len;
    for (uint32_t s = 0; s < b.n_seqs; ++s) {
        const uint64_t n = b.lens[s];
        const uint64_t nf = n / C;
        for (uint64_t j = 0; j < nf; ++j) full.push_back(make_uint2(s, (uint32_t)j));
        if (n % C) { part.push_back(make_uint2(s, (uint32_t)nf)); part_len.push_back(n % C); }
    }
    std::vector<size_t> order(part.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return part_len[a] > part_len[c]; });
    for (size_t i : order) full.push_back(part[i]);
    return full;
}

int batch_plan_kernel(dna_batch &b, uint32_t chunk_tiles, uint32_t warps, cudaStream_t stream) {
    std::vector<uint2> ch = build_chunks(b, chunk_tiles);
    if (ch.size() > b.chunk_cap) return DNA_ERR_CAPACITY;
    if (!ch.empty())
        DNA_CUDA(cudaMemcpyAsync(b.d_chunks, ch.data(), ch.size() * sizeof(uint2), cudaMemcpyHostToDevice, stream));
    DNA_CUDA(cudaStreamSynchronize(stream));   // 'ch' is freed on return
    b.n_chunks = ch.size();
    b.chunk_tiles = chunk_tiles;
    b.warps = warps;
    BatchFn fn = batch_fn((int)warps);
    if (!fn) return DNA_ERR_INVALID_ARG;
    const size_t optin = device_props(b.device).smem_optin ? device_props(b.device).smem_optin : 232448;
    const size_t dyn = batch_smem_bytes((int)warps, b.max_states);
    if (dyn + batch_static_smem((int)warps) > optin) return DNA_ERR_CAPACITY;
    int rc = ensure_smem_optin((const void *)fn, b.device, optin - batch_static_smem((int)warps));
    if (rc) return rc;
    int per_sm = 0;
    DNA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)warps * 32, dyn));
    if (per_sm < 1) return DNA_ERR_CAPACITY;
    const uint64_t lanes = (uint64_t)warps * kBatchRows;   // chunks per group
    const uint64_t n_groups = (b.n_chunks + lanes - 1) / lanes;
    const int slots = device_props(b.device).sms * per_sm;
    // a task is several chunk groups with one automaton (one table load); aim for at
    // least ~8 tasks per resident block so the ticket balances uneven work
    const uint64_t fast = b.fast.size() ? b.fast.size() : 1;
    uint32_t gpt = 8;
    while (gpt > 1 && ((n_groups + gpt - 1) / gpt) * fast < (uint64_t)slots * 8) gpt >>= 1;
    b.groups_per_task = gpt;
    const uint64_t tasks = ((n_groups + gpt - 1) / gpt) * fast;
    b.grid = (int)std::min<uint64_t>((uint64_t)slots, tasks ? tasks : 1);
    return DNA_OK;
}

void fill_params(const dna_batch &b, BatchParams &bp, unsigned long long *out) {
    const uint64_t lanes = (uint64_t)b.warps * kBatchRows;   // chunks per group
    bp.codes = b.d_codes; bp.tflags = b.d_tflags; bp.seqs = b.d_seqs; bp.lens = b.d_lens;
    bp.tile0 = b.d_tile0; bp.chunks = b.d_chunks; bp.n_chunks = b.n_chunks;
    bp.chunk_tiles = b.chunk_tiles; bp.groups_per_task = b.groups_per_task;
    bp.n_groups = (b.n_chunks + lanes - 1) / lanes;
    bp.n_tasks = ((bp.n_groups + b.groups_per_task - 1) / b.groups_per_task) * b.fast.size();
    bp.dfas = b.d_dfas; bp.n_fast = (uint32_t)b.fast.size(); bp.out_stride = b.n_dfas;
    bp.ticket = b.d_ticket; bp.out = out; bp.max_states = b.max_states;
    bp.k1 = 1u; bp.k5 = 32u;
}

// Queues the whole batch on 'stream': zero the outputs, ingest, the persistent scan,
// then the single-sequence path for the automata that do not qualify.
int enqueue_batch(dna_batch &b, cudaStream_t stream, uint64_t *out) {
    DNA_CUDA(cudaMemsetAsync(out, 0, (size_t)b.n_seqs * b.n_dfas * 8, stream));
    if (!b.fast.empty() && b.total_tiles > 0) {
        DNA_CUDA(cudaMemsetAsync(b.d_ticket, 0, 4, stream));
        IngestParams ip;
        ip.seqs = b.d_seqs; ip.lens = b.d_lens; ip.tile0 = b.d_tile0; ip.units = b.d_units;
        ip.n_units = (uint32_t)b.n_units; ip.codes = b.d_codes; ip.tflags = b.d_tflags;
        ip.lut_lo = kLutLo; ip.lut_hi = kLutHi;
        ProfToken ti = prof_begin(stream);
        ingest_kernel<<<b.ingest_grid, 256, 0, stream>>>(ip);
        DNA_CUDA(cudaGetLastError());
        record_launch();
        prof_end(ti, stream, PROF_INGEST);
        BatchParams bp;
        fill_params(b, bp, reinterpret_cast<unsigned long long *>(out));
        if (bp.n_tasks > 0) {
            ProfToken tb = prof_begin(stream);
            batch_fn((int)b.warps)<<<b.grid, b.warps * 32, batch_smem_bytes((int)b.warps, b.max_states), stream>>>(bp);
            DNA_CUDA(cudaGetLastError());
            record_launch();
            prof_end(tb, stream, PROF_BATCH);
        }
    }
    for (uint32_t col : b.slow)
        for (uint32_t s = 0; s < b.n_seqs; ++s) {
            int rc = scan_impl(b.dfas[col], b.seqs[s], b.lens[s], stream, out + (uint64_t)s * b.n_dfas + col,
                               nullptr, 0, nullptr);
            if (rc) return rc;
        }
    return DNA_OK;
}

int autotune(dna_batch &b, cudaStream_t stream) {
    // candidate (chunk tiles, warps) pairs, timed on the batch's own data
    const uint32_t tiles_c[] = {4, 8, 16, 32};
    const uint32_t warps_c[] = {16, 24};
    uint64_t *tmp = nullptr;
    {
        const int ra = scratch_alloc(b.device, (size_t)b.n_seqs * b.n_dfas * 8, stream, (void **)&tmp);
        if (ra) return ra;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    uint32_t bt = b.chunk_tiles, bw = b.warps;
    int rc = DNA_OK;
    std::vector<uint32_t> saved_slow;
    saved_slow.swap(b.slow);   // time the persistent kernel alone
    for (uint32_t w : warps_c)
        for (uint32_t t : tiles_c) {
            if (batch_plan_kernel(b, t, w, stream) != DNA_OK) continue;
            rc = enqueue_batch(b, stream, tmp);   // warm-up (and ingest)
            if (rc) break;
            cudaEventRecord(e0, stream);
            rc = enqueue_batch(b, stream, tmp);
            cudaEventRecord(e1, stream);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = DNA_ERR_CUDA; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bt = t; bw = w; }
        }
    saved_slow.swap(b.slow);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    scratch_free(tmp, stream);
    if (rc) return rc;
    return batch_plan_kernel(b, bt, bw, stream);
}

void release(dna_batch *b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->mem) cudaFree(b->mem);
    delete b;
}

}  // namespace

// ========================================================================= C ABI

extern "C" int dna_batch_create(const dna_dfa *const *dfas, uint32_t n_dfas, const uint8_t *const *seqs,
                                const uint64_t *lens, uint32_t n_seqs, const dna_batch_opts *opts,
                                dna_stream_t stream_h, dna_batch **out) {
    if (!dfas || !seqs || !lens || !out || n_dfas == 0 || n_seqs == 0) return DNA_ERR_INVALID_ARG;
    int dev = -1;
    DNA_CUDA(cudaGetDevice(&dev));
    for (uint32_t k = 0; k < n_dfas; ++k)
        if (!dfas[k] || dfas[k]->device != dev) return DNA_ERR_INVALID_ARG;
    for (uint32_t s = 0; s < n_seqs; ++s) {
        if (lens[s] > 0 && !seqs[s]) return DNA_ERR_INVALID_ARG;
        if (lens[s] > (1ull << 40)) return DNA_ERR_INVALID_ARG;
    }
    const uint32_t req_chunk = opts ? opts->chunk_bases : 0;
    const uint32_t req_warps = opts ? opts->warps_per_cta : 0;
    if (req_chunk && (req_chunk % kBasesPerTile || req_chunk / kBasesPerTile > 256)) return DNA_ERR_INVALID_ARG;
    if (req_warps && req_warps != 8 && req_warps != 16 && req_warps != 24) return DNA_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_h;

    dna_batch *b = new (std::nothrow) dna_batch;
    if (!b) return DNA_ERR_NOMEM;
    b->device = dev;
    b->n_dfas = n_dfas;
    b->n_seqs = n_seqs;
    b->dfas.assign(dfas, dfas + n_dfas);
    b->seqs.assign(seqs, seqs + n_seqs);
    b->lens.assign(lens, lens + n_seqs);
    b->use_graph = opts && opts->use_graph;

    // which automata the persistent kernel takes: definite depth <= 64 and a table that
    // fits next to the smallest staging area (8 warps)
    const size_t optin = device_props(dev).smem_optin ? device_props(dev).smem_optin : 232448;
    const size_t fixed8 = batch_smem_bytes(8, 0) + batch_static_smem(8);
    const uint32_t cap_states = optin > fixed8 ? (uint32_t)((optin - fixed8) / (kPairRowBytes + 16)) : 0;
    for (uint32_t k = 0; k < n_dfas; ++k) {
        const dna_dfa *d = dfas[k];
        const bool ok = d->d_pair && d->definite_depth >= 0 && (uint32_t)d->definite_depth <= kBatchMaxDepth &&
                        d->n_states <= cap_states;
        (ok ? b->fast : b->slow).push_back(k);
        if (ok) b->max_states = std::max(b->max_states, d->n_states);
    }

    // layout of the packed sequences and the ingest units
    std::vector<uint64_t> tile0(n_seqs);
    std::vector<uint2> units;
    uint64_t tiles = 0;
    for (uint32_t s = 0; s < n_seqs; ++s) {
        tile0[s] = tiles;
        const uint64_t nt = (lens[s] + kBasesPerTile - 1) / kBasesPerTile;
        for (uint64_t t = 0; t < nt; t += kIngestTilesPerUnit) units.push_back(make_uint2(s, (uint32_t)t));
        tiles += nt;
    }
    b->total_tiles = tiles;
    b->n_units = units.size();
    // chunk capacity: the most chunks any candidate chunk length can give
    const uint32_t min_tiles = req_chunk ? req_chunk / kBasesPerTile : 4;
    uint64_t chunk_cap = 0;
    for (uint32_t s = 0; s < n_seqs; ++s) {
        const uint64_t C = (uint64_t)min_tiles * kBasesPerTile;
        chunk_cap += (lens[s] + C - 1) / C;
    }
    b->chunk_cap = chunk_cap;

    std::vector<BatchDfa> descs;
    for (uint32_t k : b->fast) {
        const dna_dfa *d = dfas[k];
        BatchDfa bd;
        bd.one = d->d_one; bd.pair = d->d_pair; bd.n_states = d->n_states;
        bd.lookback = ((uint32_t)d->definite_depth + 15u) / 16u * 16u;
        bd.reset_entry = d->reset_entry; bd.col = k;
        descs.push_back(bd);
    }

    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_seqs = take((size_t)n_seqs * 8), o_lens = take((size_t)n_seqs * 8);
    const size_t o_tile0 = take((size_t)n_seqs * 8), o_units = take(units.size() * 8 + 8);
    const size_t o_dfas = take(descs.size() * sizeof(BatchDfa) + 8), o_chunks = take(chunk_cap * 8 + 8);
    const size_t o_ticket = take(16), o_tflags = take(tiles + 16);
    const size_t o_codes = take(b->fast.empty() ? 16 : tiles * (size_t)kTile + 16);
    cudaError_t e = device_alloc((void **)&b->mem, off);
    if (e != cudaSuccess) { release(b); return cuda_status(e); }
    b->d_seqs = reinterpret_cast<const uint8_t **>(b->mem + o_seqs);
    b->d_lens = reinterpret_cast<uint64_t *>(b->mem + o_lens);
    b->d_tile0 = reinterpret_cast<uint64_t *>(b->mem + o_tile0);
    b->d_units = reinterpret_cast<uint2 *>(b->mem + o_units);
    b->d_dfas = reinterpret_cast<BatchDfa *>(b->mem + o_dfas);
    b->d_chunks = reinterpret_cast<uint2 *>(b->mem + o_chunks);
    b->d_ticket = reinterpret_cast<uint32_t *>(b->mem + o_ticket);
    b->d_tflags = b->mem + o_tflags;
    b->d_codes = reinterpret_cast<uint32_t *>(b->mem + o_codes);
    e = cudaMemcpyAsync(b->d_seqs, seqs, (size_t)n_seqs * 8, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_lens, lens, (size_t)n_seqs * 8, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_tile0, tile0.data(), (size_t)n_seqs * 8, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && !units.empty())
        e = cudaMemcpyAsync(b->d_units, units.data(), units.size() * 8, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && !descs.empty())
        e = cudaMemcpyAsync(b->d_dfas, descs.data(), descs.size() * sizeof(BatchDfa), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // host vectors are freed on return
    if (e != cudaSuccess) { release(b); return cuda_status(e); }
    b->ingest_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)device_props(dev).sms * 8,
                                                                    (units.size() + 7) / 8));

    int rc = DNA_OK;
    if (!b->fast.empty()) {
        uint32_t w = req_warps;
        if (!w) {
            w = 8;
            for (uint32_t c : {24u, 16u})
                if (batch_smem_bytes((int)c, b->max_states) + batch_static_smem((int)c) <= optin) { w = c; break; }
        }
        rc = batch_plan_kernel(*b, req_chunk ? req_chunk / kBasesPerTile : 8, w, stream);
        if (rc == DNA_OK && opts && opts->autotune && !req_chunk && !req_warps) rc = autotune(*b, stream);
    }
    if (rc) { release(b); return rc; }
    *out = b;
    return DNA_OK;
}

extern "C" int dna_batch_run(dna_batch *b, dna_stream_t stream_h, uint64_t *out_counts) {
    if (!b || !out_counts) return DNA_ERR_INVALID_ARG;
    int dev = -1;
    DNA_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return DNA_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_h;
    std::lock_guard<std::mutex> lk(b->mu);
    if (!b->use_graph) return enqueue_batch(*b, stream, out_counts);
    if (!b->graph || b->graph_out != out_counts) {
        // capture the batch once per output buffer; later runs replay the graph
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        cudaStream_t cs;
        DNA_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        int rc = e == cudaSuccess ? enqueue_batch(*b, cs, out_counts) : cuda_status(e);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (rc == DNA_OK && e2 != cudaSuccess) rc = cuda_status(e2);
        if (rc == DNA_OK) {
            e = cudaGraphInstantiate(&b->graph, g, 0);
            if (e != cudaSuccess) rc = cuda_status(e);
        }
        if (rc == DNA_OK) {
            // kernels per replay, for the launch counter
            size_t n = 0;
            b->graph_kernels = 0;
            if (cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess && n) {
                std::vector<cudaGraphNode_t> nodes(n);
                if (cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess)
                    for (auto nd : nodes) {
                        cudaGraphNodeType ty;
                        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                            ++b->graph_kernels;
                    }
            }
        }
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (rc) { b->graph = nullptr; return rc; }
        b->graph_out = out_counts;
    }
    DNA_CUDA(cudaGraphLaunch(b->graph, stream));
    record_launch(b->graph_kernels);
    return DNA_OK;
}

extern "C" int dna_batch_info(const dna_batch *b, dna_batch_info_t *out) {
    if (!b || !out) return DNA_ERR_INVALID_ARG;
    out->chunk_bases = b->chunk_tiles * (uint32_t)kBasesPerTile;
    out->warps_per_cta = b->warps;
    out->grid = (uint32_t)b->grid;
    out->groups_per_task = b->groups_per_task;
    out->n_fast = (uint32_t)b->fast.size();
    out->n_slow = (uint32_t)b->slow.size();
    out->n_chunks = b->n_chunks;
    out->packed_tiles = b->total_tiles;
    out->max_states = b->max_states;
    return DNA_OK;
}

extern "C" void dna_batch_free(dna_batch *b) { release(b); }

extern "C" int dna_scan_batch(const dna_dfa *const *dfas, uint32_t n_dfas, const uint8_t *const *seqs,
                              const uint64_t *lens, uint32_t n_seqs, dna_stream_t stream,
                              uint64_t *out_counts) {
    dna_batch *b = nullptr;
    int rc = dna_batch_create(dfas, n_dfas, seqs, lens, n_seqs, nullptr, stream, &b);
    if (rc) return rc;
    rc = dna_batch_run(b, stream, out_counts);
    // the plan's device memory is released once the queued work has finished
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    dna_batch_free(b);
    if (rc) return rc;
    return cuda_status(e);
}
