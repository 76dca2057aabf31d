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

namespace {

// ------------------------------------------------------------------ constants

constexpr int kTile = 128;          // bytes per chunk row staged per step
constexpr int kStages = 2;          // cp.async pipeline depth
constexpr int kStageBytes = 32 * kTile;
constexpr int kStashCap = 16;       // positions kept per chunk before a rescan
constexpr int kPairRowBytes = 16 * 32 * 4;  // 16 symbol pairs x 32 lanes x 4 bytes
constexpr uint32_t kMaxLookback = 64;
constexpr int kResolveThreads = 256;
constexpr uint32_t kMaxStates = 1u << 24;

enum Mode { MODE_PAIR = 0, MODE_ONE_SMEM = 1, MODE_ONE_GLOBAL = 2 };

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_profile{0};
std::mutex g_prof_mu;
struct ProfRec { cudaEvent_t a, b; };
std::vector<ProfRec> g_prof_pending;
double g_prof_ms = 0.0;
uint64_t g_prof_calls = 0;

// ----------------------------------------------------------- device helpers

// Byte -> code: code = (byte >> 1) & 3 gives A=0, C=1, T=2, G=3 for both cases; a byte
// is a base iff (byte | 0x20) equals the lowercase letter of its code.
__device__ __forceinline__ bool byte_is_base(uint32_t b) {
    uint32_t code = (b >> 1) & 3u;
    uint32_t expect = (0x67746361u >> (code << 3)) & 0xFFu;  // 'a','c','t','g'
    return (b | 0x20u) == expect;
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n"
                 :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" :: "n"(N) : "memory"); }

// One-symbol entry: next state in bits 0..30, bit 31 = next state accepts.
struct OneTable {
    const uint32_t *t;      // [n_states][4] in code order (A, C, T, G)
    uint32_t reset_entry;   // entry taken on a reset byte: state 0 (+ its accept bit)
    __device__ __forceinline__ uint32_t step(uint32_t q, uint32_t b) const {
        return byte_is_base(b) ? t[q * 4u + ((b >> 1) & 3u)] : reset_entry;
    }
};

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
    uint32_t *stash;        // [nseg][kStashCap] chunk-relative positions, or null
};

// Per-byte walk over bytes [k0, k1) of the lane's staged 128-byte row; 16-byte chunk c
// of the row is stored at slot c ^ (lane & 7).
template <bool kStash>
__device__ __forceinline__ uint32_t row_bytes_swz(const OneTable &T, uint32_t q, const uint8_t *srow,
                                                  int lane, int k0, int k1, uint32_t &cnt,
                                                  uint32_t row_rel, uint32_t *stash) {
    for (int k = k0; k < k1; ++k) {
        uint32_t byte = srow[(((k >> 4) ^ (lane & 7)) << 4) | (k & 15)];
        uint32_t e = T.step(q, byte);
        q = e & 0x7FFFFFFFu;
        if (e >> 31) {
            if (kStash && cnt < (uint32_t)kStashCap) stash[cnt] = row_rel + (uint32_t)k;
            ++cnt;
        }
    }
    return q;
}

template <int MODE, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
scan_kernel(ScanParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);

    // shared memory layout: [staging: WARPS*kStages*4 KB][one-symbol table][pad][pair table]
    uint8_t *stage_ptr = smem + (size_t)warp * kStages * kStageBytes;
    const uint32_t stage_addr = smem_base + (uint32_t)warp * kStages * kStageBytes;
    uint32_t *one_s = reinterpret_cast<uint32_t *>(smem + (size_t)WARPS * kStages * kStageBytes);
    OneTable T;
    T.reset_entry = p.reset_entry;
    uint32_t pair_base = 0;
    if (MODE == MODE_ONE_GLOBAL) {
        T.t = p.one;
    } else {
        const uint32_t n1 = p.n_states * 4u;
        for (uint32_t i = threadIdx.x; i < n1; i += WARPS * 32) one_s[i] = p.one[i];
        T.t = one_s;
        if (MODE == MODE_PAIR) {
            uint32_t after_one = smem_base + (uint32_t)WARPS * kStages * kStageBytes + n1 * 4u;
            pair_base = (after_one + 2047u) & ~2047u;   // bits 0..10 of the base are zero
            const uint32_t n2 = p.n_states * 16u * 32u;
            uint8_t *pair_ptr = smem + (pair_base - smem_base);
            for (uint32_t i = threadIdx.x; i < n2; i += WARPS * 32) {
                uint32_t q = i >> 9, pr = (i >> 5) & 15u, l = i & 31u;
                uint32_t e = p.pair[q * 16u + pr];
                uint32_t nx = e & 0x00FFFFFFu, c = e >> 24;
                reinterpret_cast<uint32_t *>(pair_ptr)[i] =
                    (c << 24) | (pair_base + nx * (uint32_t)kPairRowBytes + l * 4u);
                (void)q;
            }
        }
    }
    __syncthreads();

    const uint64_t seg0 = ((uint64_t)blockIdx.x * WARPS + warp) * 32u;
    if (seg0 >= p.nseg) return;   // whole warp idle (no block-wide sync follows)
    const uint64_t seg = seg0 + lane;
    const bool active = seg < p.nseg;
    const uint64_t S = p.seg_bytes;
    const uint64_t b = seg * S;   // aligned offset of this chunk
    const uint32_t ntiles = (uint32_t)(S / kTile);
    uint32_t *stash = p.stash ? p.stash + seg * kStashCap : nullptr;

    // ---- speculation: run from q0 over the lookback window in front of the chunk
    uint32_t q = 0;
    if (active && b > p.lo) {
        uint64_t from = b - p.lo > p.lookback ? b - p.lookback : p.lo;
        for (uint64_t off = from; off < b; ++off) q = T.step(q, p.abase[off]) & 0x7FFFFFFFu;
    }
    const uint32_t spec = q;
    uint32_t cnt = 0;
    uint32_t cur = pair_base + q * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u;

    // ---- staging pipeline prologue
    auto issue = [&](uint32_t t) {
        const uint32_t st = t % kStages;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int f = j * 32 + lane;
            int r = f >> 3, c = f & 7;
            uint64_t rseg = seg0 + r;
            uint64_t goff = rseg * S + (uint64_t)t * kTile + (uint64_t)c * 16u;
            bool ok = rseg < p.nseg && goff < p.hi;
            const uint8_t *src = ok ? p.abase + goff : p.abase;
            uint32_t dst = stage_addr + st * kStageBytes + r * kTile + ((c ^ (r & 7)) * 16);
            cp_async16(dst, src, ok ? 16u : 0u);
        }
    };
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if ((uint32_t)s < ntiles) issue(s);
        cp_async_commit();
    }

    for (uint32_t t = 0; t < ntiles; ++t) {
        __syncwarp();   // every lane is done with the stage the next issue overwrites
        if (t + kStages - 1 < ntiles) issue(t + kStages - 1);
        cp_async_commit();
        cp_async_wait<kStages - 1>();
        __syncwarp();   // tile t of all 32 rows is visible to the warp
        if (!active) continue;
        const uint64_t row_off = b + (uint64_t)t * kTile;
        if (row_off >= p.hi) continue;   // past the end of the sequence (last chunk)
        // the lane's row, un-swizzled: 16-byte chunk c sits at slot c ^ (lane & 7)
        const uint8_t *srow = stage_ptr + (t % kStages) * kStageBytes + lane * kTile;
        const uint32_t row_rel = (uint32_t)(t * kTile);
        const bool full = row_off >= p.lo && row_off + kTile <= p.hi;
        const int k0 = row_off < p.lo ? (int)(p.lo - row_off) : 0;
        const int k1 = row_off + kTile > p.hi ? (int)(p.hi - row_off) : kTile;

        if (MODE == MODE_PAIR) {
            bool done = false;
            if (full) {
                uint32_t w[32];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint4 v = *reinterpret_cast<const uint4 *>(srow + ((c ^ (lane & 7)) * 16));
                    w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
                }
                uint32_t acc = 0, err = 0, c2 = cur;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    uint32_t x = w[k] & 0x06060606u;
                    uint32_t y = x * 65u;
                    uint32_t e1 = lds_u32((c2 & 0x00FFFFFFu) | (y & 0x780u));
                    uint32_t e2 = lds_u32((e1 & 0x00FFFFFFu) | ((y >> 16) & 0x780u));
                    acc += e1 + e2;
                    c2 = e2;
                    // bit-exact base check: expected lowercase word from the codes
                    uint32_t z = x | (x >> 4);
                    uint32_t sel = __byte_perm(z, 0, 0x0020);
                    uint32_t expect = __byte_perm(0x00630061u, 0x00670074u, sel);
                    err |= expect ^ w[k];
                }
                if ((err & 0xDFDFDFDFu) == 0) {
                    uint32_t rc = acc >> 24;
                    if (stash && rc) {
                        uint32_t qs = ((cur & 0x00FFFFFFu) - pair_base) / (uint32_t)kPairRowBytes;
                        row_bytes_swz<true>(T, qs, srow, lane, 0, kTile, cnt, row_rel, stash);
                    } else {
                        cnt += rc;
                    }
                    cur = c2 & 0x00FFFFFFu;
                    done = true;
                }
            }
            if (!done) {
                uint32_t qs = ((cur & 0x00FFFFFFu) - pair_base) / (uint32_t)kPairRowBytes;
                if (stash) qs = row_bytes_swz<true>(T, qs, srow, lane, k0, k1, cnt, row_rel, stash);
                else qs = row_bytes_swz<false>(T, qs, srow, lane, k0, k1, cnt, row_rel, nullptr);
                cur = pair_base + qs * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u;
            }
        } else {
            if (stash) q = row_bytes_swz<true>(T, q, srow, lane, k0, k1, cnt, row_rel, stash);
            else q = row_bytes_swz<false>(T, q, srow, lane, k0, k1, cnt, row_rel, nullptr);
        }
    }
    cp_async_wait<0>();
    if (!active) return;
    uint32_t last = q;
    if (MODE == MODE_PAIR) last = ((cur & 0x00FFFFFFu) - pair_base) / (uint32_t)kPairRowBytes;
    p.spec_start[seg] = spec;
    p.last_state[seg] = last;
    p.count[seg] = cnt;
}

// ------------------------------------------------------------ resolve kernels

struct ResolveParams {
    const uint8_t *abase;
    uint64_t lo, hi, seg_bytes, nseg;
    const uint32_t *one;        // global one-symbol table
    uint32_t reset_entry;
    const uint32_t *spec_start, *last_state, *count;
    uint32_t *true_start, *true_last, *true_count;
    uint8_t *flags;             // bit0 corrected, bit1 never met, bit2 last state differs
    unsigned long long *block_sum;  // [nblocks]
    uint32_t *div_list;         // chunks whose true last state differs
    uint32_t *div_count;
    uint32_t div_cap;
};

__device__ __forceinline__ uint32_t one_step(const uint32_t *one, uint32_t reset_entry, uint32_t q,
                                             uint32_t b) {
    return byte_is_base(b) ? one[q * 4u + ((b >> 1) & 3u)] : reset_entry;
}

// Converging-point repair (Sec. III-B.3, Alg. 1): run the true start 'a' and the
// speculated start 's' in lockstep over chunk c until their states meet.
__device__ void repair_chunk(const ResolveParams &p, uint64_t c, uint32_t a, uint32_t s,
                             uint32_t spec_total, uint32_t spec_last,
                             uint32_t &out_count, uint32_t &out_last, uint8_t &out_flags) {
    uint64_t b = c * p.seg_bytes;
    uint64_t from = b > p.lo ? b : p.lo;
    uint64_t to = b + p.seg_bytes < p.hi ? b + p.seg_bytes : p.hi;
    uint32_t qa = a, qs = s, ca = 0, cs = 0;
    for (uint64_t off = from; off < to; ++off) {
        uint32_t byte = p.abase[off];
        uint32_t ea = one_step(p.one, p.reset_entry, qa, byte);
        uint32_t es = one_step(p.one, p.reset_entry, qs, byte);
        qa = ea & 0x7FFFFFFFu; qs = es & 0x7FFFFFFFu;
        ca += ea >> 31; cs += es >> 31;
        if (qa == qs) {   // converging point: the rest of the runs coincide
            out_count = ca + (spec_total - cs);
            out_last = spec_last;
            out_flags = 1;
            return;
        }
    }
    out_count = ca;
    out_last = qa;
    out_flags = (uint8_t)(1 | 2 | (qa != spec_last ? 4 : 0));
}

__global__ void __launch_bounds__(kResolveThreads) resolve_kernel(ResolveParams p) {
    __shared__ unsigned long long red[kResolveThreads / 32];
    const uint64_t c = (uint64_t)blockIdx.x * kResolveThreads + threadIdx.x;
    uint32_t tc = 0;
    if (c < p.nseg) {
        uint32_t a = c == 0 ? 0u : p.last_state[c - 1];
        uint32_t s = p.spec_start[c];
        uint32_t cnt = p.count[c], last = p.last_state[c];
        uint8_t fl = 0;
        if (a != s) {
            repair_chunk(p, c, a, s, cnt, last, cnt, last, fl);
            if (fl & 4) {
                uint32_t k = atomicAdd(p.div_count, 1u);
                if (k < p.div_cap) p.div_list[k] = (uint32_t)c;
            }
        }
        p.true_start[c] = a;
        p.true_last[c] = last;
        p.true_count[c] = cnt;
        p.flags[c] = fl;
        tc = cnt;
    }
    unsigned long long v = tc;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int i = 0; i < kResolveThreads / 32; ++i) s += red[i];
        p.block_sum[blockIdx.x] = s;
    }
}

// Sequential cascade over chunks whose true last state differs from the speculated
// one, then the exclusive scan of block sums and the total count. One block.
__global__ void __launch_bounds__(1024) finalize_kernel(ResolveParams p, uint64_t nblocks,
                                                        unsigned long long *block_off,
                                                        uint64_t *out_count) {
    __shared__ unsigned long long carry;
    __shared__ unsigned long long wsum[32];
    if (threadIdx.x == 0) {
        uint32_t nd = *p.div_count;
        if (nd > p.div_cap) {
            // list overflowed: walk every chunk sequentially from the start
            uint32_t prev_last = 0;
            for (uint64_t c = 0; c < p.nseg; ++c) {
                uint32_t a = c == 0 ? 0u : prev_last;
                if (a != p.true_start[c]) {
                    uint32_t cnt, last; uint8_t fl;
                    repair_chunk(p, c, a, p.spec_start[c], p.count[c], p.last_state[c], cnt, last, fl);
                    long long d = (long long)cnt - (long long)p.true_count[c];
                    p.block_sum[c / kResolveThreads] += (unsigned long long)d;
                    p.true_start[c] = a; p.true_count[c] = cnt; p.true_last[c] = last;
                    p.flags[c] = fl;
                }
                prev_last = p.true_last[c];
            }
        } else if (nd > 0) {
            // sort the (small) list, then walk forward from each entry until the chain agrees
            for (uint32_t i = 1; i < nd; ++i) {
                uint32_t v = p.div_list[i], j = i;
                while (j > 0 && p.div_list[j - 1] > v) { p.div_list[j] = p.div_list[j - 1]; --j; }
                p.div_list[j] = v;
            }
            uint64_t walked = 0;
            for (uint32_t i = 0; i < nd; ++i) {
                uint64_t c = p.div_list[i];
                if (c < walked) continue;
                uint32_t cur_last = p.true_last[c];
                uint64_t k = c + 1;
                while (k < p.nseg && cur_last != p.last_state[k - 1]) {
                    uint32_t cnt, last; uint8_t fl = 0;
                    uint32_t a = cur_last;
                    if (a == p.spec_start[k]) { cnt = p.count[k]; last = p.last_state[k]; }
                    else repair_chunk(p, k, a, p.spec_start[k], p.count[k], p.last_state[k], cnt, last, fl);
                    long long d = (long long)cnt - (long long)p.true_count[k];
                    p.block_sum[k / kResolveThreads] += (unsigned long long)d;
                    p.true_start[k] = a; p.true_count[k] = cnt; p.true_last[k] = last;
                    p.flags[k] = fl | 1;
                    cur_last = last;
                    ++k;
                }
                walked = k;
            }
        }
        carry = 0;
    }
    __syncthreads();
    // exclusive scan of block sums, 1024 at a time
    for (uint64_t base = 0; base < nblocks; base += 1024) {
        uint64_t i = base + threadIdx.x;
        unsigned long long v = i < nblocks ? p.block_sum[i] : 0ull;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long s = wsum[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
                if (threadIdx.x >= o) s += y;
            }
            wsum[threadIdx.x] = s;
        }
        __syncthreads();
        unsigned long long incl = x + ((threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0ull) + carry;
        if (i < nblocks) block_off[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_count = carry;
}

struct EmitParams {
    const uint8_t *abase;
    uint64_t lo, hi, seg_bytes, nseg;
    const uint32_t *one;
    uint32_t reset_entry;
    const uint32_t *true_start, *true_count, *stash;
    const uint8_t *flags;
    const unsigned long long *block_off;
    uint64_t *out;
    uint64_t cap;
};

__global__ void __launch_bounds__(kResolveThreads) emit_kernel(EmitParams p) {
    __shared__ unsigned long long wsum[kResolveThreads / 32];
    const uint64_t c = (uint64_t)blockIdx.x * kResolveThreads + threadIdx.x;
    unsigned long long v = c < p.nseg ? p.true_count[c] : 0u;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned long long before = 0;
    for (int i = 0; i < (int)(threadIdx.x >> 5); ++i) before += wsum[i];
    if (c >= p.nseg) return;
    unsigned long long off = p.block_off[blockIdx.x] + before + x - v;
    if (off >= p.cap || v == 0) return;
    const uint64_t b = c * p.seg_bytes;
    if (p.flags[c] == 0 && v <= (unsigned long long)kStashCap) {
        for (uint32_t k = 0; k < (uint32_t)v && off + k < p.cap; ++k)
            p.out[off + k] = b + p.stash[c * kStashCap + k] - p.lo;
        return;
    }
    // rescan from the true start
    uint64_t from = b > p.lo ? b : p.lo;
    uint64_t to = b + p.seg_bytes < p.hi ? b + p.seg_bytes : p.hi;
    uint32_t q = p.true_start[c];
    uint64_t k = 0;
    for (uint64_t o = from; o < to && off + k < p.cap; ++o) {
        uint32_t e = one_step(p.one, p.reset_entry, q, p.abase[o]);
        q = e & 0x7FFFFFFFu;
        if (e >> 31) { p.out[off + k] = o - p.lo; ++k; }
    }
}

__global__ void write_zero_kernel(uint64_t *out) { *out = 0; }

// ------------------------------------------------------------------ host side

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DNA_OK;
    if (e == cudaErrorMemoryAllocation) return DNA_ERR_NOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
        e == cudaErrorNoKernelImageForDevice)
        return DNA_ERR_NO_DEVICE;
    return DNA_ERR_CUDA;
}

#define DNA_CUDA(call)                                   \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_status(_e);   \
    } while (0)

struct DeviceProps {
    int sms = 0;
    size_t smem_optin = 0;
};

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

size_t scan_smem_bytes(int mode, int warps, uint32_t n_states) {
    size_t s = (size_t)warps * kStages * kStageBytes;
    if (mode == MODE_ONE_GLOBAL) return s;
    s += (size_t)n_states * 16;
    if (mode == MODE_PAIR) s += 2048 + (size_t)n_states * kPairRowBytes;
    return s;
}

using ScanFn = void (*)(ScanParams);

ScanFn scan_fn(int mode, int warps) {
#define PICK(M, W) if (mode == M && warps == W) return scan_kernel<M, W>;
    PICK(MODE_PAIR, 4) PICK(MODE_PAIR, 8) PICK(MODE_PAIR, 16)
    PICK(MODE_ONE_SMEM, 4) PICK(MODE_ONE_SMEM, 8) PICK(MODE_ONE_SMEM, 16)
    PICK(MODE_ONE_GLOBAL, 4) PICK(MODE_ONE_GLOBAL, 8) PICK(MODE_ONE_GLOBAL, 16)
#undef PICK
    return nullptr;
}

}  // namespace

struct dna_dfa {
    uint32_t n_states = 0;
    int device = 0;
    int definite_depth = -1;
    uint32_t lookback = 0;
    uint32_t placement = DNA_PLACE_AUTO;
    uint32_t accept0 = 0;
    uint32_t reset_entry = 0;
    uint32_t *d_one = nullptr;
    uint32_t *d_pair = nullptr;
};

namespace {

// code order (A, C, T, G) -> table column (A, C, G, T)
constexpr int kColOfCode[4] = {0, 1, 3, 2};

size_t max_pair_states(size_t smem_optin, int warps) {
    size_t fixed = (size_t)warps * kStages * kStageBytes + 2048;
    if (smem_optin <= fixed) return 0;
    return (smem_optin - fixed) / (kPairRowBytes + 16);
}

struct Plan {
    int mode, warps;
    uint64_t seg_bytes, nseg;
    uint32_t lookback;
    size_t smem;
    int grid;
};

int make_plan(const dna_dfa *d, uint64_t total, const dna_plan *ov, Plan &pl) {
    DeviceProps pr = device_props(d->device);
    const size_t optin = pr.smem_optin ? pr.smem_optin : 232448;
    int mode;
    uint32_t req = ov ? ov->placement : 0;
    int warps = ov && ov->warps_per_cta ? (int)ov->warps_per_cta : 0;
    if (warps && warps != 4 && warps != 8 && warps != 16) return DNA_ERR_INVALID_ARG;
    if (req == DNA_PLACE_AUTO) req = d->placement;
    if (req == DNA_PLACE_SMEM_PAIR) mode = MODE_PAIR;
    else if (req == DNA_PLACE_SMEM_ONE) mode = MODE_ONE_SMEM;
    else if (req == DNA_PLACE_GLOBAL_ONE) mode = MODE_ONE_GLOBAL;
    else return DNA_ERR_INVALID_ARG;
    if (!warps) {
        warps = 4;
        for (int w : {16, 8}) if (scan_smem_bytes(mode, w, d->n_states) <= optin) { warps = w; break; }
    }
    size_t smem = scan_smem_bytes(mode, warps, d->n_states);
    if (smem > optin) return DNA_ERR_CAPACITY;
    uint32_t lb = ov && ov->lookback ? ov->lookback : d->lookback;
    if (lb > kMaxLookback) return DNA_ERR_INVALID_ARG;
    ScanFn fn = scan_fn(mode, warps);
    if (!fn) return DNA_ERR_INVALID_ARG;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
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
    pl.mode = mode; pl.warps = warps; pl.seg_bytes = S;
    pl.nseg = (total + S - 1) / S;
    pl.lookback = lb; pl.smem = smem;
    uint64_t lanes_per_cta = (uint64_t)warps * 32;
    pl.grid = (int)((pl.nseg + lanes_per_cta - 1) / lanes_per_cta);
    return DNA_OK;
}

// device scratch carved from one stream-ordered allocation
struct Scratch {
    uint32_t *spec_start, *last_state, *count, *true_start, *true_last, *true_count, *stash;
    uint32_t *div_list, *div_count;
    uint8_t *flags;
    unsigned long long *block_sum, *block_off;
    void *base;
    size_t bytes;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void carve(Scratch &s, uint64_t nseg, uint64_t nblocks, bool positions, uint32_t div_cap, uint8_t *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) { uint8_t *p = base ? base + off : nullptr; off = align_up(off + bytes, 256); return p; };
    s.block_sum = (unsigned long long *)take(nblocks * 8);
    s.block_off = (unsigned long long *)take(nblocks * 8);
    s.spec_start = (uint32_t *)take(nseg * 4);
    s.last_state = (uint32_t *)take(nseg * 4);
    s.count = (uint32_t *)take(nseg * 4);
    s.true_start = (uint32_t *)take(nseg * 4);
    s.true_last = (uint32_t *)take(nseg * 4);
    s.true_count = (uint32_t *)take(nseg * 4);
    s.div_count = (uint32_t *)take(4);
    s.div_list = (uint32_t *)take((size_t)div_cap * 4);
    s.flags = (uint8_t *)take(nseg);
    s.stash = positions ? (uint32_t *)take(nseg * kStashCap * 4) : nullptr;
    s.bytes = off;
    s.base = base;
}

void record_launch(int n = 1) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

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
    Plan pl;
    int rc = make_plan(d, total, ov, pl);
    if (rc) return rc;
    const bool positions = out_positions != nullptr && cap > 0;
    const uint64_t nblocks = (pl.nseg + kResolveThreads - 1) / kResolveThreads;
    const uint32_t div_cap = 4096;
    Scratch s;
    carve(s, pl.nseg, nblocks, positions, div_cap, nullptr);
    void *mem = nullptr;
    DNA_CUDA(cudaMallocAsync(&mem, s.bytes, stream));
    carve(s, pl.nseg, nblocks, positions, div_cap, (uint8_t *)mem);
    cudaError_t e = cudaMemsetAsync(s.div_count, 0, 4, stream);

    ScanParams sp;
    sp.abase = abase; sp.lo = shift; sp.hi = total; sp.seg_bytes = pl.seg_bytes; sp.nseg = pl.nseg;
    sp.lookback = pl.lookback; sp.n_states = d->n_states; sp.reset_entry = d->reset_entry;
    sp.one = d->d_one; sp.pair = d->d_pair;
    sp.spec_start = s.spec_start; sp.last_state = s.last_state; sp.count = s.count;
    sp.stash = s.stash;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool prof = g_profile.load(std::memory_order_relaxed) != 0;
    if (prof && e == cudaSuccess) {
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
        cudaEventRecord(ev0, stream);
    }
    if (e == cudaSuccess) {
        scan_fn(pl.mode, pl.warps)<<<pl.grid, pl.warps * 32, pl.smem, stream>>>(sp);
        e = cudaGetLastError();
        record_launch();
    }
    if (prof && ev1) {
        cudaEventRecord(ev1, stream);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_pending.push_back({ev0, ev1});
    }
    ResolveParams rp;
    rp.abase = abase; rp.lo = shift; rp.hi = total; rp.seg_bytes = pl.seg_bytes; rp.nseg = pl.nseg;
    rp.one = d->d_one; rp.reset_entry = d->reset_entry;
    rp.spec_start = s.spec_start; rp.last_state = s.last_state; rp.count = s.count;
    rp.true_start = s.true_start; rp.true_last = s.true_last; rp.true_count = s.true_count;
    rp.flags = s.flags; rp.block_sum = s.block_sum;
    rp.div_list = s.div_list; rp.div_count = s.div_count; rp.div_cap = div_cap;
    if (e == cudaSuccess) {
        resolve_kernel<<<(unsigned)nblocks, kResolveThreads, 0, stream>>>(rp);
        e = cudaGetLastError();
        record_launch();
    }
    if (e == cudaSuccess) {
        finalize_kernel<<<1, 1024, 0, stream>>>(rp, nblocks, s.block_off, out_count);
        e = cudaGetLastError();
        record_launch();
    }
    if (e == cudaSuccess && positions) {
        EmitParams ep;
        ep.abase = abase; ep.lo = shift; ep.hi = total; ep.seg_bytes = pl.seg_bytes; ep.nseg = pl.nseg;
        ep.one = d->d_one; ep.reset_entry = d->reset_entry;
        ep.true_start = s.true_start; ep.true_count = s.true_count; ep.stash = s.stash;
        ep.flags = s.flags; ep.block_off = s.block_off; ep.out = out_positions; ep.cap = cap;
        emit_kernel<<<(unsigned)nblocks, kResolveThreads, 0, stream>>>(ep);
        e = cudaGetLastError();
        record_launch();
    }
    cudaError_t e2 = cudaFreeAsync(mem, stream);
    if (e == cudaSuccess) e = e2;
    return cuda_status(e);
}

}  // namespace

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
    if (d->definite_depth >= 0) d->lookback = (uint32_t)d->definite_depth;
    else d->lookback = 32;
    DeviceProps pr = device_props(dev);
    size_t optin = pr.smem_optin ? pr.smem_optin : 232448;
    if (n_states <= max_pair_states(optin, 4)) d->placement = DNA_PLACE_SMEM_PAIR;
    else if (scan_smem_bytes(MODE_ONE_SMEM, 4, n_states) <= optin) d->placement = DNA_PLACE_SMEM_ONE;
    else d->placement = DNA_PLACE_GLOBAL_ONE;
    cudaError_t e = cudaMalloc(&d->d_one, sizeof(uint32_t) * one.size());
    if (e == cudaSuccess) e = cudaMemcpy(d->d_one, one.data(), sizeof(uint32_t) * one.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_states <= max_pair_states(optin, 4)) {
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

extern "C" int dna_scan_planned(const dna_dfa *dfa, const uint8_t *seq, uint64_t len,
                                dna_stream_t stream, uint64_t *out_count, uint64_t *out_positions,
                                uint64_t positions_capacity, const dna_plan *plan) {
    return scan_impl(dfa, seq, len, (cudaStream_t)stream, out_count, out_positions,
                     positions_capacity, plan);
}

extern "C" int dna_scan_batch(const dna_dfa *const *dfas, uint32_t n_dfas, const uint8_t *const *seqs,
                              const uint64_t *lens, uint32_t n_seqs, dna_stream_t stream,
                              uint64_t *out_counts) {
    if (!dfas || !seqs || !lens || !out_counts || n_dfas == 0 || n_seqs == 0) return DNA_ERR_INVALID_ARG;
    for (uint32_t s = 0; s < n_seqs; ++s)
        for (uint32_t k = 0; k < n_dfas; ++k) {
            int rc = scan_impl(dfas[k], seqs[s], lens[s], (cudaStream_t)stream,
                               out_counts + (uint64_t)s * n_dfas + k, nullptr, 0, nullptr);
            if (rc) return rc;
        }
    return DNA_OK;
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

extern "C" void dna_profile_enable(int enable) { g_profile.store(enable ? 1 : 0); }

extern "C" int dna_profile_read(dna_profile_t *out, int reset) {
    if (!out) return DNA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof_pending) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_prof_ms += ms;
            ++g_prof_calls;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof_pending.clear();
    out->scan_kernel_ms = g_prof_ms;
    out->scan_kernel_calls = g_prof_calls;
    out->kernel_launches = g_launches.load();
    if (reset) {
        g_prof_ms = 0;
        g_prof_calls = 0;
        g_launches.store(0);
    }
    return DNA_OK;
}
