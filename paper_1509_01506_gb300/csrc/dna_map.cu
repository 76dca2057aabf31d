// dna_map.cu -- the chunk-map path for automata whose runs do not converge.
//
// Speculation with repair (dna_scan.cu) relies on the runs from different start states
// meeting soon (the converging point of Sec. III-B.3). Some automata never synchronise
// on DNA (permutation-like tables, counters): there every chunk's repair walks the whole
// chunk and every join cascades, serially. For those the scan follows the paper's
// possible-starting-state approach in full (Sec. III-A): a chunk is run from every state
// at once. Automata of at most 16 states keep all runs of a lane in one or two registers
// (map_nib_kernel below: a lane walks one of the chunk's 32 parts). Larger ones: a warp
// runs one chunk from 32 start states (lane q from state 32w + q for the warp's state
// block w); automata of more than 32 states give each chunk ceil(Q / 32) warps, and
// automata of at most 32 states cut the chunk into 2 parts walked side by side (two
// chains per lane), whose maps the warp composes. Each chunk yields a map (end
// state and count per start state) and, for the positions pass, the state at each of its
// 32 sub-chunk boundaries per start state. A single-block join composes the maps in order
// (chunk c starts in the end state of chunk c-1 from its true start), which gives the
// total count and every sub-chunk's exact start state. The positions come from the
// single-sequence kernels run with those exact starts.
//
// Lookups never conflict in shared memory. The register-field kernels read 8-byte rows
// of 128-byte tables (one row per symbol pair); the others give every lane its own copy
// of the table in its own bank: the two-symbol table up to about 90 states (2 KiB per
// state), a one-symbol table (512 B per state) up to kMaxMapStates.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../include/dna_dfa.h"
#include "dna_device.cuh"
#include "dna_runtime.h"

using namespace dnalib;

namespace {

constexpr int kMapWarps = 24;
constexpr int kMapTile = 512;          // bytes staged per warp per step (4 rows of 128)
constexpr uint32_t kMapSubs = 32;      // sub-chunks per chunk (one per lane in the positions pass)
constexpr int kJoinWarps = 16;
constexpr uint32_t kOneRowBytes = 4 * 32 * 4;   // replicated one-symbol row: 4 codes x 32 lanes
// replicated one-symbol entry: shared address of the next state's row for this lane
// (bits 2..6 lane, bits 9..17 row; bits 7..8 take the next code) | next state accepts (bit 0)
constexpr uint32_t kOneAddrMask = 0x3FE7Cu;

enum MapTab { TAB_PAIR = 0, TAB_ONE = 1 };

struct MapParams {
    const uint8_t *abase;       // 16-byte aligned base; sequence byte j is abase[lo + j]
    uint64_t lo, hi;
    uint64_t chunk_bytes;       // multiple of kMapSubs * kTile
    uint32_t n_chunks;
    uint32_t n_states;          // <= 32 / G for a kernel with G parts per chunk
    uint32_t wblocks;           // warps (blocks of 32 start states) per chunk
    uint32_t qp;                // row width of the map arrays: 32 * wblocks
    uint32_t reset_entry;
    const uint32_t *one;        // [n_states][4] next | accept << 31, code order A, C, T, G
    const uint32_t *pair;       // [n_states][16] compact pair entries next | count << 24 (TAB_PAIR)
    uint32_t *map_end;          // [n_chunks][qp] end state per start state
    uint32_t *map_cnt;          // [n_chunks][qp] accepting steps per start state
    uint32_t *bound;            // [n_chunks][32 sub-chunks][qp]: state at each sub-chunk start,
                                //   per state at the start of the part holding that sub-chunk
                                //   (null for a count-only scan)
    uint32_t *gstart;           // [n_chunks][G][32]: state at the start of part g per chunk start
                                //   state (G > 1; null for a count-only scan)
    uint32_t *cpre;             // map_nib_kernel, positions pass: [n_chunks][16] state at each
                                //   chunk's start per start state of its block (else null)
    uint32_t k1, k5, lut_lo, lut_hi;
};

// One warp per (chunk, block of 32 start states). Lanes form G groups of 32 / G; the
// chunk is cut into G x C equal parts and lane (g, q) runs parts g, g + G, ..., (C of
// them, side by side as independent chains) from state 32w + q (lanes at or past
// n_states run from state 0 and are ignored), so that small automata keep every lane
// busy and each lane has C lookups in flight. Each part's bytes are staged TILE at a
// time; lane k decodes word k of every part's row for the warp. At the end the warp
// composes the parts' maps, in order, into the chunk's map.
template <int G, int TAB, int C>
__global__ void __launch_bounds__(kMapWarps * 32, 1) map_kernel(MapParams p) {
    static_assert(TAB == TAB_PAIR || G * C == 1, "parts only with the two-symbol table");
    constexpr uint32_t kParts = (uint32_t)(G * C);
    constexpr uint32_t kLanes = 32u / G;               // lanes (start states) per group
    // bytes of a part per stage: 512 for one chain, else 2 KiB shared by the parts
    constexpr uint32_t TILE = C == 1 ? (uint32_t)kMapTile : 2048u / kParts;
    constexpr uint32_t kRows = TILE / kTile;           // 128-byte rows per part per stage
    constexpr uint32_t kWarpStage = 2u * kParts * TILE;   // double-buffered tile of every part
    static_assert(kRows >= 1 && (kParts * TILE) % 512 == 0, "tile shape");
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t g = (uint32_t)lane / kLanes, q = (uint32_t)lane % kLanes;
    const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);
    // shared memory: [stages: warps x 2 x parts x TILE][one-symbol table: Q x 16 B][pad]
    //                [replicated table: two-symbol 2 KiB or one-symbol 512 B per state]
    uint8_t *stage = smem + (size_t)warp * kWarpStage;
    const uint32_t stage_addr = smem_base + (uint32_t)warp * kWarpStage;
    uint32_t *one_s = reinterpret_cast<uint32_t *>(smem + (size_t)kMapWarps * kWarpStage);
    const uint32_t tab_base = (smem_base + kMapWarps * kWarpStage + p.n_states * 16u + 2047u) & ~2047u;
    uint32_t *tab_s = reinterpret_cast<uint32_t *>(smem + (tab_base - smem_base));
    for (uint32_t i = threadIdx.x; i < p.n_states * 4u; i += kMapWarps * 32) one_s[i] = p.one[i];
    if (TAB == TAB_PAIR) {
        for (uint32_t i = threadIdx.x; i < p.n_states * 16u * 32u; i += kMapWarps * 32) {
            const uint32_t e = p.pair[i >> 5];
            tab_s[i] = ((e >> 24) << kCountShift) |
                       (tab_base + (e & 0x00FFFFFFu) * (uint32_t)kPairRowBytes + (i & 31u) * 4u);
        }
    } else {
        // row of state s: [code][lane]; entry = next row's address for the lane | accept bit
        for (uint32_t i = threadIdx.x; i < p.n_states * 128u; i += kMapWarps * 32) {
            const uint32_t e = p.one[i >> 5];
            tab_s[i] = (tab_base + (e & 0x7FFFFFFFu) * kOneRowBytes + (i & 31u) * 4u) | (e >> 31);
        }
    }
    __syncthreads();
    const uint32_t task = blockIdx.x * kMapWarps + warp;
    const uint32_t c = task / p.wblocks, wb = task - c * p.wblocks;
    if (c >= p.n_chunks) return;   // warp-uniform; no barrier follows
    // decoded codes of the current row of every part (rows 36 words apart, so that parts
    // read by the same instruction sit in different banks)
    __shared__ __align__(16) uint32_t ys_all[kMapWarps][kParts][36];

    OneTable T;
    T.t = one_s;
    T.reset_entry = p.reset_entry;
    const uint64_t b = (uint64_t)c * p.chunk_bytes;
    const uint64_t part = p.chunk_bytes / kParts;      // multiple of TILE
    const uint64_t sub = p.chunk_bytes / kMapSubs;
    const uint32_t ntiles = (uint32_t)(part / TILE);   // the same for every part and warp
    const uint32_t sq = wb * 32u + q;                  // this lane's start state
    const uint32_t q0 = sq < p.n_states ? sq : 0u;
    auto cur_of = [&](uint32_t st) {
        return TAB == TAB_PAIR ? tab_base + st * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u
                               : tab_base + st * kOneRowBytes + (uint32_t)lane * 4u;
    };
    auto state_of = [&](uint32_t cv) {
        return TAB == TAB_PAIR ? ((cv & 0x3FFFFu) - tab_base) / (uint32_t)kPairRowBytes
                               : ((cv & 0x3FE00u) - tab_base) / kOneRowBytes;
    };
    // chain h of this lane: part g + G h, bytes [from[h], to[h])
    uint64_t pb[C], from[C], to[C];
    uint32_t cur[C], cnt[C];
#pragma unroll
    for (int h = 0; h < C; ++h) {
        pb[h] = b + (uint64_t)(g + (uint32_t)G * h) * part;
        from[h] = pb[h] > p.lo ? pb[h] : p.lo;
        const uint64_t pe = pb[h] + part < p.hi ? pb[h] + part : p.hi;
        to[h] = pe > from[h] ? pe : from[h];           // empty past the sequence end
        cur[h] = cur_of(q0);
        cnt[h] = 0;
    }
    // lane copies 16-byte pieces of tile t of every part (past hi: zero-filled)
    auto issue = [&](uint32_t t) {
        constexpr uint32_t kPieces = kParts * TILE / 16u / 32u;   // per lane
#pragma unroll
        for (uint32_t j = 0; j < kPieces; ++j) {
            const uint32_t idx = j * 32u + (uint32_t)lane;
            const uint32_t pp = idx / (TILE / 16u), o = (idx % (TILE / 16u)) * 16u;
            const uint64_t off = b + (uint64_t)pp * part + (uint64_t)t * TILE + o;
            const bool ok = off < p.hi;
            cp_async16(stage_addr + ((t & 1u) * kParts + pp) * TILE + o, ok ? p.abase + off : p.abase, ok ? 16u : 0u);
        }
    };
    // the pair walk of one 128-byte row (words from the decoded row 'ys') from 'cv'
    auto pair_row = [&](const uint32_t *ys, uint32_t &cv, uint32_t &cn) {
        uint32_t acc = 0, rc = 0, c2 = cv;
#pragma unroll
        for (int k4 = 0; k4 < 8; ++k4) {
            const uint4 y4 = *reinterpret_cast<const uint4 *>(ys + 4 * k4);
            const uint32_t yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * k4 + i;
                const uint32_t e1 = lds_u32(mux_pair(c2, yv[i]));
                const uint32_t e2 = lds_u32(mux_pair(e1, yv[i] >> 16));
                acc = mad_lo(e1, p.k1, acc);
                acc = mad_lo(e2, p.k1, acc);
                c2 = e2;
                if (k % 3 == 2 || k == 31) {
                    rc = mad_hi(acc, p.k5, rc);
                    acc = 0;
                }
            }
        }
        cn += rc;
        cv = c2 & 0x3FFFFu;
    };
    issue(0);
    cp_async_commit();
    for (uint32_t t = 0; t < ntiles; ++t) {
        if (t + 1 < ntiles) issue(t + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        const uint8_t *tiles = stage + (t & 1u) * kParts * TILE;
#pragma unroll 1
        for (uint32_t r = 0; r < kRows; ++r) {
            uint64_t ro[C];
#pragma unroll
            for (int h = 0; h < C; ++h) {
                ro[h] = pb[h] + (uint64_t)t * TILE + (uint64_t)r * kTile;
                if (p.bound && ro[h] < to[h] && (ro[h] - b) % sub == 0)   // a sub-chunk starts here
                    p.bound[((uint64_t)c * kMapSubs + (ro[h] - b) / sub) * p.qp + sq] = state_of(cur[h]);
            }
            // lane k decodes word k of each part's row for the warp: its codes (y, read
            // back by the part's lanes) and the base check (voted per part)
            uint32_t bad_parts = 0;
#pragma unroll
            for (uint32_t pp = 0; pp < kParts; ++pp) {
                const uint32_t wk = *reinterpret_cast<const uint32_t *>(tiles + pp * TILE + r * kTile + 4 * lane);
                const uint32_t xk = wk & 0x06060606u;
                // two-symbol table: pairs at bits 7..10 and 23..26; one-symbol: raw codes
                ys_all[warp][pp][lane] = TAB == TAB_PAIR ? mad_lo(xk, 65u, 0u) : xk;
                const uint32_t zk = xk | (xk >> 4);
                const bool bad = ((__byte_perm(p.lut_lo, p.lut_hi, __byte_perm(zk, 0, 0x0020)) ^ wk) & 0xDFDFDFDFu) != 0;
                bad_parts |= (__any_sync(0xFFFFFFFFu, bad) ? 1u : 0u) << pp;
            }
            __syncwarp();
            bool fast[C];
#pragma unroll
            for (int h = 0; h < C; ++h)
                fast[h] = ro[h] >= from[h] && ro[h] + kTile <= to[h] && !((bad_parts >> (g + G * h)) & 1u);
            if (TAB == TAB_PAIR && C == 2 && fast[0] && fast[C - 1]) {
                // both chains side by side: their lookups overlap
                const uint32_t *ya = ys_all[warp][g], *yb = ys_all[warp][g + (C - 1) * G];
                uint32_t acc0 = 0, acc1 = 0, rc0 = 0, rc1 = 0, a2 = cur[0], b2 = cur[C - 1];
#pragma unroll
                for (int k4 = 0; k4 < 8; ++k4) {
                    const uint4 y4 = *reinterpret_cast<const uint4 *>(ya + 4 * k4);
                    const uint4 z4 = *reinterpret_cast<const uint4 *>(yb + 4 * k4);
                    const uint32_t yv[4] = {y4.x, y4.y, y4.z, y4.w}, zv[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k = 4 * k4 + i;
                        const uint32_t e1 = lds_u32(mux_pair(a2, yv[i]));
                        const uint32_t f1 = lds_u32(mux_pair(b2, zv[i]));
                        const uint32_t e2 = lds_u32(mux_pair(e1, yv[i] >> 16));
                        const uint32_t f2 = lds_u32(mux_pair(f1, zv[i] >> 16));
                        acc0 = mad_lo(e1, p.k1, acc0);
                        acc1 = mad_lo(f1, p.k1, acc1);
                        acc0 = mad_lo(e2, p.k1, acc0);
                        acc1 = mad_lo(f2, p.k1, acc1);
                        a2 = e2;
                        b2 = f2;
                        if (k % 3 == 2 || k == 31) {
                            rc0 = mad_hi(acc0, p.k5, rc0);
                            rc1 = mad_hi(acc1, p.k5, rc1);
                            acc0 = 0;
                            acc1 = 0;
                        }
                    }
                }
                cnt[0] += rc0;
                cnt[C - 1] += rc1;
                cur[0] = a2 & 0x3FFFFu;
                cur[C - 1] = b2 & 0x3FFFFu;
            } else {
#pragma unroll
                for (int h = 0; h < C; ++h) {
                    const uint32_t ph = g + (uint32_t)G * h;
                    if (fast[h]) {
                        if (TAB == TAB_PAIR) {
                            pair_row(ys_all[warp][ph], cur[h], cnt[h]);
                        } else {
                            // byte j's code sits at bits 8j+1..8j+2 of y; the lookup puts it
                            // at bits 7..8 of the row address
                            const uint32_t *ys = ys_all[warp][ph];
                            uint32_t rc = 0, e = cur[h];
#pragma unroll
                            for (int k4 = 0; k4 < 8; ++k4) {
                                const uint4 y4 = *reinterpret_cast<const uint4 *>(ys + 4 * k4);
                                const uint32_t yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    const uint32_t y = yv[i];
                                    e = lds_u32((e & kOneAddrMask) | ((y << 6) & 0x180u)); rc += e & 1u;
                                    e = lds_u32((e & kOneAddrMask) | ((y >> 2) & 0x180u)); rc += e & 1u;
                                    e = lds_u32((e & kOneAddrMask) | ((y >> 10) & 0x180u)); rc += e & 1u;
                                    e = lds_u32((e & kOneAddrMask) | ((y >> 18) & 0x180u)); rc += e & 1u;
                                }
                            }
                            cnt[h] += rc;
                            cur[h] = e & ~1u;
                        }
                    } else if (ro[h] + kTile > from[h] && ro[h] < to[h]) {
                        // reset bytes or a sequence edge in this row: byte by byte
                        const uint8_t *row = tiles + ph * TILE + r * kTile;
                        uint32_t qs = state_of(cur[h]);
                        const uint32_t k0 = ro[h] < from[h] ? (uint32_t)(from[h] - ro[h]) : 0u;
                        const uint32_t k1 = ro[h] + kTile > to[h] ? (uint32_t)(to[h] - ro[h]) : (uint32_t)kTile;
                        for (uint32_t k = k0; k < k1; ++k) {
                            const uint32_t e = T.step(qs, row[k]);
                            qs = e & 0x7FFFFFFFu;
                            cnt[h] += e >> 31;
                        }
                        cur[h] = cur_of(qs);
                    }
                }
            }
            __syncwarp();   // ys is rewritten by the next row
        }
        __syncwarp();   // every lane is done with this stage before it is refilled
    }
    cp_async_wait<0>();
    // compose the parts in order: from chunk start state s, part pp starts where part
    // pp - 1 ended; part pp is chain pp / G of group pp % G
    uint32_t end[C];
#pragma unroll
    for (int h = 0; h < C; ++h) end[h] = state_of(cur[h]);
    if (kParts == 1) {
        p.map_end[(uint64_t)c * p.qp + sq] = end[0];
        p.map_cnt[(uint64_t)c * p.qp + sq] = cnt[0];
        return;
    }
    uint32_t st = q0, total = 0;
#pragma unroll
    for (uint32_t pp = 0; pp < kParts; ++pp) {
        if (p.gstart && pp > 0 && g == 0) p.gstart[((uint64_t)c * kParts + pp) * 32u + q] = st;
        const uint32_t hsel = pp / G;
        uint32_t cv = cnt[0], ev = end[0];
#pragma unroll
        for (int h = 1; h < C; ++h)
            if (hsel == (uint32_t)h) { cv = cnt[h]; ev = end[h]; }
        const int src = (int)((pp % G) * kLanes + st);
        total += __shfl_sync(0xFFFFFFFFu, cv, src);
        st = __shfl_sync(0xFFFFFFFFu, ev, src);
    }
    if (g == 0) {
        p.map_end[(uint64_t)c * 32u + q] = st;
        p.map_cnt[(uint64_t)c * 32u + q] = total;
    }
}

// ---- Automata of at most 16 states: the runs from all start states in one or two words.
//
// A lane walks one part of the chunk (a warp's 32 lanes walk its 32 parts, which are also
// the positions pass's sub-chunks) and follows every start state at once: the state of
// the run from each start sits in a 4-bit field, 8 runs to a register (W registers for
// up to 8 W states). A two-symbol step looks up the pair's rows (the state two symbols
// after state j, and the accepting steps on the way, as bytes; 8-byte rows, each kind a
// 128-byte table of the 16 pairs, so the lanes' lookups never conflict in shared memory)
// and moves every run through them with byte permutes: permute(row, fields 0..3) gives
// the new states of fields 0..3 as bytes, and permute(row, fields 4..7) those of fields
// 4..7, packed back as (fields 0..3 bytes) + (fields 4..7 bytes) x 16; the same permutes
// of the count rows give each run's accepting steps. A permute selects one of 8 bytes by
// the low 3 bits of a field and copies the byte's sign instead when the field's bit 3 is
// set, so for 16 states (W = 2) each permute is taken from the rows of states 0..7 and of
// states 8..15 with bit 3 cleared, and a permute of 0x80 bytes by the fields themselves
// (0xFF where bit 3 is set, 0x80 where not) chooses between them bit by bit.
// The packing moves the run in field i to field rotl3(i) (i = 0..3 go to 0, 2, 4, 6 and
// i = 4..7 to 1, 3, 5, 7), a permutation of period 3, so a row starts with field i holding
// the run from start 8r + i and the step number mod 3 tells where each run is; the count
// bytes are kept per step number mod 3 and sorted back to runs at the end of the row.
// At the end the lanes of a warp walk the 32 part maps in order (the chunk map, and every
// part's start per chunk start state: the positions pass's sub-chunk starts), and the
// first warp walks the block's chunk maps the same way, so the join sees one map per
// block.
constexpr int kNibWarps = 24;
constexpr uint32_t kStageBytesNib = 32u * kTile;   // one 128-byte row of each of 32 parts
constexpr uint32_t kNibMaxStates = 16;
constexpr uint32_t kNibRow = 2u + kNibMaxStates + 1u;   // composition row: 2 end words, 16 counts, pad
constexpr uint32_t kNibTotRow = kNibMaxStates + 1u;     // a lane's per-start totals (padded)
// dynamic shared memory: the warps' stages, then every lane's per-start totals
constexpr size_t kNibSmem = (size_t)kNibWarps * kStageBytesNib + (size_t)kNibWarps * 32 * kNibTotRow * 4;

// byte permute (prmt default mode)
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// bitwise m ? b : a, one lop3: with inputs (b, a, m) the table of (b & m) | (a & ~m) is
// (0xF0 & 0xAA) | (0xCC & 0x55) = 0xE4
__device__ __forceinline__ uint32_t lop3_sel(uint32_t a, uint32_t b, uint32_t m) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(b), "r"(a), "r"(m));
    return d;
}

__device__ __forceinline__ uint2 lds_v2(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

// The rows of one step: states and counts for states 0..7 (and 8..15 when W = 2).
template <int W>
struct NibRows {
    uint2 s[W], c[W];
};

template <int W>
__global__ void __launch_bounds__(kNibWarps * 32, 1) map_nib_kernel(MapParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    // pair rows, pair index = code1 + 4 x code2: [W halves][16 pairs] of 8 bytes, states
    // and counts; one-symbol rows, index code (4: a reset byte)
    __shared__ __align__(128) uint2 tab2s[W][16], tab2c[W][16];
    __shared__ __align__(16) uint2 tab1s[5][W], tab1c[5][W];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t Q = p.n_states;
    // byte j of half h: next state of state 8h + j; fields past n_states stay put
    if (threadIdx.x < 21u * W) {
        const uint32_t i = threadIdx.x % 21u, h = threadIdx.x / 21u;
        uint32_t st[2] = {0, 0}, ct[2] = {0, 0};
        for (uint32_t j = 0; j < 8; ++j) {
            const uint32_t q = 8u * h + j;
            uint32_t v = q, a = 0;
            if (q < Q) {
                if (i < 16) {
                    const uint32_t e1 = p.one[q * 4u + (i & 3u)];
                    const uint32_t e2 = p.one[(e1 & 0x7FFFFFFFu) * 4u + (i >> 2)];
                    v = e2 & 0x7FFFFFFFu;
                    a = (e1 >> 31) + (e2 >> 31);
                } else if (i < 20) {
                    const uint32_t e1 = p.one[q * 4u + (i - 16u)];
                    v = e1 & 0x7FFFFFFFu;
                    a = e1 >> 31;
                } else {
                    v = 0;                       // a reset: q0, counted when q0 accepts
                    a = p.reset_entry >> 31;
                }
            }
            st[j >> 2] |= v << (8 * (j & 3u));
            ct[j >> 2] |= a << (8 * (j & 3u));
        }
        if (i < 16) {
            tab2s[h][i] = make_uint2(st[0], st[1]);
            tab2c[h][i] = make_uint2(ct[0], ct[1]);
        } else {
            tab1s[i - 16][h] = make_uint2(st[0], st[1]);
            tab1c[i - 16][h] = make_uint2(ct[0], ct[1]);
        }
    }
    __syncthreads();
    // warps past the last chunk walk nothing (identity maps) and join the block's
    // composition below
    const uint32_t c = blockIdx.x * kNibWarps + warp;
    const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);
    uint8_t *stage_ptr = smem + (size_t)warp * kStageBytesNib;
    const uint32_t stage_addr = smem_base + (uint32_t)warp * kStageBytesNib;
    const uint32_t tab2s_addr = (uint32_t)__cvta_generic_to_shared(&tab2s[0][0]);
    const uint32_t tab2c_addr = (uint32_t)__cvta_generic_to_shared(&tab2c[0][0]);
    const uint64_t b = (uint64_t)c * p.chunk_bytes;
    const uint64_t part = p.chunk_bytes / 32u;          // multiple of kTile
    const uint64_t pb = b + (uint64_t)lane * part;
    const uint64_t from = pb > p.lo ? pb : p.lo;
    const uint64_t pe = pb + part < p.hi ? pb + part : p.hi;
    const uint64_t to = pe > from ? pe : from;           // empty past the sequence end
    const uint32_t ntiles = (uint32_t)(part / kTile);
    // run-time constants: the multiplies and high multiplies that use them (shifts) stay
    // on the multiply-add pipe, beside the byte permutes and logic on the integer pipe
    const uint32_t k1 = p.k1, k16 = p.k5 >> 1, k65 = p.k1 * 65u;
    const uint32_t h16 = p.k5 << 11, h28 = p.k5 << 23;    // high multiplies: x >> 16, x >> 4
    const uint32_t h12 = p.k5 << 7;                      // x >> 20
    // staging: tile t of the 32 parts into a swizzled [32 rows][128 B] stage (16-byte
    // column c of row r at slot c ^ (r & 7)); copy j of a lane moves column lane & 7 of
    // row 4j + lane / 8, so each copy instruction covers four whole 128-byte lines
    const uint32_t l8 = (uint32_t)lane >> 3, cc = (uint32_t)lane & 7u;
    auto issue = [&](uint32_t t) {
#pragma unroll
        for (uint32_t j = 0; j < 8; ++j) {
            const uint32_t r = 4u * j + l8;
            const uint64_t off = b + (uint64_t)r * part + (uint64_t)t * kTile + cc * 16u;
            const bool ok = off < p.hi;
            cp_async16(stage_addr + r * kTile + ((cc ^ (r & 7u)) << 4), ok ? p.abase + off : p.abase, ok ? 16u : 0u);
        }
    };
    // four fields (the low 16 bits of 'sel') through a row: their new states (or counts)
    // as bytes
    auto look = [&](const uint2 *rows, uint32_t sel, uint32_t s7, uint32_t m) {
        if constexpr (W == 1) {
            return prmt(rows[0].x, rows[0].y, sel);
        } else {
            return lop3_sel(prmt(rows[0].x, rows[0].y, s7), prmt(rows[1].x, rows[1].y, s7), m);
        }
    };
    // one step of every run: the count bytes of fields 0..3 and 4..7 of register r are
    // added to ca[r] and cb[r]
    auto step = [&](uint32_t (&R)[W], const NibRows<W> &rw, uint32_t (&ca)[W], uint32_t (&cb)[W]) {
#pragma unroll
        for (int r = 0; r < W; ++r) {
            const uint32_t sa = R[r], sb = __umulhi(R[r], h16);   // fields 0..3, 4..7
            uint32_t sa7 = sa, sb7 = sb, ma = 0, mb = 0;
            if constexpr (W > 1) {
                sa7 = sa & 0x7777u; sb7 = sb & 0x7777u;
                ma = prmt(0x80808080u, 0x80808080u, sa);
                mb = prmt(0x80808080u, 0x80808080u, sb);
            }
            const uint32_t A = look(rw.s, sa, sa7, ma), B = look(rw.s, sb, sb7, mb);
            ca[r] = mad_lo(look(rw.c, sa, sa7, ma), k1, ca[r]);
            cb[r] = mad_lo(look(rw.c, sb, sb7, mb), k1, cb[r]);
            R[r] = mad_lo(B, k16, A);   // 4-bit states in the bytes: B x 16 and A share no bit
        }
    };
    // the identity step (no counts): moves every run as a step does
    const uint2 id_rows[2] = {make_uint2(0x03020100u, 0x07060504u), make_uint2(0x0B0A0908u, 0x0F0E0D0Cu)};
    auto shuffle = [&](uint32_t (&R)[W]) {
#pragma unroll
        for (int r = 0; r < W; ++r) {
            const uint32_t sa = R[r], sb = __umulhi(R[r], h16);
            uint32_t sa7 = sa, sb7 = sb, ma = 0, mb = 0;
            if constexpr (W > 1) {
                sa7 = sa & 0x7777u; sb7 = sb & 0x7777u;
                ma = prmt(0x80808080u, 0x80808080u, sa);
                mb = prmt(0x80808080u, 0x80808080u, sb);
            }
            R[r] = mad_lo(look(id_rows, sb, sb7, mb), k16, look(id_rows, sa, sa7, ma));
        }
    };
    uint32_t R[W];
#pragma unroll
    for (int r = 0; r < W; ++r) R[r] = 0x76543210u + 0x88888888u * (uint32_t)r;   // field i: start 8r + i
    // per-start totals of this lane's part, added to once per row
    uint32_t *tot = reinterpret_cast<uint32_t *>(smem + (size_t)kNibWarps * kStageBytesNib) +
                    ((uint32_t)warp * 32u + (uint32_t)lane) * kNibTotRow;
#pragma unroll
    for (int s = 0; s < 8 * W; ++s) tot[s] = 0;
    // count bytes of one phase (step number mod 3) -> per-run byte sums: the run from
    // start 8r + s sits in field rotl3^ph(s) of register r
    auto sort_counts = [&](uint32_t ca, uint32_t cb, int ph, uint32_t &lo, uint32_t &hi) {
        const uint32_t sl = ph == 0 ? 0x3210u : ph == 1 ? 0x6420u : 0x5140u;
        const uint32_t sh = ph == 0 ? 0x7654u : ph == 1 ? 0x7531u : 0x7362u;
        lo += prmt(ca, cb, sl);
        hi += prmt(ca, cb, sh);
    };
    auto add_totals = [&](int r, uint32_t lo, uint32_t hi) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            tot[8 * r + s] += (lo >> (8 * s)) & 0xFFu;
            tot[8 * r + s + 4] += (hi >> (8 * s)) & 0xFFu;
        }
    };
    issue(0);
    cp_async_commit();
    for (uint32_t t = 0; t < ntiles; ++t) {
        cp_async_wait<0>();
        __syncwarp();
        uint32_t w[32];
        {
            const uint8_t *srow = stage_ptr + lane * kTile;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint4 v = *reinterpret_cast<const uint4 *>(srow + ((q ^ (lane & 7)) * 16));
                w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
            }
        }
        __syncwarp();   // every lane holds its row: the stage can be refilled
        if (t + 1 < ntiles) issue(t + 1);
        cp_async_commit();
        const uint64_t ro = pb + (uint64_t)t * kTile;
        if (!(ro + kTile > from && ro < to)) continue;   // no byte of this row is in the part
        const bool full = ro >= from && ro + kTile <= to;
        bool done = false;
        if (full) {
            uint32_t R0[W];
#pragma unroll
            for (int r = 0; r < W; ++r) R0[r] = R[r];
            uint32_t ca[3][W], cb[3][W], err = 0;
#pragma unroll
            for (int ph = 0; ph < 3; ++ph)
#pragma unroll
                for (int r = 0; r < W; ++r) { ca[ph][r] = 0; cb[ph][r] = 0; }
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const uint32_t x = w[k] & 0x06060606u;
                const uint32_t y = mad_lo(x, k65, 0u);   // pair codes at bits 7..10 and 23..26
                // 8-byte rows: pair x 8 from bits 7..10 (and 23..26) of y
                const uint32_t o1 = __umulhi(y, h28) & 0x78u, o2 = __umulhi(y, h12) & 0x78u;
                NibRows<W> r1, r2;
#pragma unroll
                for (int h = 0; h < W; ++h) {
                    r1.s[h] = lds_v2(tab2s_addr + 128u * h + o1);
                    r1.c[h] = lds_v2(tab2c_addr + 128u * h + o1);
                    r2.s[h] = lds_v2(tab2s_addr + 128u * h + o2);
                    r2.c[h] = lds_v2(tab2c_addr + 128u * h + o2);
                }
                step(R, r1, ca[(2 * k) % 3], cb[(2 * k) % 3]);
                step(R, r2, ca[(2 * k + 1) % 3], cb[(2 * k + 1) % 3]);
                // bit-exact base check: expected lowercase bytes selected by the codes
                const uint32_t z = mad_lo(__umulhi(x, h28), k1, x);   // x | x >> 4 (no common bits)
                err |= prmt(p.lut_lo, p.lut_hi, prmt(z, 0u, 0x0020u)) ^ w[k];
            }
            if ((err & 0xDFDFDFDFu) == 0) {
                // 64 steps: the run in field s moved to field rotl3(s); two identity steps
                // bring every run back to its own field
                shuffle(R);
                shuffle(R);
#pragma unroll
                for (int r = 0; r < W; ++r) {
                    uint32_t lo = 0, hi = 0;
                    sort_counts(ca[0][r], cb[0][r], 0, lo, hi);
                    sort_counts(ca[1][r], cb[1][r], 1, lo, hi);
                    sort_counts(ca[2][r], cb[2][r], 2, lo, hi);
                    add_totals(r, lo, hi);
                }
                done = true;
            } else {
#pragma unroll
                for (int r = 0; r < W; ++r) R[r] = R0[r];
            }
        }
        if (!done) {
            // reset bytes or a part edge in this row: one symbol per step, every run
            // brought back to its own field after each
            const uint32_t k0 = ro < from ? (uint32_t)(from - ro) : 0u;
            const uint32_t kn = ro + kTile > to ? (uint32_t)(to - ro) : (uint32_t)kTile;
            uint32_t lo[W], hi[W];
#pragma unroll
            for (int r = 0; r < W; ++r) { lo[r] = 0; hi[r] = 0; }
            for (uint32_t k = k0; k < kn; ++k) {
                const uint32_t byte = p.abase[ro + k];   // the row is in L2
                const uint32_t code = byte_is_base(byte) ? ((byte >> 1) & 3u) : 4u;
                NibRows<W> rw;
#pragma unroll
                for (int h = 0; h < W; ++h) { rw.s[h] = tab1s[code][h]; rw.c[h] = tab1c[code][h]; }
                step(R, rw, lo, hi);
                shuffle(R);
                shuffle(R);
            }
#pragma unroll
            for (int r = 0; r < W; ++r) add_totals(r, lo[r], hi[r]);
        }
    }
    cp_async_wait<0>();
    __syncwarp();
    // the part's map (end state per start, packed 8 to a word, and counts) into a row of
    // the stage; lane s < 8 W then walks the 32 part maps in order from start s
    uint32_t *rows = reinterpret_cast<uint32_t *>(stage_ptr);
    uint32_t *mine = rows + lane * kNibRow;
#pragma unroll
    for (int r = 0; r < W; ++r) mine[r] = R[r];
#pragma unroll
    for (int s = 0; s < 8 * W; ++s) mine[2 + s] = tot[s];
    __syncwarp();
    __shared__ uint32_t chunk_map[kNibWarps][kNibRow];
    const bool walker = (uint32_t)lane < 8u * W;
    if (walker) {
        uint32_t st = (uint32_t)lane, cn = 0;
        for (uint32_t k = 0; k < 32; ++k) {
            if (p.bound && c < p.n_chunks) p.bound[((uint64_t)c * 32u + k) * 32u + lane] = st;
            const uint32_t *mk = rows + k * kNibRow;
            cn += mk[2 + st];
            st = (mk[st >> 3] >> (4 * (st & 7u))) & 15u;
        }
        // the chunk's map: end states packed into fields, counts
        const uint32_t field = st << (4 * (lane & 7));
        uint32_t packed = field;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) packed |= __shfl_xor_sync((1u << (8 * W)) - 1u, packed, o, 8);
        if ((lane & 7) == 0) chunk_map[warp][lane >> 3] = packed;
        chunk_map[warp][2 + lane] = cn;
    }
    __syncthreads();
    if (warp != 0 || !walker) return;
    // the block's chunks in order from block start s = lane
    uint32_t st = (uint32_t)lane, cn = 0;
    for (uint32_t k = 0; k < (uint32_t)kNibWarps; ++k) {
        const uint32_t ck = blockIdx.x * kNibWarps + k;
        if (p.cpre && ck < p.n_chunks) p.cpre[(uint64_t)ck * kNibMaxStates + lane] = st;
        cn += chunk_map[k][2 + st];
        st = (chunk_map[k][st >> 3] >> (4 * (st & 7u))) & 15u;
    }
    p.map_end[(uint64_t)blockIdx.x * 32u + lane] = st;
    p.map_cnt[(uint64_t)blockIdx.x * 32u + lane] = cn;
}

struct JoinParams {
    const uint32_t *map_end, *map_cnt, *bound, *gstart;
    uint32_t n_chunks;
    uint32_t n_states;
    uint32_t qp;                // row width of the map arrays (32 * warps per chunk)
    uint32_t parts;             // G of the map kernel: parts per chunk
    uint32_t *given;            // [n_chunks * 32] exact start of each sub-chunk, or null
    // map_nib_kernel: the maps are per block of kNibWarps chunks (n_chunks counts the
    // blocks); cpre gives each chunk's start per block start state; else null
    const uint32_t *cpre;
    uint32_t *bstart;           // (with cpre) receives each block's start state
    uint64_t *out_count;
    uint32_t start;             // the state the sequence starts in
    uint32_t *out_last;         // null, or receives the state after the last byte
    const uint32_t *perm_inv;   // null, or device -> caller state numbering (for out_last)
};

// Single block. Chunks are taken 32 at a time: the group's 32 maps are composed for all
// start states (for maps 32 wide, a warp per group with its maps cached in shared memory
// and lane q following start q; for wider maps, one thread per (group, start state)
// reading the maps from global memory), thread 0 then chains the groups from the start,
// and (for the positions pass) each group is walked again from its true start to give
// every chunk's, and so every sub-chunk's, exact start.
__global__ void __launch_bounds__(kJoinWarps * 32, 1) map_join_kernel(JoinParams p) {
    extern __shared__ __align__(16) uint32_t jsm[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t ng = (p.n_chunks + 31) / 32;
    const uint32_t qp = p.qp;
    uint32_t *g_end = jsm;                      // [ng][qp]
    uint32_t *g_cnt = g_end + ng * qp;          // [ng][qp]
    uint32_t *g_start = g_cnt + ng * qp;        // [ng]
    // per warp (maps 32 wide): [32 chunks][32] ends, then counts; 16-byte aligned
    uint32_t *wbuf = g_start + ((ng + 3u) & ~3u);
    uint32_t *my_end = wbuf + (size_t)warp * 2048;
    uint32_t *my_cnt = my_end + 1024;
    uint32_t *kst = wbuf + (size_t)kJoinWarps * 2048 + (size_t)warp * 32;   // [32] chunk starts
    auto group_size = [&](uint32_t g) { return p.n_chunks - g * 32 < 32 ? p.n_chunks - g * 32 : 32u; };
    // a group's maps (nk x 32 words each) into shared memory: every 16-byte copy is issued
    // before the first is waited for
    auto load_group = [&](uint32_t g) {
        const uint32_t nk = group_size(g);
        const uint32_t e0 = (uint32_t)__cvta_generic_to_shared(my_end), c0 = (uint32_t)__cvta_generic_to_shared(my_cnt);
#pragma unroll
        for (uint32_t j = 0; j < 8; ++j) {
            const uint32_t i = (j * 32u + (uint32_t)lane) * 4u;   // word index of this 16-byte piece
            if (i < nk * 32u) {
                cp_async16(e0 + i * 4u, p.map_end + (uint64_t)g * 1024 + i, 16u);
                cp_async16(c0 + i * 4u, p.map_cnt + (uint64_t)g * 1024 + i, 16u);
            }
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        return nk;
    };
    if (qp == 32) {
        for (uint32_t g = warp; g < ng; g += kJoinWarps) {
            const uint32_t nk = load_group(g);
            uint32_t s = (uint32_t)lane < p.n_states ? (uint32_t)lane : 0u, cc = 0;
            for (uint32_t k = 0; k < nk; ++k) {
                cc += my_cnt[k * 32 + s];
                s = my_end[k * 32 + s];
            }
            g_end[g * 32 + lane] = s;
            g_cnt[g * 32 + lane] = cc;
            __syncwarp();
        }
    } else {
        for (uint32_t i = threadIdx.x; i < ng * qp; i += kJoinWarps * 32) {
            const uint32_t g = i / qp, s0 = i - g * qp;
            const uint32_t nk = group_size(g);
            uint32_t s = s0 < p.n_states ? s0 : 0u, cc = 0;
            for (uint32_t k = 0; k < nk; ++k) {
                const uint64_t row = ((uint64_t)g * 32 + k) * qp;
                cc += p.map_cnt[row + s];
                s = p.map_end[row + s];
            }
            g_end[i] = s;
            g_cnt[i] = cc;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = p.start;
        unsigned long long total = 0;
        for (uint32_t g = 0; g < ng; ++g) {
            g_start[g] = s;
            total += g_cnt[g * qp + s];
            s = g_end[g * qp + s];
        }
        *p.out_count = total;
        if (p.out_last) *p.out_last = p.perm_inv ? p.perm_inv[s] : s;
    }
    __syncthreads();
    if (!p.given) return;
    for (uint32_t g = warp; g < ng; g += kJoinWarps) {
        const uint32_t nk = qp == 32 ? load_group(g) : group_size(g);
        // the group's chunk starts (one lane walks the maps), then every sub-chunk's start
        // with the loads of eight chunks in flight at once
        if (p.cpre) {
            // the maps are per block: each block's start goes out for nib_given_kernel,
            // which gives every sub-chunk's start from it
            if (lane == 0) {
                uint32_t s = g_start[g];
                for (uint32_t k = 0; k < nk; ++k) {
                    p.bstart[(uint64_t)g * 32 + k] = s;
                    s = my_end[k * 32 + s];
                }
            }
            __syncwarp();
            continue;
        }
        if (lane == 0) {
            uint32_t s = g_start[g];
            for (uint32_t k = 0; k < nk; ++k) {
                kst[k] = s;
                s = qp == 32 ? my_end[k * 32 + s] : p.map_end[((uint64_t)g * 32 + k) * qp + s];
            }
        }
        __syncwarp();
        // sub-chunk 'lane' lies in part gl of its chunk; its recorded states are indexed
        // by the state at that part's start
        const uint32_t gl = (uint32_t)lane / (kMapSubs / p.parts);
#pragma unroll 8
        for (uint32_t k = 0; k < nk; ++k) {
            const uint64_t c = (uint64_t)g * 32 + k;
            const uint32_t s = kst[k];
            const uint32_t sp = gl ? p.gstart[(c * p.parts + gl) * 32u + s] : s;
            p.given[c * kMapSubs + lane] = p.bound[(c * kMapSubs + lane) * qp + sp];
        }
        __syncwarp();
    }
}

// The positions pass's start of every sub-chunk of the nibble path (a part: 32 per
// chunk): its chunk's start from the chunk's block start, then the part's start from
// the chunk's start. One thread per sub-chunk.
__global__ void nib_given_kernel(const uint32_t *bstart, const uint32_t *cpre, const uint32_t *bound,
                                 uint32_t *given, uint32_t n_chunks) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint64_t)n_chunks * kMapSubs) return;
    const uint64_t c = i / kMapSubs;
    const uint32_t sb = bstart[c / kNibWarps];
    const uint32_t sc = cpre[c * kNibMaxStates + sb];
    given[i] = bound[i * 32u + sc];
}

}  // namespace

namespace dnalib {

// The chunk-map scan of one sequence (count, and positions through scan_impl with the
// exact sub-chunk starts). Requires n_states <= kMaxMapStates. Automata of at most 8 (16)
// states walk each chunk as 4 (2) parts at once; automata of more than 32 states run
// ceil(Q / 32) warps per chunk. 'ext' (count only) supplies the scratch instead of the
// library's pool: ext_bytes of device memory; DNA_ERR_CAPACITY when it is too small.
int map_scan_impl(const dna_dfa *d, const uint8_t *seq, uint64_t len, cudaStream_t stream, uint64_t *out_count,
                  uint64_t *out_positions, uint64_t cap, uint8_t *ext, size_t ext_bytes, const LabelOut *lab,
                  const ScanFrom *from) {
    if (d->n_states > kMaxMapStates) return DNA_ERR_INVALID_ARG;
    const uint64_t shift = (uint64_t)((uintptr_t)seq & 15u);
    const uint8_t *abase = seq - shift;
    const uint64_t total = len + shift;
    const DeviceProps pr = device_props(d->device);
    const uint32_t wblocks = (d->n_states + 31) / 32;
    const uint32_t qp = 32 * wblocks;
    // one wave of warps: every chunk takes wblocks of them
    const uint64_t tasks = (uint64_t)(pr.sms ? pr.sms : 152) * (d->n_states <= kNibMaxStates ? kNibWarps : kMapWarps);
    const uint64_t unit = (uint64_t)kMapSubs * kTile;                        // 4 KiB
    // at most 16 states: every run of a part in one or two words, a lane per part
    // (map_nib_kernel); else a lane per start state, two chains per lane up to 32 states
    const bool nib = d->n_states <= kNibMaxStates;
    const uint32_t groups = 1u;
    const uint32_t chains = d->n_states <= 32 ? 2u : 1u;
    const uint32_t parts = nib ? 1u : groups * chains;
    const int tab = d->d_pair ? TAB_PAIR : TAB_ONE;
    const uint64_t want_chunks = std::max<uint64_t>(1, tasks / wblocks);
    uint64_t S = (total + want_chunks - 1) / want_chunks;
    S = (S + unit - 1) / unit * unit;
    const uint32_t n_chunks = (uint32_t)((total + S - 1) / S);
    // the positions pass also gives per-label outputs
    const bool positions = (out_positions != nullptr && cap > 0) || lab != nullptr;
    if (ext && positions) return DNA_ERR_INVALID_ARG;
    const size_t nq = (size_t)n_chunks * qp;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_end = take(nq * 4), o_cnt = take(nq * 4);
    // sub-chunk states, only for the positions pass
    const size_t o_bound = positions ? take(nq * kMapSubs * 4) : 0;
    const size_t o_gstart = positions ? take((size_t)n_chunks * 32 * parts * 4) : 0;
    const size_t o_given = positions ? take((size_t)n_chunks * kMapSubs * 4) : 0;
    const size_t o_cpre = positions && nib ? take((size_t)n_chunks * kNibMaxStates * 4) : 0;
    const size_t o_bstart = positions && nib ? take((size_t)n_chunks * 4) : 0;
    const size_t optin = pr.smem_optin ? pr.smem_optin : 232448;
    const size_t part_tile = chains == 1 ? (size_t)kMapTile : (size_t)2048 / parts;
    const size_t msmem = nib ? kNibSmem
                             : (size_t)kMapWarps * 2 * parts * part_tile + (size_t)d->n_states * 16 + 2048 +
                                   (size_t)d->n_states * (tab == TAB_PAIR ? (size_t)kPairRowBytes : (size_t)kOneRowBytes);
    void (*fn)(MapParams) = nib ? (d->n_states <= 8 ? map_nib_kernel<1> : map_nib_kernel<2>)
                          : tab == TAB_ONE ? map_kernel<1, TAB_ONE, 1>
                          : chains == 1 ? map_kernel<1, TAB_PAIR, 1>
                          : map_kernel<1, TAB_PAIR, 2>;
    // the kernel's static shared memory (its decoded rows, 3.5 KB per part) comes off the
    // block's shared memory before the dynamic part
    size_t static_smem = 0;
    {
        cudaFuncAttributes fa;
        DNA_CUDA(cudaFuncGetAttributes(&fa, (const void *)fn));
        static_smem = fa.sharedSizeBytes;
    }
    if (static_smem + 1024 >= optin || msmem > optin - static_smem - 1024) return DNA_ERR_CAPACITY;
    const uint32_t ng = (n_chunks + 31) / 32;
    const size_t jsmem = ((size_t)ng * 2 * qp + ((ng + 3) & ~(size_t)3) + (size_t)kJoinWarps * (2048 + 32)) * 4;
    if (jsmem > optin - 1024) return DNA_ERR_CAPACITY;
    void *mem = nullptr;
    if (ext) {
        if (off > ext_bytes) return DNA_ERR_CAPACITY;
        mem = ext;
    } else {
        const int ra = scratch_alloc(d->device, off, stream, &mem);
        if (ra) return ra;
    }
    uint8_t *base = (uint8_t *)mem;

    MapParams mp;
    mp.abase = abase; mp.lo = shift; mp.hi = total; mp.chunk_bytes = S; mp.n_chunks = n_chunks;
    mp.n_states = d->n_states; mp.wblocks = wblocks; mp.qp = qp;
    mp.reset_entry = d->reset_entry; mp.one = d->d_one; mp.pair = d->d_pair;
    mp.map_end = (uint32_t *)(base + o_end); mp.map_cnt = (uint32_t *)(base + o_cnt);
    mp.bound = positions ? (uint32_t *)(base + o_bound) : nullptr;
    mp.gstart = positions && parts > 1 ? (uint32_t *)(base + o_gstart) : nullptr;
    mp.cpre = positions && nib ? (uint32_t *)(base + o_cpre) : nullptr;
    mp.k1 = 1u; mp.k5 = 32u; mp.lut_lo = 0x00630061u; mp.lut_hi = 0x00670074u;
    int rc = ensure_smem_optin((const void *)fn, d->device, optin - static_smem - 1024);
    cudaError_t e = rc ? cudaErrorInvalidValue : cudaSuccess;
    if (e == cudaSuccess) {
        const uint64_t n_tasks = (uint64_t)n_chunks * wblocks;
        const ProfToken tk = prof_begin(stream);
        const int warps = nib ? kNibWarps : kMapWarps;
        fn<<<(unsigned)((n_tasks + warps - 1) / warps), warps * 32, msmem, stream>>>(mp);
        e = cudaGetLastError();
        prof_end(tk, stream, PROF_SCAN);
        record_launch();
    }
    JoinParams jp;
    jp.map_end = mp.map_end; jp.map_cnt = mp.map_cnt; jp.bound = mp.bound; jp.gstart = mp.gstart;
    // map_nib_kernel leaves one map per block of kNibWarps chunks
    const uint32_t n_blocks_nib = (n_chunks + kNibWarps - 1) / kNibWarps;
    jp.n_chunks = nib ? n_blocks_nib : n_chunks; jp.n_states = d->n_states; jp.qp = qp; jp.parts = parts;
    jp.cpre = mp.cpre;
    jp.bstart = positions && nib ? (uint32_t *)(base + o_bstart) : nullptr;
    jp.given = positions ? (uint32_t *)(base + o_given) : nullptr;
    jp.out_count = out_count;
    jp.start = from ? from->start : 0u;
    jp.out_last = from ? from->out_last : nullptr;
    jp.perm_inv = d->d_perm_inv;
    if (e == cudaSuccess) {
        rc = ensure_smem_optin((const void *)map_join_kernel, d->device, optin - 1024);
        if (rc) e = cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) {
        map_join_kernel<<<1, kJoinWarps * 32, jsmem, stream>>>(jp);
        e = cudaGetLastError();
        record_launch();
    }
    if (e == cudaSuccess && positions && nib) {
        const uint64_t n_sub = (uint64_t)n_chunks * kMapSubs;
        nib_given_kernel<<<(unsigned)((n_sub + 255) / 256), 256, 0, stream>>>(jp.bstart, jp.cpre, jp.bound,
                                                                               jp.given, n_chunks);
        e = cudaGetLastError();
        record_launch();
    }
    rc = cuda_status(e);
    if (rc == DNA_OK && positions) {
        // the single-sequence kernels with every sub-chunk's exact start: no speculation,
        // no repair; they also write the (same) count
        dna_plan pl = {};
        pl.chunk_bytes = (uint32_t)(S / kMapSubs);
        pl.placement = d->d_pair ? DNA_PLACE_SMEM_PAIR : 0u;
        rc = scan_impl_given(d, seq, len, stream, out_count, out_positions, cap, &pl, jp.given, lab,
                             from);
    }
    if (!ext) {
        const int rf = scratch_free(mem, stream);
        if (rc == DNA_OK) rc = rf;
    }
    return rc;
}

}  // namespace dnalib
