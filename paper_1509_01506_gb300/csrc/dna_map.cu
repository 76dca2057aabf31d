// dna_map.cu -- the chunk-map path for automata whose runs do not converge.
//
// Speculation with repair (dna_scan.cu) relies on the runs from different start states
// meeting soon (the converging point of Sec. III-B.3). Some automata never synchronise
// on DNA (permutation-like tables, counters): there every chunk's repair walks the whole
// chunk and every join cascades, serially. For those the scan follows the paper's
// possible-starting-state approach in full (Sec. III-A): a chunk is run from every state
// at once. A warp runs one chunk from 32 start states (lane q from state 32w + q for the
// warp's state block w); automata of more than 32 states give each chunk ceil(Q / 32)
// warps, and automata of at most 8 or 16 states cut the chunk into 4 or 2 parts walked
// side by side by lane groups, whose maps the warp composes. Each chunk yields a map (end
// state and count per start state) and, for the positions pass, the state at each of its
// 32 sub-chunk boundaries per start state. A single-block join composes the maps in order
// (chunk c starts in the end state of chunk c-1 from its true start), which gives the
// total count and every sub-chunk's exact start state. The positions come from the
// single-sequence kernels run with those exact starts.
//
// Lookups never conflict in shared memory: every lane has its own copy of the table in
// its own bank. Automata of up to about 90 states use the two-symbol table (2 KiB per
// state); larger ones, up to kMaxMapStates, a one-symbol table (512 B per state).

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
    uint32_t k1, k5, lut_lo, lut_hi;
};

// One warp per (chunk, block of 32 start states). The chunk is cut into G equal parts
// (32 / G lanes each) walked at once: lane (g, q) runs part g from state 32w + q (lanes at
// or past n_states run from state 0 and are ignored), so that small automata keep every
// lane busy. Each part's bytes are staged 512 at a time; lane k decodes word k of every
// part's row for the warp. At the end the warp composes the parts' maps into the chunk's
// map.
template <int G, int TAB>
__global__ void __launch_bounds__(kMapWarps * 32, 1) map_kernel(MapParams p) {
    static_assert(TAB == TAB_PAIR || G == 1, "parts only with the two-symbol table");
    constexpr uint32_t kLanes = 32u / G;               // lanes (start states) per part
    constexpr uint32_t kWarpStage = 2u * G * kMapTile; // double-buffered tile of every part
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t g = (uint32_t)lane / kLanes, q = (uint32_t)lane % kLanes;
    const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);
    // shared memory: [stages: warps x 2 x G x 512 B][one-symbol table: Q x 16 B][pad]
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
    __shared__ __align__(16) uint32_t ys_all[kMapWarps][G][36];
    uint32_t *ys = ys_all[warp][g];

    OneTable T;
    T.t = one_s;
    T.reset_entry = p.reset_entry;
    const uint64_t b = (uint64_t)c * p.chunk_bytes;
    const uint64_t part = p.chunk_bytes / G;           // multiple of kMapTile
    const uint64_t pb = b + g * part;                  // this lane's part
    const uint64_t from = pb > p.lo ? pb : p.lo;
    const uint64_t pe = pb + part < p.hi ? pb + part : p.hi;
    const uint64_t to = pe > from ? pe : from;         // empty past the sequence end
    const uint64_t sub = p.chunk_bytes / kMapSubs;
    const uint32_t ntiles = (uint32_t)(part / kMapTile);   // the same for every part and warp
    const uint32_t sq = wb * 32u + q;                  // this lane's start state
    const uint32_t q0 = sq < p.n_states ? sq : 0u;
    auto cur_of = [&](uint32_t s) {
        return TAB == TAB_PAIR ? tab_base + s * (uint32_t)kPairRowBytes + (uint32_t)lane * 4u
                               : tab_base + s * kOneRowBytes + (uint32_t)lane * 4u;
    };
    auto state_of = [&](uint32_t cv) {
        return TAB == TAB_PAIR ? ((cv & 0x3FFFFu) - tab_base) / (uint32_t)kPairRowBytes
                               : ((cv & 0x3FE00u) - tab_base) / kOneRowBytes;
    };
    uint32_t cur = cur_of(q0);
    uint32_t cnt = 0;
    auto issue = [&](uint32_t t) {   // lane copies 16 bytes of tile t of every part (past hi: zero-filled)
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
            const uint64_t off = b + (uint64_t)gg * part + (uint64_t)t * kMapTile + (uint64_t)lane * 16u;
            const bool ok = off < p.hi;
            cp_async16(stage_addr + ((t & 1u) * G + (uint32_t)gg) * kMapTile + (uint32_t)lane * 16u,
                       ok ? p.abase + off : p.abase, ok ? 16u : 0u);
        }
    };
    issue(0);
    cp_async_commit();
    for (uint32_t t = 0; t < ntiles; ++t) {
        if (t + 1 < ntiles) issue(t + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        const uint8_t *tiles = stage + (t & 1u) * G * kMapTile;
#pragma unroll 1
        for (int r = 0; r < kMapTile / kTile; ++r) {
            const uint64_t ro = pb + (uint64_t)t * kMapTile + (uint64_t)r * kTile;
            if (p.bound && ro < to && (ro - b) % sub == 0)   // a sub-chunk starts here: record the state
                p.bound[((uint64_t)c * kMapSubs + (ro - b) / sub) * p.qp + sq] = state_of(cur);
            const uint8_t *row = tiles + g * kMapTile + r * kTile;
            // lane k decodes word k of each part's row for the warp: its codes (y, read
            // back by the part's lanes) and the base check (voted per part)
            uint32_t bad_parts = 0;
#pragma unroll
            for (int gg = 0; gg < G; ++gg) {
                const uint32_t wk = *reinterpret_cast<const uint32_t *>(tiles + gg * kMapTile + r * kTile + 4 * lane);
                const uint32_t xk = wk & 0x06060606u;
                // two-symbol table: pairs at bits 7..10 and 23..26; one-symbol: raw codes
                ys_all[warp][gg][lane] = TAB == TAB_PAIR ? mad_lo(xk, 65u, 0u) : xk;
                const uint32_t zk = xk | (xk >> 4);
                const bool bad = ((__byte_perm(p.lut_lo, p.lut_hi, __byte_perm(zk, 0, 0x0020)) ^ wk) & 0xDFDFDFDFu) != 0;
                bad_parts |= (__any_sync(0xFFFFFFFFu, bad) ? 1u : 0u) << gg;
            }
            __syncwarp();
            const bool full = ro >= from && ro + kTile <= to;
            if (full && !((bad_parts >> g) & 1u)) {
                if (TAB == TAB_PAIR) {
                    uint32_t acc = 0, rc = 0, c2 = cur;
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
                    cnt += rc;
                    cur = c2 & 0x3FFFFu;
                } else {
                    // byte j's code sits at bits 8j+1..8j+2 of y; the lookup puts it at bits
                    // 7..8 of the row address
                    uint32_t rc = 0, e = cur;
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
                    cnt += rc;
                    cur = e & ~1u;
                }
            } else if (ro + kTile > from && ro < to) {
                // reset bytes or a sequence edge in this row: byte by byte
                uint32_t qs = state_of(cur);
                const uint32_t k0 = ro < from ? (uint32_t)(from - ro) : 0u;
                const uint32_t k1 = ro + kTile > to ? (uint32_t)(to - ro) : (uint32_t)kTile;
                for (uint32_t k = k0; k < k1; ++k) {
                    const uint32_t e = T.step(qs, row[k]);
                    qs = e & 0x7FFFFFFFu;
                    cnt += e >> 31;
                }
                cur = cur_of(qs);
            }
            __syncwarp();   // ys is rewritten by the next row
        }
        __syncwarp();   // every lane is done with this stage before it is refilled
    }
    cp_async_wait<0>();
    // compose the parts: from chunk start state s, part g starts where part g-1 ended
    const uint32_t end = state_of(cur);
    if (G == 1) {
        p.map_end[(uint64_t)c * p.qp + sq] = end;
        p.map_cnt[(uint64_t)c * p.qp + sq] = cnt;
        return;
    }
    uint32_t s = q0, total = 0;
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
        if (p.gstart && gg > 0 && g == 0) p.gstart[((uint64_t)c * G + gg) * 32u + q] = s;
        total += __shfl_sync(0xFFFFFFFFu, cnt, gg * (int)kLanes + (int)s);
        s = __shfl_sync(0xFFFFFFFFu, end, gg * (int)kLanes + (int)s);
    }
    if (g == 0) {
        p.map_end[(uint64_t)c * 32u + q] = s;
        p.map_cnt[(uint64_t)c * 32u + q] = total;
    }
}

struct JoinParams {
    const uint32_t *map_end, *map_cnt, *bound, *gstart;
    uint32_t n_chunks;
    uint32_t n_states;
    uint32_t qp;                // row width of the map arrays (32 * warps per chunk)
    uint32_t parts;             // G of the map kernel: parts per chunk
    uint32_t *given;            // [n_chunks * 32] exact start of each sub-chunk, or null
    uint64_t *out_count;
};

// Single block. Chunks are taken 32 at a time: the group's 32 maps are composed for all
// start states (for maps 32 wide, a warp per group with its maps cached in shared memory
// and lane q following start q; for wider maps, one thread per (group, start state)
// reading the maps from global memory), thread 0 then chains the groups from state 0,
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
    uint32_t *wbuf = g_start + ng;              // per warp (maps 32 wide): [32 chunks][32] ends, then counts
    uint32_t *my_end = wbuf + (size_t)warp * 2048;
    uint32_t *my_cnt = my_end + 1024;
    auto group_size = [&](uint32_t g) { return p.n_chunks - g * 32 < 32 ? p.n_chunks - g * 32 : 32u; };
    auto load_group = [&](uint32_t g) {
        const uint32_t nk = group_size(g);
        for (uint32_t i = lane; i < nk * 32; i += 32) {
            my_end[i] = p.map_end[(uint64_t)g * 1024 + i];
            my_cnt[i] = p.map_cnt[(uint64_t)g * 1024 + i];
        }
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
        uint32_t s = 0;
        unsigned long long total = 0;
        for (uint32_t g = 0; g < ng; ++g) {
            g_start[g] = s;
            total += g_cnt[g * qp + s];
            s = g_end[g * qp + s];
        }
        *p.out_count = total;
    }
    __syncthreads();
    if (!p.given) return;
    for (uint32_t g = warp; g < ng; g += kJoinWarps) {
        const uint32_t nk = qp == 32 ? load_group(g) : group_size(g);
        uint32_t s = g_start[g];
        // sub-chunk 'lane' lies in part gl of its chunk; its recorded states are indexed
        // by the state at that part's start
        const uint32_t gl = (uint32_t)lane / (kMapSubs / p.parts);
        for (uint32_t k = 0; k < nk; ++k) {
            const uint64_t c = (uint64_t)g * 32 + k;
            const uint32_t sp = gl ? p.gstart[(c * p.parts + gl) * 32u + s] : s;
            p.given[c * kMapSubs + lane] = p.bound[(c * kMapSubs + lane) * qp + sp];
            s = qp == 32 ? my_end[k * 32 + s] : p.map_end[c * qp + s];
        }
        __syncwarp();
    }
}

}  // namespace

namespace dnalib {

// The chunk-map scan of one sequence (count, and positions through scan_impl with the
// exact sub-chunk starts). Requires n_states <= kMaxMapStates. Automata of at most 8 (16)
// states walk each chunk as 4 (2) parts at once; automata of more than 32 states run
// ceil(Q / 32) warps per chunk. 'ext' (count only) supplies the scratch instead of the
// library's pool: ext_bytes of device memory; DNA_ERR_CAPACITY when it is too small.
int map_scan_impl(const dna_dfa *d, const uint8_t *seq, uint64_t len, cudaStream_t stream, uint64_t *out_count,
                  uint64_t *out_positions, uint64_t cap, uint8_t *ext, size_t ext_bytes, const LabelOut *lab) {
    if (d->n_states > kMaxMapStates) return DNA_ERR_INVALID_ARG;
    const uint64_t shift = (uint64_t)((uintptr_t)seq & 15u);
    const uint8_t *abase = seq - shift;
    const uint64_t total = len + shift;
    const DeviceProps pr = device_props(d->device);
    const uint32_t wblocks = (d->n_states + 31) / 32;
    const uint32_t qp = 32 * wblocks;
    // one wave of warps: every chunk takes wblocks of them
    const uint64_t tasks = (uint64_t)(pr.sms ? pr.sms : 152) * kMapWarps;
    const uint64_t unit = (uint64_t)kMapSubs * kTile;                        // 4 KiB
    const uint32_t parts = d->n_states <= 8 ? 4u : d->n_states <= 16 ? 2u : 1u;
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
    const size_t optin = pr.smem_optin ? pr.smem_optin : 232448;
    const size_t msmem = (size_t)kMapWarps * 2 * parts * kMapTile + (size_t)d->n_states * 16 + 2048 +
                         (size_t)d->n_states * (tab == TAB_PAIR ? (size_t)kPairRowBytes : (size_t)kOneRowBytes);
    // static shared memory: the decoded rows, about 3.5 KB per part; 16 KB is reserved
    if (msmem > optin - 16384) return DNA_ERR_CAPACITY;
    const uint32_t ng = (n_chunks + 31) / 32;
    const size_t jsmem = ((size_t)ng * (2 * qp + 1) + (qp == 32 ? (size_t)kJoinWarps * 2048 : 0)) * 4;
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
    mp.k1 = 1u; mp.k5 = 32u; mp.lut_lo = 0x00630061u; mp.lut_hi = 0x00670074u;
    void (*fn)(MapParams) = tab == TAB_ONE ? map_kernel<1, TAB_ONE>
                          : parts == 4 ? map_kernel<4, TAB_PAIR>
                          : parts == 2 ? map_kernel<2, TAB_PAIR> : map_kernel<1, TAB_PAIR>;
    int rc = ensure_smem_optin((const void *)fn, d->device, optin - 16384);
    cudaError_t e = rc ? cudaErrorInvalidValue : cudaSuccess;
    if (e == cudaSuccess) {
        const uint64_t n_tasks = (uint64_t)n_chunks * wblocks;
        const ProfToken tk = prof_begin(stream);
        fn<<<(unsigned)((n_tasks + kMapWarps - 1) / kMapWarps), kMapWarps * 32, msmem, stream>>>(mp);
        e = cudaGetLastError();
        prof_end(tk, stream, PROF_SCAN);
        record_launch();
    }
    JoinParams jp;
    jp.map_end = mp.map_end; jp.map_cnt = mp.map_cnt; jp.bound = mp.bound; jp.gstart = mp.gstart;
    jp.n_chunks = n_chunks; jp.n_states = d->n_states; jp.qp = qp; jp.parts = parts;
    jp.given = positions ? (uint32_t *)(base + o_given) : nullptr;
    jp.out_count = out_count;
    if (e == cudaSuccess) {
        rc = ensure_smem_optin((const void *)map_join_kernel, d->device, optin - 1024);
        if (rc) e = cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) {
        map_join_kernel<<<1, kJoinWarps * 32, jsmem, stream>>>(jp);
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
        rc = scan_impl_given(d, seq, len, stream, out_count, out_positions, cap, &pl, jp.given, lab);
    }
    if (!ext) {
        const int rf = scratch_free(mem, stream);
        if (rc == DNA_OK) rc = rf;
    }
    return rc;
}

}  // namespace dnalib
