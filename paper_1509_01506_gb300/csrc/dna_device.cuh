// dna_device.cuh -- device helpers shared by the library's kernels (dna_scan.cu, the
// single-sequence path, and dna_batch.cu, the batched path). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace {

constexpr int kTile = 128;                  // bytes per chunk row staged per step
constexpr int kPairRowBytes = 16 * 32 * 4;  // 16 symbol pairs x 32 lanes x 4 bytes

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

__device__ __forceinline__ uint32_t lds_u16(uint32_t addr) {
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n"
                 :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
template <int OFF>
__device__ __forceinline__ void cp_async16_full(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0+%2], [%1], 16;\n"
                 :: "r"(dst), "l"(src), "n"(OFF) : "memory");
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

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" :: "l"(p));
}

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// Pair-table entry layout (lane l's copy): bits 0..17 = shared address of the next
// state's row for lane l (row base 2048-aligned, so bits 7..10 are zero), bits 27..28 =
// accepting steps in the pair. The two codes of a pair enter at bits 7..10.
constexpr uint32_t kPairMuxMask = 0x78000780u;
constexpr int kCountShift = 27;

// Bitwise select with the pair-table mask: bits of b where kPairMuxMask is set, bits of a
// elsewhere. Written as one lop3 (lut 0xD8 = (a & ~c) | (b & c)); the C++ form of the
// same select compiles to two logic instructions.
__device__ __forceinline__ uint32_t mux_pair(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xD8;" : "=r"(d) : "r"(a), "r"(b), "n"(kPairMuxMask));
    return d;
}

__device__ __forceinline__ uint32_t one_step(const uint32_t *one, uint32_t reset_entry, uint32_t q,
                                             uint32_t b) {
    return byte_is_base(b) ? one[q * 4u + ((b >> 1) & 3u)] : reset_entry;
}

// Walks aligned offsets [from, to) of the sequence in 128-byte blocks: each block is
// fetched with eight independent 16-byte loads (a 16-byte granule is loaded only if it
// starts before 'hi', so no load leaves the sequence's last page), then f(offset, byte)
// is called in order. f returns false to stop the walk.
template <class F>
__device__ __forceinline__ void walk_range(const uint8_t *abase, uint64_t from, uint64_t to, uint64_t hi,
                                           F &&f) {
    for (uint64_t blk = from & ~(uint64_t)(kTile - 1); blk < to; blk += kTile) {
        uint4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint64_t g = blk + 16u * j;
            v[j] = g < hi ? *reinterpret_cast<const uint4 *>(abase + g) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k4 = 0; k4 < 32; ++k4) {
            const uint4 &vv = v[k4 >> 2];
            const uint32_t word = (k4 & 3) == 0 ? vv.x : (k4 & 3) == 1 ? vv.y : (k4 & 3) == 2 ? vv.z : vv.w;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint64_t o = blk + 4u * k4 + i;
                if (o >= from && o < to && !f(o, (word >> (8 * i)) & 0xFFu)) return;
            }
        }
    }
}

}  // namespace
