// dna_bench.cu -- the lookup-throughput microbenchmark behind dna_lookup_peak: the
// measured peaks that the scans' rooflines divide by (the scans are chains of dependent
// table lookups, not floating-point or streaming work). No counterpart in the paper.

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dna_dfa.h"
#include "dna_device.cuh"
#include "dna_runtime.h"

using namespace dnalib;

namespace {

constexpr int kPeakThreads = 1024;
constexpr int kPeakChains = 8;          // independent lookup chains per thread
constexpr uint32_t kPeakWords = 16384;  // 64 KiB shared-memory table
constexpr uint32_t kPeakGlobalWords = 32768;   // 128 KiB global table (the size of a large
                                               // automaton's one-symbol table)

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16; x *= 0x7FEB352Du; x ^= x >> 15; x *= 0x846CA68Bu; x ^= x >> 16;
    return x;
}

// Every thread runs kPeakChains chains of 'iters' dependent 4-byte lookups; each entry
// holds the byte offset of the next one, so no lookup can start before the previous one
// of its chain has returned.
//   mode 0: shared memory, lane l only ever reads bank l (the per-lane table copies of
//           the two-symbol scans): no bank conflict;
//   mode 1: shared memory, entries anywhere in the table (the shared one-symbol table):
//           32 lanes meet random banks;
//   mode 2: global memory, entries anywhere in a 128 KiB table read with ordinary
//           (L1-cached) loads, as the one-symbol table of automata too large for shared
//           memory is read.
__global__ void __launch_bounds__(kPeakThreads, 1)
lookup_peak_kernel(uint32_t mode, uint32_t iters, const uint32_t *gtab, unsigned long long *sink) {
    extern __shared__ __align__(16) uint32_t tab[];
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    for (uint32_t i = tid; i < kPeakWords; i += kPeakThreads) {
        const uint32_t h = mix32(i * 0x9E3779B9u + 17u);
        tab[i] = mode == 0 ? (((h & 511u) * 32u) + (i & 31u)) * 4u : (h & (kPeakWords - 1u)) * 4u;
    }
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(tab);
    uint32_t a[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) {
        const uint32_t h = mix32(blockIdx.x * 131071u + tid * kPeakChains + (uint32_t)c);
        a[c] = mode == 0 ? (((h & 511u) * 32u) + lane) * 4u : (h & (kPeakWords - 1u)) * 4u;
    }
    if (mode == 2) {
        const uint8_t *g = reinterpret_cast<const uint8_t *>(gtab);
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c)
            a[c] = (mix32(blockIdx.x * 131071u + tid * kPeakChains + (uint32_t)c) & (kPeakGlobalWords - 1u)) * 4u;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c)
                a[c] = *reinterpret_cast<const uint32_t *>(g + a[c]);
        }
    } else {
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) a[c] = lds_u32(base + a[c]);
        }
    }
    unsigned long long t = 0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) t += a[c];
    if (t == 0x123456789ull) sink[0] = t;   // keeps the chains live; practically never true
}

__global__ void fill_global_table(uint32_t *gtab) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kPeakGlobalWords) gtab[i] = (mix32(i * 0x9E3779B9u + 17u) & (kPeakGlobalWords - 1u)) * 4u;
}

}  // namespace

extern "C" int dna_lookup_peak(uint32_t mode, dna_stream_t stream_h, double *lookups_per_s) {
    if (mode > 2 || !lookups_per_s) return DNA_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_h;
    int dev = 0;
    DNA_CUDA(cudaGetDevice(&dev));
    const DeviceProps pr = device_props(dev);
    const int grid = pr.sms ? pr.sms : 152;
    const size_t smem = kPeakWords * 4;
    int rc = ensure_smem_optin((const void *)lookup_peak_kernel, dev, smem);
    if (rc) return rc;
    void *mem = nullptr;
    rc = scratch_alloc(dev, kPeakGlobalWords * 4 + 64, stream, &mem);
    if (rc) return rc;
    uint32_t *gtab = (uint32_t *)mem;
    unsigned long long *sink = (unsigned long long *)((uint8_t *)mem + kPeakGlobalWords * 4);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const uint32_t iters = mode == 2 ? 1024u : 4096u;
    float best = 3.4e38f;
    if (e == cudaSuccess) {
        fill_global_table<<<(kPeakGlobalWords + 255) / 256, 256, 0, stream>>>(gtab);
        record_launch();
        for (int r = 0; r < 4 && e == cudaSuccess; ++r) {   // the first run warms up
            e = cudaEventRecord(e0, stream);
            lookup_peak_kernel<<<grid, kPeakThreads, smem, stream>>>(mode, iters, gtab, sink);
            record_launch();
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && r > 0 && ms < best) best = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const int rf = scratch_free(mem, stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (rf) return rf;
    const double lookups = (double)grid * kPeakThreads * kPeakChains * iters;
    *lookups_per_s = lookups / (best * 1e-3);
    return DNA_OK;
}
