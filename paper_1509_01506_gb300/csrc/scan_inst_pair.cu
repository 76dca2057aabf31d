// scan_inst_pair.cu -- the MODE_PAIR variants of the chunk-scan kernel (8, 16, 24 and 32
// warps per block, with and without position records).
#include "scan_kernel.cuh"

namespace dnalib {

ScanFn scan_fn_pair(int warps, bool pos) {
    switch (warps) {
        case 8: return pos ? scan_kernel<MODE_PAIR, 8, true> : scan_kernel<MODE_PAIR, 8, false>;
        case 16: return pos ? scan_kernel<MODE_PAIR, 16, true> : scan_kernel<MODE_PAIR, 16, false>;
        case 24: return pos ? scan_kernel<MODE_PAIR, 24, true> : scan_kernel<MODE_PAIR, 24, false>;
        case 32: return pos ? scan_kernel<MODE_PAIR, 32, true> : scan_kernel<MODE_PAIR, 32, false>;
        default: return nullptr;
    }
}

}  // namespace dnalib
