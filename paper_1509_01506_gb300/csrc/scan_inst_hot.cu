// scan_inst_hot.cu -- the MODE_HOT variants of the chunk-scan kernel (hot-state two-symbol
// rows in shared memory; 8 and 16 warps per block, with and without position records).
#include "scan_kernel.cuh"

namespace dnalib {

ScanFn scan_fn_hot(int warps, bool pos) {
    switch (warps) {
        case 8: return pos ? scan_kernel<MODE_HOT, 8, true> : scan_kernel<MODE_HOT, 8, false>;
        case 16: return pos ? scan_kernel<MODE_HOT, 16, true> : scan_kernel<MODE_HOT, 16, false>;
        default: return nullptr;
    }
}

}  // namespace dnalib
