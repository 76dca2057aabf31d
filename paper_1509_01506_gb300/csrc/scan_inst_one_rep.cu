// scan_inst_one_rep.cu -- the MODE_ONE_REP variants of the chunk-scan kernel (one-symbol
// table copied once per lane in shared memory; 8, 16 and 24 warps per block, with and
// without position records).
#include "scan_kernel.cuh"

namespace dnalib {

ScanFn scan_fn_one_rep(int warps, bool pos) {
    switch (warps) {
        case 8: return pos ? scan_kernel<MODE_ONE_REP, 8, true> : scan_kernel<MODE_ONE_REP, 8, false>;
        case 16: return pos ? scan_kernel<MODE_ONE_REP, 16, true> : scan_kernel<MODE_ONE_REP, 16, false>;
        case 24: return pos ? scan_kernel<MODE_ONE_REP, 24, true> : scan_kernel<MODE_ONE_REP, 24, false>;
        default: return nullptr;
    }
}

}  // namespace dnalib
