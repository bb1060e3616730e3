// Instances of the persistent kernel for variant 0: the exact (6, 4, 3) variant, several blocks per SM (64 registers).
#include "bpsf_persistent.cuh"

namespace bpsf {

typedef void (*KernelFn)(KernelParams);

KernelFn kernel_fn_v0(bool debug, bool lay) {
    if (debug) return lay ? bpsf_persistent<6, 4, 3, true, BPSF_MIN_BLOCKS, true> : bpsf_persistent<6, 4, 3, true, BPSF_MIN_BLOCKS, false>;
    return lay ? bpsf_persistent<6, 4, 3, false, BPSF_MIN_BLOCKS, true> : bpsf_persistent<6, 4, 3, false, BPSF_MIN_BLOCKS, false>;
}

}  // namespace bpsf
