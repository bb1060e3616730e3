// Instances of the persistent kernel for variant 2: rows of at most 8, columns of at most 4.
#include "bpsf_persistent.cuh"

namespace bpsf {

typedef void (*KernelFn)(KernelParams);

KernelFn kernel_fn_v2(bool debug, bool lay) {
    if (debug) return lay ? bpsf_persistent<8, 4, 0, true, 1, true> : bpsf_persistent<8, 4, 0, true, 1, false>;
    return lay ? bpsf_persistent<8, 4, 0, false, 1, true> : bpsf_persistent<8, 4, 0, false, 1, false>;
}

}  // namespace bpsf
