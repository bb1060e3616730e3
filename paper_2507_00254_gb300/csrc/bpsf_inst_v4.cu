// Instances of the persistent kernel for variant 4: rows of at most 32, columns of at most 16.
#include "bpsf_persistent.cuh"

namespace bpsf {

typedef void (*KernelFn)(KernelParams);

KernelFn kernel_fn_v4(bool debug, bool lay) {
    if (debug) return lay ? bpsf_persistent<32, 16, 0, true, 1, true> : bpsf_persistent<32, 16, 0, true, 1, false>;
    return lay ? bpsf_persistent<32, 16, 0, false, 1, true> : bpsf_persistent<32, 16, 0, false, 1, false>;
}

}  // namespace bpsf
