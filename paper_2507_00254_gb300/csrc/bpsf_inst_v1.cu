// Instances of the persistent kernel for variant 1: rows of at most 6, columns of at most 4.
#include "bpsf_persistent.cuh"

namespace bpsf {

typedef void (*KernelFn)(KernelParams);

KernelFn kernel_fn_v1(bool debug, bool lay) {
    if (debug) return lay ? bpsf_persistent<6, 4, 0, true, 1, true> : bpsf_persistent<6, 4, 0, true, 1, false>;
    return lay ? bpsf_persistent<6, 4, 0, false, 1, true> : bpsf_persistent<6, 4, 0, false, 1, false>;
}

}  // namespace bpsf
