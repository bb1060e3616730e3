// Instances of the persistent kernel for variant 5: the exact (6, 4, 3) variant, one block per SM with the full register budget.
#include "bpsf_persistent.cuh"

namespace bpsf {

typedef void (*KernelFn)(KernelParams);

KernelFn kernel_fn_v5(bool debug, bool lay) {
    if (debug) return lay ? bpsf_persistent<6, 4, 3, true, 1, true> : bpsf_persistent<6, 4, 3, true, 1, false>;
    return lay ? bpsf_persistent<6, 4, 3, false, 1, true> : bpsf_persistent<6, 4, 3, false, 1, false>;
}

}  // namespace bpsf
