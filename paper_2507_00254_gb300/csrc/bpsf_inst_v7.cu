// Instances of the persistent kernel for variant 7: rows of at most 8 and
// columns of at most 4 (variant 2's team loop) together with the exact
// (6, 4, 3) team loop, chosen per code of the launch (mixed-code launches and
// servers over codes of both kinds, none of them layered).
#include "bpsf_persistent.cuh"

namespace bpsf {

typedef void (*KernelFn)(KernelParams);

KernelFn kernel_fn_v7(bool debug, bool lay) {
    if (lay) return nullptr;  // launches with a layered code do not use this instance
    return debug ? bpsf_persistent<8, 4, 0, true, 1, false, 2, true> : bpsf_persistent<8, 4, 0, false, 1, false, 2, true>;
}

}  // namespace bpsf
