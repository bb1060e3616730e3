// Instances of the persistent kernel for variant 6: the exact (6, 4, 3)
// variant, one block per SM with the full register budget and one-byte flip
// words (launches whose codes all have max_iter <= 127 and no layered
// schedule).  There is no layered instance: the plan never asks for one.
#include "bpsf_persistent.cuh"

namespace bpsf {

typedef void (*KernelFn)(KernelParams);

KernelFn kernel_fn_v6(bool debug, bool lay) {
    if (lay) return nullptr;
    return debug ? bpsf_persistent<6, 4, 3, true, 1, false, 1> : bpsf_persistent<6, 4, 3, false, 1, false, 1>;
}

}  // namespace bpsf
