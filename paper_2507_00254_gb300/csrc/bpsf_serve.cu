// Serving form of libbpsf (continuous batching).  Placeholder entry points
// until the request loop lands.
#include "bpsf.h"
#include "bpsf_api_internal.h"

extern "C" bpsf_status bpsf_serve_start(bpsf_server **out, bpsf_ctx *const *, int32_t, const bpsf_serve_cfg *) {
    if (out) *out = nullptr;
    return bpsf_fail(BPSF_EINVAL, "serving is not available in this build");
}
extern "C" bpsf_status bpsf_serve_submit(bpsf_server *, int32_t, int64_t, const uint32_t *, int64_t, uint64_t *) {
    return bpsf_fail(BPSF_EINVAL, "serving is not available in this build");
}
extern "C" bpsf_status bpsf_serve_poll(bpsf_server *, uint64_t, int64_t, uint32_t *, uint8_t *, int16_t *, uint8_t *) {
    return bpsf_fail(BPSF_EINVAL, "serving is not available in this build");
}
extern "C" bpsf_status bpsf_serve_stop(bpsf_server *) {
    return bpsf_fail(BPSF_EINVAL, "serving is not available in this build");
}
