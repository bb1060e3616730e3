// bpsf_decode_noalloc: the batched decode for callers that cannot allocate
// device memory when they decode -- a control loop with a hard deadline that
// must never block inside the CUDA allocator, or a host runtime that hands
// the whole device heap to another framework's allocator.  Such callers
// create their context once at set-up and then decode without any further
// allocation: the kernel's scratch (launch counters and failed-shot records)
// lives in one statically sized device array defined in this file, which
// every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "bpsf.h"
#include "bpsf_api_internal.h"
#include "bpsf_internal.h"

using namespace bpsf;

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;  // 32 MiB per device

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kMaxDevices];  // device address of the array, per device

// The array's name in host code is only a stand-in; its device address comes
// from cudaGetSymbolAddress, asked once per device with that device current.
bpsf_status noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return bpsf_fail(BPSF_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return bpsf_fail(BPSF_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_noalloc_ptr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[device];
    return BPSF_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of scratch for a ring of `ring` failed-shot records (counters first).
size_t noalloc_bytes(const bpsf_ctx *c, long long ring) {
    return align256(sizeof(StreamCounters)) + bpsf_records_bytes(ring, c->p.w, c->Ws, c->Wn, 256);
}

// The largest record ring (a power of two) that fits the static scratch for
// this code; 0 if not even one record fits.  Every record is at least 44
// bytes, so the search starts below 2^20 and no product can wrap.
long long noalloc_ring(const bpsf_ctx *c) {
    long long r = 1ll << 20;
    while (r >= 1 && noalloc_bytes(c, r) > kNoallocScratchBytes) r >>= 1;
    return r;
}

}  // namespace

// A batch of n shots needs a ring of at least n records.
extern "C" int64_t bpsf_noalloc_max_shots(const bpsf_ctx *c) {
    if (!c) return -1;
    return noalloc_ring(c);
}

extern "C" bpsf_status bpsf_decode_noalloc(bpsf_ctx *c, int64_t n, const uint32_t *synd, int32_t ss, uint32_t *corr,
                                           int32_t cs, uint8_t *conv, int16_t *iters, uint8_t *stage, void *stream) {
    if (!c) return bpsf_fail(BPSF_EINVAL, "ctx is NULL");
    if (n < 0) return bpsf_fail(BPSF_EINVAL, "n_shots must be >= 0");
    // The bound comes first (no size arithmetic depends on n beyond it).
    const long long max_n = bpsf_noalloc_max_shots(c);
    if (n > max_n)
        return bpsf_fail(BPSF_EINVAL,
                         "n_shots = %lld does not fit the static scratch of %zu bytes "
                         "(at most %lld shots of this code per call)",
                         (long long)n, kNoallocScratchBytes, max_n);
    if (bpsf_check_trials(c) != BPSF_OK) return BPSF_EINVAL;
    if (n == 0) return BPSF_OK;
    if (!synd || !corr || !conv || !iters) return bpsf_fail(BPSF_EINVAL, "NULL input or output pointer");
    if (ss < c->Ws) return bpsf_fail(BPSF_EINVAL, "synd_stride_words %d < Ws = %d", ss, c->Ws);
    if (cs < c->Wn) return bpsf_fail(BPSF_EINVAL, "corr_stride_words %d < Wn = %d", cs, c->Wn);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    unsigned char *base = nullptr;
    bpsf_status st = noalloc_scratch(c->device, &base);
    if (st != BPSF_OK) return st;
    bpsf_plan pl;
    bpsf_ctx *cs1[1] = {c};
    st = bpsf_make_plan(cs1, 1, &c->tune, false, &pl);
    if (st != BPSF_OK) return st;
    // Carve the counters and the record ring out of the array.
    const long long ring = bpsf_record_ring(n);
    StreamCounters *ctr = reinterpret_cast<StreamCounters *>(base);
    Records rec = bpsf_records_carve(base + align256(sizeof(StreamCounters)), ring, c->p.w, c->Ws, c->Wn, 256);
    // The array keeps the previous call's contents: the counters must start
    // at zero and every record free.  Every other record field is written
    // before it is read.
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(ctr, 0, sizeof(StreamCounters), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rec.qseq, 0, 8 * (size_t)ring, s);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    JobDev job{synd, corr, conv, iters, stage, n, ss, cs};
    StreamDev sd = bpsf_make_stream(c, job, nullptr, 0);
    sd.ctr = ctr;
    sd.rec = rec;
    bpsf_launch_plan(pl, false, &sd, 1, pl.grid, stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    // The next call reuses the array's counters, so this call's counters go
    // to the context's own block, in stream order after the kernel (a copy
    // between device buffers, no allocation); bpsf_sync reads them there
    // even when another no-allocation call has run since.
    e = cudaMemcpyAsync(c->d_ctr, ctr, sizeof(StreamCounters), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "counter copy: %s", cudaGetErrorString(e));
    c->d_ctr_last = c->d_ctr;
    c->last_shards = 1;
    c->last_launch_n = n;
    return BPSF_OK;
}
