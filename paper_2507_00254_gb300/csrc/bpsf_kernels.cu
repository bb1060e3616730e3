// Dispatch over the persistent kernel's variants and instances, and the two
// small harness kernels (syndrome, error sampler) of libbpsf.  The kernel's
// device code is in bpsf_persistent.cuh; each variant is instantiated in its
// own translation unit (bpsf_inst_*.cu).
#include <cuda_runtime.h>

#include <cstdint>

#include "bpsf_internal.h"

namespace bpsf {

typedef void (*KernelFn)(KernelParams);

// Per-variant instance tables (bpsf_inst_*.cu): the kernel for (debug, layered).
KernelFn kernel_fn_v0(bool debug, bool lay);
KernelFn kernel_fn_v1(bool debug, bool lay);
KernelFn kernel_fn_v2(bool debug, bool lay);
KernelFn kernel_fn_v3(bool debug, bool lay);
KernelFn kernel_fn_v4(bool debug, bool lay);
KernelFn kernel_fn_v5(bool debug, bool lay);
KernelFn kernel_fn_v6(bool debug, bool lay);
KernelFn kernel_fn_v7(bool debug, bool lay);

// ---------------------------------------------------------------------------
// Variants and launch helpers.
// ---------------------------------------------------------------------------

struct Variant {
    int dc, dvs, dvx;  // row-degree bound, column table width, exact column degree (0 = any)
};
// Index 5 is the full-register instance of variant 0 and index 6 the same
// with one-byte flip words; index 7 is variant 2 with the exact (6, 4, 3)
// path for the codes that have it (none is chosen by kernel_variant; see
// kernel_variant_full_regs, kernel_variant_byte_flips and
// kernel_variant_mixed).
static const Variant kVariants[] = {{6, 4, 3}, {6, 4, 0}, {8, 4, 0}, {16, 8, 0}, {32, 16, 0}, {6, 4, 3}, {6, 4, 3},
                                    {8, 4, 0}};
static const int kNumVariants = 5;

// Smallest variant that fits.  The exact-degree variant serves codes with
// exactly dc ones in every row and dvx in every column; the caller marks
// such codes by passing dc_max = -dc.
int kernel_variant(int dc_max, int dv_max) {
    const bool regular = dc_max < 0;
    const int dc = regular ? -dc_max : dc_max;
    for (int v = 0; v < kNumVariants; ++v) {
        const Variant &k = kVariants[v];
        if (k.dvx > 0) {
            if (regular && dc == k.dc && dv_max == k.dvx) return v;
            continue;
        }
        if (dc <= k.dc && dv_max <= k.dvs) return v;
    }
    return -1;
}

static KernelFn kernel_fn(int variant, bool debug, bool lay) {
    switch (variant) {
        case 0: return kernel_fn_v0(debug, lay);
        case 1: return kernel_fn_v1(debug, lay);
        case 2: return kernel_fn_v2(debug, lay);
        case 3: return kernel_fn_v3(debug, lay);
        case 4: return kernel_fn_v4(debug, lay);
        case 5: return kernel_fn_v5(debug, lay);
        case 6: return kernel_fn_v6(debug, lay);
        default: return kernel_fn_v7(debug, lay);
    }
}

int kernel_variant_dv(int variant) { return kVariants[variant].dvs; }

// The full-register instance of a variant (itself when it has only one).
int kernel_variant_full_regs(int variant) { return variant == 0 ? 5 : variant; }

// The instance with one-byte flip words (full registers, no layered path), or -1.
int kernel_variant_byte_flips(int variant) { return (variant == 0 || variant == 5) ? 6 : -1; }

// The instance that runs variant 2's codes together with exact (6, 4, 3)
// codes on their own path, or -1.
int kernel_variant_mixed(int variant) { return variant == 2 ? 7 : -1; }

const void *persistent_kernel_ptr(int variant, bool debug, bool layered) {
    return reinterpret_cast<const void *>(kernel_fn(variant, debug, layered));
}

void launch_persistent(int variant, bool debug, bool layered, int grid, int block, int smem, const LaunchArgs &args,
                       void *stream) {
    KernelParams kp;
    for (int k = 0; k < args.n_streams; ++k) kp.streams[k] = args.streams[k];
    kp.n_streams = args.n_streams;
    kp.Q = args.Q;
    kp.wait_ns = args.wait_ns;
    kernel_fn(variant, debug, layered)<<<grid, block, smem, (cudaStream_t)stream>>>(kp);
}

// ---------------------------------------------------------------------------
// Harness kernels.
// ---------------------------------------------------------------------------

// s = H e (mod 2): one thread per (shot, syndrome word).
__global__ void syndrome_kernel(const uint16_t *row_ptr, const uint16_t *csr_col, int M, int Ws, long long n,
                                const uint32_t *err, int err_stride, uint32_t *synd, int synd_stride) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * Ws) return;
    const long long shot = t / Ws;
    const int w = (int)(t - shot * Ws);
    const uint32_t *e = err + shot * err_stride;
    unsigned out = 0;
    for (int b = 0; b < 32; ++b) {
        const int j = 32 * w + b;
        if (j >= M) break;
        unsigned par = 0;
        for (int k = row_ptr[j]; k < row_ptr[j + 1]; ++k) {
            const int c = csr_col[k];
            par ^= (__ldg(e + (c >> 5)) >> (c & 31)) & 1u;
        }
        out |= par << b;
    }
    synd[shot * synd_stride + w] = out;
}

// Product-internal error sampler for the autotuner (independent hash).
__device__ __forceinline__ unsigned long long hash64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

__global__ void sample_errors_kernel(long long n, int nbits, unsigned long long thr, unsigned long long seed,
                                     uint32_t *err, int stride) {
    const int Wn = (nbits + 31) / 32;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * Wn) return;
    const long long shot = t / Wn;
    const int w = (int)(t - shot * Wn);
    unsigned out = 0;
    for (int b = 0; b < 32 && 32 * w + b < nbits; ++b) {
        const unsigned long long u = hash64(seed ^ ((unsigned long long)shot * 0x9E3779B97F4A7C15ull) ^
                                            (unsigned long long)(32 * w + b) * 0xD1B54A32D192ED03ull);
        out |= ((u >> 11) < thr ? 1u : 0u) << b;
    }
    err[shot * stride + w] = out;
}

void launch_syndrome(const CodeDev &cd, long long n, const uint32_t *err, int err_stride, uint32_t *synd,
                     int synd_stride, void *stream) {
    const long long total = n * cd.Ws;
    if (total <= 0) return;
    const int block = 256;
    const long long grid = (total + block - 1) / block;
    syndrome_kernel<<<(unsigned)grid, block, 0, (cudaStream_t)stream>>>(cd.row_ptr, cd.csr_col, cd.M, cd.Ws, n, err,
                                                                       err_stride, synd, synd_stride);
}

void launch_sample_errors(long long n, int nbits, double p, unsigned long long seed, uint32_t *err, int stride,
                          void *stream) {
    const int Wn = (nbits + 31) / 32;
    const long long total = n * Wn;
    if (total <= 0) return;
    const unsigned long long thr = (unsigned long long)(p * 9007199254740992.0);
    const int block = 256;
    const long long grid = (total + block - 1) / block;
    sample_errors_kernel<<<(unsigned)grid, block, 0, (cudaStream_t)stream>>>(n, nbits, thr, seed, err, stride);
}

}  // namespace bpsf
