// Host-side context of libbpsf, shared by the decode and serving code.
#pragma once

#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bpsf.h"
#include "bpsf_internal.h"

// NVTX range over a host entry point or one of its steps (shown by profilers
// that record NVTX; a no-op otherwise).
struct BpsfRange {
    explicit BpsfRange(const char *name) { nvtxRangePushA(name); }
    ~BpsfRange() { nvtxRangePop(); }
    BpsfRange(const BpsfRange &) = delete;
    BpsfRange &operator=(const BpsfRange &) = delete;
};

struct bpsf_ctx {
    int device = 0, sm_count = 0, smem_optin = 0;
    int M = 0, N = 0, nnz = 0, Ws = 0, Wn = 0, dc_max = 0, dv_max = 0, n_trials = 0, variant = 0;
    int P = 0, vstride = 0, regular = 0;
    bpsf_params p{};
    std::vector<int32_t> csr_ptr, csr_col;  // host copy of H (CSR, ascending columns)
    void *d_code = nullptr;                 // one allocation for all code arrays
    void *d_trials = nullptr;               // trial list set by bpsf_set_trials (else the default in d_code)
    void *d_layouts = nullptr;              // per-slot-count message layouts (CodeDev::lay)
    const unsigned long long *default_masks = nullptr;
    int default_n_trials = 0;
    bpsf::CodeDev code{};
    bpsf::StreamCounters *d_ctr = nullptr;  // per-launch counters, one block per shard (kMaxStreams)
    bpsf::StreamCounters *d_ctr_last = nullptr;  // counters of the most recent launch (read by bpsf_sync)
    bpsf::StreamCounters *h_ctr = nullptr;  // pinned copy read by bpsf_sync
    bpsf::StreamCounters *h_preset = nullptr;
    uint8_t *h_flag = nullptr;              // pinned flag read by the plain form
    void *d_rec = nullptr;                  // failed-shot records
    bpsf::Records rec{};
    long long rec_cap = 0;
    void *d_host_stage = nullptr;           // device buffers of bpsf_decode_host
    size_t host_stage_bytes = 0;
    bpsf_tuning tune{};
    bpsf_work last{};
    long long last_launch_n = 0;
    int last_shards = 1;                    // shards of the last launch (counter blocks bpsf_sync adds up)
};

// A batch is decoded as up to kMaxShards shards: contiguous shot ranges, each
// its own stream of the launch with its own counters and its own slice of the
// record ring (so the blocks' claims spread over several sets of counters).
constexpr int kMaxShards = 4;
constexpr long long kMinShardShots = 8192;
constexpr int kMaxShardNnz = 2048;  // larger codes: few, long runs per block, and a costly table reload per stream
int bpsf_batch_shards(const bpsf_ctx *c, long long n, int n_jobs);
// Workspace for n shots in `shards` shards; *shard_cap = records per shard.
bpsf_status bpsf_ensure_workspace_sharded(bpsf_ctx *c, long long n, int shards, long long *shard_cap);
// The streams of one job's shards (counters and ring slices of ctx c).
void bpsf_shard_streams(const bpsf_ctx *c, const bpsf::JobDev &job, int shards, long long shard_cap,
                        const bpsf::DebugDev *dbg, bpsf::StreamDev *out);

// Launch plan of the persistent kernel for one or several codes.
struct bpsf_plan {
    int variant = 0, Q = 0, block = 0, smem = 0, grid = 0;
    bool layered = false;  // some code of the launch uses the layered schedule
    int S_code[bpsf::kMaxStreams] = {0};      // slots per team, per code of the launch
    int W_code[bpsf::kMaxStreams] = {0};      // warps per team, per code
    int teams_code[bpsf::kMaxStreams] = {0};  // teams per block, per code
    int chunk_code[bpsf::kMaxStreams] = {0};  // iterations between refills, per code
};

bpsf_status bpsf_fail(bpsf_status s, const char *fmt, ...);

// Records for n shots: the smallest power of two >= n (a batch has at most n
// failed shots, a server at most its admitted shots in flight).
inline long long bpsf_record_ring(long long n) {
    long long r = 1;
    while (r < n) r <<= 1;
    return r;
}

// A ring of `rows` failed-shot records in one block of memory, each array
// aligned to `al` bytes: bytes needed, and the arrays carved from `base`.
inline size_t bpsf_records_bytes(long long rows, int w, int Ws, int Wn, size_t al) {
    const size_t r = (size_t)(rows > 0 ? rows : 1), ww = (size_t)(w > 0 ? w : 1);
    auto A = [al](size_t x) { return (x + al - 1) / al * al; };
    return A(8 * r) + A(8 * r) + A(4 * r) + A(8 * r) + A(8 * r * (size_t)Wn) + A(4 * r * ww) + A(4 * r * (size_t)Ws);
}
inline bpsf::Records bpsf_records_carve(void *base, long long rows, int w, int Ws, int Wn, size_t al) {
    const size_t r = (size_t)(rows > 0 ? rows : 1), ww = (size_t)(w > 0 ? w : 1);
    auto A = [al](size_t x) { return (x + al - 1) / al * al; };
    unsigned char *p = static_cast<unsigned char *>(base);
    bpsf::Records rec;
    rec.qseq = reinterpret_cast<unsigned long long *>(p);
    p += A(8 * r);
    rec.qshot = reinterpret_cast<long long *>(p);
    p += A(8 * r);
    rec.done = reinterpret_cast<unsigned *>(p);
    p += A(4 * r);
    rec.best = reinterpret_cast<unsigned long long *>(p);
    p += A(8 * r);
    rec.win = reinterpret_cast<unsigned long long *>(p);
    p += A(8 * r * (size_t)Wn);
    rec.phi = reinterpret_cast<int32_t *>(p);
    p += A(4 * r * ww);
    rec.synd = reinterpret_cast<uint32_t *>(p);
    rec.cap = (long long)r;
    return rec;
}

// Index of the layout for S slots per team (S a power of two, 1..32).
inline int layout_index(int S) {
    int i = 0;
    while ((1 << i) < S && i < bpsf::kNumLayouts - 1) ++i;
    return i;
}

// Make the layout for S slots per team the active one of a code descriptor.
inline void bpsf_activate_layout(bpsf::CodeDev &cd, int S) {
    const bpsf::LayoutS &ly = cd.lay[layout_index(S)];
    cd.Mp = ly.Mp;
    cd.P = ly.P;
    cd.vpos = ly.vpos;
    cd.lch_pos = ly.lch_pos;
    cd.pos_var = ly.pos_var;
}

// A context with trials (w > 0) decodes only with a non-empty trial set.
inline bpsf_status bpsf_check_trials(const bpsf_ctx *c) {
    if (c->p.w > 0 && c->n_trials == 0)
        return bpsf_fail(BPSF_EINVAL, "the default trial set is too large; give a trial list (bpsf_set_trials)");
    return BPSF_OK;
}
bpsf_status bpsf_ensure_workspace(bpsf_ctx *c, long long n);
bpsf_status bpsf_ensure_kernel_attrs(int variant, int smem_optin);
// Plan one launch over n_codes codes; tunes[k] is code k's team shape (a
// single tuning for a one-code launch).  With shrink, a code whose block does
// not fit gets fewer slots per team, then fewer teams.
bpsf_status bpsf_make_plan(bpsf_ctx *const *codes, int n_codes, const bpsf_tuning *tunes, bool debug,
                           bpsf_plan *out, bool shrink = false);
void bpsf_launch_plan(const bpsf_plan &pl, bool debug, bpsf::StreamDev *sds, int n, int grid, void *stream);
bool bpsf_tuning_cache_lookup(const bpsf_ctx *c, bpsf_tuning *out);
bpsf::StreamDev bpsf_make_stream(const bpsf_ctx *c, const bpsf::JobDev &job, const bpsf::DebugDev *dbg,
                                 unsigned flags);
extern const unsigned long long kBpsfWaitNs;
