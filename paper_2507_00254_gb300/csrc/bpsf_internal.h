// Internal layout shared by the host side and the kernels of libbpsf.
#pragma once

#include <cstdint>

namespace bpsf {

constexpr int kMaxW = 16;       // largest |Phi|
constexpr int kMaxSlots = 32;   // work items per team (one lane of the team's first warp each)
constexpr int kMaxStreams = 16; // codes per launch
constexpr int kMaxNamedTeams = 15;

// Device error bits (StreamCounters::status).
enum : unsigned {
    kDevReadyTimeout = 1u,  // a trial waited too long for its record
    kDevIdleTimeout = 2u,   // a block waited too long for other blocks
    kDevRecordOverflow = 4u // more failed shots than record slots
};

// Stream flags.
enum : unsigned {
    kNoTickets = 1u,  // do not run trials (plain form, first launch)
    kServe = 2u       // shots come from a growing request queue
};

// One code's Tanner graph in the order the kernels read it, plus the
// decoder constants.  Edges are numbered twice: CSR order (row-major,
// ascending column inside a row) and CSC order (column-major, ascending row
// inside a column); the permutations map one numbering to the other.
struct CodeDev {
    int M, N, nnz, Ws, Wn, dc_max, dv_max;
    int max_iter, short_iter, w, n_trials, select;
    float alpha;
    const uint16_t *row_ptr;     // M+1, offsets into CSR order
    const uint16_t *csr_to_csc;  // nnz
    const uint16_t *col_ptr;     // N+1, offsets into CSC order
    const uint16_t *csc_to_csr;  // nnz
    const uint16_t *csc_chk;     // nnz, check of each CSC edge
    const uint16_t *csr_col;     // nnz, column of each CSR edge
    const float *lch;            // N, channel LLRs (FP32)
    const float *lch_csr;        // nnz, channel LLR of each CSR edge's variable
    const uint32_t *trial_mask;  // n_trials subset masks over Phi, ascending
};

// Per-launch counters of one stream (64 bytes, zeroed before a launch).
struct StreamCounters {
    unsigned long long shot_next;    // next unclaimed shot
    unsigned long long init_done;    // initial runs finished
    unsigned long long ticket_next;  // trial tickets claimed
    unsigned long long iters_total;  // iterations run (all runs)
    unsigned long long trial_runs;   // trial runs finished
    unsigned int rec_count;          // failed-shot records allocated
    unsigned int status;             // kDev* bits
    unsigned long long pad[2];
};
static_assert(sizeof(StreamCounters) == 64, "counter block is one 64-byte line");

// Records of failed shots (capacity `cap`), structure of arrays.
struct Records {
    long long *shot;            // cap
    unsigned int *ready;        // cap, 1 once the record is written
    unsigned int *done;         // cap, trials finished
    unsigned long long *best;   // cap, min over converged trials of the selection key
    int32_t *phi;               // cap x w
    uint32_t *synd;             // cap x Ws, the shot's syndrome
    uint32_t *corr;             // cap x n_trials x Wn, e' xor t of converged trials
    int16_t *iters;             // cap x n_trials
    long long cap;
};

struct JobDev {
    const uint32_t *synd;
    uint32_t *corr;
    uint8_t *conv;
    int16_t *iters;
    uint8_t *stage;
    long long n_shots;
    int synd_stride, corr_stride;
};

struct DebugDev {
    float *lout;
    uint16_t *flips;
    int32_t *phi;
    uint32_t *trial_synd;
    uint8_t *trial_conv;
    int16_t *trial_iters;
};

// Serving: per-code request ring in host-mapped memory.  Shots get global
// sequence numbers; request k covers [base, base + n).
struct ServeReq {
    long long base;       // first global shot number
    long long n;          // shots
    long long arena_off;  // first arena row of its syndromes / outputs
    unsigned long long ticket;
};

struct ServeDev {
    volatile long long *published;   // shots published by the host (mapped)
    volatile ServeReq *reqs;         // request ring (mapped)
    volatile int *stop;              // host asks the loop to end when idle (mapped)
    unsigned long long *done_shots;  // per request ring slot: shots finished (device)
    volatile unsigned int *req_done; // per request ring slot: completion sequence (mapped)
    long long arena_rows;            // rows in the syndrome / output arena
    int req_cap;                     // request ring size
    long long idle_ns;               // exit after this long without work
};

struct StreamDev {
    CodeDev code;
    JobDev job;
    Records rec;
    StreamCounters *ctr;
    DebugDev dbg;
    ServeDev serve;
    int W, S;        // warps per team, slots per team
    unsigned flags;  // kNoTickets, kServe
    int pad;
};

struct LaunchArgs {
    const StreamDev *streams;
    int n_streams;
    int warps_per_block;
    unsigned long long wait_ns;  // bound on any device-side wait
};

// ---------------------------------------------------------------------------
// Shared-memory layout (identical on host and device).
// ---------------------------------------------------------------------------

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Block header: stream choice and command.
constexpr int kBlockHeaderBytes = 64;

struct LayoutOffsets {
    int row_ptr, csr_to_csc, col_ptr, csc_to_csr, lch, total;
};

__host__ __device__ inline LayoutOffsets layout_offsets(int M, int N, int nnz) {
    LayoutOffsets o;
    int p = 0;
    o.row_ptr = p;      p = align_up(p + 2 * (M + 1), 4);
    o.csr_to_csc = p;   p = align_up(p + 2 * nnz, 4);
    o.col_ptr = p;      p = align_up(p + 2 * (N + 1), 4);
    o.csc_to_csr = p;   p = align_up(p + 2 * nnz, 4);
    o.lch = p;          p = align_up(p + 4 * N, 16);
    o.total = p;
    return o;
}

// Per-slot state in shared memory (64 bytes).
struct SlotState {
    int kind;        // 0 empty, 1 initial run, 2 trial run
    int fresh;       // 1 until the first iteration has run
    int iter;        // iterations completed
    int limit;       // iteration cap of this run
    long long shot;  // shot index in the job
    int rec;         // record (trial runs)
    int kidx;        // trial index (trial runs)
    uint16_t phi[kMaxW];
};

// Team control block (32 bytes).
struct TeamCtl {
    long long chunk_next, chunk_end;  // shots claimed by the team, not yet started
    unsigned act_mask, fresh_mask, init_mask;
    int exit;
};

struct TeamOffsets {
    int ctl, state, syn, mism, ebits, flips, q, r, total;
};

__host__ __device__ inline TeamOffsets team_offsets(int S, int M, int N, int nnz, int Ws) {
    TeamOffsets o;
    int p = 0;
    o.ctl = p;    p += 32;
    o.state = p;  p += 64 * S;
    o.syn = p;    p += 4 * S * Ws;
    o.mism = p;   p += 4 * S * Ws;
    o.ebits = p;  p += 4 * ((S * N + 31) / 32 + 1);
    o.flips = p;  p = align_up(p + 2 * S * N, 16);
    o.q = p;      p += 4 * S * nnz;
    o.r = p;      p += 4 * S * nnz;
    o.total = align_up(p, 16);
    return o;
}

__host__ __device__ inline int block_smem_bytes(int M, int N, int nnz, int Ws, int S, int teams) {
    return kBlockHeaderBytes + layout_offsets(M, N, nnz).total + teams * team_offsets(S, M, N, nnz, Ws).total;
}

// Kernel entry points (bpsf_kernels.cu).
struct KernelShape {
    int dc, dv;
};
int kernel_variant(int dc_max, int dv_max);  // index of the smallest variant that fits, -1 if none
int kernel_variant_dc(int v);
int kernel_variant_dv(int v);
const void *persistent_kernel_ptr(int variant, bool debug);
void launch_persistent(int variant, bool debug, int grid, int block, int smem, const LaunchArgs &args,
                       void *stream);
void launch_syndrome(const CodeDev &cd, long long n, const uint32_t *err, int err_stride, uint32_t *synd,
                     int synd_stride, void *stream);
void launch_sample_errors(long long n, int nbits, double p, unsigned long long seed, uint32_t *err, int stride,
                          void *stream);

}  // namespace bpsf
