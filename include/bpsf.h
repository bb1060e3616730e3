/*
 * bpsf.h — C ABI of libbpsf, a GB300 (sm_103a) decoder for quantum LDPC codes
 * implementing BP-SF: normalised min-sum belief propagation with oscillation
 * tracking, followed by speculative syndrome-flip trials, from
 * "Fully Parallelized BP Decoding for Quantum LDPC Codes Can Outperform
 * BP-OSD" (Wang, Li, Mueller; arXiv 2507.00254).
 *
 * The problem (Section II-B, "Decoding Problem"): given a parity-check matrix
 * H in F_2^{M x N} and a syndrome s in F_2^M, find e in F_2^N with
 * e H^T = s.  The decoder is Algorithm 1 (BP-SF): an initial min-sum run
 * (Section II-B, Eq. c2v) with per-bit flip counters; if it does not
 * converge, Phi = the |Phi| = w most-flipped bits, every non-empty subset t
 * of Phi with |t| <= w_max gives a trial syndrome s' = s xor t H^T, each
 * trial is decoded by a fresh short BP, and a converged trial returns e' xor t.
 *
 * Conventions used by every entry point:
 *   - Bit vectors are packed into uint32 words, least significant bit first:
 *     bit i of a vector lives in word i / 32 at position i % 32.  A syndrome
 *     takes Ws = ceil(M / 32) words, a correction Wn = ceil(N / 32) words.
 *     Rows of a batch are `stride` words apart (stride >= Ws or Wn).
 *   - Pointers named d_* are device pointers on the current CUDA device;
 *     h_* are host pointers.  The caller owns every input and output buffer.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Device calls are asynchronous on that stream; bpsf_sync() waits and
 *     reports errors the device found (timeouts, record overflow).
 *   - Every function returns a bpsf_status and never aborts or throws; on
 *     failure bpsf_last_error() gives a message for the calling thread.
 *   - A context holds per-launch counters and workspace: decode calls on one
 *     context must not overlap (one thread, one stream at a time).  Servers
 *     keep their own device state and may run beside such calls.
 *   - Messages are FP32.  Each add and multiply is rounded on its own, in
 *     one fixed order (V2C and posterior sums fold from the channel LLR over
 *     the checks of a column in ascending check index), so results do not
 *     depend on the launch shape.
 */
#ifndef BPSF_H
#define BPSF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BPSF_OK = 0,
    BPSF_EINVAL = 1,    /* invalid argument (message in bpsf_last_error) */
    BPSF_ENOMEM = 2,    /* device or pinned allocation failed, or a cap was hit */
    BPSF_ECUDA = 3,     /* a CUDA runtime call failed */
    BPSF_ETIMEOUT = 4,  /* a bounded wait ran out (device spin or host poll) */
    BPSF_EBUSY = 5,     /* no room right now (serving admission) */
    BPSF_ECLOSED = 6,   /* the server was stopped */
    BPSF_EDEVICE = 7    /* the device reported an internal error */
} bpsf_status;

typedef enum { BPSF_CSR = 0, BPSF_CSC = 1 } bpsf_layout;

enum { BPSF_SELECT_MIN_WEIGHT = 0, BPSF_SELECT_FIRST = 1 };
enum { BPSF_FLAG_LAYERED = 1 };

/*
 * Decoder parameters (Algorithm 1 inputs plus the min-sum settings of
 * Section II-B).
 *   max_iter   iterations of the initial run (i_max of Algorithm 1), 1..32767.
 *   alpha      normalisation factor of Eq. (c2v), finite and > 0; or 0 for
 *              adaptive damping alpha_t = 1 - 2^-t at iteration t = 1, 2, ...
 *              of every run (Section V's schedule, printed there as
 *              "1 - 2^i"), rounded once to float.  C2V magnitudes are
 *              clamped at 2^100 (never reached with a fixed alpha at the
 *              configurations; with alpha_t -> 1 it keeps messages finite).
 *   w          |Phi|, the number of oscillating bits used for trials,
 *              0..64; 0 means plain BP with no post-processing.
 *   w_max      largest trial weight, 1..min(w, 16); 0 means w.  The default
 *              trial set is every non-empty subset of Phi of weight <= w_max;
 *              bpsf_set_trials replaces it.  When that set would exceed 4096
 *              trials it is left empty, and decoding (every form) returns
 *              BPSF_EINVAL until a list is given.
 *   short_iter iterations of each trial run, 1..max_iter.
 *   select     BPSF_SELECT_MIN_WEIGHT: the converged trial whose e' xor t has
 *              the smallest Hamming weight, ties to the earlier trial (the
 *              default set is in ascending subset mask);
 *              BPSF_SELECT_FIRST: the earliest converged trial (the paper's
 *              "first valid" rule made deterministic).
 *   flags      BPSF_FLAG_LAYERED: the layered schedule (the paper's variant for
 *              the [[288]] code) instead of flooding: rows are coloured
 *              greedily in ascending order into layers of rows that share no
 *              variable; layer by layer, each row takes its V2C messages out
 *              of the running posterior (q = L - r), computes its C2V
 *              messages by Eq. (c2v) and puts them back (L = q + r).  Other
 *              bits must be 0.
 */
typedef struct {
    int32_t max_iter;
    float alpha;
    int32_t w;
    int32_t w_max;
    int32_t short_iter;
    int32_t select;
    uint32_t flags;
} bpsf_params;

typedef struct bpsf_ctx bpsf_ctx;

/*
 * Create a decoder for one code (H) and one prior vector.
 *   M, N       rows (checks) and columns (variables) of H, 1..65535.
 *   nnz        ones in H, 1..65535.
 *   layout     BPSF_CSR: ptr has M+1 entries and idx holds column indices;
 *              BPSF_CSC: ptr has N+1 entries and idx holds row indices.
 *   ptr, idx   host arrays, copied; indices in range, no duplicates.  Every
 *              row needs at least two ones (a check of degree one has no
 *              "other" variable in Eq. c2v); rows of degree > 32 or columns
 *              of degree > 16 are rejected.
 *   priors     host array of N error probabilities p_i in (0, 0.5); the
 *              channel LLR log((1 - p_i) / p_i) (Section II-B, step 1) is
 *              computed in double and rounded once to float.
 *   params     decoder parameters (see bpsf_params).
 * The context allocates device memory on the current device and owns it.
 */
bpsf_status bpsf_create(bpsf_ctx **out, int32_t M, int32_t N, int64_t nnz, int32_t layout, const int32_t *ptr,
                        const int32_t *idx, const double *priors, const bpsf_params *params);

/* Release a context and its device memory (NULL is ignored).  Wait for the
 * context's work to finish first. */
void bpsf_destroy(bpsf_ctx *ctx);

/*
 * Batched BP-SF (Algorithm 1 on every shot): one persistent launch decodes
 * all n_shots syndromes and all of their trial runs.  Work items are the
 * initial runs and the trials of failed shots; thread teams take items from
 * a device-wide queue, retire converged runs early and refill free slots.
 *   d_synd       n_shots rows of Ws words (padding bits beyond M ignored).
 *   d_corr       n_shots rows of Wn words: the returned correction e.
 *   d_converged  n_shots bytes: 1 if e H^T = s holds for the returned e.
 *   d_iters      n_shots int16: iterations of the run whose e is returned.
 *   d_stage      n_shots bytes (nullable): 0 initial run converged, 1 a
 *                trial converged, 2 failure (the initial run's e is returned).
 * Results depend only on the inputs (not on timing or launch shape).  The
 * workspace holds one record per failed shot, in failure order (a power of
 * two >= n_shots records, about 100 bytes each for [[144,12,12]] at w = 6);
 * a call with a larger n_shots than before grows it, so capture such calls
 * in a CUDA graph only after a warm-up call.  A batch of at least 16384
 * shots of a code with at most 2048 edges runs as 2 or 4 shards (contiguous
 * shot ranges with their own claim counters and record slices, one launch);
 * this changes no result, and bpsf_last_work reports their sums.
 */
bpsf_status bpsf_decode(bpsf_ctx *ctx, int64_t n_shots, const uint32_t *d_synd, int32_t synd_stride_words,
                        uint32_t *d_corr, int32_t corr_stride_words, uint8_t *d_converged, int16_t *d_iters,
                        uint8_t *d_stage, void *stream);

/*
 * Plain per-shot form (the baseline the batched form is compared with):
 * for each shot, launch the initial run alone, synchronise and read its
 * stage; on failure launch that shot's trial sweep and synchronise again.
 * Same arguments and results as bpsf_decode; returns after the last shot.
 */
bpsf_status bpsf_decode_plain(bpsf_ctx *ctx, int64_t n_shots, const uint32_t *d_synd, int32_t synd_stride_words,
                              uint32_t *d_corr, int32_t corr_stride_words, uint8_t *d_converged, int16_t *d_iters,
                              uint8_t *d_stage, void *stream);

/*
 * End-to-end form with HOST buffers: copies the syndromes to the device,
 * runs bpsf_decode and copies the results back, all on `stream`, and
 * returns when the results are in the host buffers.  Pinned buffers give
 * full copy bandwidth.  h_stage is nullable.
 */
bpsf_status bpsf_decode_host(bpsf_ctx *ctx, int64_t n_shots, const uint32_t *h_synd, int32_t synd_stride_words,
                             uint32_t *h_corr, int32_t corr_stride_words, uint8_t *h_converged, int16_t *h_iters,
                             uint8_t *h_stage, void *stream);

/* One batch of one code for bpsf_decode_multi (fields as in bpsf_decode). */
typedef struct {
    bpsf_ctx *ctx;
    int64_t n_shots;
    const uint32_t *d_synd;
    int32_t synd_stride_words;
    uint32_t *d_corr;
    int32_t corr_stride_words;
    uint8_t *d_converged;
    int16_t *d_iters;
    uint8_t *d_stage;
} bpsf_job;

/*
 * Mixed-code batch: all jobs (codes of different sizes) decode in ONE
 * persistent launch; thread blocks move to another code when theirs runs
 * out of work.  At most 16 jobs; all contexts on the current device.
 */
bpsf_status bpsf_decode_multi(int32_t n_jobs, const bpsf_job *jobs, void *stream);

/*
 * End-to-end mixed-code batch with HOST buffers: the jobs' five array fields
 * hold host addresses here (pinned memory gives full copy bandwidth).  Each
 * job's syndromes are copied into its context's device staging buffer, all
 * jobs decode in ONE bpsf_decode_multi launch, and the results are copied
 * back, all on `stream`; the call returns when the results are in the host
 * buffers.  Same limits and results as bpsf_decode_multi; jobs with
 * n_shots = 0 are checked and then left out of the launch.  A context's
 * staging buffer is shared with bpsf_decode_host: calls on one context must
 * not overlap.
 */
bpsf_status bpsf_decode_multi_host(int32_t n_jobs, const bpsf_job *jobs, void *stream);

/*
 * Batched decode that allocates nothing.  The paper has no counterpart: this
 * serves callers that cannot allocate device memory when they decode (a
 * control loop with a hard deadline that must not block in the CUDA
 * allocator, or a runtime whose own allocator owns the whole device heap).
 * It runs the same kernel as bpsf_decode with the same
 * arguments and results, but the kernel's scratch (launch counters and the
 * ring of records of failed shots in flight) lives in one static 32 MiB
 * device array that every GPU loading this library holds until the process
 * exits.
 *   - At most bpsf_noalloc_max_shots(ctx) shots per call (the records the
 *     array holds for this code: 262144 for [[144,12,12]] at w = 6, 32768 for
 *     its 12-round phenomenological code); larger batches get BPSF_EINVAL and
 *     nothing runs.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents;
 *     each call clears what must start at zero.  Calls that overlap on the
 *     GPU (on different streams, or from several contexts) race on the
 *     array: order them on one stream.
 *   - The context must already exist (bpsf_create allocates at set-up).
 * After the kernel, the call copies its launch counters into ctx's own
 * counter block on `stream` (a device-to-device copy), so bpsf_sync(ctx,
 * stream) and bpsf_last_work report this call's device-side errors and work
 * even when further no-allocation calls have been queued since.
 */
bpsf_status bpsf_decode_noalloc(bpsf_ctx *ctx, int64_t n_shots, const uint32_t *d_synd, int32_t synd_stride_words,
                                uint32_t *d_corr, int32_t corr_stride_words, uint8_t *d_converged, int16_t *d_iters,
                                uint8_t *d_stage, void *stream);

/* Largest n_shots bpsf_decode_noalloc accepts for this context (-1 for NULL,
 * 0 if not even one record of this code fits the static array). */
int64_t bpsf_noalloc_max_shots(const bpsf_ctx *ctx);

/* Wait for `stream` and report device-side errors of ctx's last launches
 * (BPSF_ETIMEOUT for a bounded device wait that ran out, BPSF_EDEVICE for an
 * internal error).  Clears the device error word. */
bpsf_status bpsf_sync(bpsf_ctx *ctx, void *stream);

/*
 * Launch shape of the batched kernel for one context (the autotuner's
 * search space).  A team of warps_per_team warps decodes slots_per_team work
 * items in lock step (interleaved in shared memory, so each lane serves one
 * fixed slot); warps_per_block / warps_per_team teams share a block
 * together with one manager warp that writes results and refills slots;
 * blocks_per_sm blocks per SM (0 = as many as fit); iter_chunk bounds how
 * often a team stops to refill finished slots.  bpsf_set_tuning
 * returns BPSF_EINVAL for a shape whose block does not fit in shared memory.
 * For codes of row weight 6 and column weight 3 with max_iter <= 127 and no
 * layered schedule, a kernel instance with one-byte flip counters makes
 * room for shapes that two-byte counters do not fit (for example 13 teams of
 * 8 slots on [[144,12,12]]).
 */
typedef struct {
    int32_t warps_per_team;  /* 1, 2, 4 or 8 */
    int32_t slots_per_team;  /* 1, 2, 4, 8, 16 or 32 */
    int32_t warps_per_block; /* compute warps: a multiple of warps_per_team, <= 15 */
    int32_t blocks_per_sm;   /* 0 = occupancy limit */
    int32_t iter_chunk;      /* 0 or 1: refill a finished slot after the iteration it finished in; k in 2..64:
                                a team refills its finished slots at most every k iterations (finished slots
                                wait, the team's other slots keep iterating).  Every run still stops at the
                                first iteration whose decision satisfies its syndrome, so results do not
                                depend on it. */
} bpsf_tuning;

bpsf_status bpsf_get_tuning(const bpsf_ctx *ctx, bpsf_tuning *out);
bpsf_status bpsf_set_tuning(bpsf_ctx *ctx, const bpsf_tuning *t);

/*
 * Autotuner: times bpsf_decode over candidate launch shapes on n_sample
 * syndromes of random errors drawn at rate p_sample (device generator):
 * threads per shot (warps per team over slots per team), shots per block
 * (slots per team x teams), then the iteration chunk for the fastest shape.
 * Keeps the fastest, sets it on ctx and caches it per code shape (M, N, nnz,
 * degrees, parameters) for the process; a context created later for the same
 * code shape starts with it.  Synchronises `stream`.  chosen is nullable.
 */
bpsf_status bpsf_autotune(bpsf_ctx *ctx, double p_sample, int64_t n_sample, void *stream, bpsf_tuning *chosen);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of a request stream (mixed codes).        */
/* ---------------------------------------------------------------------- */

/*
 * A server keeps one persistent decode loop on the device over several codes
 * (the paper's streaming setting: syndromes arrive one request at a time,
 * Section VI).  Each code has max_inflight_shots rows, each with its shot's
 * device-side records (the state of a failed shot's trials); a request takes
 * consecutive rows and is admitted only when they are free (admission by
 * device memory).  Submitting writes the syndromes into a host-mapped input
 * arena and publishes them with a release store that the device reads with
 * system-scope acquire loads: no copy and no driver call per request.  Shots
 * of requests that arrive while others run join the same device work pool as
 * slots free up; results are written to host-mapped rows and each request's
 * completion is posted by the device.
 * The device loop leaves after idle_exit_us without work and a host thread
 * relaunches it when admitted work is pending, so no device wait is unbounded.
 * While the loop runs it holds the SMs: other kernels on the same device wait.
 *
 *   max_inflight_shots  rows per code (default 65536).
 *   blocks              persistent blocks of the loop (0 = as many as fit).
 *   idle_exit_us        device idle time before the loop leaves (default 20000).
 *   max_requests        requests admitted and not yet polled (default 4096).
 *   flags               reserved, must be 0.
 */
typedef struct {
    int64_t max_inflight_shots;
    int32_t blocks;
    int32_t idle_exit_us;
    int32_t max_requests;
    uint32_t flags;
} bpsf_serve_cfg;

typedef struct bpsf_server bpsf_server;

/* Start a server over n_codes contexts (1..16; not owned, they must outlive
 * the server; all on the current device).  cfg is nullable (defaults). */
bpsf_status bpsf_serve_start(bpsf_server **out, bpsf_ctx *const *codes, int32_t n_codes, const bpsf_serve_cfg *cfg);

/*
 * Submit n shots of code index `code` (h_synd: n rows of that code's Ws words,
 * host memory, copied to the device before return).  Waits while the code's
 * rows or the request slots are full, up to timeout_us (<= 0: do not wait);
 * then BPSF_EBUSY.  n larger than the arena is BPSF_EINVAL.  On success
 * *ticket identifies the request.  Thread-safe.
 */
bpsf_status bpsf_serve_submit(bpsf_server *s, int32_t code, int64_t n, const uint32_t *h_synd, int64_t timeout_us,
                              uint64_t *ticket);

/*
 * Wait up to timeout_us for a request (BPSF_ETIMEOUT if not done; the ticket
 * stays valid), then copy its results (Wn words per shot, converged bytes,
 * int16 iterations, stage bytes; each output pointer nullable), release the
 * request's rows and the ticket.  Unknown tickets: BPSF_EINVAL.  Thread-safe.
 */
bpsf_status bpsf_serve_poll(bpsf_server *s, uint64_t ticket, int64_t timeout_us, uint32_t *h_corr,
                            uint8_t *h_converged, int16_t *h_iters, uint8_t *h_stage);

/*
 * Open-loop replay of a request trace (latency measurement, thread-safe
 * against other clients).  Request i (code[i], n_shots[i] rows at synd[i])
 * is submitted at arrival_s[i] seconds (non-decreasing) after the call
 * starts, by one host thread, while another polls every outstanding request;
 * results are dropped.  On return latency_s[i] = completion time - scheduled
 * arrival of request i, and *span_s (nullable) = time from the start to the
 * last completion.  arrival_s NULL replays the trace closed loop instead:
 * request i is submitted when request i - 1 has completed, and latency_s[i]
 * is its own submit-to-results time.  Times come from the host's monotonic
 * clock (std::chrono::steady_clock), as in bpsf_plain_replay.
 */
bpsf_status bpsf_serve_replay(bpsf_server *s, int64_t n_req, const double *arrival_s, const int32_t *code,
                              const int64_t *n_shots, const uint32_t *const *synd, double *latency_s, double *span_s);

/*
 * The plain per-shot form serving the same kind of trace, on the same clock:
 * one host thread takes request i (code index code[i] into codes[], n_shots[i]
 * host rows at synd[i]) at arrival_s[i] (or, with arrival_s NULL, when request
 * i - 1 is done), copies its syndromes to the device, decodes its shots one at
 * a time with bpsf_decode_plain (each shot: initial-run launch, synchronise,
 * read the flag, on failure the trial-sweep launch, synchronise) and copies
 * the results back.  latency_s[i] = completion - scheduled arrival (closed
 * loop: its own service time); *span_s (nullable) = start to last completion.
 * Requests wait in arrival order while earlier ones are decoded, so an
 * offered load above the form's rate shows as growing latency.  Allocates
 * its staging buffers for the call.  codes: 1..16 contexts on one device.
 */
bpsf_status bpsf_plain_replay(bpsf_ctx *const *codes, int32_t n_codes, int64_t n_req, const double *arrival_s,
                              const int32_t *code, const int64_t *n_shots, const uint32_t *const *synd,
                              double *latency_s, double *span_s);

/* Stop: new submits get BPSF_ECLOSED, admitted requests finish on the device
 * (bounded wait), the device loop ends and the server is freed.  Results not
 * yet polled are dropped.  Returns BPSF_ETIMEOUT if a device wait ran out. */
bpsf_status bpsf_serve_stop(bpsf_server *s);

/* ---------------------------------------------------------------------- */
/* Code builders and helpers                                              */
/* ---------------------------------------------------------------------- */

/*
 * Bivariate bicycle code (Appendix "Code Construction", BB codes):
 * x = S_l (x) I_m, y = I_l (x) S_m with S_l the cyclic shift, A = a(x, y),
 * B = b(x, y), H_X = [A | B] (which = 0) or H_Z = [B^T | A^T] (which = 1).
 * Terms are monomials x^{a_x[t]} y^{a_y[t]}; repeated terms cancel mod 2.
 * m = 1 gives the generalised bicycle codes of the same appendix.
 * Output in CSR: ptr_out has l*m + 1 entries, idx_out room for idx_cap
 * column indices (ascending per row); *nnz_out = ones written.
 */
bpsf_status bpsf_bb_code(int32_t l, int32_t m, int32_t n_a, const int32_t *a_x, const int32_t *a_y, int32_t n_b,
                         const int32_t *b_x, const int32_t *b_y, int32_t which, int32_t *ptr_out, int32_t *idx_out,
                         int64_t idx_cap, int64_t *nnz_out);

/*
 * R-round phenomenological detector matrix built from one round's H0
 * (M0 x N0, CSR): H = [I_R (x) H0 | B_R (x) I_M0] with B_R lower bidiagonal;
 * detector row t*M0 + j compares rounds t and t-1 of check j; columns are
 * R*N0 data errors (round-major) then R*M0 measurement errors.  The
 * phenomenological model is not in the paper; see the project notes.
 * Output CSR with R*M0 rows; idx_cap bounds idx_out.
 */
bpsf_status bpsf_phenom_code(int32_t M0, int32_t N0, const int32_t *ptr0, const int32_t *idx0, int32_t rounds,
                             int32_t *ptr_out, int32_t *idx_out, int64_t idx_cap, int64_t *nnz_out);

/* s = H e (mod 2) for n packed error vectors on the device (harness). */
bpsf_status bpsf_syndrome(const bpsf_ctx *ctx, int64_t n, const uint32_t *d_err, int32_t err_stride_words,
                          uint32_t *d_synd, int32_t synd_stride_words, void *stream);

/*
 * Debug/test hook: batched decode that also dumps internal values.  All
 * outputs are device arrays indexed by shot (nullable):
 *   d_lout        n x N float: posterior LLRs of the initial run's last iteration.
 *   d_flips       n x N uint16: flip counters of the initial run.
 *   d_phi         n x w int32: Phi of failed shots (untouched otherwise).
 *   d_trial_synd  n x T x Ws uint32: trial syndromes s' (T = trials per shot).
 *   d_trial_conv  n x T bytes: trial converged flags (failed shots only).
 *   d_trial_iters n x T int16: trial iterations (failed shots only).
 * It runs the same kernels as bpsf_decode with the dump stores enabled.
 */
bpsf_status bpsf_decode_debug(bpsf_ctx *ctx, int64_t n_shots, const uint32_t *d_synd, int32_t synd_stride_words,
                              uint32_t *d_corr, int32_t corr_stride_words, uint8_t *d_converged, int16_t *d_iters,
                              uint8_t *d_stage, float *d_lout, uint16_t *d_flips, int32_t *d_phi,
                              uint32_t *d_trial_synd, uint8_t *d_trial_conv, int16_t *d_trial_iters, void *stream);

/*
 * Failure-detection self test (no paper counterpart).  Runs the trial sweep
 * of one failed shot whose record is never published, so every device wait
 * for it must give up after wait_us (1..10^7) instead of spinning forever;
 * the kernel then records the timeout in its status word and ends normally.
 * Synchronises `stream` and returns BPSF_ETIMEOUT when the bounded waits
 * worked (BPSF_OK would mean a wait did not run).  Nothing faults or hangs.
 */
bpsf_status bpsf_selftest_wait(bpsf_ctx *ctx, int64_t wait_us, void *stream);

/* Number of trials per failed shot (the default set or the given list). */
int32_t bpsf_num_trials(const bpsf_ctx *ctx);

/*
 * Replace the trial set of ctx (Algorithm 1's trial vectors t as subsets of
 * Phi): n masks, bit j of mask k selects Phi[j] (j < w); each mask
 * non-empty with at most 16 bits; n <= 4096.  Trials are decoded and
 * selected in list order: the minimum-weight rule breaks ties, and the
 * first-success rule picks, by list index.  The sampled variant of
 * Section V (n_s random trial vectors per weight 1..w_max over a larger
 * Phi) is such a list.  n = 0 restores the default set.  Host array,
 * copied.  Not while a decode or a server uses ctx; the next decode
 * re-sizes the failed-shot workspace.
 */
bpsf_status bpsf_set_trials(bpsf_ctx *ctx, int32_t n, const uint64_t *masks);

/* Work counters of the last decode on ctx (after bpsf_sync): runs started,
 * failed shots (records), iterations and edge-updates (iterations x nnz
 * summed over runs), and the slot-iterations the teams offered while they
 * had work (team iterations with a running slot x slots per team);
 * iterations / slot_capacity is the slot occupancy of the launch; and the
 * trials cancelled because they could not win (first-success rule: a trial
 * after the earliest converged one is not started, or is stopped at its
 * next iteration); trial_runs counts the trials run to their end. */
typedef struct {
    int64_t initial_runs;
    int64_t failed_shots;
    int64_t trial_runs;
    int64_t iterations;
    int64_t edge_updates;
    int64_t slot_capacity;
    int64_t trials_cancelled;
} bpsf_work;
bpsf_status bpsf_last_work(bpsf_ctx *ctx, bpsf_work *out);

const char *bpsf_status_str(bpsf_status s);
const char *bpsf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BPSF_H */
