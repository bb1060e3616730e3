// Internal layout shared by the host side and the kernels of libbpsf.
#pragma once

#include <cstdint>

namespace bpsf {

constexpr int kMaxW = 16;         // most bits a trial vector flips (entries of a work item's bit list)
constexpr int kMaxPhi = 64;       // |Phi|: trial masks are 64-bit
constexpr int kMaxTrials = 4096;  // trials per failed shot
constexpr int kMaxSlots = 32;     // work items per team
constexpr int kMaxStreams = 16;   // codes per launch
constexpr int kMaxComputeWarps = 15;  // plus one manager warp: <= 512 threads per block
constexpr int kMaxNamedTeams = 15;    // named barriers 1..15 for multi-warp teams
constexpr int kDVP = 4;           // column entries stored per variable for dv <= 4 codes

// Device error bits (StreamCounters::status).
enum : unsigned {
    kDevReadyTimeout = 1u,   // a trial waited too long for its record
    kDevIdleTimeout = 2u,    // a block waited too long for other blocks
    kDevRecordOverflow = 4u  // more failed shots than record slots
};

// Stream flags.
enum : unsigned {
    kNoTickets = 1u,  // do not run trials (plain form, first launch)
    kServe = 2u       // shots come from a growing request queue
};

// One code's Tanner graph in the order the kernels read it, plus the
// decoder constants.  Messages of one work item live in one array of P
// floats, one position per edge, given by the layout of the launch's slot
// count (LayoutS): a check-node thread reads and writes its row at stride Mp
// (one word per bank for consecutive rows).  vpos lists, for each column,
// the positions of its edges in ascending check order (the order the V2C and
// posterior sums are folded in).
// Message layout for one slot count S = 1 << index: edge of row j with
// rank r sits at position r*Mp + j (Mp >= M, P = dc_max * Mp positions); the
// rank stride and the rank of each edge within its row are chosen at create
// so that the column phase's gathered accesses meet few shared-memory bank
// conflicts for that S (the row phase is exact for any rank order).
struct LayoutS {
    int Mp, P;
    const uint16_t *vpos;     // N x vstride positions
    const float *lch_pos;     // P, channel LLR of the variable at each position
    const uint16_t *pos_var;  // P, variable at each position (0xffff: unused)
};
constexpr int kNumLayouts = 6;  // S = 1, 2, 4, 8, 16, 32

struct CodeDev {
    int M, N, nnz, Ws, Wn;
    int DC, dv_max, P, regular;  // regular: every row has DC ones, every column dv_max
    int vstride;                 // entries per column in vpos / vchk (>= dv_max)
    int max_iter, short_iter, w, n_trials, select;
    float alpha;
    const uint8_t *row_deg;      // M, ones per row
    const uint16_t *vpos;        // N x vstride, message positions (0xffff padding), active layout
    const uint16_t *vchk;        // N x vstride, check indices
    const float *lch;            // N, channel LLRs (FP32)
    const float *lch_pos;        // P, channel LLR of the variable at each position, active layout
    const uint16_t *row_ptr;     // M+1, CSR (syndrome kernel)
    const uint16_t *csr_col;     // nnz
    const unsigned long long *trial_mask;  // n_trials subset masks over Phi (bit j selects Phi[j]), list order
    int Mp;                      // rank stride of the active layout (see LayoutS)
    const uint16_t *pos_var;     // active layout: variable at each position
    LayoutS lay[kNumLayouts];    // per slot count; a launch activates the one of its S
    int layered;                 // 1: layered schedule
    int n_layers;
    const uint16_t *layer_ptr;   // n_layers+1, rows of layer l are layer_rows[layer_ptr[l] .. layer_ptr[l+1])
    const uint16_t *layer_rows;  // M, rows grouped by layer, ascending within a layer
};

// Per-launch counters of one stream (64 bytes, zeroed before a launch).
struct StreamCounters {
    unsigned long long shot_next;    // next unclaimed shot
    unsigned long long init_done;    // initial runs finished
    unsigned long long ticket_next;  // trial tickets claimed
    unsigned long long iters_total;  // iterations run (all runs)
    unsigned long long trial_runs;   // trial runs finished
    unsigned long long rec_count;    // failed shots published
    unsigned int status;             // kDev* bits
    unsigned int pad0;
    unsigned long long slot_capacity;  // slot-iterations offered: team iterations with work x S
    unsigned long long trials_cancelled; // trials not run, or stopped, because they could not win
    unsigned long long pad[7];
};
static_assert(sizeof(StreamCounters) == 128, "counter block is two 64-byte lines");

// Failed-shot records: a ring of `cap` records (a power of two) in failure
// order.  The team whose initial run fails claims the next failure number q
// (rec_count), checks that record q % cap is free, writes Phi, the syndrome,
// an empty selection and the shot's provisional output, and then publishes
// it (qseq = q + 1); trial tickets walk the failure numbers, and the last
// trial of a shot frees its record (qseq = 0).  A batch's ring has at least
// as many records as the batch has shots, so it never wraps within a launch
// and the records are written densely in failure order; a server's ring has
// at least its admitted shots (so it wraps only over freed records).  A
// record found busy is waited for (bounded) and reported (kDevRecordOverflow).
//
// Only the winning trial's correction is kept.  A converged trial's
// selection key (kSelKeyBits bits: weight << 12 | list index, or the list
// index under the first-success rule; unique per trial) goes into the top
// half of 64-bit words merged with atomicMin: best = key << 32 | iterations,
// and word w of the correction as key << 32 | (e' xor t)_w.  Each word's
// minimum is then the smallest key's own word, whatever order the trials
// finish in, with no lock.
struct Records {
    unsigned long long *qseq;   // cap: q + 1 while the record holds failure q, 0 when free
    long long *qshot;           // cap: the failed shot
    unsigned int *done;         // cap: its trials finished
    unsigned long long *best;   // cap: min over converged trials of key << 32 | iterations
    unsigned long long *win;    // cap x Wn: min over converged trials of key << 32 | correction word
    int32_t *phi;               // cap x w
    uint32_t *synd;             // cap x Ws: the shot's syndrome
    long long cap;              // records in the ring (a power of two)
};

constexpr int kSelKeyBits = 28;  // weight (16 bits, N <= 65535) above a 12-bit list index (n_trials <= 4096)

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

// Serving: shots carry global sequence numbers g; shot g uses arena row
// g % rows.  The host writes a request's syndromes into its rows of the
// host-mapped arena and then stores the new published count with release
// semantics; the device reads the count with system-scope acquire loads
// before it reads the rows, and posts g + 1 to the row's completion word
// once the shot's results are in the host-mapped output rows.
struct ServeDev {
    volatile long long *published;   // shots published for this code (host-mapped)
    volatile int *stop;              // host asks the loop to end (host-mapped)
    volatile unsigned *row_done;     // rows: (g + 1) once the shot's results are out (host-mapped)
    long long rows;                  // arena rows
    long long idle_ns;               // leave the loop after this long without work
};

struct StreamDev {
    CodeDev code;
    JobDev job;
    Records rec;
    StreamCounters *ctr;
    DebugDev dbg;
    ServeDev serve;
    unsigned flags;  // kNoTickets, kServe
    int S, W, teams; // team shape for this code: teams of W warps with S slots each
    int chunk;       // team iterations between refills of finished slots (>= 1)
};

// Launch: the team shape is set per stream (StreamDev::S, W, teams); each
// block has one manager warp besides; Q ready-queue entries.
struct LaunchArgs {
    const StreamDev *streams;
    int n_streams;
    int Q;
    unsigned long long wait_ns;  // bound on any device-side wait
};

// ---------------------------------------------------------------------------
// Shared-memory layout (identical on host and device).
// ---------------------------------------------------------------------------

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

constexpr int kBlockHeaderBytes = 64;

struct LayoutOffsets {
    int row_deg, vpos, lch, lch_pos, total;
};

__host__ __device__ inline LayoutOffsets layout_offsets(int M, int N, int vstride, int P) {
    LayoutOffsets o;
    int p = 0;
    o.row_deg = p;  p = align_up(p + M, 16);
    o.vpos = p;     p = align_up(p + 2 * N * vstride, 16);
    o.lch = p;      p = align_up(p + 4 * N, 16);
    o.lch_pos = p;  p = align_up(p + 4 * P, 16);
    o.total = p;
    return o;
}

// Slot states.  Only the slot's team writes them: RUNNING while a run is in
// progress, PENDING once it has finished and until its facts are in the
// slot's outbox, EMPTY when the slot may take the item in its inbox.
enum : int { kSlotEmpty = 0, kSlotRunning = 1, kSlotPending = 2 };

// Per-slot state in shared memory (80 bytes), owned by the slot's team.
struct SlotState {
    int state;       // kSlot*
    int kind;        // 1 initial run, 2 trial run
    int start;       // team iteration at which the current run's first iteration ran
    int outcome;     // 1 converged, 2 iteration cap, 3 stopped (cannot win); valid when PENDING
    int iter;        // iterations completed
    int limit;       // iteration cap of this run
    int kidx;        // trial index (trial runs)
    int rec;         // record of the shot (trial runs)
    long long shot;  // shot index in the job (global sequence number when serving)
    long long cancel;  // manager -> team: shot * n_trials + kidx + 1 of a trial run that cannot win
};
static_assert(sizeof(SlotState) == 48, "slot state is 48 bytes");

// A finished run's facts, handed from the team to the manager (32 bytes;
// the packed hard decision goes with it in the team's ebits words).  The
// team fills an outbox whose flag is 0 and then sets it; the manager writes
// the results out and clears it.  A failed initial run's Phi =
// top(flip_count, w) goes to the shot's record directly; a trial's flipped
// bits are the record's Phi[j] that the trial mask selects, so neither the
// items nor the outboxes carry them.
struct OutBox {
    int full;
    int kind;
    int kidx;
    int outcome;
    int iter;
    int rec;  // record of the shot (trial runs)
    long long shot;
};
static_assert(sizeof(OutBox) == 32, "outbox is 32 bytes");

// Team control block (64 bytes).  run_mask, init_mask and exit are written
// by the team's warp 0 at a service step and read by the whole team after the
// barrier that follows; stop_mask[t & 1] holds the slots whose run ends after
// team iteration t whatever its syndrome (iteration cap, or a trial asked to
// stop), written by warp 0 before the iteration's first barrier and read by
// every warp after its last, so consecutive iterations use different words.
struct TeamCtl {
    unsigned run_mask, init_mask;
    int exit;
    unsigned stop_mask[2];
    unsigned last_beat;              // idle team (warp 0): the manager's heartbeat last seen,
    unsigned long long idle_since;   //   when it started idling (0: it runs),
    unsigned idle_ns, idle_looks;    //   its current sleep and the looks that found nothing
    unsigned long long iters;  // iterations run by this team (all slots)
    unsigned long long cap;    // team iterations with a running slot, times S
};
static_assert(sizeof(TeamCtl) <= 64, "team control block fits its 64 bytes");

// Work items of the manager's ready queue and of the slots' inboxes: 16
// bytes of fields plus Ws syndrome words (a trial's words are s' = s xor t H^T).  kind 1 = initial run of a shot,
// 2 = trial run, 0 = nothing to run (an item dropped after a timed-out wait).
struct QEntry {
    int16_t kind;
    int16_t kidx;  // < 4096
    int rec;       // record of the shot (trial runs)
    long long shot;
};
static_assert(sizeof(QEntry) == 16, "queue entry header is 16 bytes");

__host__ __device__ inline int qentry_bytes(int Ws) { return align_up((int)sizeof(QEntry) + 4 * Ws, 16); }

// Per-team shared memory.  The S slots of a team (S a power of two <= 32)
// are interleaved: item x of slot s sits at x*S + s, so lane l always serves
// slot l mod S and the 32 lanes of a warp touch 32 consecutive items.
//   syn, mism : bit j*S + s = s_j, resp. the residual syndrome (s xor H e)_j,
//               of slot s, in (S*M + 31)/32 words each
//   ebits     : S x Wn words, the hard decision of a finished run, packed
//               (part of the slot's outbox)
//   flips     : flip word i*S + s (fb bytes) = decision (top bit) and flip
//               count of variable i in slot s
//   m         : float k*S + s = the message of edge position k = r*Mp + j
//               (edge of row j with rank r) in slot s: V2C and C2V alternately
//   outbox    : S OutBox entries
//   inflag    : S flags, 1 while the slot's inbox holds an item
//   inbox     : S work items (qentry_bytes(Ws) each), filled by the manager
//               ahead of time and installed by the team as soon as the slot
//               is free, so a slot does not wait for the manager between runs
//   post      : layered schedule only: float i*S + s = running posterior L_i
//               of slot s (the message array then holds the C2V messages)
struct TeamOffsets {
    int ctl, state, syn, mism, ebits, flips, m, outbox, inflag, inbox, ibstride, post, total;
};

__host__ __device__ inline TeamOffsets team_offsets(int S, int M, int N, int P, int Ws, int layered, int fb = 2) {
    TeamOffsets o;
    const int sw = (S * M + 31) / 32;
    int p = 0;
    o.ctl = p;     p += 64;
    o.state = p;   p += (int)sizeof(SlotState) * S;
    o.outbox = p;  p += (int)sizeof(OutBox) * S;
    o.syn = p;     p += 4 * sw;
    o.mism = p;    p += 4 * sw;
    o.ebits = p;   p += 4 * S * ((N + 31) / 32);
    o.inflag = p;  p = align_up(p + 4 * S, 16);
    o.ibstride = qentry_bytes(Ws);
    o.inbox = p;   p += o.ibstride * S;
    o.flips = p;   p = align_up(p + fb * S * N, 16);
    o.m = p;       p += 4 * S * P;
    o.post = p;    p += layered ? 4 * S * N : 0;
    o.total = align_up(p, 16);
    return o;
}

__host__ __device__ inline int block_smem_bytes(int M, int N, int P, int Ws, int vstride, int S, int teams, int Q,
                                                int layered, int fb = 2) {
    return kBlockHeaderBytes + layout_offsets(M, N, vstride, P).total + Q * qentry_bytes(Ws) +
           teams * team_offsets(S, M, N, P, Ws, layered, fb).total;
}

// Arguments of one persistent launch: the streams (codes) it serves, by value.
struct KernelParams {
    StreamDev streams[kMaxStreams];
    int n_streams;
    int Q;
    unsigned long long wait_ns;
};

// Kernel entry points (bpsf_kernels.cu).
int kernel_variant(int dc_max, int dv_max);  // smallest variant that fits, -1 if none
int kernel_variant_dv(int variant);          // column table width of a variant
int kernel_variant_full_regs(int variant);   // its one-block, full-register instance
int kernel_variant_byte_flips(int variant);  // its one-block instance with one-byte flip words, -1 if none
int kernel_variant_mixed(int variant);       // its instance with the exact (6, 4, 3) path as well, -1 if none
const void *persistent_kernel_ptr(int variant, bool debug, bool layered);
void launch_persistent(int variant, bool debug, bool layered, int grid, int block, int smem, const LaunchArgs &args,
                       void *stream);
void launch_syndrome(const CodeDev &cd, long long n, const uint32_t *err, int err_stride, uint32_t *synd,
                     int synd_stride, void *stream);
void launch_sample_errors(long long n, int nbits, double p, unsigned long long seed, uint32_t *err, int stride,
                          void *stream);

}  // namespace bpsf
