// Device code of libbpsf: the persistent BP-SF kernel (Algorithm 1 of
// arXiv 2507.00254) and two small harness kernels (syndrome, error sampler).
//
// Execution model.  A *team* of W warps decodes S work items ("slots") in
// lock step, one BP iteration at a time.  A work item is either the initial
// run of a shot (with oscillation counters) or one trial of a failed shot.
// Per iteration the team runs
//   C phase : one thread per (slot, check): min1 / min2 / sign product over
//             the row (Eq. c2v), one FP32 multiply by alpha, C2V messages
//             written to their CSC positions;
//   V phase : one thread per (slot, variable): V2C messages for the next
//             iteration (Section II-B step 2, explicit exclusion), posterior
//             LLR and hard decision (step 4), a warp ballot packs e into
//             words, changed bits update the flip counters (Algorithm 1) and
//             toggle the slot's residual syndrome s xor H e by shared atomics;
//   decide  : a slot whose residual syndrome is zero converged; a slot at its
//             iteration cap is exhausted.  Finished slots are written out and
//             refilled from the device-wide queue at once.
// A failed initial run picks Phi = top(flip_count, w), writes a record (Phi,
// s) and publishes its trials as tickets; any team may claim them.  Each
// converged trial stores e' xor t and takes an atomicMin on (weight, index);
// the last trial of a record writes the winner.  All messages and per-slot
// state live in shared memory; HBM only sees syndromes, outputs and records.
#include <cuda_runtime.h>

#include <cstdint>

#include "bpsf_internal.h"

namespace bpsf {

#define FULLMASK 0xffffffffu

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_vol_u64(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ unsigned ld_vol_u32(const unsigned *p) {
    return *reinterpret_cast<const volatile unsigned *>(p);
}

__device__ __forceinline__ void team_sync(int W, int bar_id) {
    if (W == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(W * 32) : "memory");
    }
}

struct LayoutMem {
    const uint16_t *row_ptr, *csr_to_csc, *col_ptr, *csc_to_csr;
    const float *lch;
};

struct TeamMem {
    TeamCtl *ctl;
    SlotState *st;
    uint32_t *syn, *mism, *ebits;
    uint16_t *flips;
    float *q, *r;
};

// ---------------------------------------------------------------------------
// C phase: check-node update, Eq. (c2v).  For row j with V2C inputs q_k:
//   neg = s_j xor (xor_k [q_k < 0]),  m1 = min |q_k| (first argmin k1),
//   m2 = min over k != k1,  r_k = (neg xor [q_k < 0]) ? -a : a,
//   a = alpha * (k == k1 ? m2 : m1),
// which equals the explicit "min and sign product over the other variables"
// bit for bit (min is exact; the sign factors are exact).
// ---------------------------------------------------------------------------
template <int DC>
__device__ __forceinline__ void c_phase(const CodeDev &cd, const LayoutMem &L, const TeamMem &T, int S, int tid,
                                        int nthreads) {
    const unsigned act = T.ctl->act_mask, fresh = T.ctl->fresh_mask;
    const int M = cd.M, nnz = cd.nnz, Ws = cd.Ws;
    const int total = S * M;
    const float alpha = cd.alpha;
    int s = tid / M, j = tid - s * M;
    for (int tau = tid; tau < total; tau += nthreads) {
        if ((act >> s) & 1u) {
            const bool fr = (fresh >> s) & 1u;
            const int e0 = L.row_ptr[j];
            const int deg = L.row_ptr[j + 1] - e0;
            unsigned neg = (T.syn[s * Ws + (j >> 5)] >> (j & 31)) & 1u;
            const float *qs = T.q + s * nnz + e0;
            float v[DC];
#pragma unroll
            for (int k = 0; k < DC; ++k) v[k] = (k < deg) ? (fr ? __ldg(cd.lch_csr + e0 + k) : qs[k]) : 0.f;
            float m1 = __int_as_float(0x7f800000), m2 = m1;
            int k1 = 0;
#pragma unroll
            for (int k = 0; k < DC; ++k) {
                if (k < deg) {
                    const float a = fabsf(v[k]);
                    if (a < m1) {
                        m2 = m1;
                        m1 = a;
                        k1 = k;
                    } else if (a < m2) {
                        m2 = a;
                    }
                    neg ^= (v[k] < 0.f) ? 1u : 0u;
                }
            }
            const float g1 = __fmul_rn(alpha, m1), g2 = __fmul_rn(alpha, m2);
            float *rs = T.r + s * nnz;
#pragma unroll
            for (int k = 0; k < DC; ++k) {
                if (k < deg) {
                    const float mag = (k == k1) ? g2 : g1;
                    const unsigned ng = neg ^ ((v[k] < 0.f) ? 1u : 0u);
                    rs[L.csr_to_csc[e0 + k]] = ng ? -mag : mag;
                }
            }
        }
        j += nthreads;
        while (j >= M) {
            j -= M;
            ++s;
        }
    }
}

// ---------------------------------------------------------------------------
// V phase: variable-node update (Section II-B steps 2 and 4) and oscillation
// tracking (Algorithm 1).  For column i with C2V inputs r_0..r_{d-1} in
// ascending check order:
//   q_k   = l_ch + sum_{k' != k} r_k'   (left fold, ascending k'),
//   l_out = l_ch + sum_k r_k            (left fold),  e_i = [l_out <= 0].
// ---------------------------------------------------------------------------
template <int DV, bool DEBUG>
__device__ __forceinline__ void v_phase(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int S, int tid,
                                        int nthreads) {
    const CodeDev &cd = sd.code;
    const unsigned act = T.ctl->act_mask, fresh = T.ctl->fresh_mask, initm = T.ctl->init_mask;
    const int N = cd.N, nnz = cd.nnz, Ws = cd.Ws;
    const int total = S * N;
    const int lane = tid & 31;
    int tau = tid;
    int s = tau / N, i = tau - s * N;
    for (int base = tid - lane; base < total; base += nthreads) {
        const bool valid = tau < total;
        const bool a = valid && ((act >> s) & 1u);
        const bool fr = a && ((fresh >> s) & 1u);
        const bool ini = a && ((initm >> s) & 1u);
        unsigned ebit = 0;
        int f0 = 0, f1 = 0;
        if (a) {
            f0 = L.col_ptr[i];
            f1 = L.col_ptr[i + 1];
            const int deg = f1 - f0;
            const float lc = L.lch[i];
            const float *rs = T.r + s * nnz + f0;
            float rv[DV];
#pragma unroll
            for (int k = 0; k < DV; ++k) rv[k] = (k < deg) ? rs[k] : 0.f;
            float *qs = T.q + s * nnz;
#pragma unroll
            for (int k = 0; k < DV; ++k) {
                if (k < deg) {
                    float acc = lc;
#pragma unroll
                    for (int k2 = 0; k2 < DV; ++k2)
                        if (k2 != k && k2 < deg) acc = __fadd_rn(acc, rv[k2]);
                    qs[L.csc_to_csr[f0 + k]] = acc;
                }
            }
            float lo = lc;
#pragma unroll
            for (int k = 0; k < DV; ++k)
                if (k < deg) lo = __fadd_rn(lo, rv[k]);
            ebit = (lo <= 0.f) ? 1u : 0u;
            if (DEBUG && ini && sd.dbg.lout) sd.dbg.lout[T.st[s].shot * N + i] = lo;
        }
        const int widx = base >> 5;
        const unsigned old = T.ebits[widx];
        const unsigned am = __ballot_sync(FULLMASK, a);
        const unsigned nb = __ballot_sync(FULLMASK, ebit != 0);
        __syncwarp();
        if (lane == 0) T.ebits[widx] = (nb & am) | (old & ~am);
        if (a) {
            const unsigned prev = fr ? 0u : ((old >> lane) & 1u);
            const unsigned flip = prev ^ ebit;
            if (ini) T.flips[tau] = fr ? (uint16_t)flip : (uint16_t)(T.flips[tau] + flip);
            if (flip) {
                for (int f = f0; f < f1; ++f) {
                    const int c = __ldg(cd.csc_chk + f);
                    atomicXor(&T.mism[s * Ws + (c >> 5)], 1u << (c & 31));
                }
            }
        }
        tau += nthreads;
        i += nthreads;
        while (i >= N) {
            i -= N;
            ++s;
        }
    }
}

// Word w of slot s's hard decision, from the team's flattened bit array.
__device__ __forceinline__ unsigned slot_word(const TeamMem &T, int N, int s, int w) {
    const int bit0 = s * N + 32 * w;
    const int wi = bit0 >> 5, sh = bit0 & 31;
    unsigned v = T.ebits[wi] >> sh;
    if (sh) v |= T.ebits[wi + 1] << (32 - sh);
    const int rem = N - 32 * w;
    if (rem < 32) v &= (1u << rem) - 1u;
    return v;
}

// Write out one finished slot (whole first warp of the team).
template <bool DEBUG>
__device__ void finalize_slot(const StreamDev &sd, const TeamMem &T, int s, bool conv, int lane,
                              unsigned long long &init_local, unsigned long long &trials_local) {
    const CodeDev &cd = sd.code;
    const JobDev &job = sd.job;
    SlotState *ss = &T.st[s];
    const int kind = ss->kind, iter = ss->iter;
    const long long shot = ss->shot;
    const int N = cd.N, Wn = cd.Wn, Ws = cd.Ws;
    if (kind == 1) {
        if (DEBUG && sd.dbg.flips)
            for (int i = lane; i < N; i += 32) sd.dbg.flips[shot * N + i] = T.flips[s * N + i];
        uint32_t *out = job.corr + shot * job.corr_stride;
        for (int w = lane; w < Wn; w += 32) out[w] = slot_word(T, N, s, w);
        if (lane == 0) {
            job.conv[shot] = conv ? 1 : 0;
            job.iters[shot] = (int16_t)(conv ? iter : cd.max_iter);
            if (job.stage) job.stage[shot] = conv ? 0 : 2;
        }
        if (!conv && cd.w > 0) {
            // Phi = top(flip_count, w): keys (count << 16 | 0xffff - i) are
            // distinct, so each round takes the largest key below the last.
            unsigned thr = 0xffffffffu;
            int my_phi = 0;
            for (int r = 0; r < cd.w; ++r) {
                unsigned best = 0;
                for (int i = lane; i < N; i += 32) {
                    const unsigned key = ((unsigned)T.flips[s * N + i] << 16) | (0xffffu - (unsigned)i);
                    if (key < thr && key > best) best = key;
                }
                best = __reduce_max_sync(FULLMASK, best);
                if (lane == r) my_phi = (int)(0xffffu - (best & 0xffffu));
                thr = best;
            }
            unsigned rec = 0;
            if (lane == 0) rec = atomicAdd(&sd.ctr->rec_count, 1u);
            rec = __shfl_sync(FULLMASK, rec, 0);
            if ((long long)rec < sd.rec.cap) {
                if (lane == 0) {
                    sd.rec.shot[rec] = shot;
                    sd.rec.done[rec] = 0u;
                    sd.rec.best[rec] = ~0ull;
                }
                if (lane < cd.w) sd.rec.phi[(long long)rec * cd.w + lane] = my_phi;
                for (int w = lane; w < Ws; w += 32) sd.rec.synd[(long long)rec * Ws + w] = T.syn[s * Ws + w];
                if (DEBUG && sd.dbg.phi && lane < cd.w) sd.dbg.phi[shot * cd.w + lane] = my_phi;
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release_u32(&sd.rec.ready[rec], 1u);
            } else if (lane == 0) {
                atomicOr(&sd.ctr->status, kDevRecordOverflow);
            }
        }
        if (lane == 0) ++init_local;
    } else {
        const int C = cd.n_trials, kidx = ss->kidx, rec = ss->rec;
        const unsigned mask = __ldg(cd.trial_mask + kidx);
        if (conv) {
            // Undo the flip (Algorithm 1): return e' xor t.
            unsigned wsum = 0;
            for (int w = lane; w < Wn; w += 32) {
                unsigned v = slot_word(T, N, s, w);
                for (int j = 0; j < cd.w; ++j) {
                    if ((mask >> j) & 1u) {
                        const int b = ss->phi[j];
                        if ((b >> 5) == w) v ^= 1u << (b & 31);
                    }
                }
                sd.rec.corr[((long long)rec * C + kidx) * Wn + w] = v;
                wsum += __popc(v);
            }
            wsum = __reduce_add_sync(FULLMASK, wsum);
            if (lane == 0) sd.rec.iters[(long long)rec * C + kidx] = (int16_t)iter;
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                const unsigned long long key =
                    cd.select == 0 ? (((unsigned long long)wsum << 32) | (unsigned)kidx) : (unsigned long long)kidx;
                atomicMin(&sd.rec.best[rec], key);
            }
        }
        if (DEBUG && lane == 0) {
            if (sd.dbg.trial_conv) sd.dbg.trial_conv[shot * C + kidx] = conv ? 1 : 0;
            if (sd.dbg.trial_iters) sd.dbg.trial_iters[shot * C + kidx] = (int16_t)iter;
        }
        unsigned d = 0;
        if (lane == 0) {
            __threadfence();
            d = atomicAdd(&sd.rec.done[rec], 1u) + 1u;
        }
        d = __shfl_sync(FULLMASK, d, 0);
        if (d == (unsigned)C) {
            // Last trial of this shot: the winner is settled.
            __threadfence();
            unsigned long long best = 0;
            if (lane == 0) best = atomicAdd(&sd.rec.best[rec], 0ull);
            best = __shfl_sync(FULLMASK, best, 0);
            if (best != ~0ull) {
                const int kw = (int)(best & 0xffffffffu);
                uint32_t *out = job.corr + shot * job.corr_stride;
                for (int w = lane; w < Wn; w += 32) out[w] = __ldcg(sd.rec.corr + ((long long)rec * C + kw) * Wn + w);
                if (lane == 0) {
                    job.conv[shot] = 1;
                    job.iters[shot] = __ldcg(sd.rec.iters + (long long)rec * C + kw);
                    if (job.stage) job.stage[shot] = 1;
                }
            }
        }
        if (lane == 0) ++trials_local;
    }
    if (lane == 0) ss->kind = 0;
    __syncwarp();
}

// Start the initial run of `shot` in slot s (one lane).
__device__ __forceinline__ void init_shot(const StreamDev &sd, const TeamMem &T, int s, long long shot) {
    const CodeDev &cd = sd.code;
    SlotState *ss = &T.st[s];
    ss->kind = 1;
    ss->fresh = 1;
    ss->iter = 0;
    ss->limit = cd.max_iter;
    ss->shot = shot;
    ss->rec = -1;
    ss->kidx = -1;
    const uint32_t *src = sd.job.synd + shot * sd.job.synd_stride;
    const int Ws = cd.Ws, tail = cd.M & 31;
    for (int w = 0; w < Ws; ++w) {
        unsigned v = __ldcg(src + w);
        if (w == Ws - 1 && tail) v &= (1u << tail) - 1u;
        T.syn[s * Ws + w] = v;
        T.mism[s * Ws + w] = v;
    }
}

// Start trial `ticket` (record ticket / T, trial ticket % T) in slot s (one lane).
template <bool DEBUG>
__device__ __forceinline__ void init_trial(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int s,
                                           unsigned long long ticket, unsigned long long wait_ns) {
    const CodeDev &cd = sd.code;
    const int C = cd.n_trials, Ws = cd.Ws;
    const long long rec = (long long)(ticket / (unsigned long long)C);
    const int kidx = (int)(ticket - (unsigned long long)rec * C);
    if (ld_acquire_u32(&sd.rec.ready[rec]) == 0u) {
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire_u32(&sd.rec.ready[rec]) == 0u) {
            if (globaltimer_ns() - t0 > wait_ns) {
                atomicOr(&sd.ctr->status, kDevReadyTimeout);
                return;
            }
            __nanosleep(128);
        }
    }
    SlotState *ss = &T.st[s];
    const long long shot = __ldcg(sd.rec.shot + rec);
    for (int j = 0; j < cd.w; ++j) ss->phi[j] = (uint16_t)__ldcg(sd.rec.phi + rec * cd.w + j);
    for (int w = 0; w < Ws; ++w) T.syn[s * Ws + w] = __ldcg(sd.rec.synd + rec * Ws + w);
    // s' = s xor t H^T (Algorithm 1): flip the checks of every selected bit.
    const unsigned mask = __ldg(cd.trial_mask + kidx);
    for (int j = 0; j < cd.w; ++j) {
        if ((mask >> j) & 1u) {
            const int v = ss->phi[j];
            for (int f = L.col_ptr[v]; f < L.col_ptr[v + 1]; ++f) {
                const int c = __ldg(cd.csc_chk + f);
                T.syn[s * Ws + (c >> 5)] ^= 1u << (c & 31);
            }
        }
    }
    for (int w = 0; w < Ws; ++w) {
        T.mism[s * Ws + w] = T.syn[s * Ws + w];
        if (DEBUG && sd.dbg.trial_synd) sd.dbg.trial_synd[(shot * C + kidx) * Ws + w] = T.syn[s * Ws + w];
    }
    ss->kind = 2;
    ss->fresh = 1;
    ss->iter = 0;
    ss->limit = cd.short_iter;
    ss->shot = shot;
    ss->rec = (int)rec;
    ss->kidx = kidx;
}

// Decide every active slot after an iteration and write out finished ones
// (first warp of the team).
template <bool DEBUG>
__device__ __forceinline__ void decide(const StreamDev &sd, const TeamMem &T, int S, int lane,
                                       unsigned long long &init_local, unsigned long long &iters_local,
                                       unsigned long long &trials_local) {
    const int Ws = sd.code.Ws;
    int outcome = 0;
    bool active = false;
    if (lane < S) {
        SlotState *ss = &T.st[lane];
        if (ss->kind) {
            active = true;
            ss->fresh = 0;
            const int it = ss->iter + 1;
            ss->iter = it;
            unsigned any = 0;
            for (int w = 0; w < Ws; ++w) any |= T.mism[lane * Ws + w];
            outcome = (any == 0u) ? 1 : (it >= ss->limit ? 2 : 0);
        }
    }
    const unsigned am = __ballot_sync(FULLMASK, active);
    unsigned fin = __ballot_sync(FULLMASK, outcome != 0);
    const unsigned cvm = __ballot_sync(FULLMASK, outcome == 1);
    if (lane == 0) iters_local += __popc(am);
    __syncwarp();
    while (fin) {
        const int s = __ffs(fin) - 1;
        fin &= fin - 1u;
        finalize_slot<DEBUG>(sd, T, s, (cvm >> s) & 1u, lane, init_local, trials_local);
    }
}

// Fill empty slots: trial tickets first (they finish failed shots), then new
// shots from the team's claimed chunk (first warp of the team).
template <bool DEBUG>
__device__ __forceinline__ void refill(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int S, int lane,
                                       unsigned long long &init_local, unsigned long long wait_ns) {
    const CodeDev &cd = sd.code;
    TeamCtl *ctl = T.ctl;
    const bool empty = lane < S && T.st[lane].kind == 0;
    const unsigned em = __ballot_sync(FULLMASK, empty);
    const int n_empty = __popc(em);
    const int rank = __popc(em & ((1u << lane) - 1u));
    unsigned long long t0 = 0;
    int take = 0;
    if (n_empty && cd.w > 0 && !(sd.flags & kNoTickets)) {
        if (lane == 0) {
            for (int att = 0; att < 4; ++att) {
                const unsigned long long cur = ld_vol_u64(&sd.ctr->ticket_next);
                const unsigned long long rc = ld_vol_u32(&sd.ctr->rec_count);
                const unsigned long long rcap = rc < (unsigned long long)sd.rec.cap ? rc : (unsigned long long)sd.rec.cap;
                const unsigned long long total = rcap * (unsigned long long)cd.n_trials;
                if (cur >= total) break;
                const unsigned long long want = (total - cur) < (unsigned long long)n_empty ? (total - cur)
                                                                                             : (unsigned long long)n_empty;
                if (atomicCAS(&sd.ctr->ticket_next, cur, cur + want) == cur) {
                    t0 = cur;
                    take = (int)want;
                    break;
                }
            }
        }
        t0 = __shfl_sync(FULLMASK, t0, 0);
        take = __shfl_sync(FULLMASK, take, 0);
    }
    const int need = n_empty - take;
    long long s0 = 0;
    int got = 0;
    if (need > 0) {
        if (lane == 0) {
            long long cn = ctl->chunk_next, ce = ctl->chunk_end;
            const long long n = sd.job.n_shots;
            if (cn >= ce && (long long)ld_vol_u64(&sd.ctr->shot_next) < n) {
                const long long ch = (2 * S > 4) ? 2 * S : 4;
                const long long c0 = (long long)atomicAdd(&sd.ctr->shot_next, (unsigned long long)ch);
                cn = c0 < n ? c0 : n;
                ce = (c0 + ch) < n ? (c0 + ch) : n;
            }
            const long long avail = ce - cn;
            got = (int)((long long)need < avail ? need : avail);
            s0 = cn;
            ctl->chunk_next = cn + got;
            ctl->chunk_end = ce;
            if (got < need && init_local) {
                __threadfence();
                atomicAdd(&sd.ctr->init_done, init_local);
                init_local = 0;
            }
        }
        s0 = __shfl_sync(FULLMASK, s0, 0);
        got = __shfl_sync(FULLMASK, got, 0);
    }
    if (empty) {
        if (rank < take)
            init_trial<DEBUG>(sd, L, T, lane, t0 + (unsigned long long)rank, wait_ns);
        else if (rank < take + got)
            init_shot(sd, T, lane, s0 + (rank - take));
    }
    __syncwarp();
    const bool actv = lane < S && T.st[lane].kind != 0;
    const unsigned am = __ballot_sync(FULLMASK, actv);
    const unsigned fm = __ballot_sync(FULLMASK, actv && T.st[lane].fresh);
    const unsigned im = __ballot_sync(FULLMASK, actv && T.st[lane].kind == 1);
    if (lane == 0) {
        ctl->act_mask = am;
        ctl->fresh_mask = fm;
        ctl->init_mask = im;
        ctl->exit = (am == 0u) ? 1 : 0;
    }
    __syncwarp();
}

template <int DC, int DV, bool DEBUG>
__device__ void team_loop(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int S, int W, int tid,
                          int bar_id, unsigned long long wait_ns) {
    const int lane = tid & 31, wt = tid >> 5, nthreads = 32 * W;
    unsigned long long init_local = 0, iters_local = 0, trials_local = 0;
    if (wt == 0) {
        if (lane < S) T.st[lane].kind = 0;
        if (lane == 0) {
            T.ctl->chunk_next = 0;
            T.ctl->chunk_end = 0;
        }
        __syncwarp();
        refill<DEBUG>(sd, L, T, S, lane, init_local, wait_ns);
    }
    team_sync(W, bar_id);
    while (!T.ctl->exit) {
        c_phase<DC>(sd.code, L, T, S, tid, nthreads);
        team_sync(W, bar_id);
        v_phase<DV, DEBUG>(sd, L, T, S, tid, nthreads);
        team_sync(W, bar_id);
        if (wt == 0) {
            decide<DEBUG>(sd, T, S, lane, init_local, iters_local, trials_local);
            refill<DEBUG>(sd, L, T, S, lane, init_local, wait_ns);
        }
        team_sync(W, bar_id);
    }
    if (wt == 0 && lane == 0) {
        if (init_local) {
            __threadfence();
            atomicAdd(&sd.ctr->init_done, init_local);
        }
        if (iters_local) atomicAdd(&sd.ctr->iters_total, iters_local);
        if (trials_local) atomicAdd(&sd.ctr->trial_runs, trials_local);
    }
}

struct KernelParams {
    StreamDev streams[kMaxStreams];
    int n_streams;
    int warps_per_block;
    unsigned long long wait_ns;
};

template <int DC, int DV, bool DEBUG>
__global__ void __launch_bounds__(512, 1) bpsf_persistent(const __grid_constant__ KernelParams kp) {
    extern __shared__ __align__(16) unsigned char smem[];
    volatile int *hdr = reinterpret_cast<volatile int *>(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    int cur = -1;
    bool waiting = false;
    unsigned long long wait_start = 0;
    for (;;) {
        if (tid == 0) {
            int pick = -1;
            bool all_done = true;
            const int ns = kp.n_streams;
            const int start = (cur >= 0) ? cur : (int)(blockIdx.x % (unsigned)ns);
            for (int k = 0; k < ns; ++k) {
                const int sid = (start + k) % ns;
                const StreamDev &sd = kp.streams[sid];
                const StreamCounters *c = sd.ctr;
                const unsigned long long n = (unsigned long long)sd.job.n_shots;
                const unsigned long long shot_next = ld_vol_u64(&c->shot_next);
                const unsigned long long init_done = ld_vol_u64(&c->init_done);
                __threadfence();
                const unsigned long long rc = ld_vol_u32(&c->rec_count);
                const unsigned long long tk = ld_vol_u64(&c->ticket_next);
                const bool trials = sd.code.w > 0 && !(sd.flags & kNoTickets);
                const unsigned long long rcap = rc < (unsigned long long)sd.rec.cap ? rc : (unsigned long long)sd.rec.cap;
                const unsigned long long ttot = trials ? rcap * (unsigned long long)sd.code.n_trials : 0ull;
                const bool claimable = shot_next < n || tk < ttot;
                const bool done = shot_next >= n && init_done >= n && tk >= ttot;
                if (claimable && pick < 0) pick = sid;
                if (!done) all_done = false;
            }
            hdr[0] = pick;
            hdr[1] = pick >= 0 ? 1 : (all_done ? 2 : 0);
        }
        __syncthreads();
        const int cmd = hdr[1], sid = hdr[0];
        __syncthreads();
        if (cmd == 2) break;
        if (cmd == 0) {
            // Other blocks still run initial runs that may publish trials.
            if (tid == 0) {
                const unsigned long long now = globaltimer_ns();
                if (!waiting) {
                    waiting = true;
                    wait_start = now;
                } else if (now - wait_start > kp.wait_ns) {
                    for (int k = 0; k < kp.n_streams; ++k) atomicOr(&kp.streams[k].ctr->status, kDevIdleTimeout);
                    hdr[1] = 3;
                }
                __nanosleep(1000);
            }
            __syncthreads();
            const int abort_now = hdr[1] == 3;
            __syncthreads();
            if (abort_now) break;
            continue;
        }
        waiting = false;
        const StreamDev &sd = kp.streams[sid];
        const CodeDev &cd = sd.code;
        const LayoutOffsets lo = layout_offsets(cd.M, cd.N, cd.nnz);
        unsigned char *lay = smem + kBlockHeaderBytes;
        if (sid != cur) {
            uint16_t *rp = reinterpret_cast<uint16_t *>(lay + lo.row_ptr);
            uint16_t *c2c = reinterpret_cast<uint16_t *>(lay + lo.csr_to_csc);
            uint16_t *cp = reinterpret_cast<uint16_t *>(lay + lo.col_ptr);
            uint16_t *c2r = reinterpret_cast<uint16_t *>(lay + lo.csc_to_csr);
            float *lc = reinterpret_cast<float *>(lay + lo.lch);
            for (int k = tid; k <= cd.M; k += blockDim.x) rp[k] = cd.row_ptr[k];
            for (int k = tid; k <= cd.N; k += blockDim.x) cp[k] = cd.col_ptr[k];
            for (int k = tid; k < cd.nnz; k += blockDim.x) {
                c2c[k] = cd.csr_to_csc[k];
                c2r[k] = cd.csc_to_csr[k];
            }
            for (int k = tid; k < cd.N; k += blockDim.x) lc[k] = cd.lch[k];
            cur = sid;
            __syncthreads();
        }
        LayoutMem L;
        L.row_ptr = reinterpret_cast<const uint16_t *>(lay + lo.row_ptr);
        L.csr_to_csc = reinterpret_cast<const uint16_t *>(lay + lo.csr_to_csc);
        L.col_ptr = reinterpret_cast<const uint16_t *>(lay + lo.col_ptr);
        L.csc_to_csr = reinterpret_cast<const uint16_t *>(lay + lo.csc_to_csr);
        L.lch = reinterpret_cast<const float *>(lay + lo.lch);
        const int W = sd.W, S = sd.S;
        const int teams = kp.warps_per_block / W;
        const int team = warp / W;
        if (team < teams) {
            const TeamOffsets to = team_offsets(S, cd.M, cd.N, cd.nnz, cd.Ws);
            unsigned char *tb = lay + lo.total + team * to.total;
            TeamMem T;
            T.ctl = reinterpret_cast<TeamCtl *>(tb + to.ctl);
            T.st = reinterpret_cast<SlotState *>(tb + to.state);
            T.syn = reinterpret_cast<uint32_t *>(tb + to.syn);
            T.mism = reinterpret_cast<uint32_t *>(tb + to.mism);
            T.ebits = reinterpret_cast<uint32_t *>(tb + to.ebits);
            T.flips = reinterpret_cast<uint16_t *>(tb + to.flips);
            T.q = reinterpret_cast<float *>(tb + to.q);
            T.r = reinterpret_cast<float *>(tb + to.r);
            team_loop<DC, DV, DEBUG>(sd, L, T, S, W, tid - team * W * 32, 1 + team, kp.wait_ns);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Variants and launch helpers.
// ---------------------------------------------------------------------------

static const int kVariantDC[] = {6, 8, 16, 32};
static const int kVariantDV[] = {3, 3, 8, 16};
static const int kNumVariants = 4;

int kernel_variant(int dc_max, int dv_max) {
    for (int v = 0; v < kNumVariants; ++v)
        if (dc_max <= kVariantDC[v] && dv_max <= kVariantDV[v]) return v;
    return -1;
}
int kernel_variant_dc(int v) { return kVariantDC[v]; }
int kernel_variant_dv(int v) { return kVariantDV[v]; }

typedef void (*KernelFn)(KernelParams);

static KernelFn kernel_fn(int variant, bool debug) {
    switch (variant * 2 + (debug ? 1 : 0)) {
        case 0: return bpsf_persistent<6, 3, false>;
        case 1: return bpsf_persistent<6, 3, true>;
        case 2: return bpsf_persistent<8, 3, false>;
        case 3: return bpsf_persistent<8, 3, true>;
        case 4: return bpsf_persistent<16, 8, false>;
        case 5: return bpsf_persistent<16, 8, true>;
        case 6: return bpsf_persistent<32, 16, false>;
        default: return bpsf_persistent<32, 16, true>;
    }
}

const void *persistent_kernel_ptr(int variant, bool debug) {
    return reinterpret_cast<const void *>(kernel_fn(variant, debug));
}

void launch_persistent(int variant, bool debug, int grid, int block, int smem, const LaunchArgs &args, void *stream) {
    KernelParams kp;
    for (int k = 0; k < args.n_streams; ++k) kp.streams[k] = args.streams[k];
    kp.n_streams = args.n_streams;
    kp.warps_per_block = args.warps_per_block;
    kp.wait_ns = args.wait_ns;
    kernel_fn(variant, debug)<<<grid, block, smem, (cudaStream_t)stream>>>(kp);
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
