// Device code of the persistent BP-SF kernel (Algorithm 1 of arXiv
// 2507.00254), included by the translation units that instantiate it
// (bpsf_inst_*.cu): one unit per kernel variant, so the instances compile in
// parallel.  The dispatch over variants and the harness kernels are in
// bpsf_kernels.cu.
//
// Execution model.  A block holds one MANAGER warp and `teams` compute teams
// of W warps.  A team decodes S work items ("slots") in lock step, one BP
// iteration at a time; a work item is the initial run of a shot (with
// oscillation counters) or one trial of a failed shot.  Per iteration a team
// runs
//   C phase : one thread per (slot, check): min1 / min2 / sign product over
//             the row (Eq. c2v), one FP32 multiply by alpha, C2V messages
//             written in place of the V2C messages they were computed from;
//   V phase : one thread per (slot, variable): V2C messages for the next
//             iteration (Section II-B step 2, explicit exclusion), posterior
//             LLR and hard decision (step 4), kept with the variable's flip
//             counter (Algorithm 1) in one 16-bit word; a changed decision
//             bumps the counter and toggles the slot's residual syndrome
//             s xor H e at the column's checks by shared atomics;
//   decide  : a slot whose residual syndrome is zero has converged, a slot at
//             its iteration cap is exhausted (a trial the manager found
//             unable to win under the first-success rule is stopped); the
//             slot then waits for its team's service step.
// Each message is read and written by exactly one thread in each phase, so
// one array of P floats per slot holds V2C and C2V messages alternately.
// The S slots of a team are interleaved item by item (S is a power of two):
// task tau = j*S + s (row j) or i*S + s (column i) addresses its data
// directly and a warp's lanes touch consecutive words.  A lane serves one
// slot, or 2 or 4 adjacent slots with 64- or 128-bit accesses (vector
// phases).  Installing a slot sets its messages to the channel LLRs, so the
// phases have no first-iteration special case.  With the layered schedule
// the C and V phases are replaced by layer-by-layer row updates against a
// running posterior (vector lanes for six-wide rows, else one slot per lane).
//
// Service (the team's warp 0, after an iteration in which a slot finished or
// while a slot is empty): a finished slot packs its decision into words and
// its run's facts into its outbox; a failed initial run also fills a record
// of the failure ring (Phi = top(flip_count, w), the syndrome, the shot's
// provisional output) and publishes its trials; then the slot installs the
// item the manager staged in its inbox and runs again at once.
//
// The manager warp does the rest of the global-memory work: it writes the
// outboxes out, resolves the winner of each failed shot (minimum over
// converged trials of (weight, index), merged into the shot's record by
// atomicMin), claims new shots and trial tickets ahead of time into a small
// ready queue and fills the inboxes from it.  Compute warps touch global
// memory only when a run fails (its record) or changes a decision (the
// column's check list, in L1).
#pragma once
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

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release_sys_u32(volatile unsigned *p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long ld_acquire_sys_s64(const volatile long long *p) {
    long long v;
    asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_vol_u64(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ void team_sync(int W, int bar_id) {
    if (W == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(W * 32) : "memory");
    }
}

struct BlockHdr {
    int stream, cmd;
    volatile int exit;            // manager -> teams: leave the team loop
    volatile unsigned heartbeat;  // manager passes; idle teams give up only if it stalls
    int pad[12];
};

struct LayoutMem {
    const uint8_t *row_deg;
    const uint16_t *vpos;
    const float *lch;
    const float *lch_pos;
};

struct TeamMem {
    TeamCtl *ctl;
    SlotState *st;
    uint32_t *syn, *mism, *ebits;
    unsigned char *flips;  // flip words, FB bytes each (see FlipW)
    float *m;
    OutBox *ob;         // per slot: a finished run's facts for the manager
    int *ibf;           // per slot: 1 while the inbox holds an item
    unsigned char *ib;  // per slot: the next work item
    int ibstride;
    float *post;        // layered schedule: running posterior per (variable, slot)
};

__device__ __forceinline__ TeamMem team_mem(unsigned char *tb, const TeamOffsets &to) {
    TeamMem T;
    T.ctl = reinterpret_cast<TeamCtl *>(tb + to.ctl);
    T.st = reinterpret_cast<SlotState *>(tb + to.state);
    T.syn = reinterpret_cast<uint32_t *>(tb + to.syn);
    T.mism = reinterpret_cast<uint32_t *>(tb + to.mism);
    T.ebits = reinterpret_cast<uint32_t *>(tb + to.ebits);
    T.flips = tb + to.flips;
    T.m = reinterpret_cast<float *>(tb + to.m);
    T.ob = reinterpret_cast<OutBox *>(tb + to.outbox);
    T.ibf = reinterpret_cast<int *>(tb + to.inflag);
    T.ib = tb + to.inbox;
    T.ibstride = to.ibstride;
    T.post = reinterpret_cast<float *>(tb + to.post);
    return T;
}

__device__ __forceinline__ volatile int *vstate(SlotState *s) { return reinterpret_cast<volatile int *>(&s->state); }
__device__ __forceinline__ volatile int *vflag(int *f) { return reinterpret_cast<volatile int *>(f); }

// Flip words: FB bytes per (variable, slot).  The top bit is the current hard
// decision, the bits below it count its flips (Algorithm 1): up to 32767 in
// two bytes, up to 127 in one (used only when max_iter <= 127).  Installing
// a slot zeroes them (e = 0, count 0).
template <int FB> struct FlipW;
template <> struct FlipW<2> { typedef uint16_t W; };
template <> struct FlipW<1> { typedef uint8_t W; };
template <int FB>
__device__ __forceinline__ typename FlipW<FB>::W *flipw(const TeamMem &T) {
    return reinterpret_cast<typename FlipW<FB>::W *>(T.flips);
}
template <int FB> __device__ __forceinline__ unsigned flip_dec(unsigned f) { return (f >> (8 * FB - 1)) & 1u; }
template <int FB> __device__ __forceinline__ unsigned flip_count(unsigned f) { return f & ((1u << (8 * FB - 1)) - 1u); }
// Toggle the decision and count one flip (the count is below max_iter before
// the increment, so no carry reaches the decision bit).
template <int FB> __device__ __forceinline__ unsigned flip_bump(unsigned f) { return (f ^ (1u << (8 * FB - 1))) + 1u; }

// ---------------------------------------------------------------------------
// C phase: check-node update, Eq. (c2v).  For row j with V2C inputs q_k:
//   neg = s_j xor (xor_k [q_k < 0]),  m1 = min |q_k| (first argmin k1),
//   m2 = min over k != k1,  r_k = (neg xor [q_k < 0]) ? -a : a,
//   a = alpha * (k == k1 ? m2 : m1),
// which equals the explicit "min and sign product over the other variables"
// bit for bit (min is exact; the sign factors are exact), independently of
// the order the row's edges are stored in.  V2C messages are never -0 (each
// is a fold that starts at a channel LLR > 0, and an exact cancellation
// rounds to +0), so the sign bit of q_k is [q_k < 0] and the sign product is
// an XOR of sign bits.  m2 = min(m2, max(m1, a)) keeps the second smallest
// value branch-free, equal to m1 on ties.
// ---------------------------------------------------------------------------
// C2V magnitudes are clamped here (2^100): never reached with a fixed alpha at
// the configurations; keeps messages finite when adaptive damping tends to 1.
constexpr float kMagClamp = 0x1p100f;

// Back-off of an idle team's service loop (ns), after kIdleLooks looks that
// found nothing; the manager backs off after kIdleLooks passes without progress.
constexpr unsigned kIdleMinNs = 100, kIdleMaxNs = 2048, kIdleLooks = 16;

// Damping factor of iteration t (1-based) of a run: the fixed alpha, or the
// adaptive 1 - 2^-t (alpha == 0), an exactly rounded float subtraction
// (2^-t is exact; t >= 25 rounds to 1).
__device__ __forceinline__ float damping(const CodeDev &cd, int t) {
    const float tiny = __int_as_float((127 - min(t, 126)) << 23);
    return cd.alpha > 0.f ? cd.alpha : __fsub_rn(1.0f, tiny);
}

template <int DC, bool REG>
struct CTask {
    float v[DC];
    float *p;       // message of edge rank 0 of this (row, slot); rank k sits k*M*S further
    unsigned sall;  // bit 31: s_j xor the sign bits of all inputs
    int deg;
    bool on;
};

// Task tau = j*S + s of the interleaved team layout: row j of slot s.
template <int DC, bool REG>
__device__ __forceinline__ void c_load(CTask<DC, REG> &t, const LayoutMem &L, const TeamMem &T, int MS, int lgS,
                                       int tau, bool on) {
    t.on = on;
    if (!on) return;
    t.deg = REG ? DC : (int)L.row_deg[tau >> lgS];
    t.p = T.m + tau;
    t.sall = (T.syn[tau >> 5] >> (tau & 31)) << 31;
#pragma unroll
    for (int k = 0; k < DC; ++k)
        if (REG || k < t.deg) t.v[k] = t.p[k * MS];
}

template <int DC, bool REG>
__device__ __forceinline__ void c_compute_store(CTask<DC, REG> &t, int MS, float alpha) {
    if (!t.on) return;
    // m1 <= m2 are the two smallest |q_k| (equal on ties).  The message to
    // edge k excludes k itself: alpha * m2 if |q_k| == m1, else alpha * m1
    // (on a tie m2 == m1, so either choice gives the same value).
    float m1 = __int_as_float(0x7f800000), m2 = m1;
    unsigned sx = t.sall;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (REG || k < t.deg) {
            const float a = fabsf(t.v[k]);
            m2 = fminf(m2, fmaxf(m1, a));
            m1 = fminf(m1, a);
            sx ^= __float_as_uint(t.v[k]);
        }
    }
    // The row's sign product goes into both magnitudes (they are >= 0); each
    // output then flips it by its own input's sign bit.
    sx &= 0x80000000u;
    const unsigned g1 = __float_as_uint(fminf(__fmul_rn(alpha, m1), kMagClamp)) | sx;
    const unsigned g2 = __float_as_uint(fminf(__fmul_rn(alpha, m2), kMagClamp)) | sx;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (REG || k < t.deg) {
            const unsigned mag = (fabsf(t.v[k]) == m1) ? g2 : g1;
            t.p[k * MS] = __uint_as_float(mag ^ (__float_as_uint(t.v[k]) & 0x80000000u));
        }
    }
}

// Rows (C phase) and columns (V phase) a thread handles per step: their
// loads are all issued before any of their stores, for instruction-level
// parallelism (the tasks of one step touch disjoint messages).
// Teams with S >= 2 slots run the vector phases: a lane serves up to
// BPSF_VEC adjacent slots (2 or 4); BPSF_PAIRS = 0 keeps one slot per lane.
#ifndef BPSF_PAIRS
#define BPSF_PAIRS 1
#endif
#ifndef BPSF_VEC
#define BPSF_VEC 4
#endif
#ifndef BPSF_CU
#define BPSF_CU 1
#endif
#ifndef BPSF_VU
#define BPSF_VU 1
#endif

template <int DC, bool REG>
__device__ __forceinline__ void c_phase(const CodeDev &cd, const LayoutMem &L, const TeamMem &T, int lgS, float alpha,
                                        int tid, int nthreads) {
    const int MS = cd.Mp << lgS;  // rank stride of the active layout
    const int nt = cd.M << lgS;   // row tasks (rows M..Mp-1 of the stride are padding)
    for (int tau = tid; tau < nt; tau += BPSF_CU * nthreads) {
        CTask<DC, REG> t[BPSF_CU];
#pragma unroll
        for (int u = 0; u < BPSF_CU; ++u) c_load<DC, REG>(t[u], L, T, MS, lgS, tau + u * nthreads, tau + u * nthreads < nt);
#pragma unroll
        for (int u = 0; u < BPSF_CU; ++u) c_compute_store<DC, REG>(t[u], MS, alpha);
    }
}

// ---------------------------------------------------------------------------
// V phase: variable-node update (Section II-B steps 2 and 4) and oscillation
// tracking (Algorithm 1).  For column i with C2V inputs r_0..r_{d-1} in
// ascending check order:
//   q_k   = l_ch + sum_{k' != k} r_k'   (left fold, ascending k'),
//   l_out = l_ch + sum_k r_k            (left fold),  e_i = [l_out <= 0].
// ---------------------------------------------------------------------------
template <int DVS>
struct VTask {
    uint16_t pos[DVS];  // edge positions r*Mp + j of the column's checks
    float r[DVS];
    float lc;
    unsigned f;  // decision (bit 15) and flip count of (variable, slot)
    int tau;
    bool on;
};

// Task tau = i*S + s of the interleaved team layout: column i of slot s
// (s is the lane's fixed slot).
template <int DVS, int DVX, int FB>
__device__ __forceinline__ void v_load(VTask<DVS> &t, const LayoutMem &L, const TeamMem &T, int lgS, int s, int tau,
                                       bool on) {
    t.on = on;
    if (!on) return;
    t.tau = tau;
    const int i = tau >> lgS;
    const uint16_t *vp = L.vpos + i * DVS;
    if (DVS == 4) {
        const uint2 raw = *reinterpret_cast<const uint2 *>(vp);
        t.pos[0] = (uint16_t)(raw.x & 0xffffu);
        t.pos[1] = (uint16_t)(raw.x >> 16);
        t.pos[2] = (uint16_t)(raw.y & 0xffffu);
        t.pos[3] = (uint16_t)(raw.y >> 16);
    } else {
#pragma unroll
        for (int k = 0; k < DVS; ++k) t.pos[k] = vp[k];
    }
    t.lc = L.lch[i];
    const float *ms = T.m + s;
#pragma unroll
    for (int k = 0; k < DVS; ++k)
        if (DVX > 0 ? (k < DVX) : true)
            t.r[k] = (DVX > 0 || t.pos[k] != 0xffffu) ? ms[(int)t.pos[k] << lgS] : 0.f;
    t.f = (unsigned)flipw<FB>(T)[tau];
}

template <int DVS, int DVX, bool DEBUG, int FB>
__device__ __forceinline__ void v_compute_store(const VTask<DVS> &t, const StreamDev &sd, const TeamMem &T, int lgS,
                                                int s, unsigned initm) {
    if (!t.on) return;
    float *ms = T.m + s;
    float lo;
    if (DVX == 3) {
        // Three checks: shared prefix l_ch + r0.
        const float t0 = __fadd_rn(t.lc, t.r[0]);
        const float q2 = __fadd_rn(t0, t.r[1]);
        lo = __fadd_rn(q2, t.r[2]);
        const float q1 = __fadd_rn(t0, t.r[2]);
        const float q0 = __fadd_rn(__fadd_rn(t.lc, t.r[1]), t.r[2]);
        ms[(int)t.pos[0] << lgS] = q0;
        ms[(int)t.pos[1] << lgS] = q1;
        ms[(int)t.pos[2] << lgS] = q2;
    } else {
#pragma unroll
        for (int k = 0; k < DVS; ++k) {
            if (t.pos[k] != 0xffffu) {
                float acc = t.lc;
#pragma unroll
                for (int k2 = 0; k2 < DVS; ++k2)
                    if (k2 != k && t.pos[k2] != 0xffffu) acc = __fadd_rn(acc, t.r[k2]);
                ms[(int)t.pos[k] << lgS] = acc;
            }
        }
        lo = t.lc;
#pragma unroll
        for (int k = 0; k < DVS; ++k)
            if (t.pos[k] != 0xffffu) lo = __fadd_rn(lo, t.r[k]);
    }
    const unsigned ebit = (lo <= 0.f) ? 1u : 0u;
    const int i = t.tau >> lgS;
    if (DEBUG && ((initm >> s) & 1u) && sd.dbg.lout) sd.dbg.lout[T.st[s].shot * sd.code.N + i] = lo;
    // The (variable, slot) flip word: decision and flip count (FlipW).
    if (flip_dec<FB>(t.f) != ebit) {
        flipw<FB>(T)[t.tau] = (typename FlipW<FB>::W)flip_bump<FB>(t.f);
        // The residual syndrome s xor H e toggles at this column's checks
        // (bit c*S + s of the team's residual-syndrome words).
        const uint16_t *vc = sd.code.vchk + i * DVS;
#pragma unroll
        for (int k = 0; k < DVS; ++k) {
            if (DVX > 0 ? (k < DVX) : (t.pos[k] != 0xffffu)) {
                const int b = ((int)__ldg(vc + k) << lgS) + s;
                atomicXor(&T.mism[b >> 5], 1u << (b & 31));
            }
        }
    }
}

template <int DVS, int DVX, bool DEBUG, int FB>
__device__ __forceinline__ void v_phase(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int lgS,
                                        unsigned initm, int tid, int nthreads) {
    const int total = sd.code.N << lgS;
    const int s = tid & ((1 << lgS) - 1);
    for (int tau = tid; tau < total; tau += BPSF_VU * nthreads) {
        VTask<DVS> t[BPSF_VU];
#pragma unroll
        for (int u = 0; u < BPSF_VU; ++u)
            v_load<DVS, DVX, FB>(t[u], L, T, lgS, s, tau + u * nthreads, tau + u * nthreads < total);
#pragma unroll
        for (int u = 0; u < BPSF_VU; ++u) v_compute_store<DVS, DVX, DEBUG, FB>(t[u], sd, T, lgS, s, initm);
    }
}

// ---------------------------------------------------------------------------
// Vector phases (S >= V, V = 2 or 4): lane l serves the V adjacent slots
// V*q .. V*q + V-1, q = l mod S/V.  Their items are adjacent words, so one
// 64- or 128-bit access moves all V slots' messages; column tables, LLRs,
// addresses and loop control are shared, and the V slots' residual-syndrome
// bits of a check sit in one word.  A slot of the group that is not running
// is computed on its own stale data and its messages are rewritten
// harmlessly (an install resets them); its decision/flip word and syndrome
// bits are left alone.
// ---------------------------------------------------------------------------
template <int V> struct VecF;
template <> struct VecF<2> { typedef float2 T; };
template <> struct VecF<4> { typedef float4 T; };

// The flip words of V adjacent slots packed in one integer U (slot c in the
// c-th FB-byte field).  dmask: their decision bits as a mask with bit c for
// slot c.  bump: toggle the decision and add one flip in the fields selected
// by mask bm; a count is below max_iter before the increment, so no carry
// leaves its field.
template <int FB, int V> struct FlipPack;
template <> struct FlipPack<2, 2> {
    typedef uint32_t U;
    static __device__ __forceinline__ unsigned dmask(U w) { return ((w >> 15) & 1u) | ((w >> 30) & 2u); }
    static __device__ __forceinline__ U bump(U w, unsigned bm) {
        return (w ^ (((bm & 1u) << 15) | ((bm & 2u) << 30))) + ((bm & 1u) | ((bm & 2u) << 15));
    }
};
template <> struct FlipPack<2, 4> {
    typedef uint2 U;
    static __device__ __forceinline__ unsigned dmask(U w) {
        return FlipPack<2, 2>::dmask(w.x) | (FlipPack<2, 2>::dmask(w.y) << 2);
    }
    static __device__ __forceinline__ U bump(U w, unsigned bm) {
        return make_uint2(FlipPack<2, 2>::bump(w.x, bm & 3u), FlipPack<2, 2>::bump(w.y, bm >> 2));
    }
};
template <> struct FlipPack<1, 2> {
    typedef uint16_t U;
    static __device__ __forceinline__ unsigned dmask(U w) {
        const unsigned x = w;
        return ((x >> 7) & 1u) | ((x >> 14) & 2u);
    }
    static __device__ __forceinline__ U bump(U w, unsigned bm) {
        const unsigned sp = (bm & 1u) | ((bm & 2u) << 7);
        return (U)(((unsigned)w ^ (sp << 7)) + sp);
    }
};
template <> struct FlipPack<1, 4> {
    typedef uint32_t U;
    static __device__ __forceinline__ unsigned dmask(U w) {
        return ((w >> 7) & 1u) | ((w >> 14) & 2u) | ((w >> 21) & 4u) | ((w >> 28) & 8u);
    }
    static __device__ __forceinline__ U bump(U w, unsigned bm) {
        const unsigned sp = (bm & 1u) | ((bm & 2u) << 7) | ((bm & 4u) << 14) | ((bm & 8u) << 21);
        return (w ^ (sp << 7)) + sp;
    }
};

template <int V>
__device__ __forceinline__ float &comp(typename VecF<V>::T &v, int c) { return reinterpret_cast<float *>(&v)[c]; }
template <int V>
__device__ __forceinline__ float compc(const typename VecF<V>::T &v, int c) {
    return reinterpret_cast<const float *>(&v)[c];
}

template <int DC, bool REG, int V>
__device__ __forceinline__ void c_row_vec(const LayoutMem &L, const TeamMem &T, int MQ, int lgQ, int tauv,
                                          const float (&alpha)[V]) {
    typedef typename VecF<V>::T VT;
    VT *pv = reinterpret_cast<VT *>(T.m) + tauv;  // tauv = j*(S/V) + q
    const int deg = REG ? DC : (int)L.row_deg[tauv >> lgQ];
    const unsigned sb = T.syn[(V * tauv) >> 5] >> ((V * tauv) & 31);
    VT v[DC];
#pragma unroll
    for (int k = 0; k < DC; ++k)
        if (REG || k < deg) v[k] = pv[k * MQ];
    float m1[V], m2[V];
    unsigned sx[V];
#pragma unroll
    for (int c = 0; c < V; ++c) {
        m1[c] = __int_as_float(0x7f800000);
        m2[c] = m1[c];
        sx[c] = ((sb >> c) & 1u) << 31;
    }
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (REG || k < deg) {
#pragma unroll
            for (int c = 0; c < V; ++c) {
                const float a = fabsf(compc<V>(v[k], c));
                m2[c] = fminf(m2[c], fmaxf(m1[c], a));
                m1[c] = fminf(m1[c], a);
                sx[c] ^= __float_as_uint(compc<V>(v[k], c));
            }
        }
    }
    unsigned g1[V], g2[V];
#pragma unroll
    for (int c = 0; c < V; ++c) {
        sx[c] &= 0x80000000u;
        g1[c] = __float_as_uint(fminf(__fmul_rn(alpha[c], m1[c]), kMagClamp)) | sx[c];
        g2[c] = __float_as_uint(fminf(__fmul_rn(alpha[c], m2[c]), kMagClamp)) | sx[c];
    }
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (REG || k < deg) {
            VT o;
#pragma unroll
            for (int c = 0; c < V; ++c) {
                const float x = compc<V>(v[k], c);
                comp<V>(o, c) = __uint_as_float(((fabsf(x) == m1[c]) ? g2[c] : g1[c]) ^ (__float_as_uint(x) & 0x80000000u));
            }
            pv[k * MQ] = o;
        }
    }
}

template <int DC, bool REG, int V>
__device__ __forceinline__ void c_phase_vec(const CodeDev &cd, const LayoutMem &L, const TeamMem &T, int lgS,
                                            const float (&alpha)[V], int tid, int nthreads) {
    const int lgQ = lgS - (V == 4 ? 2 : 1);
    const int MQ = cd.Mp << lgQ;  // rank stride of the active layout, in V-slot groups
    const int nt = cd.M << lgQ;   // row tasks (rows M..Mp-1 of the stride are padding)
    for (int tauv = tid; tauv < nt; tauv += nthreads) c_row_vec<DC, REG, V>(L, T, MQ, lgQ, tauv, alpha);
}

template <int DVS, int DVX, bool DEBUG, int V, int FB>
__device__ __forceinline__ void v_phase_vec(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int lgS,
                                            unsigned onm, unsigned initm, int tid, int nthreads) {
    typedef typename VecF<V>::T VT;
    typedef typename FlipPack<FB, V>::U UT;
    const CodeDev &cd = sd.code;
    const int lgQ = lgS - (V == 4 ? 2 : 1);
    const int total = cd.N << lgQ;
    const int q = tid & ((1 << lgQ) - 1);
    const int s0 = V * q;
    VT *mv = reinterpret_cast<VT *>(T.m) + q;
    UT *fv = reinterpret_cast<UT *>(T.flips);
    for (int tauv = tid; tauv < total; tauv += nthreads) {
        const int i = tauv >> lgQ;
        uint16_t pos[DVS];
        const uint16_t *vp = L.vpos + i * DVS;
        if (DVS == 4) {
            const uint2 raw = *reinterpret_cast<const uint2 *>(vp);
            pos[0] = (uint16_t)(raw.x & 0xffffu);
            pos[1] = (uint16_t)(raw.x >> 16);
            pos[2] = (uint16_t)(raw.y & 0xffffu);
            pos[3] = (uint16_t)(raw.y >> 16);
        } else {
#pragma unroll
            for (int k = 0; k < DVS; ++k) pos[k] = vp[k];
        }
        const float lc = L.lch[i];
        VT r[DVS];
#pragma unroll
        for (int k = 0; k < DVS; ++k)
            if (DVX > 0 ? (k < DVX) : (pos[k] != 0xffffu)) r[k] = mv[(int)pos[k] << lgQ];
        const UT fw = fv[tauv];
        float lo[V];
        if (DVX == 3) {
            VT q0, q1, q2;
#pragma unroll
            for (int c = 0; c < V; ++c) {
                const float t0 = __fadd_rn(lc, compc<V>(r[0], c));
                const float a2 = __fadd_rn(t0, compc<V>(r[1], c));
                lo[c] = __fadd_rn(a2, compc<V>(r[2], c));
                comp<V>(q0, c) = __fadd_rn(__fadd_rn(lc, compc<V>(r[1], c)), compc<V>(r[2], c));
                comp<V>(q1, c) = __fadd_rn(t0, compc<V>(r[2], c));
                comp<V>(q2, c) = a2;
            }
            mv[(int)pos[0] << lgQ] = q0;
            mv[(int)pos[1] << lgQ] = q1;
            mv[(int)pos[2] << lgQ] = q2;
        } else {
#pragma unroll
            for (int k = 0; k < DVS; ++k) {
                if (pos[k] != 0xffffu) {
                    VT acc;
#pragma unroll
                    for (int c = 0; c < V; ++c) comp<V>(acc, c) = lc;
#pragma unroll
                    for (int k2 = 0; k2 < DVS; ++k2)
                        if (k2 != k && pos[k2] != 0xffffu)
#pragma unroll
                            for (int c = 0; c < V; ++c) comp<V>(acc, c) = __fadd_rn(compc<V>(acc, c), compc<V>(r[k2], c));
                    mv[(int)pos[k] << lgQ] = acc;
                }
            }
#pragma unroll
            for (int c = 0; c < V; ++c) lo[c] = lc;
#pragma unroll
            for (int k = 0; k < DVS; ++k)
                if (pos[k] != 0xffffu)
#pragma unroll
                    for (int c = 0; c < V; ++c) lo[c] = __fadd_rn(lo[c], compc<V>(r[k], c));
        }
        // Decision (bit 15) and flip count of each slot's 16-bit word: the
        // running slots whose decision changed, as a mask.
        unsigned em = 0;
#pragma unroll
        for (int c = 0; c < V; ++c) {
            em |= ((lo[c] <= 0.f) ? 1u : 0u) << c;
            if (DEBUG && sd.dbg.lout && ((onm >> c) & 1u) && ((initm >> (s0 + c)) & 1u))
                sd.dbg.lout[T.st[s0 + c].shot * cd.N + i] = lo[c];
        }
        const unsigned bm = (em ^ FlipPack<FB, V>::dmask(fw)) & onm;
        if (bm) {
            fv[tauv] = FlipPack<FB, V>::bump(fw, bm);
            const uint16_t *vc = cd.vchk + i * DVS;
#pragma unroll
            for (int k = 0; k < DVS; ++k) {
                if (DVX > 0 ? (k < DVX) : (pos[k] != 0xffffu)) {
                    const int b = ((int)__ldg(vc + k) << lgS) + s0;
                    atomicXor(&T.mism[b >> 5], bm << (b & 31));
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Layered schedule (one slot per lane).  Layer by layer (rows of a layer
// share no variable, so they run in parallel and in any order), each row j
// of slot s: q_k = L_i - r_k for its edges k (i = the k-th variable of the
// row, r_k its C2V message from the previous iteration), new C2V messages
// from the q_k by Eq. (c2v) as in the C phase, then L_i = q_k + r_k.  After
// all layers L is the posterior: hard decision, flip counters and residual
// syndrome as in the V phase.
// ---------------------------------------------------------------------------
template <int DC>
__device__ __forceinline__ void layered_row(const CodeDev &cd, const LayoutMem &L, const TeamMem &T, int lgS, int j,
                                            int s, float alpha) {
    const int S = 1 << lgS, M = cd.Mp;  // rank stride of the active layout
    const int deg = (int)L.row_deg[j];
    float q[DC];
    int vi[DC];
    float *mj = T.m + (j << lgS) + s;  // edge k of row j at ((k*M + j)*S + s)
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (k < deg) {
            vi[k] = (int)__ldg(cd.pos_var + k * M + j);
            q[k] = __fsub_rn(T.post[(vi[k] << lgS) + s], mj[k * M * S]);
        }
    }
    float m1 = __int_as_float(0x7f800000), m2 = m1;
    unsigned sx = ((T.syn[((j << lgS) + s) >> 5] >> (((j << lgS) + s) & 31)) & 1u) << 31;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (k < deg) {
            const float a = fabsf(q[k]);
            m2 = fminf(m2, fmaxf(m1, a));
            m1 = fminf(m1, a);
            sx ^= __float_as_uint(q[k]);
        }
    }
    sx &= 0x80000000u;
    const unsigned g1 = __float_as_uint(fminf(__fmul_rn(alpha, m1), kMagClamp)) | sx;
    const unsigned g2 = __float_as_uint(fminf(__fmul_rn(alpha, m2), kMagClamp)) | sx;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (k < deg) {
            const float r = __uint_as_float(((fabsf(q[k]) == m1) ? g2 : g1) ^ (__float_as_uint(q[k]) & 0x80000000u));
            mj[k * M * S] = r;
            T.post[(vi[k] << lgS) + s] = __fadd_rn(q[k], r);
        }
    }
}

template <int DC, int DVS, int DVX, bool DEBUG, int FB>
__device__ __forceinline__ void layered_iteration(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int lgS,
                                                  bool lane_on, float alpha, unsigned initm, int tid, int nthreads,
                                                  int W, int bar_id) {
    const CodeDev &cd = sd.code;
    const int S = 1 << lgS;
    const int s = tid & (S - 1);
    for (int layer = 0; layer < cd.n_layers; ++layer) {
        const int r0 = (int)__ldg(cd.layer_ptr + layer), r1 = (int)__ldg(cd.layer_ptr + layer + 1);
        const int total = (r1 - r0) << lgS;
        if (lane_on)
            for (int tau = tid; tau < total; tau += nthreads)
                layered_row<DC>(cd, L, T, lgS, (int)__ldg(cd.layer_rows + r0 + (tau >> lgS)), s, alpha);
        team_sync(W, bar_id);
    }
    if (!lane_on) return;
    const int N = cd.N;
    for (int tau = tid; tau < (N << lgS); tau += nthreads) {
        const int i = tau >> lgS;
        const float lo = T.post[tau];
        const unsigned ebit = (lo <= 0.f) ? 1u : 0u;
        if (DEBUG && ((initm >> s) & 1u) && sd.dbg.lout) sd.dbg.lout[T.st[s].shot * N + i] = lo;
        const unsigned f = (unsigned)flipw<FB>(T)[tau];
        if (flip_dec<FB>(f) != ebit) {
            flipw<FB>(T)[tau] = (typename FlipW<FB>::W)flip_bump<FB>(f);
            const uint16_t *vc = cd.vchk + i * DVS;
#pragma unroll
            for (int k = 0; k < DVS; ++k) {
                const int c = (int)__ldg(vc + k);
                if (DVX > 0 ? (k < DVX) : (c != 0xffff)) {
                    const int b = (c << lgS) + s;
                    atomicXor(&T.mism[b >> 5], 1u << (b & 31));
                }
            }
        }
    }
}

// Layered schedule with V adjacent slots per lane (the slots' words are
// adjacent in the interleaved layout): the same row and posterior updates as
// layered_row, on V slots at once with vector loads and stores.  Slots of the
// group that are not running compute on stale values; their results are
// never read (a slot's messages and posterior are set up again when it takes
// its next item).
template <int DC, int V>
__device__ __forceinline__ void layered_row_vec(const CodeDev &cd, const LayoutMem &L, const TeamMem &T, int lgQ, int j,
                                                int q, const float (&alpha)[V]) {
    typedef typename VecF<V>::T VT;
    const int M = cd.Mp, MQ = cd.Mp << lgQ;  // rank stride of the active layout (in V-slot groups: MQ)
    const int deg = (int)L.row_deg[j];
    VT *mj = reinterpret_cast<VT *>(T.m) + (j << lgQ) + q;  // edge k of row j at (k*M + j)*Q + q
    VT *pv = reinterpret_cast<VT *>(T.post) + q;             // posterior of variable i at i*Q + q
    VT qv[DC];
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (k < deg) {
            const VT lp = pv[(int)__ldg(cd.pos_var + k * M + j) << lgQ], r = mj[k * MQ];
#pragma unroll
            for (int c = 0; c < V; ++c) comp<V>(qv[k], c) = __fsub_rn(compc<V>(lp, c), compc<V>(r, c));
        }
    }
    const int b0 = (j << (lgQ + (V == 4 ? 2 : 1))) + V * q;  // syndrome bit of row j, first slot of the group
    const unsigned sb = T.syn[b0 >> 5] >> (b0 & 31);
    float m1[V], m2[V];
    unsigned sx[V];
#pragma unroll
    for (int c = 0; c < V; ++c) {
        m1[c] = __int_as_float(0x7f800000);
        m2[c] = m1[c];
        sx[c] = ((sb >> c) & 1u) << 31;
    }
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (k < deg) {
#pragma unroll
            for (int c = 0; c < V; ++c) {
                const float a = fabsf(compc<V>(qv[k], c));
                m2[c] = fminf(m2[c], fmaxf(m1[c], a));
                m1[c] = fminf(m1[c], a);
                sx[c] ^= __float_as_uint(compc<V>(qv[k], c));
            }
        }
    }
    unsigned g1[V], g2[V];
#pragma unroll
    for (int c = 0; c < V; ++c) {
        sx[c] &= 0x80000000u;
        g1[c] = __float_as_uint(fminf(__fmul_rn(alpha[c], m1[c]), kMagClamp)) | sx[c];
        g2[c] = __float_as_uint(fminf(__fmul_rn(alpha[c], m2[c]), kMagClamp)) | sx[c];
    }
#pragma unroll
    for (int k = 0; k < DC; ++k) {
        if (k < deg) {
            VT r, np;
#pragma unroll
            for (int c = 0; c < V; ++c) {
                const float x = compc<V>(qv[k], c);
                comp<V>(r, c) = __uint_as_float(((fabsf(x) == m1[c]) ? g2[c] : g1[c]) ^ (__float_as_uint(x) & 0x80000000u));
                comp<V>(np, c) = __fadd_rn(x, compc<V>(r, c));
            }
            mj[k * MQ] = r;
            pv[(int)__ldg(cd.pos_var + k * M + j) << lgQ] = np;  // the variable is read again: fewer live registers
        }
    }
}

template <int DC, int DVS, int DVX, bool DEBUG, int V, int FB>
__device__ __forceinline__ void layered_iteration_vec(const StreamDev &sd, const LayoutMem &L, const TeamMem &T,
                                                      int lgS, unsigned onm, const float (&alpha)[V], unsigned initm,
                                                      int tid, int nthreads, int W, int bar_id) {
    typedef typename VecF<V>::T VT;
    typedef typename FlipPack<FB, V>::U UT;
    const CodeDev &cd = sd.code;
    const int lgQ = lgS - (V == 4 ? 2 : 1);
    const int q = tid & ((1 << lgQ) - 1);  // the lane's slot group: slots V*q .. V*q + V-1
    const int s0 = V * q;
    for (int layer = 0; layer < cd.n_layers; ++layer) {
        const int r0 = (int)__ldg(cd.layer_ptr + layer), r1 = (int)__ldg(cd.layer_ptr + layer + 1);
        const int total = (r1 - r0) << lgQ;
        if (onm)
            for (int tauv = tid; tauv < total; tauv += nthreads)
                layered_row_vec<DC, V>(cd, L, T, lgQ, (int)__ldg(cd.layer_rows + r0 + (tauv >> lgQ)), q, alpha);
        team_sync(W, bar_id);
    }
    if (!onm) return;
    const int N = cd.N;
    const VT *pv = reinterpret_cast<const VT *>(T.post);
    UT *fv = reinterpret_cast<UT *>(T.flips);
    for (int tauv = tid; tauv < (N << lgQ); tauv += nthreads) {
        const int i = tauv >> lgQ;
        const VT lo = pv[tauv];
        const UT fw = fv[tauv];
        unsigned em = 0;
#pragma unroll
        for (int c = 0; c < V; ++c) {
            em |= ((compc<V>(lo, c) <= 0.f) ? 1u : 0u) << c;
            if (DEBUG && sd.dbg.lout && ((onm >> c) & 1u) && ((initm >> (s0 + c)) & 1u))
                sd.dbg.lout[T.st[s0 + c].shot * N + i] = compc<V>(lo, c);
        }
        const unsigned bm = (em ^ FlipPack<FB, V>::dmask(fw)) & onm;
        if (bm) {
            fv[tauv] = FlipPack<FB, V>::bump(fw, bm);
            const uint16_t *vc = cd.vchk + i * DVS;
#pragma unroll
            for (int k = 0; k < DVS; ++k) {
                const int c = (int)__ldg(vc + k);
                if (DVX > 0 ? (k < DVX) : (c != 0xffff)) {
                    const int b = (c << lgS) + s0;
                    atomicXor(&T.mism[b >> 5], bm << (b & 31));
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Team-side slot service (warp 0 of the team, all lanes).  A finished slot
// (PENDING) hands its facts to its outbox as soon as the manager has drained
// the previous ones; a free slot (EMPTY) installs the item the manager put
// in its inbox.  The slot therefore runs again at the team's next iteration,
// without a round trip through the manager.
// ---------------------------------------------------------------------------

// Pack finished slot s into its outbox: the hard decision into words and the
// run's facts.  A failed initial run (with trials) also gets its record
// here: Phi = top(flip_count, w) (keys (count << 16 | 0xffff - i) are
// distinct, so each round takes the largest key below the previous one:
// count descending, index ascending), the shot's syndrome, an empty
// selection and the provisional output (the initial run's e, not
// converged), and only then is the record published for the trials.
template <bool DEBUG, int FB>
__device__ __forceinline__ void team_pack(const StreamDev &sd, const TeamMem &T, int lgS, int s, int lane,
                                          unsigned long long wait_ns) {
    const CodeDev &cd = sd.code;
    const int N = cd.N, Wn = cd.Wn;
    const SlotState *ss = &T.st[s];
    OutBox *ob = &T.ob[s];
    for (int w = 0; w < Wn; ++w) {
        const int i = 32 * w + lane;
        const unsigned b = i < N ? flip_dec<FB>((unsigned)flipw<FB>(T)[(i << lgS) + s]) : 0u;
        const unsigned word = __ballot_sync(FULLMASK, b != 0u);
        if (lane == 0) T.ebits[s * Wn + w] = word;
    }
    const int kind = ss->kind, outcome = ss->outcome;
    if (kind == 1 && outcome == 2 && cd.w > 0) {
        const JobDev &job = sd.job;
        const long long shot = ss->shot;
        const long long row = (sd.flags & kServe) ? (shot % sd.serve.rows) : shot;
        // Phi into lane registers: lane r % 32 holds Phi[r] (r < 32 in phi0, else phi1).
        int phi0 = -1, phi1 = -1;
        unsigned thr = 0xffffffffu;
        for (int r = 0; r < cd.w; ++r) {
            unsigned best = 0;
            for (int i = lane; i < N; i += 32) {
                const unsigned key =
                    (flip_count<FB>((unsigned)flipw<FB>(T)[(i << lgS) + s]) << 16) | (0xffffu - (unsigned)i);
                if (key < thr && key > best) best = key;
            }
            best = __reduce_max_sync(FULLMASK, best);
            const int phi_r = (int)(0xffffu - (best & 0xffffu));
            if (lane == (r & 31)) {
                if (r < 32)
                    phi0 = phi_r;
                else
                    phi1 = phi_r;
            }
            if (DEBUG && lane == 0 && sd.dbg.phi) sd.dbg.phi[shot * cd.w + r] = phi_r;
            thr = best;
        }
        // The next failure number and its record, once free (a bounded wait;
        // more failed shots in flight than records is reported).
        unsigned long long q = 0;
        if (lane == 0) {
            q = atomicAdd(&sd.ctr->rec_count, 1ull);
            const unsigned long long *qs = sd.rec.qseq + (q & (unsigned long long)(sd.rec.cap - 1));
            if (ld_acquire_u64(qs) != 0ull) {
                const unsigned long long t0 = globaltimer_ns();
                while (ld_acquire_u64(qs) != 0ull) {
                    if (globaltimer_ns() - t0 > wait_ns) {
                        atomicOr(&sd.ctr->status, kDevRecordOverflow);
                        break;
                    }
                    __nanosleep(256);
                }
            }
        }
        q = __shfl_sync(FULLMASK, q, 0);
        const long long rs = (long long)(q & (unsigned long long)(sd.rec.cap - 1));
        if (lane < cd.w) sd.rec.phi[rs * cd.w + lane] = phi0;
        if (lane + 32 < cd.w) sd.rec.phi[rs * cd.w + lane + 32] = phi1;
        // The slot's syndrome (check j sits at bit j*S + s of the team's words).
        for (int w = 0; w < cd.Ws; ++w) {
            const int j = 32 * w + lane;
            const int b = (j << lgS) + s;
            const unsigned bit = j < cd.M ? (T.syn[b >> 5] >> (b & 31)) & 1u : 0u;
            const unsigned word = __ballot_sync(FULLMASK, bit != 0u);
            if (lane == 0) sd.rec.synd[rs * cd.Ws + w] = word;
        }
        __syncwarp();  // lane 0's decision words are visible to the warp
        uint32_t *out = job.corr + row * job.corr_stride;
        for (int w = lane; w < Wn; w += 32) {
            sd.rec.win[rs * Wn + w] = ~0ull;
            out[w] = T.ebits[s * Wn + w];
        }
        if (lane == 0) {
            job.conv[row] = 0;
            job.iters[row] = (int16_t)cd.max_iter;
            if (job.stage) job.stage[row] = 2;
            sd.rec.done[rs] = 0u;
            sd.rec.best[rs] = ~0ull;
            sd.rec.qshot[rs] = shot;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_u64(sd.rec.qseq + rs, q + 1ull);
    }
    if (DEBUG && kind == 1 && sd.dbg.flips)
        for (int i = lane; i < N; i += 32)
            sd.dbg.flips[ss->shot * N + i] = (uint16_t)flip_count<FB>((unsigned)flipw<FB>(T)[(i << lgS) + s]);
    if (lane == 0) {
        ob->kind = kind;
        ob->kidx = ss->kidx;
        ob->rec = ss->rec;
        ob->outcome = outcome;
        ob->iter = ss->iter;
        ob->shot = ss->shot;
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        *vflag(&ob->full) = 1;
    }
    __syncwarp();
}

// Install slot s's inbox item: the slot's bits of the syndrome and
// residual-syndrome words (atomic toggles of the bits that differ: lanes
// share words), its V2C messages set to the channel LLRs (the first C phase
// reads l_ch on every edge), its decision and flip-count words zeroed.
template <int FB>
__device__ __forceinline__ void team_install(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int S, int s,
                                             int lane) {
    const CodeDev &cd = sd.code;
    const QEntry *e = reinterpret_cast<const QEntry *>(T.ib + s * T.ibstride);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(T.ib + s * T.ibstride + sizeof(QEntry));
    SlotState *ss = &T.st[s];
    volatile uint32_t *vsyn = T.syn, *vmism = T.mism;
    for (int j = lane; j < cd.M; j += 32) {
        const unsigned want = (src[j >> 5] >> (j & 31)) & 1u;
        const int b = j * S + s;
        const unsigned m = 1u << (b & 31);
        if (((vsyn[b >> 5] & m) != 0u) != (want != 0u)) atomicXor(&T.syn[b >> 5], m);
        if (((vmism[b >> 5] & m) != 0u) != (want != 0u)) atomicXor(&T.mism[b >> 5], m);
    }
    if (cd.layered) {
        // Layered schedule: C2V messages start at zero, the posterior at l_ch.
        for (int k = lane; k < cd.P; k += 32) T.m[k * S + s] = 0.f;
        for (int i = lane; i < cd.N; i += 32) T.post[i * S + s] = L.lch[i];
    } else {
        for (int k = lane; k < cd.P; k += 32) T.m[k * S + s] = L.lch_pos[k];
    }
    for (int i = lane; i < cd.N; i += 32) flipw<FB>(T)[i * S + s] = 0;
    if (lane == 0) {
        ss->kind = e->kind;
        ss->kidx = e->kidx;
        ss->rec = e->rec;
        ss->shot = e->shot;
        ss->iter = 0;
        ss->start = -1;  // set by the team at the service that starts the run
        ss->outcome = 0;
        ss->cancel = 0;
        ss->limit = e->kind == 1 ? cd.max_iter : cd.short_iter;
    }
    __syncwarp();
}

template <bool DEBUG, int FB>
__device__ __forceinline__ void team_service(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, int S, int lgS,
                                             int lane, unsigned long long wait_ns) {
    const int stv = lane < S ? *vstate(&T.st[lane]) : kSlotRunning;
    const bool obf = lane < S && *vflag(&T.ob[lane].full) != 0;
    unsigned pm = __ballot_sync(FULLMASK, stv == kSlotPending && !obf);
    if (pm) __threadfence_block();  // the manager's reads of the drained outboxes are done
    while (pm) {
        const int s = __ffs(pm) - 1;
        pm &= pm - 1u;
        team_pack<DEBUG, FB>(sd, T, lgS, s, lane, wait_ns);
        // team_pack set the outbox flag before the slot reads EMPTY (the
        // manager's exit test reads the state first, then the outbox flag).
        if (lane == 0) {
            __threadfence_block();
            *vstate(&T.st[s]) = kSlotEmpty;
        }
    }
    __syncwarp();
    const bool want = lane < S && *vstate(&T.st[lane]) == kSlotEmpty && *vflag(&T.ibf[lane]) != 0;
    unsigned im = __ballot_sync(FULLMASK, want);
    if (im) __threadfence_block();  // the inbox items are visible
    while (im) {
        const int s = __ffs(im) - 1;
        im &= im - 1u;
        const int kind = reinterpret_cast<const QEntry *>(T.ib + s * T.ibstride)->kind;
        if (kind != 0) team_install<FB>(sd, L, T, S, s, lane);
        __syncwarp();
        if (lane == 0) {
            // RUNNING before the inbox reads empty: the manager's exit test
            // reads the inbox flag first, then the state.
            __threadfence_block();
            if (kind != 0) *vstate(&T.st[s]) = kSlotRunning;
            __threadfence_block();
            *vflag(&T.ibf[s]) = 0;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Compute team loop.
//
// A team iteration is: C phase, barrier, V phase, barrier, decision.  The
// decision needs no further barrier: every warp reads the residual-syndrome
// words (stable until the next V phase, which lies beyond the next barrier)
// and the iteration's stop mask (written by warp 0 before the first barrier,
// one word per iteration parity), so all warps agree on which slots are done.
// The service step (a barrier, warp 0 packs finished slots and installs new
// items, a barrier) runs only after an iteration in which a slot finished, or
// while a slot is empty, and with an iteration chunk k > 1 at most every k
// iterations while some slot still runs; a team whose slots all keep running
// goes from one iteration to the next with two barriers.
// ---------------------------------------------------------------------------
template <int DC, int DVS, int DVX, bool DEBUG, int MINB, bool LAY, int FB>
__device__ void team_loop(const StreamDev &sd, const LayoutMem &L, const TeamMem &T, BlockHdr *hdr, int S, int W,
                          int tid, int bar_id, unsigned long long wait_ns) {
    const int lane = tid & 31, wt = tid >> 5, nthreads = 32 * W;
    const CodeDev &cd = sd.code;
    const int lgS = __ffs(S) - 1;
    const int my_slot = lane & (S - 1);             // the slot this lane serves in every phase
    const int n_rwords = ((cd.M << lgS) + 31) >> 5;  // residual-syndrome words of the team
    const unsigned full = S >= 32 ? 0xffffffffu : ((1u << S) - 1u);
    constexpr bool kVec = BPSF_PAIRS && DC <= 16;  // the widest rows keep one slot per lane (registers)
    // Four slots per lane: exact-degree rows with the full register budget (one block).
    constexpr bool kVec4 = kVec && MINB == 1 && DVX == 3 && BPSF_VEC >= 4;
    // Layered schedule: vector lanes in the full-register instances only.
    constexpr bool kLayV2 = LAY && kVec && MINB == 1 && DC <= 6, kLayV4 = kLayV2 && kVec4;
    const bool lay = LAY && cd.layered;
    // Slots per lane in the phases (vs) and the lane's first slot (s0).
    const int vs = lay ? ((kLayV4 && S >= 4) ? 4 : ((kLayV2 && S >= 2) ? 2 : 1))
                       : ((kVec4 && S >= 4) ? 4 : ((kVec && S >= 2) ? 2 : 1));
    const int s0 = vs * (lane & ((S / vs) - 1));
    unsigned run = 0u, initm = 0u;
    int tt = 0;  // team iterations run (the same in every warp)
    // Every warp, lane l < S: the team iteration after which slot l's run
    // reaches its iteration cap.
    int l_end = 0;
    // Warp 0, lane 0: iterations run since the last service, and the team
    // iteration of that service (added to the control block at the next one).
    unsigned n_iters = 0;
    int tt_flush = 0;
    const bool first_rule = cd.select == 1;
    const bool adaptive = !(cd.alpha > 0.f);  // alpha_t = 1 - 2^-t needs each run's iteration number
    bool svc = true;
    const int chunk = sd.chunk > 1 ? sd.chunk : 1;  // iterations between refills of finished slots
    int since = 0;                                  // team iterations since the last service
    // The idle state (warp 0 only, rarely used) lives in the control block.
    if (wt == 0 && lane == 0) {
        T.ctl->idle_since = 0;
        T.ctl->idle_ns = kIdleMinNs;
        T.ctl->idle_looks = 0;
    }
    for (;;) {
        if (svc) {
            // Every warp has made the previous decision (read the residual
            // words, which an install rewrites) and has read the control
            // block of the previous service.
            team_sync(W, bar_id);
            if (wt == 0) {
                // The work counters first: the manager adds them up once every
                // slot of the block reads empty, which the service below may make so.
                if (lane == 0 && tt != tt_flush) {
                    T.ctl->iters += n_iters;
                    T.ctl->cap += (unsigned long long)(tt - tt_flush) * (unsigned)S;
                    n_iters = 0;
                    tt_flush = tt;
                }
                team_service<DEBUG, FB>(sd, L, T, S, lgS, lane, wait_ns);
                SlotState *ss = &T.st[lane < S ? lane : 0];
                const int stv = lane < S ? *vstate(ss) : kSlotEmpty;
                const bool r = stv == kSlotRunning;
                __threadfence_block();
                const unsigned rm = __ballot_sync(FULLMASK, r);
                const unsigned im = __ballot_sync(FULLMASK, r && ss->kind == 1);
                // A run installed at this service starts with the next iteration.
                if (r && ss->start < 0) ss->start = tt;
                int ex = 0;
                if (rm == 0u) {
                    if (hdr->exit) {
                        ex = 1;
                    } else {
                        // Never wait forever: give up only if the manager has made
                        // no pass for twice the bound on any of its own waits.
                        const unsigned long long now = globaltimer_ns();
                        const unsigned beat = hdr->heartbeat;
                        unsigned long long since_ns = T.ctl->idle_since;
                        if (since_ns == 0 || beat != T.ctl->last_beat) since_ns = now;
                        if (now - since_ns > 2 * wait_ns) ex = 1;
                        // A team idle for more than a few looks backs off (up
                        // to 2 us), so the warps of the block that do run keep
                        // the issue slots; short gaps between runs keep the
                        // short sleep.
                        unsigned ns = T.ctl->idle_ns;
                        const unsigned looks = T.ctl->idle_looks + 1;
                        __nanosleep(ns);
                        if (looks > kIdleLooks) ns = ns < kIdleMaxNs ? 2 * ns : kIdleMaxNs;
                        __syncwarp();
                        if (lane == 0) {
                            T.ctl->idle_since = since_ns;
                            T.ctl->last_beat = beat;
                            T.ctl->idle_ns = ns;
                            T.ctl->idle_looks = looks;
                        }
                    }
                } else if (lane == 0) {
                    T.ctl->idle_since = 0;
                    T.ctl->idle_ns = kIdleMinNs;
                    T.ctl->idle_looks = 0;
                }
                if (lane == 0) {
                    T.ctl->run_mask = rm;
                    T.ctl->init_mask = im;
                    T.ctl->exit = ex;
                }
            }
            team_sync(W, bar_id);
            run = T.ctl->run_mask;
            initm = T.ctl->init_mask;
            const int ex = T.ctl->exit;
            if (ex) break;
            if (run == 0u) continue;
            if (lane < S) l_end = T.st[lane].start + T.st[lane].limit - 1;
            svc = false;
            since = 0;
        }
        // First-success rule: warp 0 publishes the trials the manager asked to
        // stop (they cannot win), read by every warp after this iteration.
        if (first_rule && wt == 0) {
            bool cancel = false;
            if (lane < S && ((run >> lane) & 1u) && T.st[lane].kind == 2)
                cancel = *reinterpret_cast<volatile long long *>(&T.st[lane].cancel) ==
                         T.st[lane].shot * (long long)cd.n_trials + T.st[lane].kidx + 1;
            const unsigned cm = __ballot_sync(FULLMASK, cancel);
            if (lane == 0) T.ctl->stop_mask[tt & 1] = cm;
        }
        // Damping of iteration it = tt - start + 1 of each of the lane's slots
        // (the start is read only under adaptive damping).
        float al[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
            al[c] = adaptive && c < vs ? damping(cd, tt - T.st[s0 + c].start + 1) : cd.alpha;
        if (lay) {
            if (kLayV4 && vs == 4) {
                float a4[4] = {al[0], al[1], al[2], al[3]};
                layered_iteration_vec<DC, DVS, DVX, DEBUG, 4, FB>(sd, L, T, lgS, (run >> s0) & 0xfu, a4, initm, tid,
                                                              nthreads, W, bar_id);
            } else if (kLayV2 && vs == 2) {
                float a2[2] = {al[0], al[1]};
                layered_iteration_vec<DC, DVS, DVX, DEBUG, 2, FB>(sd, L, T, lgS, (run >> s0) & 0x3u, a2, initm, tid,
                                                              nthreads, W, bar_id);
            } else {
                const bool lane_on = (run >> my_slot) & 1u;
                layered_iteration<DC, DVS, DVX, DEBUG, FB>(sd, L, T, lgS, lane_on, al[0], initm, tid, nthreads, W,
                                                       bar_id);
            }
            team_sync(W, bar_id);
        } else if (kVec4 && vs == 4) {
            const unsigned onm = (run >> s0) & 0xfu;
            float a4[4] = {al[0], al[1], al[2], al[3]};
            if (onm) c_phase_vec<DC, (DVX > 0), 4>(cd, L, T, lgS, a4, tid, nthreads);
            team_sync(W, bar_id);
            if (onm) v_phase_vec<DVS, DVX, DEBUG, 4, FB>(sd, L, T, lgS, onm, initm, tid, nthreads);
            team_sync(W, bar_id);
        } else if (kVec && vs == 2) {
            const unsigned onm = (run >> s0) & 0x3u;
            float a2[2] = {al[0], al[1]};
            if (onm) c_phase_vec<DC, (DVX > 0), 2>(cd, L, T, lgS, a2, tid, nthreads);
            team_sync(W, bar_id);
            if (onm) v_phase_vec<DVS, DVX, DEBUG, 2, FB>(sd, L, T, lgS, onm, initm, tid, nthreads);
            team_sync(W, bar_id);
        } else {
            const bool lane_on = (run >> my_slot) & 1u;
            if (lane_on) c_phase<DC, (DVX > 0)>(cd, L, T, lgS, al[0], tid, nthreads);
            team_sync(W, bar_id);
            if (lane_on) v_phase<DVS, DVX, DEBUG, FB>(sd, L, T, lgS, initm, tid, nthreads);
            team_sync(W, bar_id);
        }
        // Decision, in every warp: slot s owns bits s, s + S, s + 2S, ... of
        // every residual-syndrome word, so OR-folding the words down to S
        // bits leaves bit s set iff slot s's residual syndrome is not zero.
        unsigned acc = 0;
        for (int w = lane; w < n_rwords; w += 32) acc |= T.mism[w];
        acc = __reduce_or_sync(FULLMASK, acc);
        for (int sh = 16; sh >= S; sh >>= 1) acc |= acc >> sh;
        const unsigned nconv = acc & full;
        // Runs at their iteration cap (every warp knows every slot's cap), and
        // trials asked to stop.
        const unsigned capped = __ballot_sync(FULLMASK, lane < S && tt >= l_end);
        const unsigned cancelled = first_rule ? T.ctl->stop_mask[tt & 1] : 0u;
        const unsigned done = run & (~nconv | capped | cancelled);
        if (wt == 0) {
            if ((done >> lane) & 1u) {
                SlotState *ss = &T.st[lane];
                ss->iter = tt - ss->start + 1;
                ss->outcome = !((nconv >> lane) & 1u) ? 1 : (((cancelled >> lane) & 1u) ? 3 : 2);
                // Finished slots are packed by the next service step.
                *vstate(ss) = kSlotPending;
            }
            n_iters += __popc(run);
        }
        // Finished slots leave the run mask at once (their decisions and flip
        // counts stay as they were) and wait for the next service, which comes
        // after the iteration chunk, or at once when no slot is left running.
        ++tt;
        ++since;
        run &= ~done;
        svc = run == 0u || (since >= chunk && run != full);
    }
}

// ---------------------------------------------------------------------------
// Manager warp.
// ---------------------------------------------------------------------------

// Manager state: head and tail are warp-uniform; the two counters are per
// lane (each lane counts the slots it wrote out) and are summed over the
// warp before they are added to the global counters.
struct MgrState {
    int head, tail;          // ready queue (ring of Q entries)
    unsigned init_local;     // finished initial runs not yet counted globally
    unsigned trials_local;   // finished trial runs not yet counted globally
    unsigned trials_cancelled; // trials not run or stopped because they could not win
};

__device__ __forceinline__ QEntry *qentry(unsigned char *q, int idx, int stride) {
    return reinterpret_cast<QEntry *>(q + idx * stride);
}

__device__ __forceinline__ uint32_t *qsyn(QEntry *e) {
    return reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(e) + sizeof(QEntry));
}

// Word w of finished slot s's hard decision (packed by its team).
__device__ __forceinline__ unsigned slot_word(const uint32_t *ebits, int Wn, int s, int w) { return ebits[s * Wn + w]; }


__device__ __forceinline__ long long row_of(const StreamDev &sd, long long shot) {
    return (sd.flags & kServe) ? (shot % sd.serve.rows) : shot;
}

// One shot's final output is out: when serving, post it to the row's
// completion word (the outputs live in host-mapped memory, hence the
// system-scope fence before the release).
__device__ __forceinline__ void shot_complete(const StreamDev &sd, long long row, long long shot) {
    if (!(sd.flags & kServe)) return;
    __threadfence_system();
    st_release_sys_u32(sd.serve.row_done + row, (unsigned)(shot + 1));
}

// One trial of a failed shot is over (run, or cancelled because it cannot
// win): count it; the last one settles the winner (the minimum key of the
// shot's converged trials) and completes the shot.
__device__ __forceinline__ void trial_done(const StreamDev &sd, long long rs, long long row, long long shot) {
    const CodeDev &cd = sd.code;
    const JobDev &job = sd.job;
    const int C = cd.n_trials, Wn = cd.Wn;
    __threadfence();
    const unsigned d = atomicAdd(&sd.rec.done[rs], 1u) + 1u;
    if (d == (unsigned)C) {
        __threadfence();
        const unsigned long long best = atomicAdd(&sd.rec.best[rs], 0ull);
        if (best != ~0ull) {
            // Every converged trial merged its words before it counted itself
            // done, so each word now holds the winner's (smallest key's) word.
            uint32_t *out = job.corr + row * job.corr_stride;
            const unsigned long long *src = sd.rec.win + rs * Wn;
            for (int w = 0; w < Wn; ++w) out[w] = (uint32_t)(__ldcg(src + w) & 0xffffffffull);
            job.conv[row] = 1;
            job.iters[row] = (int16_t)(best & 0xffffull);
            if (job.stage) job.stage[row] = 1;
        }
        // The record is free for a later failure once its reads are done.
        __threadfence();
        st_release_u64(sd.rec.qseq + rs, 0ull);
        shot_complete(sd, row, shot);
    }
}

// Under the first-success rule (select = 1) the winner is the earliest
// converged trial: once trial k* has converged, no later trial can win.
__device__ __forceinline__ bool trial_cannot_win(const StreamDev &sd, long long rs, int kidx) {
    if (sd.code.select != 1) return false;
    const unsigned long long best = __ldcg(sd.rec.best + rs);
    return best != ~0ull && (long long)(best >> 32) < (long long)kidx;
}

// Lane-parallel write-out of outboxes that need no warp cooperation:
// converged or uncorrectable initial runs, and trial runs.
template <bool DEBUG>
__device__ __forceinline__ void finalize_simple(const StreamDev &sd, TeamMem T, int s, MgrState &mg) {
    const CodeDev &cd = sd.code;
    const JobDev &job = sd.job;
    const OutBox *ss = &T.ob[s];
    const int kind = ss->kind, iter = ss->iter;
    const bool conv = ss->outcome == 1;
    const long long shot = ss->shot;
    const long long row = row_of(sd, shot);
    const int Wn = cd.Wn;
    if (kind == 1) {
        mg.init_local += 1;
        // A failed run with trials already has its record and provisional
        // output (written by its team before it published the trials).
        if (!conv && cd.w > 0) return;
        uint32_t *out = job.corr + row * job.corr_stride;
        for (int w = 0; w < Wn; ++w) out[w] = slot_word(T.ebits, Wn, s, w);
        job.conv[row] = conv ? 1 : 0;
        job.iters[row] = (int16_t)(conv ? iter : cd.max_iter);
        if (job.stage) job.stage[row] = conv ? 0 : 2;
        shot_complete(sd, row, shot);
        return;
    }
    // Trial run: undo the flip (Algorithm 1) and take part in the selection.
    const int C = cd.n_trials, kidx = ss->kidx;
    const long long rs = ss->rec;
    if (conv) {
        // e' xor t, in the slot's packed decision (the outbox is this lane's
        // until it is released): t flips the record's Phi[j] for the bits j
        // of the trial's mask.
        uint32_t *ew = T.ebits + s * Wn;
        const unsigned long long mask = __ldg(cd.trial_mask + kidx);
        for (int j = 0; j < cd.w; ++j) {
            if (!((mask >> j) & 1ull)) continue;
            const int b = __ldcg(sd.rec.phi + rs * cd.w + j);
            ew[b >> 5] ^= 1u << (b & 31);
        }
        unsigned wsum = 0;
        for (int w = 0; w < Wn; ++w) wsum += __popc(ew[w]);
        // Selection key (unique per trial): weight, then list index; or the
        // list index alone under the first-success rule.
        const unsigned long long key = cd.select == 0 ? (((unsigned long long)wsum << 12) | (unsigned)kidx)
                                                      : (unsigned long long)kidx;
        const unsigned long long old = atomicMin(&sd.rec.best[rs], (key << 32) | (unsigned)iter);
        // Only a trial that held the smallest key so far merges its words: the
        // final winner always does, and merges of others cannot beat it.
        if ((old >> 32) > key) {
            unsigned long long *win = sd.rec.win + rs * Wn;
            for (int w = 0; w < Wn; ++w) atomicMin(win + w, (key << 32) | ew[w]);
        }
    }
    if (DEBUG) {
        if (sd.dbg.trial_conv) sd.dbg.trial_conv[shot * C + kidx] = conv ? 1 : 0;
        if (sd.dbg.trial_iters) sd.dbg.trial_iters[shot * C + kidx] = (int16_t)iter;
    }
    if (ss->outcome == 3)
        mg.trials_cancelled += 1;  // stopped: it could not win
    else
        mg.trials_local += 1;
    trial_done(sd, rs, row, shot);
}

// Shots that may be claimed now.
__device__ __forceinline__ long long shots_available(const StreamDev &sd) {
    if (sd.flags & kServe) return ld_acquire_sys_s64(sd.serve.published);
    return sd.job.n_shots;
}

// Fill the ready queue: trial tickets first, then new shots.
template <bool DEBUG>
__device__ __forceinline__ bool prefetch(const StreamDev &sd, unsigned char *qbase, int Q, int qstride, int lane,
                                         MgrState &mg, int n_empty, unsigned long long wait_ns) {
    const CodeDev &cd = sd.code;
    const int Ws = cd.Ws;
    bool got_any = false;
    int space = Q - (mg.tail - mg.head);
    if (space > 0 && cd.w > 0 && !(sd.flags & kNoTickets)) {
        unsigned long long t0 = 0;
        int take = 0;
        if (lane == 0) {
            for (int att = 0; att < 4; ++att) {
                const unsigned long long cur = ld_vol_u64(&sd.ctr->ticket_next);
                const unsigned long long total = ld_vol_u64(&sd.ctr->rec_count) * (unsigned long long)cd.n_trials;
                if (cur >= total) break;
                unsigned long long want = total - cur;
                unsigned long long lim = space < 32 ? (unsigned long long)space : 32ull;
                // Few tickets left (the tail of a failed shot's trials): take
                // no more than the slots free now, so they spread over blocks.
                if (want < 128ull && lim > (unsigned long long)n_empty) lim = (unsigned long long)n_empty;
                if (lim == 0ull) break;
                if (want > lim) want = lim;
                if (atomicCAS(&sd.ctr->ticket_next, cur, cur + want) == cur) {
                    t0 = cur;
                    take = (int)want;
                    break;
                }
            }
        }
        t0 = __shfl_sync(FULLMASK, t0, 0);
        take = __shfl_sync(FULLMASK, take, 0);
        if (lane < take) {
            const unsigned long long ticket = t0 + lane;
            const unsigned long long qi = ticket / (unsigned long long)cd.n_trials;
            const int kidx = (int)(ticket - qi * (unsigned long long)cd.n_trials);
            const long long slot_q = (long long)(qi % (unsigned long long)sd.rec.cap);
            bool ok = true, timed_out = false;
            if (ld_acquire_u64(sd.rec.qseq + slot_q) != qi + 1ull) {
                const unsigned long long start = globaltimer_ns();
                while (ld_acquire_u64(sd.rec.qseq + slot_q) != qi + 1ull) {
                    if (globaltimer_ns() - start > wait_ns) {
                        atomicOr(&sd.ctr->status, kDevReadyTimeout);
                        ok = false;
                        timed_out = true;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            QEntry *e = qentry(qbase, (mg.tail + lane) % Q, qstride);
            if (ok && trial_cannot_win(sd, slot_q, kidx)) ok = false;  // early cancel: counted, not run
            if (ok) {
                const long long shot = __ldcg(sd.rec.qshot + slot_q);
                e->kind = 2;
                e->kidx = (int16_t)kidx;
                e->rec = (int)slot_q;
                e->shot = shot;
                // The trial vector t: the bits Phi[j] its mask selects.
                const unsigned long long mask = __ldg(cd.trial_mask + kidx);
                uint32_t *sy = qsyn(e);
                for (int w = 0; w < Ws; ++w) sy[w] = __ldcg(sd.rec.synd + slot_q * Ws + w);
                // s' = s xor t H^T (Algorithm 1): flip the checks of every selected bit.
                for (int j = 0; j < cd.w; ++j) {
                    if (!((mask >> j) & 1ull)) continue;
                    const int v = __ldcg(sd.rec.phi + slot_q * cd.w + j);
                    for (int k = 0; k < cd.vstride; ++k) {
                        const int c = __ldg(cd.vchk + v * cd.vstride + k);
                        if (c == 0xffff) break;
                        sy[c >> 5] ^= 1u << (c & 31);
                    }
                }
                if (DEBUG && sd.dbg.trial_synd)
                    for (int w = 0; w < Ws; ++w)
                        sd.dbg.trial_synd[(shot * cd.n_trials + kidx) * Ws + w] = sy[w];
            } else {
                // Dropped.  A trial that cannot win is counted as done now; after a
                // timed-out wait the record never settles and the status reports it.
                if (!timed_out) {
                    const long long shot = __ldcg(sd.rec.qshot + slot_q);
                    trial_done(sd, slot_q, row_of(sd, shot), shot);
                    ++mg.trials_cancelled;
                }
                e->kind = 0;
            }
        }
        __syncwarp();
        mg.tail += take;
        space -= take;
        got_any = take > 0;
    }
    if (space > 0) {
        long long c0 = 0;
        int got = 0;
        if (lane == 0) {
            const long long avail = shots_available(sd);
            const long long want = space < 32 ? space : 32;
            if (sd.flags & kServe) {
                for (int att = 0; att < 4; ++att) {
                    const long long cur = (long long)ld_vol_u64(&sd.ctr->shot_next);
                    if (cur >= avail) break;
                    const long long nw = (avail - cur) < want ? (avail - cur) : want;
                    if ((long long)atomicCAS(&sd.ctr->shot_next, (unsigned long long)cur,
                                             (unsigned long long)(cur + nw)) == cur) {
                        c0 = cur;
                        got = (int)nw;
                        break;
                    }
                }
            } else if ((long long)ld_vol_u64(&sd.ctr->shot_next) < avail) {
                c0 = (long long)atomicAdd(&sd.ctr->shot_next, (unsigned long long)want);
                const long long hi = (c0 + want) < avail ? (c0 + want) : avail;
                got = c0 < avail ? (int)(hi - c0) : 0;
            }
        }
        c0 = __shfl_sync(FULLMASK, c0, 0);
        got = __shfl_sync(FULLMASK, got, 0);
        // Lane 0's acquire of the published count orders the other lanes'
        // reads of the rows too (when serving, the host writes the rows
        // before it publishes them).
        __syncwarp();
        if (lane < got) {
            const long long shot = c0 + lane;
            const long long row = row_of(sd, shot);
            QEntry *e = qentry(qbase, (mg.tail + lane) % Q, qstride);
            e->kind = 1;
            e->kidx = 0;
            e->rec = -1;
            e->shot = shot;
            const uint32_t *src = sd.job.synd + row * sd.job.synd_stride;
            uint32_t *sy = qsyn(e);
            for (int w = 0; w < Ws; ++w) sy[w] = __ldcg(src + w);
        }
        __syncwarp();
        mg.tail += got;
        got_any = got_any || got > 0;
    }
    return got_any;
}

template <bool DEBUG>
__device__ void manager_loop(const StreamDev &sd, const LayoutMem &L, unsigned char *team_base, int team_bytes,
                             const TeamOffsets &to, int teams, int S, unsigned char *qbase, int Q, BlockHdr *hdr,
                             int lane, unsigned long long wait_ns) {
    const CodeDev &cd = sd.code;
    const int qstride = qentry_bytes(cd.Ws);
    const int nslots = teams * S;
    MgrState mg{0, 0, 0u, 0u, 0u};
    unsigned idle_ns = 32;     // back-off after passes that found nothing to do
    unsigned idle_passes = 0;  // consecutive passes without progress
    for (;;) {
        bool progress = false;
        bool busy = false;
        int n_empty = 0;  // idle slots of the block with an empty inbox (warp-uniform)
        if (lane == 0) hdr->heartbeat = hdr->heartbeat + 1u;
        // (A) write out the outboxes the teams filled.
        for (int g0 = 0; g0 < nslots; g0 += 32) {
            const int g = g0 + lane;
            const bool inr = g < nslots;
            const int t = inr ? g / S : 0, s = inr ? g - t * S : 0;
            TeamMem T = team_mem(team_base + t * team_bytes, to);
            const int stv = inr ? *vstate(&T.st[s]) : kSlotEmpty;
            const bool fin = inr && *vflag(&T.ob[s].full) != 0;
            __threadfence_block();
            if (__any_sync(FULLMASK, stv != kSlotEmpty)) busy = true;
            // First-success rule: ask running trials that can no longer win to stop.
            if (cd.select == 1 && stv == kSlotRunning && T.st[s].kind == 2) {
                const long long shot = T.st[s].shot;
                const int kidx = T.st[s].kidx;
                const long long key = shot * (long long)cd.n_trials + kidx + 1;
                if (T.st[s].cancel != key && trial_cannot_win(sd, T.st[s].rec, kidx))
                    *reinterpret_cast<volatile long long *>(&T.st[s].cancel) = key;
            }
            if (fin) finalize_simple<DEBUG>(sd, T, s, mg);
            __syncwarp();
            if (fin) {
                __threadfence_block();
                *vflag(&T.ob[s].full) = 0;
            }
            if (__any_sync(FULLMASK, fin)) progress = true;
        }
        __syncwarp();
        // (B) fill empty inboxes from the ready queue: idle slots first (they
        // start at once), then running ones (their next run).  Count the
        // slots left idle with nothing in their inbox.
        for (int pass = 0; pass < 2; ++pass) {
            for (int g0 = 0; g0 < nslots && (pass == 1 || mg.tail > mg.head); g0 += 32) {
                const int g = g0 + lane;
                const bool inr = g < nslots;
                const int t = inr ? g / S : 0, s = inr ? g - t * S : 0;
                TeamMem T = team_mem(team_base + t * team_bytes, to);
                const bool idle = inr && *vstate(&T.st[s]) == kSlotEmpty;
                const bool open = inr && *vflag(&T.ibf[s]) == 0 && (pass == 1 || idle);
                const unsigned om = __ballot_sync(FULLMASK, open);
                const int rank = __popc(om & ((1u << lane) - 1u));
                const int avail = mg.tail - mg.head;
                const bool take = open && rank < avail;
                if (take) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(qentry(qbase, (mg.head + rank) % Q, qstride));
                    uint4 *dst = reinterpret_cast<uint4 *>(T.ib + s * T.ibstride);
                    for (int k = 0; k < qstride / 16; ++k) dst[k] = src[k];
                    __threadfence_block();
                    *vflag(&T.ibf[s]) = 1;
                }
                const int used = __popc(om) < avail ? __popc(om) : avail;
                mg.head += used;
                if (used) progress = true;
                if (pass == 1) n_empty += __popc(__ballot_sync(FULLMASK, open && !take && idle));
            }
        }
        __syncwarp();
        // (C) claim work ahead.
        if (prefetch<DEBUG>(sd, qbase, Q, qstride, lane, mg, n_empty, wait_ns)) progress = true;
        // Count finished initial runs once no new shot can be claimed.
        if (!(sd.flags & kServe)) {
            int exhausted = 0;
            if (lane == 0) exhausted = (long long)ld_vol_u64(&sd.ctr->shot_next) >= sd.job.n_shots;
            exhausted = __shfl_sync(FULLMASK, exhausted, 0);
            if (exhausted) {
                const unsigned tot = __reduce_add_sync(FULLMASK, mg.init_local);
                mg.init_local = 0;
                if (lane == 0 && tot) {
                    __threadfence();
                    atomicAdd(&sd.ctr->init_done, (unsigned long long)tot);
                }
            }
        }
        // (D) leave when nothing is running, queued, boxed or claimable.
        if (!busy && !progress && mg.tail == mg.head) {
            bool any_slot = false;
            for (int g0 = 0; g0 < nslots; g0 += 32) {
                const int g = g0 + lane;
                const int t = g < nslots ? g / S : 0, s = g < nslots ? g - t * S : 0;
                TeamMem T = team_mem(team_base + t * team_bytes, to);
                // Read order matters: inbox flag, state, outbox flag (the
                // team writes state before clearing the inbox flag, and the
                // outbox flag before the state).
                bool occ = false;
                if (g < nslots) {
                    occ = *vflag(&T.ibf[s]) != 0;
                    __threadfence_block();
                    occ = occ || *vstate(&T.st[s]) != kSlotEmpty;
                    __threadfence_block();
                    occ = occ || *vflag(&T.ob[s].full) != 0;
                }
                if (__any_sync(FULLMASK, occ)) any_slot = true;
            }
            // Nothing left for this code: hand the block back, which then
            // waits across all codes (serving) or for other blocks' trials.
            if (!any_slot) break;
        }
        // A run of passes that find nothing backs off, up to 1 us (a finished
        // slot then waits that long at most for its write-out); any progress
        // resets it.
        if (progress) {
            idle_ns = 32;
            idle_passes = 0;
        } else {
            __nanosleep(idle_ns);
            if (++idle_passes > kIdleLooks) idle_ns = idle_ns < 1024 ? 2 * idle_ns : 1024;
        }
    }
    // Flush counters and release the teams.
    const unsigned init_tot = __reduce_add_sync(FULLMASK, mg.init_local);
    const unsigned trial_tot = __reduce_add_sync(FULLMASK, mg.trials_local);
    const unsigned skip_tot = __reduce_add_sync(FULLMASK, mg.trials_cancelled);
    if (lane == 0) {
        if (init_tot) {
            __threadfence();
            atomicAdd(&sd.ctr->init_done, (unsigned long long)init_tot);
        }
        if (trial_tot) atomicAdd(&sd.ctr->trial_runs, (unsigned long long)trial_tot);
        if (skip_tot) atomicAdd(&sd.ctr->trials_cancelled, (unsigned long long)skip_tot);
        unsigned long long it = 0, cap = 0;
        for (int t = 0; t < teams; ++t) {
            TeamMem T = team_mem(team_base + t * team_bytes, to);
            it += T.ctl->iters;
            cap += T.ctl->cap;
            T.ctl->iters = 0;
            T.ctl->cap = 0;
        }
        if (it) atomicAdd(&sd.ctr->iters_total, it);
        if (cap) atomicAdd(&sd.ctr->slot_capacity, cap);
        __threadfence_block();
        hdr->exit = 1;
    }
    __syncwarp();
}

// MINB: minimum resident blocks per SM the register allocation must allow.
// Two caps registers at 64 per thread, so two 512-thread blocks (or three
// smaller ones) fit on an SM; one keeps the full budget, which four slots
// per lane need.  The exact-degree variant has both instances (the launch
// plan picks by the blocks that fit); the others (wider rows, irregular
// codes whose shared-memory needs allow few slots per SM anyway) have one.
#ifndef BPSF_MIN_BLOCKS
#define BPSF_MIN_BLOCKS 2
#endif

// LAY: the instance also runs codes with the layered schedule (a launch
// with no such code uses the instance without that path and its registers).
// FB: bytes per flip word (FlipW): 2, or 1 for launches whose codes all have
// max_iter <= 127 (an instance that leaves more shared memory for slots).
// MIX: the instance also carries the exact (6, 4, 3) team loop and runs it
// for codes with exactly six ones per row and three per column, so such codes
// keep their specialised path in a launch that mixes them with codes of
// wider rows (the layouts agree: both have column tables of width DVS).
template <int DC, int DVS, int DVX, bool DEBUG, int MINB, bool LAY, int FB = 2, bool MIX = false>
__global__ void __launch_bounds__(512, MINB) bpsf_persistent(const __grid_constant__ KernelParams kp) {
    extern __shared__ __align__(16) unsigned char smem[];
    BlockHdr *hdr = reinterpret_cast<BlockHdr *>(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Q = kp.Q;
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
                if (sd.flags & kServe) {
                    const long long pub = ld_acquire_sys_s64(sd.serve.published);
                    const long long sn = (long long)ld_vol_u64(&c->shot_next);
                    const unsigned long long ttot = ld_vol_u64(&c->rec_count) * (unsigned long long)sd.code.n_trials;
                    const bool claimable = sn < pub || ld_vol_u64(&c->ticket_next) < ttot;
                    if (claimable && pick < 0) pick = sid;
                    if (claimable || !*sd.serve.stop) all_done = false;
                    continue;
                }
                const unsigned long long n = (unsigned long long)sd.job.n_shots;
                const unsigned long long shot_next = ld_vol_u64(&c->shot_next);
                const unsigned long long init_done = ld_vol_u64(&c->init_done);
                __threadfence();
                const unsigned long long rc = ld_vol_u64(&c->rec_count);
                const unsigned long long tk = ld_vol_u64(&c->ticket_next);
                const bool trials = sd.code.w > 0 && !(sd.flags & kNoTickets);
                const unsigned long long ttot = trials ? rc * (unsigned long long)sd.code.n_trials : 0ull;
                const bool claimable = shot_next < n || tk < ttot;
                const bool done = shot_next >= n && init_done >= n && tk >= ttot;
                if (claimable && pick < 0) pick = sid;
                if (!done) all_done = false;
            }
            hdr->stream = pick;
            hdr->cmd = pick >= 0 ? 1 : (all_done ? 2 : 0);
        }
        __syncthreads();
        const int cmd = hdr->cmd, sid = hdr->stream;
        __syncthreads();
        if (cmd == 2) break;
        if (cmd == 0) {
            // Other blocks still run initial runs that may publish trials, or
            // a serving loop waits for requests.
            if (tid == 0) {
                const unsigned long long now = globaltimer_ns();
                bool serve_any = false, serve_quit = true;
                for (int k = 0; k < kp.n_streams; ++k)
                    if (kp.streams[k].flags & kServe) {
                        serve_any = true;
                        if (!*kp.streams[k].serve.stop &&
                            (!waiting || now - wait_start <= (unsigned long long)kp.streams[k].serve.idle_ns))
                            serve_quit = false;
                    }
                if (!waiting) {
                    waiting = true;
                    wait_start = now;
                } else if (serve_any) {
                    if (serve_quit) hdr->cmd = 3;
                } else if (now - wait_start > kp.wait_ns) {
                    for (int k = 0; k < kp.n_streams; ++k) atomicOr(&kp.streams[k].ctr->status, kDevIdleTimeout);
                    hdr->cmd = 3;
                }
                __nanosleep(1000);
            }
            __syncthreads();
            const int quit = hdr->cmd == 3;
            __syncthreads();
            if (quit) break;
            continue;
        }
        waiting = false;
        const StreamDev &sd = kp.streams[sid];
        const CodeDev &cd = sd.code;
        const int S = sd.S, W = sd.W, teams = sd.teams;
        const LayoutOffsets lo = layout_offsets(cd.M, cd.N, DVS, cd.P);
        unsigned char *lay = smem + kBlockHeaderBytes;
        if (sid != cur) {
            uint8_t *rd = lay + lo.row_deg;
            uint16_t *vp = reinterpret_cast<uint16_t *>(lay + lo.vpos);
            float *lc = reinterpret_cast<float *>(lay + lo.lch);
            float *lp = reinterpret_cast<float *>(lay + lo.lch_pos);
            for (int k = tid; k < cd.M; k += blockDim.x) rd[k] = cd.row_deg[k];
            for (int k = tid; k < cd.N * DVS; k += blockDim.x) vp[k] = cd.vpos[k];
            for (int k = tid; k < cd.N; k += blockDim.x) lc[k] = cd.lch[k];
            for (int k = tid; k < cd.P; k += blockDim.x) lp[k] = cd.lch_pos[k];
            cur = sid;
        }
        // Every slot starts empty; teams start idle.
        const TeamOffsets to = team_offsets(S, cd.M, cd.N, cd.P, cd.Ws, cd.layered, FB);
        unsigned char *qbase = lay + lo.total;
        unsigned char *team_base = qbase + Q * qentry_bytes(cd.Ws);
        for (int k = tid; k < teams * S; k += blockDim.x) {
            unsigned char *tb = team_base + (k / S) * to.total;
            SlotState *ss = reinterpret_cast<SlotState *>(tb + to.state) + (k % S);
            ss->state = kSlotEmpty;
            ss->kind = 0;
            ss->cancel = 0;
            reinterpret_cast<OutBox *>(tb + to.outbox)[k % S].full = 0;
            reinterpret_cast<int *>(tb + to.inflag)[k % S] = 0;
        }
        for (int t = tid; t < teams; t += blockDim.x) {
            TeamCtl *ctl = reinterpret_cast<TeamCtl *>(team_base + t * to.total + to.ctl);
            ctl->iters = 0;
            ctl->cap = 0;
            ctl->exit = 0;
        }
        // Syndrome and residual-syndrome words start at zero: installs toggle
        // only their own slot's bits, and the padding bits past S*M are read
        // by the convergence test.
        {
            const int sw = (to.mism - to.syn) / 4;
            for (int k = tid; k < teams * 2 * sw; k += blockDim.x) {
                const int t = k / (2 * sw), w = k - t * 2 * sw;
                reinterpret_cast<uint32_t *>(team_base + t * to.total + to.syn)[w] = 0u;
            }
        }
        if (tid == 0) {
            hdr->exit = 0;
            hdr->heartbeat = 0u;
        }
        __syncthreads();
        LayoutMem L;
        L.row_deg = lay + lo.row_deg;
        L.vpos = reinterpret_cast<const uint16_t *>(lay + lo.vpos);
        L.lch = reinterpret_cast<const float *>(lay + lo.lch);
        L.lch_pos = reinterpret_cast<const float *>(lay + lo.lch_pos);
        if (warp == 0) {
            manager_loop<DEBUG>(sd, L, team_base, to.total, to, teams, S, qbase, Q, hdr, lane, kp.wait_ns);
        } else {
            const int team = (warp - 1) / W;
            if (team < teams) {
                TeamMem T = team_mem(team_base + team * to.total, to);
                const int ttid = tid - 32 - team * W * 32;
                if (MIX && cd.regular && cd.DC == 6 && cd.dv_max == 3)
                    team_loop<6, DVS, 3, DEBUG, MINB, LAY, FB>(sd, L, T, hdr, S, W, ttid, 1 + team, kp.wait_ns);
                else
                    team_loop<DC, DVS, DVX, DEBUG, MINB, LAY, FB>(sd, L, T, hdr, S, W, ttid, 1 + team, kp.wait_ns);
            }
        }
        __syncthreads();
    }
}

}  // namespace bpsf
