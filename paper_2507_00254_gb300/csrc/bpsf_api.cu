// Host side of libbpsf: argument checking, Tanner-graph layout, device
// workspace, the batched / plain / host-buffer / mixed-code decode forms,
// launch-shape tuning and the autotuner.  See include/bpsf.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "bpsf.h"
#include "bpsf_api_internal.h"
#include "bpsf_internal.h"

using namespace bpsf;

static thread_local std::string g_err;

bpsf_status bpsf_fail(bpsf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

extern "C" const char *bpsf_last_error(void) { return g_err.c_str(); }

extern "C" const char *bpsf_status_str(bpsf_status s) {
    switch (s) {
        case BPSF_OK: return "ok";
        case BPSF_EINVAL: return "invalid argument";
        case BPSF_ENOMEM: return "out of memory";
        case BPSF_ECUDA: return "CUDA error";
        case BPSF_ETIMEOUT: return "timeout";
        case BPSF_EBUSY: return "busy";
        case BPSF_ECLOSED: return "closed";
        case BPSF_EDEVICE: return "device error";
    }
    return "unknown status";
}

// Bound on any device-side wait (a trial waiting for its record, a block
// waiting for other blocks to publish trials).
const unsigned long long kBpsfWaitNs = 5ull * 1000 * 1000 * 1000;

static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// ---------------------------------------------------------------------------
// Context lifetime
// ---------------------------------------------------------------------------

static void free_workspace(bpsf_ctx *c) {
    if (c->d_rec) cudaFree(c->d_rec);
    c->d_rec = nullptr;
    c->rec = Records{};
    c->rec_cap = 0;
}

extern "C" void bpsf_destroy(bpsf_ctx *c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    free_workspace(c);
    if (c->d_code) cudaFree(c->d_code);
    if (c->d_trials) cudaFree(c->d_trials);
    if (c->d_layouts) cudaFree(c->d_layouts);
    if (c->d_ctr) cudaFree(c->d_ctr);
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    if (c->h_flag) cudaFreeHost(c->h_flag);
    if (c->h_preset) cudaFreeHost(c->h_preset);
    if (c->d_host_stage) cudaFree(c->d_host_stage);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

bpsf_status bpsf_ensure_kernel_attrs(int variant, int smem_optin) {
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    for (int k4 = 0; k4 < 4; ++k4) {  // debug x layered instances
        const int k = variant * 4 + k4;
        if (done[k]) continue;
        const void *fn = persistent_kernel_ptr(variant, (k4 & 1) != 0, (k4 & 2) != 0);
        if (!fn) continue;  // an instance the variant does not have
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        done[k] = true;
    }
    return BPSF_OK;
}

// ---------------------------------------------------------------------------
// Launch plans
// ---------------------------------------------------------------------------

// The slots' inboxes hold one item each besides the ready queue, so the
// queue only covers claim batches.
static int plan_queue(int teams, int S) { return std::min(32, std::max(16, teams * S / 2)); }

static int plan_smem(const bpsf_ctx *c, int vstride, int S, int teams, int Q, int fb = 2) {
    return block_smem_bytes(c->M, c->N, c->code.lay[layout_index(S)].P, c->Ws, vstride, S, teams, Q, c->code.layered,
                            fb);
}

static bpsf_status check_shape(const bpsf_tuning &t) {
    const int W = t.warps_per_team, S = t.slots_per_team, B = t.warps_per_block;
    if (!(W == 1 || W == 2 || W == 4 || W == 8)) return bpsf_fail(BPSF_EINVAL, "warps_per_team must be 1, 2, 4 or 8");
    if (S < 1 || S > kMaxSlots || (S & (S - 1)))
        return bpsf_fail(BPSF_EINVAL, "slots_per_team must be a power of two in 1..%d", kMaxSlots);
    if (B < W || B > kMaxComputeWarps || B % W)
        return bpsf_fail(BPSF_EINVAL, "warps_per_block must be a multiple of warps_per_team, at most %d",
                         kMaxComputeWarps);
    if (t.blocks_per_sm < 0) return bpsf_fail(BPSF_EINVAL, "blocks_per_sm must be >= 0");
    if (t.iter_chunk < 0 || t.iter_chunk > 64) return bpsf_fail(BPSF_EINVAL, "iter_chunk must be in 0..64");
    return BPSF_OK;
}

// Resident blocks per SM of a kernel instance at a block size and shared
// memory size, queried once and remembered: a plan made while a stream is
// being captured into a CUDA graph then makes no query.
static cudaError_t blocks_per_sm(const void *fn, int block, int smem, int *occ) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int>, int> cache;
    const auto key = std::make_tuple(fn, block, smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *occ = it->second;
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, block, smem);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = *occ;
    }
    return e;
}

bpsf_status bpsf_make_plan(bpsf_ctx *const *codes, int n_codes, const bpsf_tuning *tunes, bool debug,
                           bpsf_plan *out, bool shrink) {
    // One kernel variant must fit every code of the launch.
    bool all_regular = true, layered = false;
    int dc = 0, dv = 0, B = 0, bps = 0;
    for (int k = 0; k < n_codes; ++k) layered = layered || codes[k]->code.layered;
    for (int k = 0; k < n_codes; ++k) {
        bpsf_status st = check_shape(tunes[k]);
        if (st != BPSF_OK) return st;
        all_regular = all_regular && codes[k]->regular && codes[k]->dc_max == codes[0]->dc_max &&
                      codes[k]->dv_max == codes[0]->dv_max;
        dc = std::max(dc, codes[k]->dc_max);
        dv = std::max(dv, codes[k]->dv_max);
        B = std::max(B, tunes[k].warps_per_block);
        if (tunes[k].blocks_per_sm > 0) bps = bps > 0 ? std::min(bps, tunes[k].blocks_per_sm) : tunes[k].blocks_per_sm;
    }
    int variant = kernel_variant(all_regular ? -dc : dc, std::max(dv, 1));
    if (variant < 0) return bpsf_fail(BPSF_EINVAL, "no kernel variant for row degree %d, column degree %d", dc, dv);
    const int vstride = kernel_variant_dv(variant);
    const bpsf_ctx *c0 = codes[0];
    int Q = 32;
    for (int k = 0; k < n_codes; ++k)
        Q = std::max(Q, plan_queue(tunes[k].warps_per_block / tunes[k].warps_per_team, tunes[k].slots_per_team));
    // Team shape per code: its own tuning; when shrinking, fewer slots per
    // team first, then fewer teams, until the code's block fits.  fb: bytes
    // per flip word of the instance the sizes are for.
    int smem = 0;
    for (int k = 0; k < n_codes; ++k)
        if (codes[k]->vstride != vstride)
            return bpsf_fail(BPSF_EINVAL, "codes of one launch need the same column table width (%d vs %d)",
                             codes[k]->vstride, vstride);
    auto size_codes = [&](int fb, bool allow_shrink) -> bool {
        smem = 0;
        for (int k = 0; k < n_codes; ++k) {
            const int W = tunes[k].warps_per_team;
            int S = tunes[k].slots_per_team, teams = tunes[k].warps_per_block / W;
            while (allow_shrink && plan_smem(codes[k], vstride, S, teams, Q, fb) > c0->smem_optin) {
                if (S > 1)
                    S >>= 1;
                else if (teams > 1)
                    --teams;
                else
                    break;
            }
            const int need = plan_smem(codes[k], vstride, S, teams, Q, fb);
            if (need > c0->smem_optin) return false;
            out->S_code[k] = S;
            out->W_code[k] = W;
            out->teams_code[k] = teams;
            out->chunk_code[k] = std::max(1, tunes[k].iter_chunk);
            smem = std::max(smem, need);
        }
        return true;
    };
    // One-byte flip words fit a shape that two-byte words do not: every code is
    // of the exact (6, 4, 3) variant with max_iter <= 127 and none is layered.
    bool byte_flips_ok = kernel_variant_byte_flips(variant) >= 0 && !layered;
    for (int k = 0; k < n_codes; ++k) byte_flips_ok = byte_flips_ok && codes[k]->p.max_iter <= 127;
    bool byte_flips = false;
    if (!size_codes(2, false)) {
        if (byte_flips_ok && size_codes(1, false))
            byte_flips = true;
        else if (!(shrink && size_codes(2, true)))
            return bpsf_fail(BPSF_EINVAL, "launch shape needs more than %d bytes of shared memory", c0->smem_optin);
    }
    for (int k = 0; k < n_codes; ++k)
        if (out->W_code[k] > 1 && out->teams_code[k] > kMaxNamedTeams)
            return bpsf_fail(BPSF_EINVAL, "too many multi-warp teams");
    if (byte_flips) variant = kernel_variant_byte_flips(variant);
    // Exact (6, 4, 3) codes in a launch that needs wider rows keep their own path.
    if (!all_regular && !layered && kernel_variant_mixed(variant) >= 0) {
        bool any_exact = false;
        for (int k = 0; k < n_codes; ++k)
            any_exact = any_exact || (codes[k]->regular && codes[k]->dc_max == 6 && codes[k]->dv_max == 3);
        if (any_exact) variant = kernel_variant_mixed(variant);
    }
    bpsf_status st = bpsf_ensure_kernel_attrs(variant, c0->smem_optin);
    if (st != BPSF_OK) return st;
    const int block = 32 * (B + 1);
    int occ = 0;
    cudaError_t e = blocks_per_sm(persistent_kernel_ptr(variant, debug, layered), block, smem, &occ);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
    if (bps > 0) occ = std::min(occ, bps);
    // Fewer than two blocks per SM: the variant's full-register instance runs the
    // same work with more registers per thread (and four slots per lane).
    const int full = kernel_variant_full_regs(variant);
    if (occ < 2 && full != variant) {
        st = bpsf_ensure_kernel_attrs(full, c0->smem_optin);
        if (st != BPSF_OK) return st;
        int occ1 = 0;
        e = blocks_per_sm(persistent_kernel_ptr(full, debug, layered), block, smem, &occ1);
        if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
        if (occ1 >= 1) {
            variant = full;
            occ = 1;
        }
    }
    if (occ <= 0) return bpsf_fail(BPSF_EINVAL, "launch shape does not fit on an SM");
    out->variant = variant;
    out->layered = layered;
    out->Q = Q;
    out->block = block;
    out->smem = smem;
    out->grid = occ * c0->sm_count;
    return BPSF_OK;
}

static bpsf_tuning default_tuning(bpsf_ctx *c) {
    // Small codes: single-warp teams with a few slots each; large codes:
    // multi-warp teams.  Shrink until the block fits.
    const int Wc[] = {1, 1, 1, 2, 4, 8};
    const int Sc[] = {4, 2, 1, 2, 1, 1};
    for (int k = 0; k < 6; ++k) {
        if (c->nnz > 2048 && Wc[k] < 4) continue;
        for (int B = kMaxComputeWarps; B >= Wc[k]; --B) {
            if (B % Wc[k]) continue;
            bpsf_tuning t{Wc[k], Sc[k], B, 0};
            bpsf_plan pl;
            bpsf_ctx *cs[1] = {c};
            if (bpsf_make_plan(cs, 1, &t, false, &pl) == BPSF_OK) return t;
        }
    }
    return bpsf_tuning{1, 1, 1, 0};
}

// ---------------------------------------------------------------------------
// Context creation
// ---------------------------------------------------------------------------

// Default trial list of Algorithm 1: every non-empty subset of Phi of weight
// <= w_max, as masks (bit j selects Phi[j]) in ascending order.
static long long default_trial_count(int w, int w_max) {
    long long n = 0, c = 1;  // c = C(w, k)
    for (int k = 1; k <= w_max && k <= w; ++k) {
        c = c * (w - k + 1) / k;
        n += c;
        if (n > (1ll << 40)) break;
    }
    return n;
}

static void add_subsets(std::vector<unsigned long long> &out, int w, int k, int start, unsigned long long m) {
    if (k == 0) {
        if (m) out.push_back(m);
        return;
    }
    for (int b = start; b <= w - k; ++b) add_subsets(out, w, k - 1, b + 1, m | (1ull << b));
}

static std::vector<unsigned long long> default_trials(int w, int w_max) {
    std::vector<unsigned long long> out;
    for (int k = 1; k <= w_max && k <= w; ++k) add_subsets(out, w, k, 0, 0ull);
    std::sort(out.begin(), out.end());
    return out;
}

// ---------------------------------------------------------------------------
// Message layout per slot count (see LayoutS).  The column phase gathers the
// messages of consecutive variables; with slots interleaved, the lanes of
// one shared-memory access phase (32 lanes for 32-bit accesses, 16 for
// 64-bit, 8 for 128-bit) hit bank group (chunk mod 32/V), chunk = (r*Mp + j)
// * (S/V) + q for the q-th V-slot group.  Distinct chunks in one group
// serialise.  A deterministic local search over the rank stride (M plus a
// small pad) and the order of the edges within each row minimises the
// number of wavefronts; any choice decodes identically.
// ---------------------------------------------------------------------------
struct LayoutSearch {
    int M, N, dv, S, V, Q, lpp, G;
    const std::vector<std::vector<int>> *rows;
    const std::vector<std::vector<std::pair<int, int>>> *cols;  // (check, index in the sorted row)
    std::vector<int> row_off;                                   // first edge id of each row
    std::vector<int> edge_k;                                    // edge id -> its index in its column
};

// Wavefronts of one access phase: the k-th column edge of the lanes tau in
// [ph, ph + lpp), lane tau serving V-slot group q = tau % Q of variable tau / Q.
static int phase_cost(const LayoutSearch &L, const std::vector<int> &rank, int Mp, int k, int ph) {
    int chunks[32][32];  // per bank group, the distinct chunks seen (at most lpp)
    int cnt[32];
    for (int g = 0; g < L.G; ++g) cnt[g] = 0;
    int worst = 0;
    const int end = std::min(ph + L.lpp, L.N * L.Q);
    for (int tau = ph; tau < end; ++tau) {
        const int i = tau / L.Q, q = tau % L.Q;
        const auto &ci = (*L.cols)[i];
        if (k >= (int)ci.size()) continue;
        const int j = ci[k].first, e = L.row_off[j] + ci[k].second;
        const int chunk = (rank[e] * Mp + j) * L.Q + q, g = chunk % L.G;
        bool seen = false;
        for (int a = 0; a < cnt[g]; ++a) seen = seen || chunks[g][a] == chunk;
        if (!seen) chunks[g][cnt[g]++] = chunk;
        worst = std::max(worst, cnt[g]);
    }
    return worst;
}

static void search_layout(const LayoutSearch &L, int max_pad_dc, int &Mp_out, std::vector<int> &rank_out) {
    const int nnz = L.row_off.back();
    std::vector<int> rank0(nnz);
    for (int j = 0; j < L.M; ++j)
        for (int t = 0; t < (int)(*L.rows)[j].size(); ++t) rank0[L.row_off[j] + t] = t;
    Mp_out = L.M;
    rank_out = rank0;
    if (L.Q >= L.G || L.M < 2) return;  // a phase holds one variable's slots: no conflicts to remove
    auto total = [&](const std::vector<int> &rk, int Mp) {
        long long t = 0;
        for (int k = 0; k < L.dv; ++k)
            for (int ph = 0; ph < L.N * L.Q; ph += L.lpp) t += phase_cost(L, rk, Mp, k, ph);
        return t;
    };
    long long best = total(rank0, L.M);
    // A swap of two edges of one row moves exactly two messages, each read in
    // one phase, so only those phases are re-costed.
    const int iters = std::min(12000, 16 * nnz);
    const int pads[] = {0, 1, 3, 5};
    for (int pad : pads) {
        const int Mp = L.M + pad;
        if ((long long)max_pad_dc * Mp > 65534) continue;
        std::vector<int> rk = rank0;
        long long cur = total(rk, Mp);
        unsigned long long x = 0x9E3779B97F4A7C15ull ^ (unsigned long long)(L.S * 131 + pad);
        for (int it = 0; it < iters; ++it) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            const int j = (int)((x >> 33) % (unsigned long long)L.M);
            const int deg = (int)(*L.rows)[j].size();
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            const int a = (int)((x >> 33) % (unsigned long long)deg);
            int b = (int)((x >> 13) % (unsigned long long)(deg - 1));
            if (b >= a) ++b;
            const int ea = L.row_off[j] + a, eb = L.row_off[j] + b;
            const int ka = L.edge_k[ea], kb = L.edge_k[eb];
            const int pa = ((*L.rows)[j][a] * L.Q) / L.lpp * L.lpp, pb = ((*L.rows)[j][b] * L.Q) / L.lpp * L.lpp;
            const bool same = ka == kb && pa == pb;
            const int before = phase_cost(L, rk, Mp, ka, pa) + (same ? 0 : phase_cost(L, rk, Mp, kb, pb));
            std::swap(rk[ea], rk[eb]);
            const int after = phase_cost(L, rk, Mp, ka, pa) + (same ? 0 : phase_cost(L, rk, Mp, kb, pb));
            if (after <= before)
                cur += after - before;
            else
                std::swap(rk[ea], rk[eb]);
        }
        if (cur < best) {
            best = cur;
            Mp_out = Mp;
            rank_out = rk;
        }
    }
}

extern "C" bpsf_status bpsf_create(bpsf_ctx **out, int32_t M, int32_t N, int64_t nnz, int32_t layout,
                                   const int32_t *ptr, const int32_t *idx, const double *priors,
                                   const bpsf_params *params) {
    if (!out) return bpsf_fail(BPSF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ptr || !idx || !priors || !params) return bpsf_fail(BPSF_EINVAL, "NULL array or params");
    if (M < 1 || M > 65535 || N < 1 || N > 65535) return bpsf_fail(BPSF_EINVAL, "M and N must be in 1..65535");
    if (nnz < 1 || nnz > 65535) return bpsf_fail(BPSF_EINVAL, "nnz must be in 1..65535");
    if (layout != BPSF_CSR && layout != BPSF_CSC) return bpsf_fail(BPSF_EINVAL, "layout must be BPSF_CSR or BPSF_CSC");
    const bpsf_params p = *params;
    if (p.flags & ~(uint32_t)BPSF_FLAG_LAYERED) return bpsf_fail(BPSF_EINVAL, "params.flags: unknown bits");
    if (p.max_iter < 1 || p.max_iter > 32767) return bpsf_fail(BPSF_EINVAL, "max_iter must be in 1..32767");
    if (!(p.alpha >= 0.f) || !std::isfinite(p.alpha))
        return bpsf_fail(BPSF_EINVAL, "alpha must be finite and > 0, or 0 for adaptive damping");
    if (p.w < 0 || p.w > kMaxPhi) return bpsf_fail(BPSF_EINVAL, "w must be in 0..%d", kMaxPhi);
    if (p.w > N) return bpsf_fail(BPSF_EINVAL, "w must not exceed N");
    if (p.w > 0) {
        if (p.w_max < 0 || p.w_max > p.w) return bpsf_fail(BPSF_EINVAL, "w_max must be in 0..w");
        if ((p.w_max == 0 ? p.w : p.w_max) > kMaxW)
            return bpsf_fail(BPSF_EINVAL, "w_max must be at most %d (a trial flips at most %d bits)", kMaxW, kMaxW);
        if (p.short_iter < 1 || p.short_iter > p.max_iter)
            return bpsf_fail(BPSF_EINVAL, "short_iter must be in 1..max_iter");
    }
    if (p.select != BPSF_SELECT_MIN_WEIGHT && p.select != BPSF_SELECT_FIRST)
        return bpsf_fail(BPSF_EINVAL, "select must be 0 or 1");
    const int outer = layout == BPSF_CSR ? M : N, inner = layout == BPSF_CSR ? N : M;
    if (ptr[0] != 0 || ptr[outer] != nnz) return bpsf_fail(BPSF_EINVAL, "ptr[0] must be 0 and ptr[last] must be nnz");
    std::vector<std::vector<int>> rows(M);
    for (int a = 0; a < outer; ++a) {
        if (ptr[a + 1] < ptr[a]) return bpsf_fail(BPSF_EINVAL, "ptr must be non-decreasing");
        for (int k = ptr[a]; k < ptr[a + 1]; ++k) {
            const int b = idx[k];
            if (b < 0 || b >= inner) return bpsf_fail(BPSF_EINVAL, "index %d out of range at position %d", b, k);
            if (layout == BPSF_CSR)
                rows[a].push_back(b);
            else
                rows[b].push_back(a);
        }
    }
    for (int i = 0; i < N; ++i) {
        const double pi = priors[i];
        if (!(pi > 0.0 && pi < 0.5)) return bpsf_fail(BPSF_EINVAL, "prior %d = %g is not in (0, 0.5)", i, pi);
    }
    int dc = 0;
    for (int j = 0; j < M; ++j) {
        std::sort(rows[j].begin(), rows[j].end());
        for (size_t k = 1; k < rows[j].size(); ++k)
            if (rows[j][k] == rows[j][k - 1]) return bpsf_fail(BPSF_EINVAL, "duplicate entry (%d, %d)", j, rows[j][k]);
        if (rows[j].size() < 2)
            return bpsf_fail(BPSF_EINVAL, "row %d has degree %d; every check needs degree >= 2", j, (int)rows[j].size());
        dc = std::max(dc, (int)rows[j].size());
    }
    // Columns list their checks in ascending order (rows are visited in order).
    std::vector<std::vector<std::pair<int, int>>> cols(N);  // (check, rank of the edge in its row)
    for (int j = 0; j < M; ++j)
        for (int k = 0; k < (int)rows[j].size(); ++k) cols[rows[j][k]].push_back({j, k});
    int dv = 0;
    for (int i = 0; i < N; ++i) dv = std::max(dv, (int)cols[i].size());
    bool regular = true;
    for (int j = 0; j < M; ++j) regular = regular && (int)rows[j].size() == dc;
    for (int i = 0; i < N; ++i) regular = regular && (int)cols[i].size() == dv;
    if (dc > 32 || dv > 16)
        return bpsf_fail(BPSF_EINVAL, "row degree %d or column degree %d too large (limits 32, 16)", dc, dv);
    const int variant = kernel_variant(regular ? -dc : dc, std::max(dv, 1));
    if (variant < 0) return bpsf_fail(BPSF_EINVAL, "no kernel variant for row degree %d, column degree %d", dc, dv);
    const int vstride = kernel_variant_dv(variant);
    const long long P = (long long)dc * M;
    if (P > 65534) return bpsf_fail(BPSF_EINVAL, "max row degree x M = %lld exceeds 65534", P);

    bpsf_ctx *c = new bpsf_ctx();
    c->M = M;
    c->N = N;
    c->nnz = (int)nnz;
    c->Ws = (M + 31) / 32;
    c->Wn = (N + 31) / 32;
    c->dc_max = dc;
    c->dv_max = dv;
    c->regular = regular ? 1 : 0;
    c->variant = variant;
    c->vstride = vstride;
    c->P = (int)P;
    c->p = p;
    if (c->p.w > 0 && c->p.w_max == 0) c->p.w_max = c->p.w;
    c->csr_ptr.assign(M + 1, 0);
    for (int j = 0; j < M; ++j) {
        for (int v : rows[j]) c->csr_col.push_back(v);
        c->csr_ptr[j + 1] = (int)c->csr_col.size();
    }
    // Check table per column (ascending check order); message positions are per layout below.
    std::vector<uint8_t> row_deg(M);
    std::vector<uint16_t> vchk((size_t)N * vstride, 0xffff);
    std::vector<uint16_t> row_ptr(M + 1), csr_col(nnz);
    std::vector<float> lch(N);
    for (int j = 0; j < M; ++j) row_deg[j] = (uint8_t)rows[j].size();
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < (int)cols[i].size(); ++k) vchk[(size_t)i * vstride + k] = (uint16_t)cols[i][k].first;
    for (int j = 0; j <= M; ++j) row_ptr[j] = (uint16_t)c->csr_ptr[j];
    for (int e = 0; e < nnz; ++e) csr_col[e] = (uint16_t)c->csr_col[e];
    // Channel LLR (Section II-B, step 1) in double, rounded once to float.
    for (int i = 0; i < N; ++i) lch[i] = (float)std::log((1.0 - priors[i]) / priors[i]);
    cudaGetDevice(&c->device);
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, c->device);
    if (e != cudaSuccess) {
        delete c;
        return bpsf_fail(BPSF_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    }
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = (int)prop.sharedMemPerBlockOptin;
    // Per-slot-count layouts (LayoutS): rank stride and edge ranks from the search.
    std::vector<int> row_off(M + 1, 0);
    for (int j = 0; j < M; ++j) row_off[j + 1] = row_off[j] + (int)rows[j].size();
    std::vector<int> edge_k(nnz);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < (int)cols[i].size(); ++k) edge_k[row_off[cols[i][k].first] + cols[i][k].second] = k;
    std::vector<std::vector<uint16_t>> lay_vpos(kNumLayouts), lay_var(kNumLayouts);
    std::vector<std::vector<float>> lay_lch(kNumLayouts);
    int lay_Mp[kNumLayouts];
    for (int li = 0; li < kNumLayouts; ++li) {
        const int S = 1 << li;
        // Slots per lane in the column phase: 4 for the exact-degree variant, 2 for
        // rows up to 16 wide, else 1.
        const int V = (variant == 0) ? std::min(S, 4) : (dc <= 16 ? std::min(S, 2) : 1);
        LayoutSearch L;
        L.M = M; L.N = N; L.dv = dv; L.S = S; L.V = V; L.Q = S / V; L.lpp = 32 / V; L.G = 32 / V;
        L.rows = &rows; L.cols = &cols; L.row_off = row_off; L.edge_k = edge_k;
        int Mp = M;
        std::vector<int> rank;
        search_layout(L, dc, Mp, rank);
        lay_Mp[li] = Mp;
        const size_t PS = (size_t)dc * Mp;
        lay_vpos[li].assign((size_t)N * vstride, 0xffff);
        lay_lch[li].assign(PS, 0.f);
        lay_var[li].assign(PS, 0xffff);
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < (int)cols[i].size(); ++k) {
                const int j = cols[i][k].first, r = rank[row_off[j] + cols[i][k].second];
                lay_vpos[li][(size_t)i * vstride + k] = (uint16_t)(r * Mp + j);
            }
        for (int j = 0; j < M; ++j)
            for (int t = 0; t < (int)rows[j].size(); ++t) {
                const size_t pos = (size_t)rank[row_off[j] + t] * Mp + j;
                lay_lch[li][pos] = lch[rows[j][t]];
                lay_var[li][pos] = (uint16_t)rows[j][t];
            }
    }
    // A default set beyond kMaxTrials is left empty: decoding then needs a list.
    std::vector<unsigned long long> masks;
    if (default_trial_count(c->p.w, c->p.w_max) <= kMaxTrials) masks = default_trials(c->p.w, c->p.w_max);
    c->n_trials = (int)masks.size();
    if (masks.empty()) masks.push_back(0);


    // Layered schedule: rows coloured greedily in ascending order, each taking the
    // smallest layer not used by an earlier row that shares a variable with it.
    std::vector<uint16_t> layer_ptr(1, 0), layer_rows;
    int n_layers = 0;
    if (p.flags & BPSF_FLAG_LAYERED) {
        std::vector<int> layer(M, 0);
        std::vector<char> used;
        for (int j = 0; j < M; ++j) {
            used.assign(M + 1, 0);
            for (int v : rows[j])
                for (const auto &ck : cols[v])
                    if (ck.first < j) used[layer[ck.first]] = 1;
            int l = 0;
            while (used[l]) ++l;
            layer[j] = l;
            n_layers = std::max(n_layers, l + 1);
        }
        layer_ptr.assign(n_layers + 1, 0);
        for (int j = 0; j < M; ++j) ++layer_ptr[layer[j] + 1];
        for (int l = 0; l < n_layers; ++l) layer_ptr[l + 1] = (uint16_t)(layer_ptr[l + 1] + layer_ptr[l]);
        layer_rows.assign(M, 0);
        std::vector<int> fill(layer_ptr.begin(), layer_ptr.end() - 1);
        for (int j = 0; j < M; ++j) layer_rows[fill[layer[j]]++] = (uint16_t)j;
    } else {
        layer_rows.assign(1, 0);
    }

    // One allocation for all code arrays.
    const void *srcs[8] = {row_deg.data(), vchk.data(), lch.data(), row_ptr.data(), csr_col.data(),
                           masks.data(), layer_ptr.data(), layer_rows.data()};
    const size_t sizes[8] = {(size_t)M, 2 * vchk.size(), 4 * (size_t)N, 2 * (size_t)(M + 1), 2 * (size_t)nnz,
                             8 * masks.size(), 2 * layer_ptr.size(), 2 * layer_rows.size()};
    size_t off[8], sz = 0;
    for (int k = 0; k < 8; ++k) {
        off[k] = sz;
        sz += align16(sizes[k]);
    }
    e = cudaMalloc(&c->d_code, sz);
    if (e != cudaSuccess) {
        delete c;
        return bpsf_fail(BPSF_ENOMEM, "cudaMalloc(code): %s", cudaGetErrorString(e));
    }
    std::vector<unsigned char> hbuf(sz, 0);
    for (int k = 0; k < 8; ++k) std::memcpy(hbuf.data() + off[k], srcs[k], sizes[k]);
    e = cudaMemcpy(c->d_code, hbuf.data(), sz, cudaMemcpyHostToDevice);
    unsigned char *base = (unsigned char *)c->d_code;
    CodeDev &cd = c->code;
    cd.M = M;
    cd.N = N;
    cd.nnz = (int)nnz;
    cd.Ws = c->Ws;
    cd.Wn = c->Wn;
    cd.DC = dc;
    cd.dv_max = dv;
    cd.P = (int)P;
    cd.regular = c->regular;
    cd.vstride = vstride;
    cd.max_iter = p.max_iter;
    cd.short_iter = c->p.w > 0 ? p.short_iter : 1;
    cd.w = c->p.w;
    cd.n_trials = c->n_trials;
    cd.select = p.select;
    cd.alpha = p.alpha;
    cd.row_deg = (const uint8_t *)(base + off[0]);
    cd.vchk = (const uint16_t *)(base + off[1]);
    cd.lch = (const float *)(base + off[2]);
    cd.row_ptr = (const uint16_t *)(base + off[3]);
    cd.csr_col = (const uint16_t *)(base + off[4]);
    cd.trial_mask = (const unsigned long long *)(base + off[5]);
    c->default_masks = cd.trial_mask;
    cd.layered = (p.flags & BPSF_FLAG_LAYERED) ? 1 : 0;
    cd.n_layers = n_layers;
    cd.layer_ptr = (const uint16_t *)(base + off[6]);
    cd.layer_rows = (const uint16_t *)(base + off[7]);
    c->default_n_trials = c->n_trials;
    // The per-slot-count layouts: one allocation.
    {
        size_t lsz = 0;
        size_t lo[kNumLayouts][3];
        for (int li = 0; li < kNumLayouts; ++li) {
            lo[li][0] = lsz; lsz += align16(2 * lay_vpos[li].size());
            lo[li][1] = lsz; lsz += align16(4 * lay_lch[li].size());
            lo[li][2] = lsz; lsz += align16(2 * lay_var[li].size());
        }
        if (e == cudaSuccess) e = cudaMalloc(&c->d_layouts, lsz);
        if (e == cudaSuccess) {
            std::vector<unsigned char> lb(lsz, 0);
            for (int li = 0; li < kNumLayouts; ++li) {
                std::memcpy(lb.data() + lo[li][0], lay_vpos[li].data(), 2 * lay_vpos[li].size());
                std::memcpy(lb.data() + lo[li][1], lay_lch[li].data(), 4 * lay_lch[li].size());
                std::memcpy(lb.data() + lo[li][2], lay_var[li].data(), 2 * lay_var[li].size());
            }
            e = cudaMemcpy(c->d_layouts, lb.data(), lsz, cudaMemcpyHostToDevice);
            unsigned char *lbase = (unsigned char *)c->d_layouts;
            for (int li = 0; li < kNumLayouts; ++li) {
                LayoutS &ly = cd.lay[li];
                ly.Mp = lay_Mp[li];
                ly.P = (int)lay_lch[li].size();
                ly.vpos = (const uint16_t *)(lbase + lo[li][0]);
                ly.lch_pos = (const float *)(lbase + lo[li][1]);
                ly.pos_var = (const uint16_t *)(lbase + lo[li][2]);
            }
            bpsf_activate_layout(cd, 1);
        }
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_ctr, kMaxStreams * sizeof(StreamCounters));
    if (e == cudaSuccess) e = cudaMemset(c->d_ctr, 0, kMaxStreams * sizeof(StreamCounters));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_ctr, kMaxStreams * sizeof(StreamCounters));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_flag, 64);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_preset, sizeof(StreamCounters));
    if (e != cudaSuccess) {
        bpsf_destroy(c);
        return bpsf_fail(BPSF_ECUDA, "context allocation: %s", cudaGetErrorString(e));
    }
    std::memset(c->h_ctr, 0, kMaxStreams * sizeof(StreamCounters));
    c->tune = default_tuning(c);
    bpsf_tuning cached;
    if (bpsf_tuning_cache_lookup(c, &cached)) c->tune = cached;
    *out = c;
    return BPSF_OK;
}

// ---------------------------------------------------------------------------
// Workspace: one record row per shot (capacity = the largest batch so far).
// ---------------------------------------------------------------------------

bpsf_status bpsf_ensure_workspace(bpsf_ctx *c, long long n) {
    long long cap_s = 0;
    return bpsf_ensure_workspace_sharded(c, n, 1, &cap_s);
}

// Shards of a batch of n shots in a launch of n_jobs jobs: a power of two, at
// most kMaxShards, with no more than kMaxStreams streams in the launch and at
// least kMinShardShots shots per shard; codes of more than kMaxShardNnz edges
// are not sharded (their blocks claim work rarely, and a block that moves to
// another stream reloads the code's tables).
int bpsf_batch_shards(const bpsf_ctx *c, long long n, int n_jobs) {
    int k = 1;
    if (c->nnz > kMaxShardNnz) return 1;
    while (2 * k <= kMaxShards && (long long)n_jobs * 2 * k <= kMaxStreams && n / (2 * k) >= kMinShardShots) k *= 2;
    return k;
}

bpsf_status bpsf_ensure_workspace_sharded(bpsf_ctx *c, long long n, int shards, long long *shard_cap) {
    const long long per = (std::max<long long>(n, 1) + shards - 1) / shards;
    const long long cap_s = bpsf_record_ring(per);
    *shard_cap = cap_s;
    const long long cap = cap_s * shards;  // a power of two: shards is one
    if (cap <= c->rec_cap) return BPSF_OK;
    const size_t total = bpsf_records_bytes(cap, c->p.w, c->Ws, c->Wn, 16);
    free_workspace(c);
    void *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, total);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ENOMEM, "workspace of %zu bytes: %s", total, cudaGetErrorString(e));
    c->d_rec = mem;
    c->rec = bpsf_records_carve(mem, cap, c->p.w, c->Ws, c->Wn, 16);
    c->rec_cap = cap;
    return BPSF_OK;
}

// Every record of the ring reads free before a launch.
static bpsf_status clear_queue(bpsf_ctx *c, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(c->rec.qseq, 0, 8 * (size_t)c->rec.cap, s);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return BPSF_OK;
}

void bpsf_shard_streams(const bpsf_ctx *c, const JobDev &job, int shards, long long shard_cap, const DebugDev *dbg,
                        StreamDev *out) {
    const long long n = job.n_shots;
    const long long ww = c->p.w > 0 ? c->p.w : 1;
    for (int j = 0; j < shards; ++j) {
        const long long a = n * j / shards, b = n * (j + 1) / shards;
        JobDev jj = job;
        jj.synd = job.synd + a * job.synd_stride;
        jj.corr = job.corr + a * job.corr_stride;
        jj.conv = job.conv + a;
        jj.iters = job.iters + a;
        jj.stage = job.stage ? job.stage + a : nullptr;
        jj.n_shots = b - a;
        StreamDev sd = bpsf_make_stream(c, jj, dbg, 0);
        sd.ctr = c->d_ctr + j;
        const long long r0 = (long long)j * shard_cap;
        Records &r = sd.rec;
        r.qseq = c->rec.qseq + r0;
        r.qshot = c->rec.qshot + r0;
        r.done = c->rec.done + r0;
        r.best = c->rec.best + r0;
        r.win = c->rec.win + r0 * c->Wn;
        r.phi = c->rec.phi + r0 * ww;
        r.synd = c->rec.synd + r0 * c->Ws;
        r.cap = shard_cap;
        out[j] = sd;
    }
}

StreamDev bpsf_make_stream(const bpsf_ctx *c, const JobDev &job, const DebugDev *dbg, unsigned flags) {
    StreamDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.code = c->code;
    sd.job = job;
    sd.rec = c->rec;
    sd.ctr = c->d_ctr;
    if (dbg) sd.dbg = *dbg;
    sd.flags = flags;
    return sd;
}

void bpsf_launch_plan(const bpsf_plan &pl, bool debug, StreamDev *sds, int n, int grid, void *stream) {
    for (int k = 0; k < n; ++k) {
        sds[k].S = pl.S_code[k];
        bpsf_activate_layout(sds[k].code, pl.S_code[k]);
        sds[k].W = pl.W_code[k];
        sds[k].teams = pl.teams_code[k];
        sds[k].chunk = pl.chunk_code[k];
    }
    LaunchArgs la{sds, n, pl.Q, kBpsfWaitNs};
    launch_persistent(pl.variant, debug, pl.layered, grid, pl.block, pl.smem, la, stream);
}

static bpsf_status check_io(const bpsf_ctx *c, int64_t n, const void *synd, int32_t ss, const void *corr, int32_t cs,
                            const void *conv, const void *iters) {
    if (!c) return bpsf_fail(BPSF_EINVAL, "ctx is NULL");
    if (bpsf_check_trials(c) != BPSF_OK) return BPSF_EINVAL;
    if (n < 0) return bpsf_fail(BPSF_EINVAL, "n_shots must be >= 0");
    if (n > (1ll << 40)) return bpsf_fail(BPSF_EINVAL, "n_shots too large");
    if (n == 0) return BPSF_OK;
    if (!synd || !corr || !conv || !iters) return bpsf_fail(BPSF_EINVAL, "NULL input or output pointer");
    if (ss < c->Ws) return bpsf_fail(BPSF_EINVAL, "synd_stride_words %d < Ws = %d", ss, c->Ws);
    if (cs < c->Wn) return bpsf_fail(BPSF_EINVAL, "corr_stride_words %d < Wn = %d", cs, c->Wn);
    return BPSF_OK;
}

static bpsf_status decode_impl(bpsf_ctx *c, int64_t n, const uint32_t *synd, int32_t ss, uint32_t *corr, int32_t cs,
                               uint8_t *conv, int16_t *iters, uint8_t *stage, const DebugDev *dbg, void *stream) {
    BpsfRange range("bpsf_decode");
    bpsf_status st = check_io(c, n, synd, ss, corr, cs, conv, iters);
    if (st != BPSF_OK || n == 0) return st;
    cudaSetDevice(c->device);
    bpsf_plan pl;
    bpsf_ctx *cs1[1] = {c};
    st = bpsf_make_plan(cs1, 1, &c->tune, dbg != nullptr, &pl);
    if (st != BPSF_OK) return st;
    // Shards (the debug dump indexes its arrays by shot, so it keeps one).
    const int K = dbg ? 1 : bpsf_batch_shards(c, n, 1);
    if (K > 1) {
        bpsf_ctx *ck[kMaxShards];
        bpsf_tuning tk[kMaxShards];
        for (int j = 0; j < K; ++j) {
            ck[j] = c;
            tk[j] = c->tune;
        }
        st = bpsf_make_plan(ck, K, tk, false, &pl);
        if (st != BPSF_OK) return st;
    }
    long long cap_s = 0;
    st = bpsf_ensure_workspace_sharded(c, n, K, &cap_s);
    if (st != BPSF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(c->d_ctr, 0, K * sizeof(StreamCounters), s);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    st = clear_queue(c, s);
    if (st != BPSF_OK) return st;
    JobDev job{synd, corr, conv, iters, stage, n, ss, cs};
    StreamDev sds[kMaxShards];
    bpsf_shard_streams(c, job, K, cap_s, dbg, sds);
    bpsf_launch_plan(pl, dbg != nullptr, sds, K, pl.grid, stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    c->d_ctr_last = c->d_ctr;
    c->last_shards = K;
    c->last_launch_n = n;
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_decode(bpsf_ctx *c, int64_t n, const uint32_t *synd, int32_t ss, uint32_t *corr,
                                   int32_t cs, uint8_t *conv, int16_t *iters, uint8_t *stage, void *stream) {
    return decode_impl(c, n, synd, ss, corr, cs, conv, iters, stage, nullptr, stream);
}

extern "C" bpsf_status bpsf_decode_debug(bpsf_ctx *c, int64_t n, const uint32_t *synd, int32_t ss, uint32_t *corr,
                                         int32_t cs, uint8_t *conv, int16_t *iters, uint8_t *stage, float *lout,
                                         uint16_t *flips, int32_t *phi, uint32_t *tsynd, uint8_t *tconv,
                                         int16_t *titers, void *stream) {
    DebugDev d{lout, flips, phi, tsynd, tconv, titers};
    return decode_impl(c, n, synd, ss, corr, cs, conv, iters, stage, &d, stream);
}

extern "C" bpsf_status bpsf_sync(bpsf_ctx *c, void *stream) {
    if (!c) return bpsf_fail(BPSF_EINVAL, "ctx is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
    StreamCounters *dc = c->d_ctr_last ? c->d_ctr_last : c->d_ctr;
    const int K = std::max(1, c->last_shards);
    e = cudaMemcpy(c->h_ctr, dc, K * sizeof(StreamCounters), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    // The launch's shards add up.
    bpsf_work w{};
    unsigned stv = 0;
    for (int j = 0; j < K; ++j) {
        const StreamCounters &k = c->h_ctr[j];
        w.initial_runs += (int64_t)k.init_done;
        w.failed_shots += (int64_t)k.rec_count;
        w.trial_runs += (int64_t)k.trial_runs;
        w.iterations += (int64_t)k.iters_total;
        w.slot_capacity += (int64_t)k.slot_capacity;
        w.trials_cancelled += (int64_t)k.trials_cancelled;
        stv |= k.status;
    }
    w.edge_updates = w.iterations * c->nnz;
    c->last = w;
    if (stv) {
        for (int j = 0; j < K; ++j)
            if (c->h_ctr[j].status) cudaMemsetAsync(&dc[j].status, 0, sizeof(unsigned), (cudaStream_t)stream);
        cudaStreamSynchronize((cudaStream_t)stream);
        if (stv & (kDevReadyTimeout | kDevIdleTimeout))
            return bpsf_fail(BPSF_ETIMEOUT, "a bounded device wait ran out (status 0x%x)", stv);
        return bpsf_fail(BPSF_EDEVICE, "device error (status 0x%x)", stv);
    }
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_last_work(bpsf_ctx *c, bpsf_work *out) {
    if (!c || !out) return bpsf_fail(BPSF_EINVAL, "NULL argument");
    *out = c->last;
    return BPSF_OK;
}

extern "C" int32_t bpsf_num_trials(const bpsf_ctx *c) { return c ? c->n_trials : -1; }

extern "C" bpsf_status bpsf_set_trials(bpsf_ctx *c, int32_t n, const uint64_t *masks) {
    if (!c) return bpsf_fail(BPSF_EINVAL, "ctx is NULL");
    if (c->p.w <= 0) return bpsf_fail(BPSF_EINVAL, "the context has no trials (w = 0)");
    if (n < 0 || n > kMaxTrials) return bpsf_fail(BPSF_EINVAL, "n must be in 0..%d", kMaxTrials);
    if (n > 0 && !masks) return bpsf_fail(BPSF_EINVAL, "masks is NULL");
    for (int k = 0; k < n; ++k) {
        const unsigned long long m = masks[k];
        if (m == 0ull) return bpsf_fail(BPSF_EINVAL, "mask %d is empty", k);
        if (c->p.w < 64 && (m >> c->p.w) != 0ull) return bpsf_fail(BPSF_EINVAL, "mask %d selects a bit >= w", k);
        if (__builtin_popcountll(m) > kMaxW) return bpsf_fail(BPSF_EINVAL, "mask %d has more than %d bits", k, kMaxW);
    }
    cudaSetDevice(c->device);
    // Records hold per-trial rows: the workspace is re-sized at the next decode.
    free_workspace(c);
    if (c->d_trials) cudaFree(c->d_trials);
    c->d_trials = nullptr;
    if (n == 0) {
        c->code.trial_mask = c->default_masks;
        c->n_trials = c->default_n_trials;
    } else {
        cudaError_t e = cudaMalloc(&c->d_trials, 8 * (size_t)n);
        if (e == cudaSuccess) e = cudaMemcpy(c->d_trials, masks, 8 * (size_t)n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (c->d_trials) cudaFree(c->d_trials);
            c->d_trials = nullptr;
            c->code.trial_mask = c->default_masks;
            c->n_trials = c->default_n_trials;
            return bpsf_fail(BPSF_ENOMEM, "trial list: %s", cudaGetErrorString(e));
        }
        c->code.trial_mask = (const unsigned long long *)c->d_trials;
        c->n_trials = n;
    }
    c->code.n_trials = c->n_trials;
    return BPSF_OK;
}

// ---------------------------------------------------------------------------
// Plain per-shot form: launch, synchronise, read the flag, launch the trial
// sweep on failure, synchronise.
// ---------------------------------------------------------------------------

extern "C" bpsf_status bpsf_decode_plain(bpsf_ctx *c, int64_t n, const uint32_t *synd, int32_t ss, uint32_t *corr,
                                         int32_t cs, uint8_t *conv, int16_t *iters, uint8_t *stage, void *stream) {
    BpsfRange range("bpsf_decode_plain");
    bpsf_status st = check_io(c, n, synd, ss, corr, cs, conv, iters);
    if (st != BPSF_OK || n == 0) return st;
    cudaSetDevice(c->device);
    st = bpsf_ensure_workspace(c, 1);
    if (st != BPSF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    bpsf_ctx *cs1[1] = {c};
    // Launch A: one block, one team, one slot, the initial run of one shot.
    bpsf_plan plA, plB;
    bpsf_tuning tA{c->tune.warps_per_team, 1, c->tune.warps_per_team, 0, 1};
    st = bpsf_make_plan(cs1, 1, &tA, false, &plA);
    if (st != BPSF_OK) return st;
    // Launch B: the shot's trials spread over blocks of the tuned shape.
    st = bpsf_make_plan(cs1, 1, &c->tune, false, &plB);
    if (st != BPSF_OK) return st;
    const int trials = std::max(c->n_trials, 1);
    const int per_block = plB.teams_code[0] * plB.S_code[0];
    const int gridB = std::max(1, std::min(plB.grid, (trials + per_block - 1) / per_block));
    StreamCounters preset;
    std::memset(&preset, 0, sizeof(preset));
    preset.shot_next = 1;
    preset.init_done = 1;
    preset.rec_count = 1;
    *c->h_preset = preset;
    long long iters_total = 0, trial_runs = 0, failed = 0, cap = 0, cancelled = 0;
    for (int64_t i = 0; i < n; ++i) {
        JobDev job{synd + i * ss, corr + i * cs, conv + i, iters + i, stage ? stage + i : nullptr, 1, ss, cs};
        cudaError_t e = cudaMemsetAsync(c->d_ctr, 0, sizeof(StreamCounters), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->rec.qseq, 0, 8, s);
        if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        BpsfRange shot_range("plain shot");
        StreamDev sdA = bpsf_make_stream(c, job, nullptr, kNoTickets);
        bpsf_launch_plan(plA, false, &sdA, 1, 1, stream);
        e = cudaMemcpyAsync(c->h_flag, conv + i, 1, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(StreamCounters), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "plain initial run: %s", cudaGetErrorString(e));
        iters_total += (long long)c->h_ctr->iters_total;
        cap += (long long)c->h_ctr->slot_capacity;
        if (c->h_flag[0] == 0 && c->p.w > 0) {
            ++failed;
            e = cudaMemcpyAsync(c->d_ctr, c->h_preset, sizeof(StreamCounters), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
            BpsfRange trial_range("plain trial sweep");
            StreamDev sdB = bpsf_make_stream(c, job, nullptr, 0);
            bpsf_launch_plan(plB, false, &sdB, 1, gridB, stream);
            e = cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(StreamCounters), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "plain trial sweep: %s", cudaGetErrorString(e));
            if (c->h_ctr->status)
                return bpsf_fail(BPSF_ETIMEOUT, "device status 0x%x in the trial sweep", c->h_ctr->status);
            trial_runs += (long long)c->h_ctr->trial_runs;
            iters_total += (long long)c->h_ctr->iters_total;
            cap += (long long)c->h_ctr->slot_capacity;
            cancelled += (long long)c->h_ctr->trials_cancelled;
        }
    }
    c->last = bpsf_work{n, failed, trial_runs, iters_total, iters_total * c->nnz, cap, cancelled};
    c->d_ctr_last = c->d_ctr;
    c->last_shards = 1;
    return BPSF_OK;
}

// ---------------------------------------------------------------------------
// Host-buffer form.
// ---------------------------------------------------------------------------

// Device staging for a host-buffer call: syndromes, corrections, converged
// flags, iterations and stages of n shots, in the context's own buffer
// (grown when too small, kept for the next call).
struct HostStage {
    uint32_t *synd, *corr;
    uint8_t *conv, *stage;
    int16_t *it;
    size_t b_synd, b_corr, b_conv, b_it;
};

static bpsf_status host_stage(bpsf_ctx *c, int64_t n, int32_t ss, int32_t cs, HostStage *h) {
    h->b_synd = 4 * (size_t)n * ss;
    h->b_corr = 4 * (size_t)n * cs;
    h->b_conv = (size_t)n;
    h->b_it = 2 * (size_t)n;
    const size_t need = align16(h->b_synd) + align16(h->b_corr) + align16(h->b_conv) + align16(h->b_it) +
                        align16(h->b_conv);
    if (need > c->host_stage_bytes) {
        if (c->d_host_stage) cudaFree(c->d_host_stage);
        c->d_host_stage = nullptr;
        c->host_stage_bytes = 0;
        cudaError_t e = cudaMalloc(&c->d_host_stage, need);
        if (e != cudaSuccess) return bpsf_fail(BPSF_ENOMEM, "staging buffers: %s", cudaGetErrorString(e));
        c->host_stage_bytes = need;
    }
    unsigned char *p = (unsigned char *)c->d_host_stage;
    h->synd = (uint32_t *)p;
    p += align16(h->b_synd);
    h->corr = (uint32_t *)p;
    p += align16(h->b_corr);
    h->conv = p;
    p += align16(h->b_conv);
    h->it = (int16_t *)p;
    p += align16(h->b_it);
    h->stage = p;
    return BPSF_OK;
}

static bpsf_status host_results(const HostStage &h, uint32_t *h_corr, uint8_t *h_conv, int16_t *h_iters,
                                uint8_t *h_stage, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(h_corr, h.corr, h.b_corr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_conv, h.conv, h.b_conv, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_iters, h.it, h.b_it, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_stage) e = cudaMemcpyAsync(h_stage, h.stage, h.b_conv, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "D2H: %s", cudaGetErrorString(e));
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_decode_host(bpsf_ctx *c, int64_t n, const uint32_t *h_synd, int32_t ss, uint32_t *h_corr,
                                        int32_t cs, uint8_t *h_conv, int16_t *h_iters, uint8_t *h_stage,
                                        void *stream) {
    bpsf_status st = check_io(c, n, h_synd, ss, h_corr, cs, h_conv, h_iters);
    if (st != BPSF_OK || n == 0) return st;
    cudaSetDevice(c->device);
    HostStage h;
    st = host_stage(c, n, ss, cs, &h);
    if (st != BPSF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h.synd, h_synd, h.b_synd, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "H2D: %s", cudaGetErrorString(e));
    st = decode_impl(c, n, h.synd, ss, h.corr, cs, h.conv, h.it, h.stage, nullptr, stream);
    if (st != BPSF_OK) return st;
    st = host_results(h, h_corr, h_conv, h_iters, h_stage, s);
    if (st != BPSF_OK) return st;
    return bpsf_sync(c, stream);
}

extern "C" bpsf_status bpsf_decode_multi_host(int32_t n_jobs, const bpsf_job *jobs, void *stream) {
    BpsfRange range("bpsf_decode_multi_host");
    if (n_jobs < 1 || n_jobs > kMaxStreams || !jobs) return bpsf_fail(BPSF_EINVAL, "n_jobs must be in 1..%d", kMaxStreams);
    for (int k = 0; k < n_jobs; ++k) {
        const bpsf_job &j = jobs[k];
        bpsf_status st = check_io(j.ctx, j.n_shots, j.d_synd, j.synd_stride_words, j.d_corr, j.corr_stride_words,
                                  j.d_converged, j.d_iters);
        if (st != BPSF_OK) return st;
        for (int q = 0; q < k; ++q)
            if (jobs[q].ctx == j.ctx) return bpsf_fail(BPSF_EINVAL, "a context appears twice in one launch");
        if (j.ctx->device != jobs[0].ctx->device) return bpsf_fail(BPSF_EINVAL, "contexts on different devices");
    }
    cudaSetDevice(jobs[0].ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // Stage every non-empty job's syndromes, then one launch over the device copies.
    std::vector<HostStage> hs(n_jobs);
    std::vector<bpsf_job> dj;
    std::vector<int> live;
    for (int k = 0; k < n_jobs; ++k) {
        const bpsf_job &j = jobs[k];
        if (j.n_shots == 0) continue;  // empty jobs take no part in the launch
        bpsf_status st = host_stage(j.ctx, j.n_shots, j.synd_stride_words, j.corr_stride_words, &hs[k]);
        if (st != BPSF_OK) return st;
        cudaError_t e = cudaMemcpyAsync(hs[k].synd, j.d_synd, hs[k].b_synd, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "H2D: %s", cudaGetErrorString(e));
        bpsf_job d = j;
        d.d_synd = hs[k].synd;
        d.d_corr = hs[k].corr;
        d.d_converged = hs[k].conv;
        d.d_iters = hs[k].it;
        d.d_stage = hs[k].stage;
        dj.push_back(d);
        live.push_back(k);
    }
    if (dj.empty()) return BPSF_OK;
    bpsf_status st = bpsf_decode_multi((int32_t)dj.size(), dj.data(), stream);
    if (st != BPSF_OK) return st;
    for (int k : live) {
        const bpsf_job &j = jobs[k];
        st = host_results(hs[k], j.d_corr, j.d_converged, j.d_iters, j.d_stage, s);
        if (st != BPSF_OK) return st;
    }
    for (int k : live) {
        st = bpsf_sync(jobs[k].ctx, stream);
        if (st != BPSF_OK) return st;
    }
    return BPSF_OK;
}

// ---------------------------------------------------------------------------
// Mixed-code batch: one launch over up to kMaxStreams codes.
// ---------------------------------------------------------------------------

extern "C" bpsf_status bpsf_decode_multi(int32_t n_jobs, const bpsf_job *jobs, void *stream) {
    BpsfRange range("bpsf_decode_multi");
    if (n_jobs < 1 || n_jobs > kMaxStreams || !jobs) return bpsf_fail(BPSF_EINVAL, "n_jobs must be in 1..%d", kMaxStreams);
    std::vector<bpsf_ctx *> codes(n_jobs);
    for (int k = 0; k < n_jobs; ++k) {
        const bpsf_job &j = jobs[k];
        bpsf_status st = check_io(j.ctx, j.n_shots, j.d_synd, j.synd_stride_words, j.d_corr, j.corr_stride_words,
                                  j.d_converged, j.d_iters);
        if (st != BPSF_OK) return st;
        for (int q = 0; q < k; ++q)
            if (jobs[q].ctx == j.ctx) return bpsf_fail(BPSF_EINVAL, "a context appears twice in one launch");
        if (j.ctx->device != jobs[0].ctx->device) return bpsf_fail(BPSF_EINVAL, "contexts on different devices");
        codes[k] = j.ctx;
    }
    bpsf_ctx *c0 = codes[0];
    cudaSetDevice(c0->device);
    // Each code keeps its own team shape (shrunk if its block does not fit);
    // each job is split into shards (streams of the launch with their own
    // counters and ring slices).
    std::vector<int> shards(n_jobs);
    std::vector<bpsf_ctx *> scodes;
    std::vector<bpsf_tuning> tunes;
    for (int k = 0; k < n_jobs; ++k) {
        shards[k] = bpsf_batch_shards(codes[k], std::max<int64_t>(jobs[k].n_shots, 1), n_jobs);
        for (int q = 0; q < shards[k]; ++q) {
            scodes.push_back(codes[k]);
            tunes.push_back(codes[k]->tune);
        }
    }
    const int n_streams = (int)scodes.size();
    bpsf_plan pl;
    bpsf_status st = bpsf_make_plan(scodes.data(), n_streams, tunes.data(), false, &pl, true);
    if (st != BPSF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<StreamDev> sds(n_streams);
    int at = 0;
    for (int k = 0; k < n_jobs; ++k) {
        bpsf_ctx *c = codes[k];
        const bpsf_job &j = jobs[k];
        long long cap_s = 0;
        st = bpsf_ensure_workspace_sharded(c, std::max<int64_t>(j.n_shots, 1), shards[k], &cap_s);
        if (st != BPSF_OK) return st;
        cudaError_t e = cudaMemsetAsync(c->d_ctr, 0, shards[k] * sizeof(StreamCounters), s);
        if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        st = clear_queue(c, s);
        if (st != BPSF_OK) return st;
        JobDev job{j.d_synd, j.d_corr, j.d_converged, j.d_iters, j.d_stage, j.n_shots, j.synd_stride_words,
                   j.corr_stride_words};
        bpsf_shard_streams(c, job, shards[k], cap_s, nullptr, sds.data() + at);
        at += shards[k];
        c->last_launch_n = j.n_shots;
        c->d_ctr_last = c->d_ctr;
        c->last_shards = shards[k];
    }
    bpsf_launch_plan(pl, false, sds.data(), n_streams, pl.grid, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return BPSF_OK;
}

// ---------------------------------------------------------------------------
// Tuning and autotuner.
// ---------------------------------------------------------------------------

extern "C" bpsf_status bpsf_get_tuning(const bpsf_ctx *c, bpsf_tuning *out) {
    if (!c || !out) return bpsf_fail(BPSF_EINVAL, "NULL argument");
    *out = c->tune;
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_set_tuning(bpsf_ctx *c, const bpsf_tuning *t) {
    if (!c || !t) return bpsf_fail(BPSF_EINVAL, "NULL argument");
    bpsf_plan pl;
    bpsf_ctx *cs1[1] = {c};
    bpsf_status st = bpsf_make_plan(cs1, 1, t, false, &pl);
    if (st != BPSF_OK) return st;
    c->tune = *t;
    return BPSF_OK;
}

// Cache key: the code's shape and the parameters that set the work per shot.
typedef std::tuple<int, int, int, int, int, int, int, int, int, unsigned> ShapeKey;
static std::mutex g_tune_mu;
static std::map<ShapeKey, bpsf_tuning> g_tune_cache;

static ShapeKey shape_key(const bpsf_ctx *c) {
    return ShapeKey(c->M, c->N, c->nnz, c->dc_max, c->dv_max, c->p.max_iter, c->p.w, c->n_trials, c->p.short_iter,
                    c->p.flags);
}

bool bpsf_tuning_cache_lookup(const bpsf_ctx *c, bpsf_tuning *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(shape_key(c));
    if (it == g_tune_cache.end()) return false;
    *out = it->second;
    return true;
}

extern "C" bpsf_status bpsf_autotune(bpsf_ctx *c, double p_sample, int64_t n_sample, void *stream,
                                     bpsf_tuning *chosen) {
    BpsfRange range("bpsf_autotune");
    if (!c) return bpsf_fail(BPSF_EINVAL, "ctx is NULL");
    if (!(p_sample > 0.0 && p_sample < 0.5)) return bpsf_fail(BPSF_EINVAL, "p_sample must be in (0, 0.5)");
    if (n_sample < 1 || n_sample > (1 << 24)) return bpsf_fail(BPSF_EINVAL, "n_sample must be in 1..2^24");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b_err = 4 * (size_t)n_sample * c->Wn, b_synd = 4 * (size_t)n_sample * c->Ws;
    const size_t b_corr = b_err, b_conv = (size_t)n_sample, b_it = 2 * (size_t)n_sample;
    void *buf = nullptr;
    const size_t total = align16(b_err) + align16(b_synd) + align16(b_corr) + align16(b_conv) + align16(b_it);
    cudaError_t e = cudaMalloc(&buf, total);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ENOMEM, "autotune buffers: %s", cudaGetErrorString(e));
    unsigned char *p = (unsigned char *)buf;
    uint32_t *err = (uint32_t *)p;
    p += align16(b_err);
    uint32_t *synd = (uint32_t *)p;
    p += align16(b_synd);
    uint32_t *corr = (uint32_t *)p;
    p += align16(b_corr);
    uint8_t *conv = p;
    p += align16(b_conv);
    int16_t *it = (int16_t *)p;
    launch_sample_errors(n_sample, c->N, p_sample, 0x5eed5eedull, err, c->Wn, stream);
    launch_syndrome(c->code, n_sample, err, c->Wn, synd, c->Ws, stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bpsf_tuning saved = c->tune;
    bpsf_tuning best = saved;
    float best_ms = 1e30f;
    bpsf_status st = BPSF_OK;
    bpsf_ctx *cs1[1] = {c};
    // Time one shape: the best of two decodes after a warm-up decode.
    auto time_shape = [&](const bpsf_tuning &t) -> float {
        c->tune = t;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 3 && st == BPSF_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = bpsf_decode(c, n_sample, synd, c->Ws, corr, c->Wn, conv, it, nullptr, stream);
            cudaEventRecord(e1, s);
            if (st == BPSF_OK) st = bpsf_sync(c, stream);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_min = std::min(ms_min, ms);
        }
        return ms_min;
    };
    // Threads per shot and shots per block: warps per team, slots per team and
    // compute warps per block, every shape that fits.
    const int Ws_[] = {1, 2, 4, 8};
    const int Ss_[] = {1, 2, 4, 8, 16, 32};
    const int Bs_[] = {1, 2, 3, 4, 6, 7, 8, 10, 12, 13, 14, 15};
    for (int W : Ws_)
        for (int S : Ss_)
            for (int B : Bs_) {
                if (st != BPSF_OK) break;
                bpsf_tuning t{W, S, B, 0, 1};
                if (B % W) continue;
                bpsf_plan pl;
                if (bpsf_make_plan(cs1, 1, &t, false, &pl) != BPSF_OK) continue;
                const float ms = time_shape(t);
                if (st == BPSF_OK && ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
    // The iteration chunk of the fastest shape.
    for (int k : {2, 4, 8}) {
        if (st != BPSF_OK || best_ms >= 1e30f) break;
        bpsf_tuning t = best;
        t.iter_chunk = k;
        const float ms = time_shape(t);
        if (st == BPSF_OK && ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    c->tune = (st == BPSF_OK) ? best : saved;
    if (st != BPSF_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[shape_key(c)] = best;
    }
    if (chosen) *chosen = best;
    return BPSF_OK;
}

// ---------------------------------------------------------------------------
// Bounded-wait self test: trial tickets of a record that is never published.
// ---------------------------------------------------------------------------

extern "C" bpsf_status bpsf_selftest_wait(bpsf_ctx *c, int64_t wait_us, void *stream) {
    if (!c) return bpsf_fail(BPSF_EINVAL, "ctx is NULL");
    if (wait_us < 1 || wait_us > 10000000) return bpsf_fail(BPSF_EINVAL, "wait_us must be in 1..10^7");
    if (c->p.w <= 0) return bpsf_fail(BPSF_EINVAL, "the context has no trials (w = 0)");
    cudaSetDevice(c->device);
    bpsf_status st = bpsf_ensure_workspace(c, 1);
    if (st != BPSF_OK) return st;
    bpsf_plan pl;
    bpsf_ctx *cs1[1] = {c};
    st = bpsf_make_plan(cs1, 1, &c->tune, false, &pl);
    if (st != BPSF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // One failed shot is announced (rec_count = 1) but its queue entry is
    // never written, so claimed tickets wait for it in vain.
    StreamCounters preset;
    std::memset(&preset, 0, sizeof(preset));
    preset.shot_next = 1;
    preset.init_done = 1;
    preset.rec_count = 1;
    *c->h_preset = preset;
    cudaError_t e = cudaMemcpyAsync(c->d_ctr, c->h_preset, sizeof(StreamCounters), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->rec.qseq, 0, 8, s);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "self test set-up: %s", cudaGetErrorString(e));
    // Outputs of the (never settled) shot go to the workspace's own rows.
    JobDev job{c->rec.synd, reinterpret_cast<uint32_t *>(c->rec.win), reinterpret_cast<uint8_t *>(c->rec.done),
               reinterpret_cast<int16_t *>(c->rec.done), nullptr, 1, c->Ws, c->Wn};
    StreamDev sd = bpsf_make_stream(c, job, nullptr, 0);
    sd.S = pl.S_code[0];
    bpsf_activate_layout(sd.code, pl.S_code[0]);
    sd.W = pl.W_code[0];
    sd.teams = pl.teams_code[0];
    sd.chunk = pl.chunk_code[0];
    LaunchArgs la{&sd, 1, pl.Q, (unsigned long long)wait_us * 1000ull};
    launch_persistent(pl.variant, false, pl.layered, 1, pl.block, pl.smem, la, stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    c->d_ctr_last = c->d_ctr;
    c->last_shards = 1;
    return bpsf_sync(c, stream);
}

// ---------------------------------------------------------------------------
// Harness helper.
// ---------------------------------------------------------------------------

extern "C" bpsf_status bpsf_syndrome(const bpsf_ctx *c, int64_t n, const uint32_t *d_err, int32_t es,
                                     uint32_t *d_synd, int32_t ss, void *stream) {
    if (!c || n < 0) return bpsf_fail(BPSF_EINVAL, "bad ctx or n");
    if (n == 0) return BPSF_OK;
    if (!d_err || !d_synd) return bpsf_fail(BPSF_EINVAL, "NULL pointer");
    if (es < c->Wn || ss < c->Ws) return bpsf_fail(BPSF_EINVAL, "stride too small");
    launch_syndrome(c->code, n, d_err, es, d_synd, ss, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "syndrome kernel: %s", cudaGetErrorString(e));
    return BPSF_OK;
}
