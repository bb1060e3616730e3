// Serving form of libbpsf: continuous batching of a request stream over
// several codes.
//
// Each code owns an arena of `rows` shot rows.  A request of n shots takes n
// consecutive rows of its code's ring (admission by device memory: a request
// waits until rows are free).  Submitting copies the syndromes into the
// device arena, notes each row's request, and raises the code's published
// shot count in host-mapped memory.  The persistent kernel (the batched
// kernel with kServe streams) claims published shots as slots free up, so
// requests that arrive while others run join the same device work pool; trial
// tickets of failed shots keep priority over new shots.  The kernel writes
// results into host-mapped output rows and, when the last shot of a request
// is out, posts the request's tag to its completion flag.  Polling waits for
// that flag, copies the rows out and releases them (rows are released in
// order).  The kernel leaves after idle_exit_us without work; a host pump
// thread relaunches it whenever admitted work is unfinished.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "bpsf.h"
#include "bpsf_api_internal.h"
#include "bpsf_internal.h"

using namespace bpsf;

namespace {

size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

struct SrvCode {
    bpsf_ctx *ctx = nullptr;
    long long rows = 0;
    uint32_t *d_synd = nullptr;                  // rows x Ws, device
    void *h_out = nullptr;                       // mapped output rows
    uint32_t *h_corr = nullptr, *m_corr = nullptr;
    uint8_t *h_conv = nullptr, *m_conv = nullptr;
    int16_t *h_iters = nullptr, *m_iters = nullptr;
    uint8_t *h_stage = nullptr, *m_stage = nullptr;
    int *h_row_req = nullptr, *m_row_req = nullptr;  // mapped: request slot of each row
    long long *h_pub = nullptr, *m_pub = nullptr;    // mapped: published shot count
    StreamCounters *d_ctr = nullptr;
    void *d_rec = nullptr;
    Records rec{};
    long long next_g = 0;                        // next global shot number
    long long released = 0;                      // shots below this have free rows
    std::map<long long, long long> polled;       // polled requests not yet released: g0 -> n
};

struct SrvReq {
    int code = -1;
    long long g0 = 0, n = 0;
    uint64_t ticket = 0;
    unsigned tag = 0;
    bool live = false;
};

}  // namespace

struct bpsf_server {
    int device = 0, n_codes = 0, max_req = 0, grid = 0;
    SrvCode codes[kMaxStreams];
    unsigned *d_req_left = nullptr;                       // device: shots left per request slot
    unsigned *h_left = nullptr;                           // pinned staging for d_req_left
    unsigned *h_req_tag = nullptr, *m_req_tag = nullptr;  // mapped
    unsigned *h_req_flag = nullptr, *m_req_flag = nullptr;  // mapped, written by the device
    int *h_stop = nullptr, *m_stop = nullptr;             // mapped
    std::vector<SrvReq> reqs;
    std::vector<int> free_slots;
    std::map<uint64_t, int> by_ticket;
    uint64_t next_ticket = 1;
    unsigned next_tag = 1;
    cudaStream_t kstream = nullptr, cstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool launched = false;
    long long idle_ns = 0;
    bpsf_plan plan;
    StreamDev sds[kMaxStreams];
    std::mutex mu;
    std::condition_variable cv;
    std::thread pump;
    std::atomic<bool> quit{false}, closing{false};
    std::atomic<int> unfinished{0};  // admitted requests whose flag has not been seen
};

// Relaunch the persistent kernel if it has left and admitted work is pending.
static bpsf_status ensure_running(bpsf_server *s) {
    if (s->launched) {
        const cudaError_t q = cudaEventQuery(s->kdone);
        if (q == cudaErrorNotReady) return BPSF_OK;
        if (q != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "serving kernel: %s", cudaGetErrorString(q));
        s->launched = false;
    }
    bpsf_launch_plan(s->plan, false, s->sds, s->n_codes, s->grid, s->kstream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(s->kdone, s->kstream);
    if (e != cudaSuccess) return bpsf_fail(BPSF_ECUDA, "serving kernel launch: %s", cudaGetErrorString(e));
    s->launched = true;
    return BPSF_OK;
}

static bool request_done(const bpsf_server *s, int q) {
    return *reinterpret_cast<volatile unsigned *>(s->h_req_flag + q) == s->reqs[q].tag;
}

static void pump_loop(bpsf_server *s) {
    cudaSetDevice(s->device);
    while (!s->quit.load()) {
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        std::lock_guard<std::mutex> lk(s->mu);
        bool pending = false;
        int unf = 0;
        for (int q = 0; q < s->max_req; ++q)
            if (s->reqs[q].live && !request_done(s, q)) {
                pending = true;
                ++unf;
            }
        s->unfinished.store(unf);
        if (pending) ensure_running(s);
    }
}

static void free_server(bpsf_server *s) {
    for (int k = 0; k < s->n_codes; ++k) {
        SrvCode &c = s->codes[k];
        if (c.d_synd) cudaFree(c.d_synd);
        if (c.h_out) cudaFreeHost(c.h_out);
        if (c.d_ctr) cudaFree(c.d_ctr);
        if (c.d_rec) cudaFree(c.d_rec);
    }
    if (s->d_req_left) cudaFree(s->d_req_left);
    if (s->h_left) cudaFreeHost(s->h_left);
    if (s->h_req_tag) cudaFreeHost(s->h_req_tag);
    if (s->h_req_flag) cudaFreeHost(s->h_req_flag);
    if (s->h_stop) cudaFreeHost(s->h_stop);
    if (s->kdone) cudaEventDestroy(s->kdone);
    if (s->kstream) cudaStreamDestroy(s->kstream);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    delete s;
}

template <typename T>
static cudaError_t host_mapped(T **h, T **m, size_t bytes) {
    void *p = nullptr;
    cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    std::memset(p, 0, bytes);
    *h = static_cast<T *>(p);
    void *dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, p, 0);
    *m = static_cast<T *>(dp);
    return e;
}

extern "C" bpsf_status bpsf_serve_start(bpsf_server **out, bpsf_ctx *const *codes, int32_t n_codes,
                                        const bpsf_serve_cfg *cfg) {
    if (!out) return bpsf_fail(BPSF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!codes || n_codes < 1 || n_codes > kMaxStreams)
        return bpsf_fail(BPSF_EINVAL, "n_codes must be in 1..%d", kMaxStreams);
    bpsf_serve_cfg c = cfg ? *cfg : bpsf_serve_cfg{};
    if (c.flags != 0) return bpsf_fail(BPSF_EINVAL, "cfg.flags must be 0");
    if (c.max_inflight_shots <= 0) c.max_inflight_shots = 1 << 16;
    if (c.max_inflight_shots > (1ll << 26)) return bpsf_fail(BPSF_EINVAL, "max_inflight_shots too large");
    if (c.idle_exit_us <= 0) c.idle_exit_us = 20000;
    if (c.max_requests <= 0) c.max_requests = 4096;
    if (c.max_requests > (1 << 20)) return bpsf_fail(BPSF_EINVAL, "max_requests too large");
    if (c.blocks < 0) return bpsf_fail(BPSF_EINVAL, "blocks must be >= 0");
    for (int k = 0; k < n_codes; ++k) {
        if (!codes[k]) return bpsf_fail(BPSF_EINVAL, "code %d is NULL", k);
        for (int q = 0; q < k; ++q)
            if (codes[q] == codes[k]) return bpsf_fail(BPSF_EINVAL, "a context appears twice");
        if (codes[k]->device != codes[0]->device) return bpsf_fail(BPSF_EINVAL, "contexts on different devices");
    }
    bpsf_server *s = new bpsf_server();
    s->device = codes[0]->device;
    s->n_codes = n_codes;
    s->max_req = c.max_requests;
    s->idle_ns = (long long)c.idle_exit_us * 1000;
    cudaSetDevice(s->device);
    // One launch shape for all codes: the first code's tuning, slots per team
    // shrunk per code to fit, fewer warps if still needed.
    std::vector<bpsf_ctx *> cs(codes, codes + n_codes);
    bpsf_tuning t = codes[0]->tune;
    bpsf_status st = bpsf_make_plan(cs.data(), n_codes, t, false, &s->plan, true);
    while (st == BPSF_EINVAL && t.warps_per_block > t.warps_per_team) {
        t.warps_per_block -= t.warps_per_team;
        st = bpsf_make_plan(cs.data(), n_codes, t, false, &s->plan, true);
    }
    if (st != BPSF_OK) {
        delete s;
        return st;
    }
    s->grid = c.blocks > 0 ? std::min(c.blocks, s->plan.grid) : s->plan.grid;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_req_left, 4 * (size_t)s->max_req);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_left, 4 * (size_t)s->max_req);
    if (e == cudaSuccess) e = host_mapped(&s->h_req_tag, &s->m_req_tag, 4 * (size_t)s->max_req);
    if (e == cudaSuccess) e = host_mapped(&s->h_req_flag, &s->m_req_flag, 4 * (size_t)s->max_req);
    if (e == cudaSuccess) e = host_mapped(&s->h_stop, &s->m_stop, 64);
    for (int k = 0; k < n_codes && e == cudaSuccess; ++k) {
        SrvCode &sc = s->codes[k];
        bpsf_ctx *x = codes[k];
        sc.ctx = x;
        sc.rows = c.max_inflight_shots;
        const size_t R = (size_t)sc.rows;
        e = cudaMalloc((void **)&sc.d_synd, 4 * R * x->Ws);
        if (e != cudaSuccess) break;
        // Mapped outputs and bookkeeping: corr | conv | iters | stage | row_req | published.
        const size_t o_corr = 0, o_conv = a16(o_corr + 4 * R * x->Wn), o_it = a16(o_conv + R), o_st = a16(o_it + 2 * R),
                     o_rq = a16(o_st + R), o_pub = a16(o_rq + 4 * R), total = a16(o_pub + 64);
        unsigned char *h = nullptr, *m = nullptr;
        e = host_mapped(&h, &m, total);
        if (e != cudaSuccess) break;
        sc.h_out = h;
        sc.h_corr = (uint32_t *)(h + o_corr);
        sc.m_corr = (uint32_t *)(m + o_corr);
        sc.h_conv = h + o_conv;
        sc.m_conv = m + o_conv;
        sc.h_iters = (int16_t *)(h + o_it);
        sc.m_iters = (int16_t *)(m + o_it);
        sc.h_stage = h + o_st;
        sc.m_stage = m + o_st;
        sc.h_row_req = (int *)(h + o_rq);
        sc.m_row_req = (int *)(m + o_rq);
        sc.h_pub = (long long *)(h + o_pub);
        sc.m_pub = (long long *)(m + o_pub);
        e = cudaMalloc((void **)&sc.d_ctr, sizeof(StreamCounters));
        if (e == cudaSuccess) e = cudaMemset(sc.d_ctr, 0, sizeof(StreamCounters));
        if (e != cudaSuccess) break;
        // Records at each arena row; the publication queue is a ring of R
        // entries (pending failed shots never outnumber admitted shots).
        const int w = std::max(x->p.w, 1), T = std::max(x->n_trials, 1);
        const size_t sz[8] = {a16(8 * R), a16(8 * R), a16(4 * R), a16(8 * R), a16(4 * R * w), a16(4 * R * x->Ws),
                              a16(4 * R * T * x->Wn), a16(2 * R * T)};
        size_t tot = 0;
        for (size_t v : sz) tot += v;
        e = cudaMalloc(&sc.d_rec, tot);
        if (e != cudaSuccess) break;
        unsigned char *p = (unsigned char *)sc.d_rec;
        sc.rec.qseq = (unsigned long long *)p;
        p += sz[0];
        sc.rec.qshot = (long long *)p;
        p += sz[1];
        sc.rec.done = (unsigned *)p;
        p += sz[2];
        sc.rec.best = (unsigned long long *)p;
        p += sz[3];
        sc.rec.phi = (int32_t *)p;
        p += sz[4];
        sc.rec.synd = (uint32_t *)p;
        p += sz[5];
        sc.rec.corr = (uint32_t *)p;
        p += sz[6];
        sc.rec.iters = (int16_t *)p;
        sc.rec.cap = (long long)R;
        e = cudaMemset(sc.rec.qseq, 0, 8 * R);
        // The serving stream of this code.
        JobDev job{sc.d_synd, sc.m_corr, sc.m_conv, sc.m_iters, sc.m_stage, 0, x->Ws, x->Wn};
        StreamDev sd = bpsf_make_stream(x, job, nullptr, kServe);
        sd.rec = sc.rec;
        sd.ctr = sc.d_ctr;
        sd.serve.published = sc.m_pub;
        sd.serve.stop = s->m_stop;
        sd.serve.row_req = sc.m_row_req;
        sd.serve.req_left = s->d_req_left;
        sd.serve.req_tag = s->m_req_tag;
        sd.serve.req_flag = s->m_req_flag;
        sd.serve.rows = sc.rows;
        sd.serve.idle_ns = s->idle_ns;
        s->sds[k] = sd;
    }
    if (e != cudaSuccess) {
        free_server(s);
        return bpsf_fail(BPSF_ENOMEM, "serving buffers: %s", cudaGetErrorString(e));
    }
    s->reqs.assign(s->max_req, SrvReq{});
    for (int q = s->max_req - 1; q >= 0; --q) s->free_slots.push_back(q);
    s->pump = std::thread(pump_loop, s);
    *out = s;
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_serve_submit(bpsf_server *s, int32_t code, int64_t n, const uint32_t *h_synd,
                                         int64_t timeout_us, uint64_t *ticket) {
    if (!s) return bpsf_fail(BPSF_EINVAL, "server is NULL");
    if (s->closing.load()) return bpsf_fail(BPSF_ECLOSED, "server is stopping");
    if (code < 0 || code >= s->n_codes) return bpsf_fail(BPSF_EINVAL, "code index %d out of range", code);
    if (n < 1 || !h_synd || !ticket) return bpsf_fail(BPSF_EINVAL, "need n >= 1, syndromes and a ticket pointer");
    SrvCode &sc = s->codes[code];
    if (n > sc.rows) return bpsf_fail(BPSF_EINVAL, "request of %lld shots exceeds %lld rows", (long long)n, sc.rows);
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max<int64_t>(timeout_us, 0));
    auto fits = [&] { return !s->free_slots.empty() && sc.rows - (sc.next_g - sc.released) >= n; };
    while (!fits()) {
        if (s->closing.load()) return bpsf_fail(BPSF_ECLOSED, "server is stopping");
        if (timeout_us <= 0 || s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (fits()) break;
            return bpsf_fail(BPSF_EBUSY, "no room for %lld shots (admission by device rows)", (long long)n);
        }
    }
    cudaSetDevice(s->device);
    const int q = s->free_slots.back();
    s->free_slots.pop_back();
    const long long g0 = sc.next_g;
    const int Ws = sc.ctx->Ws;
    const long long r0 = g0 % sc.rows, first = std::min<long long>(n, sc.rows - r0);
    cudaError_t e = cudaMemcpyAsync(sc.d_synd + r0 * Ws, h_synd, 4 * (size_t)first * Ws, cudaMemcpyHostToDevice,
                                    s->cstream);
    if (e == cudaSuccess && first < n)
        e = cudaMemcpyAsync(sc.d_synd, h_synd + first * Ws, 4 * (size_t)(n - first) * Ws, cudaMemcpyHostToDevice,
                            s->cstream);
    s->h_left[q] = (unsigned)n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_req_left + q, s->h_left + q, 4, cudaMemcpyHostToDevice, s->cstream);
    for (long long i = 0; i < n; ++i) sc.h_row_req[(g0 + i) % sc.rows] = q;
    const unsigned tag = s->next_tag++;
    if (s->next_tag == 0) s->next_tag = 1;
    reinterpret_cast<volatile unsigned *>(s->h_req_flag)[q] = 0u;
    reinterpret_cast<volatile unsigned *>(s->h_req_tag)[q] = tag;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cstream);
    if (e != cudaSuccess) {
        s->free_slots.push_back(q);
        return bpsf_fail(BPSF_ECUDA, "request copy: %s", cudaGetErrorString(e));
    }
    SrvReq &r = s->reqs[q];
    r.code = code;
    r.g0 = g0;
    r.n = n;
    r.ticket = s->next_ticket++;
    r.tag = tag;
    r.live = true;
    s->by_ticket[r.ticket] = q;
    sc.next_g = g0 + n;
    // Publish: every write above is visible before the new count.
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *reinterpret_cast<volatile long long *>(sc.h_pub) = g0 + n;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    s->unfinished.fetch_add(1);
    bpsf_status st = ensure_running(s);
    if (st != BPSF_OK) return st;
    *ticket = r.ticket;
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_serve_poll(bpsf_server *s, uint64_t ticket, int64_t timeout_us, uint32_t *h_corr,
                                       uint8_t *h_conv, int16_t *h_iters, uint8_t *h_stage) {
    if (!s) return bpsf_fail(BPSF_EINVAL, "server is NULL");
    int q = -1;
    SrvReq r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->by_ticket.find(ticket);
        if (it == s->by_ticket.end())
            return bpsf_fail(s->closing.load() ? BPSF_ECLOSED : BPSF_EINVAL, "unknown ticket %llu",
                             (unsigned long long)ticket);
        q = it->second;
        r = s->reqs[q];
    }
    const auto start = std::chrono::steady_clock::now();
    long long spins = 0;
    while (*reinterpret_cast<volatile unsigned *>(s->h_req_flag + q) != r.tag) {
        const auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - start);
        if (el.count() >= timeout_us) return bpsf_fail(BPSF_ETIMEOUT, "request not finished");
        if (++spins > 2000) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    SrvCode &sc = s->codes[r.code];
    const int Wn = sc.ctx->Wn;
    for (long long i = 0; i < r.n;) {
        const long long row = (r.g0 + i) % sc.rows;
        const long long len = std::min<long long>(r.n - i, sc.rows - row);
        if (h_corr) std::memcpy(h_corr + i * Wn, sc.h_corr + row * Wn, 4 * (size_t)len * Wn);
        if (h_conv) std::memcpy(h_conv + i, sc.h_conv + row, (size_t)len);
        if (h_iters) std::memcpy(h_iters + i, sc.h_iters + row, 2 * (size_t)len);
        if (h_stage) std::memcpy(h_stage + i, sc.h_stage + row, (size_t)len);
        i += len;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->reqs[q].live = false;
        s->by_ticket.erase(ticket);
        s->free_slots.push_back(q);
        // Release rows in order.
        sc.polled[r.g0] = r.n;
        for (auto it = sc.polled.begin(); it != sc.polled.end() && it->first == sc.released;) {
            sc.released += it->second;
            it = sc.polled.erase(it);
        }
    }
    s->cv.notify_all();
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_serve_stop(bpsf_server *s) {
    if (!s) return bpsf_fail(BPSF_EINVAL, "server is NULL");
    s->closing.store(true);
    s->cv.notify_all();
    // Let admitted requests finish on the device (bounded).
    const auto start = std::chrono::steady_clock::now();
    bpsf_status st = BPSF_OK;
    for (;;) {
        bool pending = false;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int q = 0; q < s->max_req; ++q)
                if (s->reqs[q].live && !request_done(s, q)) pending = true;
        }
        if (!pending) break;
        if (std::chrono::steady_clock::now() - start > std::chrono::seconds(30)) {
            st = bpsf_fail(BPSF_ETIMEOUT, "admitted requests did not finish");
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    s->quit.store(true);
    if (s->pump.joinable()) s->pump.join();
    *reinterpret_cast<volatile int *>(s->h_stop) = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    cudaSetDevice(s->device);
    cudaError_t e = cudaStreamSynchronize(s->kstream);
    if (e != cudaSuccess && st == BPSF_OK) st = bpsf_fail(BPSF_ECUDA, "serving kernel: %s", cudaGetErrorString(e));
    for (int k = 0; k < s->n_codes && st == BPSF_OK; ++k) {
        StreamCounters h;
        if (cudaMemcpy(&h, s->codes[k].d_ctr, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess && h.status)
            st = bpsf_fail(BPSF_ETIMEOUT, "device status 0x%x while serving", h.status);
    }
    free_server(s);
    return st;
}
