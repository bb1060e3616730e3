// Serving form of libbpsf: continuous batching of a request stream over
// several codes.
//
// Each code owns an arena of `rows` shot rows.  A request of n shots takes n
// consecutive rows of its code's ring (admission by arena rows: a request
// waits until rows are free).  The arena and the code's published shot count
// live in host memory mapped into the device's address space: submitting
// writes the syndromes into the rows and then stores the new count with
// release semantics, and the device reads the count with system-scope
// acquire loads before it reads the rows, so a request reaches the device
// without a copy, a stream operation or a driver call.  The
// persistent kernel (the batched kernel with kServe streams) claims published
// shots as slots free up, so requests that arrive while others run join the
// same device work pool; trial tickets of failed shots keep priority over new
// shots.  The kernel writes results into host-mapped output rows and then
// posts g + 1 to the row's completion word.  Polling waits for those words,
// copies the rows out and releases them (rows are released in order).  The
// kernel leaves after idle_exit_us without work; a host pump thread
// relaunches it whenever admitted work is unfinished.
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
    void *h_in = nullptr;                            // mapped input block: published count, then the arena
    long long *h_pub = nullptr, *m_pub = nullptr;    // published shot count (host / device address)
    uint32_t *h_synd = nullptr, *m_synd = nullptr;   // rows x Ws arena (host / device address)
    void *h_out = nullptr;                           // mapped output rows
    uint32_t *h_corr = nullptr, *m_corr = nullptr;
    uint8_t *h_conv = nullptr, *m_conv = nullptr;
    int16_t *h_iters = nullptr, *m_iters = nullptr;
    uint8_t *h_stage8 = nullptr, *m_stage8 = nullptr;
    unsigned *h_done = nullptr, *m_done = nullptr;   // mapped: completion word per row
    StreamCounters *d_ctr = nullptr;
    void *d_rec = nullptr;
    Records rec{};
    long long next_g = 0;                            // next global shot number
    long long released = 0;                          // shots below this have free rows
    std::map<long long, long long> polled;           // polled requests not yet released: g0 -> n
};

struct SrvReq {
    int code = -1;
    long long g0 = 0, n = 0;
    long long checked = 0;  // rows known to be done (from the start of the request)
    uint64_t ticket = 0;
    bool live = false;
};

}  // namespace

struct bpsf_server {
    int device = 0, n_codes = 0, max_req = 0, grid = 0;
    SrvCode codes[kMaxStreams];
    int *h_stop = nullptr, *m_stop = nullptr;  // mapped
    std::vector<SrvReq> reqs;
    std::vector<int> free_slots;
    std::map<uint64_t, int> by_ticket;
    uint64_t next_ticket = 1;
    cudaStream_t kstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool launched = false;
    long long idle_ns = 0;
    bpsf_plan plan;
    StreamDev sds[kMaxStreams];
    std::mutex mu;
    std::condition_variable cv;
    std::thread pump;
    std::atomic<bool> quit{false}, closing{false};
};

// Relaunch the persistent kernel if it has left (the caller holds mu).
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

// True once every shot of request q has posted its completion word; advances
// the request's cursor over rows already seen done.
static bool request_done(bpsf_server *s, int q) {
    SrvReq &r = s->reqs[q];
    SrvCode &sc = s->codes[r.code];
    const volatile unsigned *done = sc.h_done;
    while (r.checked < r.n) {
        const long long g = r.g0 + r.checked;
        if (done[g % sc.rows] != (unsigned)(g + 1)) return false;
        ++r.checked;
    }
    return true;
}

static void pump_loop(bpsf_server *s) {
    cudaSetDevice(s->device);
    while (!s->quit.load()) {
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        std::lock_guard<std::mutex> lk(s->mu);
        bool pending = false;
        for (int q = 0; q < s->max_req && !pending; ++q)
            if (s->reqs[q].live && !request_done(s, q)) pending = true;
        if (pending) ensure_running(s);
    }
}

static void free_server(bpsf_server *s) {
    for (int k = 0; k < s->n_codes; ++k) {
        SrvCode &c = s->codes[k];
        if (c.h_in) cudaFreeHost(c.h_in);
        if (c.h_out) cudaFreeHost(c.h_out);
        if (c.d_ctr) cudaFree(c.d_ctr);
        if (c.d_rec) cudaFree(c.d_rec);
    }
    if (s->h_stop) cudaFreeHost(s->h_stop);
    if (s->kdone) cudaEventDestroy(s->kdone);
    if (s->kstream) cudaStreamDestroy(s->kstream);
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
        if (bpsf_check_trials(codes[k]) != BPSF_OK) return BPSF_EINVAL;
    }
    bpsf_server *s = new bpsf_server();
    s->device = codes[0]->device;
    s->n_codes = n_codes;
    s->max_req = c.max_requests;
    s->idle_ns = (long long)c.idle_exit_us * 1000;
    cudaSetDevice(s->device);
    // Each code keeps its own team shape (shrunk if its block does not fit).
    std::vector<bpsf_ctx *> cs(codes, codes + n_codes);
    std::vector<bpsf_tuning> tunes(n_codes);
    for (int k = 0; k < n_codes; ++k) tunes[k] = codes[k]->tune;
    bpsf_status st = bpsf_make_plan(cs.data(), n_codes, tunes.data(), false, &s->plan, true);
    if (st != BPSF_OK) {
        delete s;
        return st;
    }
    s->grid = c.blocks > 0 ? std::min(c.blocks, s->plan.grid) : s->plan.grid;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming);
    if (e == cudaSuccess) e = host_mapped(&s->h_stop, &s->m_stop, 64);
    for (int k = 0; k < n_codes && e == cudaSuccess; ++k) {
        SrvCode &sc = s->codes[k];
        bpsf_ctx *x = codes[k];
        sc.ctx = x;
        sc.rows = c.max_inflight_shots;
        const size_t R = (size_t)sc.rows;
        // Mapped inputs: the published count (its own 128-byte line), then the arena.
        {
            unsigned char *h = nullptr, *m = nullptr;
            e = host_mapped(&h, &m, 128 + 4 * R * x->Ws);
            if (e != cudaSuccess) break;
            sc.h_in = h;
            sc.h_pub = reinterpret_cast<long long *>(h);
            sc.m_pub = reinterpret_cast<long long *>(m);
            sc.h_synd = reinterpret_cast<uint32_t *>(h + 128);
            sc.m_synd = reinterpret_cast<uint32_t *>(m + 128);
        }
        // Mapped outputs: corr | conv | iters | stage | completion words.
        const size_t o_corr = 0, o_conv = a16(o_corr + 4 * R * x->Wn), o_it = a16(o_conv + R), o_st = a16(o_it + 2 * R),
                     o_dn = a16(o_st + R), total = a16(o_dn + 4 * R);
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
        sc.h_stage8 = h + o_st;
        sc.m_stage8 = m + o_st;
        sc.h_done = (unsigned *)(h + o_dn);
        sc.m_done = (unsigned *)(m + o_dn);
        e = cudaMalloc((void **)&sc.d_ctr, sizeof(StreamCounters));
        if (e == cudaSuccess) e = cudaMemset(sc.d_ctr, 0, sizeof(StreamCounters));
        if (e != cudaSuccess) break;
        // A ring of failed-shot records (failed shots in flight never
        // outnumber admitted shots), all free.
        const long long RR = bpsf_record_ring((long long)R);
        e = cudaMalloc(&sc.d_rec, bpsf_records_bytes(RR, x->p.w, x->Ws, x->Wn, 16));
        if (e != cudaSuccess) break;
        sc.rec = bpsf_records_carve(sc.d_rec, RR, x->p.w, x->Ws, x->Wn, 16);
        e = cudaMemset(sc.rec.qseq, 0, 8 * (size_t)RR);
        // The serving stream of this code.
        JobDev job{sc.m_synd, sc.m_corr, sc.m_conv, sc.m_iters, sc.m_stage8, 0, x->Ws, x->Wn};
        StreamDev sd = bpsf_make_stream(x, job, nullptr, kServe);
        sd.rec = sc.rec;
        sd.ctr = sc.d_ctr;
        sd.serve.published = sc.m_pub;
        sd.serve.stop = s->m_stop;
        sd.serve.row_done = sc.m_done;
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
    BpsfRange range("bpsf_serve_submit");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max<int64_t>(timeout_us, 0));
    auto fits = [&] { return !s->free_slots.empty() && sc.rows - (sc.next_g - sc.released) >= n; };
    while (!fits()) {
        if (s->closing.load()) return bpsf_fail(BPSF_ECLOSED, "server is stopping");
        if (timeout_us <= 0 || s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (fits()) break;
            return bpsf_fail(BPSF_EBUSY, "no room for %lld shots (admission by arena rows)", (long long)n);
        }
    }
    cudaSetDevice(s->device);
    const int q = s->free_slots.back();
    s->free_slots.pop_back();
    const long long g0 = sc.next_g;
    const int Ws = sc.ctx->Ws;
    // Rows first, then the count with release semantics: a device thread that
    // reads the new count (system-scope acquire) then sees the rows.  The
    // caller's buffer is free on return.
    const long long r0 = g0 % sc.rows, first = std::min<long long>(n, sc.rows - r0);
    std::memcpy(sc.h_synd + r0 * Ws, h_synd, 4 * (size_t)first * Ws);
    if (first < n) std::memcpy(sc.h_synd, h_synd + first * Ws, 4 * (size_t)(n - first) * Ws);
    __atomic_store_n(sc.h_pub, g0 + n, __ATOMIC_RELEASE);
    SrvReq &r = s->reqs[q];
    r.code = code;
    r.g0 = g0;
    r.n = n;
    r.checked = 0;
    r.ticket = s->next_ticket++;
    r.live = true;
    s->by_ticket[r.ticket] = q;
    sc.next_g = g0 + n;
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
    SrvCode &sc = s->codes[r.code];
    const volatile unsigned *done = sc.h_done;
    BpsfRange range("bpsf_serve_poll");
    const auto start = std::chrono::steady_clock::now();
    long long spins = 0, i = r.checked;
    while (i < r.n) {
        const long long g = r.g0 + i;
        if (done[g % sc.rows] == (unsigned)(g + 1)) {
            ++i;
            continue;
        }
        const auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - start);
        if (el.count() >= timeout_us) return bpsf_fail(BPSF_ETIMEOUT, "request not finished");
        if (++spins > 4000) std::this_thread::sleep_for(std::chrono::microseconds(2));
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    const int Wn = sc.ctx->Wn;
    for (long long k = 0; k < r.n;) {
        const long long row = (r.g0 + k) % sc.rows;
        const long long len = std::min<long long>(r.n - k, sc.rows - row);
        if (h_corr) std::memcpy(h_corr + k * Wn, sc.h_corr + row * Wn, 4 * (size_t)len * Wn);
        if (h_conv) std::memcpy(h_conv + k, sc.h_conv + row, (size_t)len);
        if (h_iters) std::memcpy(h_iters + k, sc.h_iters + row, 2 * (size_t)len);
        if (h_stage) std::memcpy(h_stage + k, sc.h_stage8 + row, (size_t)len);
        k += len;
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
            for (int q = 0; q < s->max_req && !pending; ++q)
                if (s->reqs[q].live && !request_done(s, q)) pending = true;
            if (pending) ensure_running(s);
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

// Open-loop trace replay for latency measurement: one thread submits request
// i at its scheduled arrival time, another polls every outstanding request
// and stamps its completion, so neither side waits on the other.
// Arguments shared by the two replays: codes in range, shots >= 1, arrivals
// non-decreasing (arrival_s NULL: closed loop).
static bpsf_status check_trace(int n_codes, int64_t n_req, const double *arrival_s, const int32_t *code,
                               const int64_t *n_shots, const uint32_t *const *synd, const double *latency_s) {
    if (n_req < 1 || !code || !n_shots || !synd || !latency_s) return bpsf_fail(BPSF_EINVAL, "bad replay arguments");
    for (int64_t i = 0; i < n_req; ++i) {
        if (code[i] < 0 || code[i] >= n_codes || n_shots[i] < 1 || !synd[i])
            return bpsf_fail(BPSF_EINVAL, "bad request %lld", (long long)i);
        if (arrival_s && i > 0 && arrival_s[i] < arrival_s[i - 1])
            return bpsf_fail(BPSF_EINVAL, "arrivals must not decrease");
    }
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_serve_replay(bpsf_server *s, int64_t n_req, const double *arrival_s, const int32_t *code,
                                         const int64_t *n_shots, const uint32_t *const *synd, double *latency_s,
                                         double *span_s) {
    if (!s) return bpsf_fail(BPSF_EINVAL, "server is NULL");
    bpsf_status cst = check_trace(s->n_codes, n_req, arrival_s, code, n_shots, synd, latency_s);
    if (cst != BPSF_OK) return cst;
    using clk = std::chrono::steady_clock;
    if (!arrival_s) {
        // Closed loop: request i is submitted once request i - 1 is done.
        const clk::time_point t0 = clk::now();
        for (int64_t i = 0; i < n_req; ++i) {
            const clk::time_point a = clk::now();
            uint64_t t = 0;
            bpsf_status st = bpsf_serve_submit(s, code[i], n_shots[i], synd[i], 60000000, &t);
            if (st == BPSF_OK) st = bpsf_serve_poll(s, t, 60000000, nullptr, nullptr, nullptr, nullptr);
            if (st != BPSF_OK) return st;
            latency_s[i] = std::chrono::duration<double>(clk::now() - a).count();
        }
        if (span_s) *span_s = std::chrono::duration<double>(clk::now() - t0).count();
        return BPSF_OK;
    }
    std::vector<uint64_t> tickets((size_t)n_req, 0);
    std::vector<std::atomic<int>> submitted((size_t)n_req);
    for (auto &a : submitted) a.store(0);
    std::atomic<int64_t> n_sub{0};
    std::atomic<bool> failed{false};
    bpsf_status sub_st = BPSF_OK;
    const clk::time_point t0 = clk::now();
    std::thread submitter([&] {
        for (int64_t i = 0; i < n_req && !failed.load(); ++i) {
            const clk::time_point at = t0 + std::chrono::nanoseconds((long long)(arrival_s[i] * 1e9));
            while (clk::now() < at) {
            }
            uint64_t t = 0;
            bpsf_status st = bpsf_serve_submit(s, code[i], n_shots[i], synd[i], 60000000, &t);
            if (st != BPSF_OK) {
                sub_st = st;
                failed.store(true);
                break;
            }
            tickets[(size_t)i] = t;
            submitted[(size_t)i].store(1, std::memory_order_release);
            n_sub.fetch_add(1);
        }
    });
    bpsf_status st = BPSF_OK;
    std::vector<int64_t> open;
    int64_t next = 0, done = 0;
    clk::time_point last = t0;
    const clk::time_point deadline = t0 + std::chrono::seconds(600);
    while (done < n_req && !failed.load()) {
        while (next < n_req && submitted[(size_t)next].load(std::memory_order_acquire)) open.push_back(next++);
        for (size_t k = 0; k < open.size();) {
            const int64_t i = open[k];
            const bpsf_status ps = bpsf_serve_poll(s, tickets[(size_t)i], 0, nullptr, nullptr, nullptr, nullptr);
            if (ps == BPSF_OK) {
                last = clk::now();
                latency_s[i] = std::chrono::duration<double>(last - t0).count() - arrival_s[i];
                ++done;
                open[k] = open.back();
                open.pop_back();
            } else if (ps == BPSF_ETIMEOUT) {
                ++k;
            } else {
                st = ps;
                failed.store(true);
                break;
            }
        }
        if (clk::now() > deadline) {
            st = bpsf_fail(BPSF_ETIMEOUT, "replay did not finish");
            failed.store(true);
        }
    }
    submitter.join();
    if (sub_st != BPSF_OK) return sub_st;
    if (st != BPSF_OK) return st;
    if (span_s) *span_s = std::chrono::duration<double>(last - t0).count();
    return BPSF_OK;
}

// ---------------------------------------------------------------------------
// The plain per-shot form as a request server, for latency comparisons on the
// same trace and the same clock as bpsf_serve_replay.
// ---------------------------------------------------------------------------

extern "C" bpsf_status bpsf_plain_replay(bpsf_ctx *const *codes, int32_t n_codes, int64_t n_req,
                                         const double *arrival_s, const int32_t *code, const int64_t *n_shots,
                                         const uint32_t *const *synd, double *latency_s, double *span_s) {
    if (!codes || n_codes < 1 || n_codes > kMaxStreams) return bpsf_fail(BPSF_EINVAL, "n_codes must be in 1..%d", kMaxStreams);
    for (int k = 0; k < n_codes; ++k)
        if (!codes[k]) return bpsf_fail(BPSF_EINVAL, "code %d is NULL", k);
    bpsf_status st = check_trace(n_codes, n_req, arrival_s, code, n_shots, synd, latency_s);
    if (st != BPSF_OK) return st;
    cudaSetDevice(codes[0]->device);
    // Per code: device rows for its largest request, and pinned host rows.
    std::vector<int64_t> max_n(n_codes, 0);
    for (int64_t i = 0; i < n_req; ++i) max_n[code[i]] = std::max(max_n[code[i]], n_shots[i]);
    struct Buf {
        void *d = nullptr, *h = nullptr;
        uint32_t *d_synd = nullptr, *d_corr = nullptr, *h_synd = nullptr, *h_corr = nullptr;
        uint8_t *d_conv = nullptr, *d_stage = nullptr, *h_small = nullptr;
        int16_t *d_it = nullptr;
    };
    std::vector<Buf> bufs(n_codes);
    cudaStream_t strm = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&strm, cudaStreamNonBlocking);
    for (int k = 0; k < n_codes && e == cudaSuccess; ++k) {
        if (max_n[k] == 0) continue;
        const bpsf_ctx *c = codes[k];
        const size_t n = (size_t)max_n[k];
        const size_t b_s = a16(4 * n * c->Ws), b_c = a16(4 * n * c->Wn), b_1 = a16(n), b_2 = a16(2 * n);
        Buf &b = bufs[k];
        e = cudaMalloc(&b.d, b_s + b_c + 2 * b_1 + b_2);
        if (e == cudaSuccess) e = cudaMallocHost(&b.h, b_s + b_c + 4 * n);
        if (e != cudaSuccess) break;
        unsigned char *p = (unsigned char *)b.d;
        b.d_synd = (uint32_t *)p;
        b.d_corr = (uint32_t *)(p + b_s);
        b.d_conv = p + b_s + b_c;
        b.d_stage = p + b_s + b_c + b_1;
        b.d_it = (int16_t *)(p + b_s + b_c + 2 * b_1);
        unsigned char *h = (unsigned char *)b.h;
        b.h_synd = (uint32_t *)h;
        b.h_corr = (uint32_t *)(h + b_s);
        b.h_small = h + b_s + b_c;
    }
    using clk = std::chrono::steady_clock;
    const clk::time_point t0 = clk::now();
    clk::time_point last = t0;
    for (int64_t i = 0; i < n_req && e == cudaSuccess && st == BPSF_OK; ++i) {
        clk::time_point a = clk::now();
        if (arrival_s) {
            a = t0 + std::chrono::nanoseconds((long long)(arrival_s[i] * 1e9));
            while (clk::now() < a) {
            }
        }
        BpsfRange req_range("plain replay request");
        bpsf_ctx *c = codes[code[i]];
        Buf &b = bufs[code[i]];
        const int64_t n = n_shots[i];
        std::memcpy(b.h_synd, synd[i], 4 * (size_t)n * c->Ws);
        e = cudaMemcpyAsync(b.d_synd, b.h_synd, 4 * (size_t)n * c->Ws, cudaMemcpyHostToDevice, strm);
        if (e != cudaSuccess) break;
        st = bpsf_decode_plain(c, n, b.d_synd, c->Ws, b.d_corr, c->Wn, b.d_conv, b.d_it, b.d_stage, strm);
        if (st != BPSF_OK) break;
        e = cudaMemcpyAsync(b.h_corr, b.d_corr, 4 * (size_t)n * c->Wn, cudaMemcpyDeviceToHost, strm);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.h_small, b.d_conv, (size_t)n, cudaMemcpyDeviceToHost, strm);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.h_small + n, b.d_it, 2 * (size_t)n, cudaMemcpyDeviceToHost, strm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
        last = clk::now();
        latency_s[i] = std::chrono::duration<double>(last - a).count();
    }
    if (e != cudaSuccess && st == BPSF_OK) st = bpsf_fail(BPSF_ECUDA, "plain replay: %s", cudaGetErrorString(e));
    if (strm) {
        cudaStreamSynchronize(strm);
        cudaStreamDestroy(strm);
    }
    for (Buf &b : bufs) {
        if (b.d) cudaFree(b.d);
        if (b.h) cudaFreeHost(b.h);
    }
    if (st == BPSF_OK && span_s) *span_s = std::chrono::duration<double>(last - t0).count();
    return st;
}
