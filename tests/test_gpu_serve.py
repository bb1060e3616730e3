"""Serving form: continuous batching through bpsf_serve_* (C ABI).

Each request's results must equal those of the same syndromes decoded alone
(bpsf_decode), whatever else is in flight; admission, back-pressure, errors
and the relaunch of the device loop after it idles out are checked too.  The
last test checks that the device's bounded waits give up and report instead
of spinning (failure detection without any fault).
"""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from paper_2507_00254_gb300 import bpsf as B  # noqa: E402
from paper_2507_00254_gb300 import build as libbuild  # noqa: E402
from paper_2507_00254_gb300 import codes  # noqa: E402

pytestmark = pytest.mark.gpu

BB_PARAMS = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
PH_PARAMS = B.Params(max_iter=200, alpha=0.625, w=5, short_iter=30)


@pytest.fixture(scope="module")
def mix():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    libbuild.build()
    out = []
    for name, p, P in (("bb72", 0.06, BB_PARAMS), ("bb144", 0.06, BB_PARAMS), ("phenom", 0.004, PH_PARAMS)):
        c = codes.phenom("bb144") if name == "phenom" else codes.bb(name)
        d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p), P)
        out.append((name, c, d, p))
    return out


def synd_host(c, d, p, n, seed):
    if c.rounds > 1:
        e = synth.phenom_error_bits(seed, 0, 0, n, 144, 72, 12, p, p)
    else:
        e = synth.bernoulli_bits(seed, 0, 0, n, c.N, p)
    pad = np.zeros((n, 32 * d.Wn), dtype=np.uint8)
    pad[:, :c.N] = e
    w = np.packbits(pad.reshape(n, d.Wn * 4, 8), axis=-1, bitorder="little").reshape(n, d.Wn * 4)
    err = torch.from_numpy(w.view(np.int32).copy()).cuda()
    return d.syndrome(err).cpu().numpy().view(np.uint32)


def alone(d, s):
    out = d.decode(torch.from_numpy(s.view(np.int32)).cuda())
    return {k: v.cpu().numpy() for k, v in out.items()}


def same(got, ref):
    assert (got["corr"].view(np.int32) == ref["corr"]).all()
    for k in ("conv", "iters", "stage"):
        assert (got[k] == ref[k]).all(), k


def test_each_result_is_the_same_alone_and_in_the_mix(mix):
    decs = [d for _, _, d, _ in mix]
    srv = B.Server(decs, max_inflight_shots=8192)
    try:
        reqs = []
        sizes = [1, 7, 130, 600, 33, 1000, 2, 257]
        for r, n in enumerate(sizes):
            for k, (name, c, d, p) in enumerate(mix):
                nn = n if name != "phenom" else max(1, n // 8)
                s = synd_host(c, d, p, nn, 7000 + 31 * r + k)
                reqs.append((k, s, srv.submit(k, s)))
        for k, s, t in reqs:
            got = srv.poll(t, s.shape[0], k)
            assert got is not None
            same(got, alone(mix[k][2], s))
    finally:
        srv.stop()


def test_first_success_rule_served_equals_alone():
    # Early cancel of trials that cannot win changes no result, served or alone.
    c = codes.bb("bb144")
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20, select=B.BPSF_SELECT_FIRST)
    d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, 0.07), P)
    srv = B.Server([d], max_inflight_shots=4096)
    try:
        reqs = []
        for r, n in enumerate((1, 50, 700, 3)):
            s = synd_host(c, d, 0.07, n, 7700 + r)
            reqs.append((s, srv.submit(0, s)))
        got = [(s, srv.poll(t, s.shape[0], 0)) for s, t in reqs]
    finally:
        srv.stop()
    for s, g in got:
        same(g, alone(d, s))


def test_admission_backpressure_and_errors(mix):
    name, c, d, p = mix[0]
    srv = B.Server([d], max_inflight_shots=256)
    try:
        s = synd_host(c, d, p, 256, 11)
        t1 = srv.submit(0, s)
        with pytest.raises(B.BpsfError) as ei:
            srv.submit(0, s[:1], timeout_us=0)  # every row is taken until t1 is polled
        assert ei.value.status == B.BPSF_EBUSY
        same(srv.poll(t1, 256, 0), alone(d, s))
        t2 = srv.submit(0, s[:1], timeout_us=0)  # rows were released
        same(srv.poll(t2, 1, 0), alone(d, s[:1]))
        big = np.zeros((257, d.Ws), dtype=np.uint32)
        with pytest.raises(B.BpsfError) as ei:
            srv.submit(0, big)
        assert ei.value.status == B.BPSF_EINVAL
        with pytest.raises(B.BpsfError) as ei:
            srv.poll(123456789, 1, 0)
        assert ei.value.status == B.BPSF_EINVAL
    finally:
        srv.stop()


def test_poll_timeout_keeps_the_ticket(mix):
    name, c, d, p = mix[2]  # phenomenological: a large request takes a while
    srv = B.Server([d], max_inflight_shots=4096)
    try:
        s = synd_host(c, d, p, 4000, 12)
        t = srv.submit(0, s)
        assert srv.poll(t, 4000, 0, timeout_us=0) is None
        same(srv.poll(t, 4000, 0), alone(d, s))
    finally:
        srv.stop()


def test_concurrent_clients(mix):
    decs = [d for _, _, d, _ in mix[:2]]
    # References first: a context serves one decode call at a time.
    work = {}
    for tid in range(4):
        for r in range(12):
            k = (tid + r) % 2
            name, c, d, p = mix[k]
            s = synd_host(c, d, p, 17 + 13 * r, 9000 + 100 * tid + r)
            work[(tid, r)] = (k, s, alone(d, s))
    srv = B.Server(decs, max_inflight_shots=2048)
    errors = []

    def client(tid):
        try:
            for r in range(12):
                k, s, ref = work[(tid, r)]
                t = srv.submit(k, s)
                got = srv.poll(t, s.shape[0], k)
                same(got, ref)
        except Exception as exc:  # pragma: no cover - reported below
            errors.append(exc)

    try:
        ths = [threading.Thread(target=client, args=(i,)) for i in range(4)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
    finally:
        srv.stop()
    assert not errors, errors


def test_device_loop_relaunches_after_idle_exit(mix):
    name, c, d, p = mix[1]
    srv = B.Server([d], max_inflight_shots=1024, idle_exit_us=500)
    try:
        for r in range(3):
            s = synd_host(c, d, p, 300, 13 + r)
            same(srv.poll(srv.submit(0, s), 300, 0), alone(d, s))
            time.sleep(0.05)  # well past the idle exit: the next submit relaunches the loop
    finally:
        srv.stop()


def test_stop_finishes_admitted_requests(mix):
    name, c, d, p = mix[1]
    srv = B.Server([d], max_inflight_shots=4096)
    s = synd_host(c, d, p, 3000, 14)
    srv.submit(0, s)
    srv.stop()  # returns once the admitted request is done on the device


def test_bounded_device_wait_reports_instead_of_spinning(mix):
    name, c, d, p = mix[0]
    t0 = time.perf_counter()
    st = B.bpsf_selftest_wait(d.handle, 2000, 0)
    assert st == B.BPSF_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    # The context stays usable.
    s = synd_host(c, d, p, 100, 15)
    alone(d, s)


def test_request_that_wraps_the_ring(mix):
    # Rows are a ring: a request that runs past the last row continues at row 0.
    name, c, d, p = mix[1]
    srv = B.Server([d], max_inflight_shots=100)
    try:
        for r, n in enumerate((70, 70, 55, 100)):
            s = synd_host(c, d, p, n, 7900 + r)
            same(srv.poll(srv.submit(0, s), n, 0), alone(d, s))
    finally:
        srv.stop()


def test_replays_time_both_forms_on_one_clock(mix):
    """bpsf_serve_replay and bpsf_plain_replay on the same requests, open loop
    and closed loop: every request gets a finite, positive latency on the
    library's monotonic clock, and the open-loop latency counts from the
    scheduled arrival."""
    decs = [d for _, _, d, _ in mix]
    reqs, which = [], []
    for r in range(24):
        k = r % len(mix)
        name, c, d, p = mix[k]
        reqs.append(synd_host(c, d, p, 1 + (r % 3), 8100 + r))
        which.append(k)
    arrivals = np.cumsum(np.full(len(reqs), 2e-4))
    lat_p, span_p = B.plain_replay(decs, arrivals, which, reqs)
    lat_pc, _ = B.plain_replay(decs, None, which, reqs)
    assert (lat_p > 0).all() and (lat_pc > 0).all() and np.isfinite(lat_p).all()
    assert span_p >= arrivals[-1]
    srv = B.Server(decs, max_inflight_shots=1024)
    try:
        lat_s, span_s = srv.replay(arrivals, which, reqs)
        lat_sc, _ = srv.replay(None, which, reqs)
    finally:
        srv.stop()
    assert (lat_s > 0).all() and (lat_sc > 0).all() and np.isfinite(lat_s).all()
    assert span_s >= arrivals[-1]
    with pytest.raises(B.BpsfError):
        B.plain_replay(decs, arrivals[::-1].copy(), which, reqs)  # arrivals must not decrease
