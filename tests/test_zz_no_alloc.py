"""bpsf_decode_noalloc against bpsf_decode through the C ABI.

The no-allocation entry point serves callers that cannot allocate device
memory while they decode (hard-deadline loops that must not block in the
allocator, runtimes whose own allocator owns the device heap).  It must give
exactly what the allocating entry point gives, call after call, although every
call reuses the same static scratch array, and the device's free memory must
not move across a call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from paper_2507_00254_gb300 import bpsf as B  # noqa: E402
from paper_2507_00254_gb300 import build as libbuild  # noqa: E402
from paper_2507_00254_gb300 import codes  # noqa: E402

pytestmark = pytest.mark.gpu


def _inputs(dec, code, p, n, seed):
    e = synth.bernoulli_bits(seed, 0, 0, n, code.N, p)
    pad = np.zeros((n, 32 * dec.Wn), dtype=np.uint8)
    pad[:, :code.N] = e
    words = np.packbits(pad.reshape(n, dec.Wn * 4, 8), axis=-1, bitorder="little").reshape(n, dec.Wn * 4)
    err = torch.from_numpy(words.view(np.int32).copy()).cuda()
    return dec.syndrome(err)


def _noalloc(dec, synd):
    n = int(synd.shape[0])
    out = dec.outputs(n)
    sh = torch.cuda.current_stream().cuda_stream
    B.bpsf_decode_noalloc(dec.handle, n, synd.data_ptr(), int(synd.shape[1]), out["corr"].data_ptr(), dec.Wn,
                          out["conv"].data_ptr(), out["iters"].data_ptr(), out["stage"].data_ptr(), sh)
    B.bpsf_sync(dec.handle, sh)
    return out


def _same(a, b):
    for key in ("corr", "conv", "iters", "stage"):
        assert torch.equal(a[key], b[key]), key


@pytest.fixture(scope="module")
def decoder():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    libbuild.build()
    c = codes.bb("bb144")
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    return c, B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, 0.07), P)


def test_noalloc_matches_decode_on_two_calls_in_a_row(decoder):
    c, dec = decoder
    cap = B.bpsf_noalloc_max_shots(dec.handle)
    assert cap >= 200000  # about 100 bytes of records per shot of [[144]]
    # A larger batch, then a smaller one over the scratch the first one left behind.
    for n, seed in ((min(cap, 50000), 901), (3000, 902)):
        synd = _inputs(dec, c, 0.07, n, seed)
        ref = dec.decode(synd)
        got = _noalloc(dec, synd)
        _same(got, ref)
        assert int((ref["stage"] == 1).sum()) > 0  # the trial records were exercised
        w = dec.last_work()
        assert w["initial_runs"] == n and w["failed_shots"] == int((ref["stage"] != 0).sum())


def test_noalloc_rejects_batches_beyond_the_scratch(decoder):
    c, dec = decoder
    cap = B.bpsf_noalloc_max_shots(dec.handle)
    synd = torch.zeros((1, dec.Ws), dtype=torch.int32, device="cuda")
    out = dec.outputs(1)
    with pytest.raises(B.BpsfError) as ei:
        B.bpsf_decode_noalloc(dec.handle, cap + 1, synd.data_ptr(), dec.Ws, out["corr"].data_ptr(), dec.Wn,
                              out["conv"].data_ptr(), out["iters"].data_ptr(), 0, 0)
    assert ei.value.status == B.BPSF_EINVAL and "scratch" in str(ei.value)


def test_noalloc_leaves_free_memory_unchanged_and_handles_a_trial_list(decoder):
    c, dec = decoder
    synd = _inputs(dec, c, 0.08, 4000, 903)
    out = dec.outputs(4000)
    sh = torch.cuda.current_stream().cuda_stream

    def call():
        B.bpsf_decode_noalloc(dec.handle, 4000, synd.data_ptr(), dec.Ws, out["corr"].data_ptr(), dec.Wn,
                              out["conv"].data_ptr(), out["iters"].data_ptr(), out["stage"].data_ptr(), sh)
        B.bpsf_sync(dec.handle, sh)

    call()  # the first call on the device looks up the array (module loading may map memory)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    call()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # A trial list of a few masks (T != 2^w - 1): a failed shot's record keeps
    # only the winning trial's correction, so the batch limit does not move.
    masks = [0b1, 0b10, 0b11, 0b100101, 0b111111]
    cap63 = B.bpsf_noalloc_max_shots(dec.handle)
    dec.set_trials(masks)
    try:
        assert B.bpsf_noalloc_max_shots(dec.handle) == cap63
        ref = dec.decode(synd)
        got = _noalloc(dec, synd)
        _same(got, ref)
        assert int((ref["stage"] == 1).sum()) > 0
    finally:
        dec.set_trials(())


def test_noalloc_reports_each_calls_own_counters(decoder):
    # Two calls queued on one stream before either is synchronised: the
    # first context's counters must be its own call's, not the second's.
    c, dec = decoder
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    dec2 = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, 0.07), P)
    try:
        s1 = _inputs(dec, c, 0.07, 3000, 904)
        s2 = _inputs(dec, c, 0.07, 1000, 905)
        o1, o2 = dec.outputs(3000), dec2.outputs(1000)
        sh = torch.cuda.current_stream().cuda_stream
        for d, s, o, n in ((dec, s1, o1, 3000), (dec2, s2, o2, 1000)):
            B.bpsf_decode_noalloc(d.handle, n, s.data_ptr(), d.Ws, o["corr"].data_ptr(), d.Wn,
                                  o["conv"].data_ptr(), o["iters"].data_ptr(), o["stage"].data_ptr(), sh)
        B.bpsf_sync(dec.handle, sh)
        B.bpsf_sync(dec2.handle, sh)
        assert dec.last_work()["initial_runs"] == 3000
        assert dec2.last_work()["initial_runs"] == 1000
        _same(o1, dec.decode(s1))
    finally:
        dec2.close()


def test_noalloc_rejects_huge_batches_before_any_size_arithmetic(decoder):
    # With a two-mask trial list a huge n would wrap the byte count; the
    # bound is checked first.  The syndrome stride is also invalid, so no
    # kernel could run even if the bound were missing.
    c, dec = decoder
    dec.set_trials([1, 2])
    try:
        buf = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
        with pytest.raises(B.BpsfError) as ei:
            B.bpsf_decode_noalloc(dec.handle, 1 << 62, buf.data_ptr(), 0, buf.data_ptr(), dec.Wn,
                                  buf.data_ptr(), buf.data_ptr(), 0, 0)
        assert ei.value.status == B.BPSF_EINVAL and "scratch" in str(ei.value)
    finally:
        dec.set_trials(())
