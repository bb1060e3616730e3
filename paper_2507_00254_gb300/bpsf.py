"""ctypes binding of libbpsf (include/bpsf.h), same names as the C ABI.

Argument marshalling only: every step of decoding runs in the CUDA kernels of
libbpsf.  The functions named like the C entry points take raw integers for
pointers and streams; :class:`Decoder` wraps them for torch tensors.  There is
no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbpsf.so")

BPSF_OK, BPSF_EINVAL, BPSF_ENOMEM, BPSF_ECUDA, BPSF_ETIMEOUT, BPSF_EBUSY, BPSF_ECLOSED, BPSF_EDEVICE = range(8)
BPSF_CSR, BPSF_CSC = 0, 1
BPSF_SELECT_MIN_WEIGHT, BPSF_SELECT_FIRST = 0, 1
BPSF_FLAG_LAYERED = 1

# Every symbol include/bpsf.h declares.
EXPORTS = (
    "bpsf_create", "bpsf_destroy", "bpsf_decode", "bpsf_decode_plain", "bpsf_decode_host", "bpsf_decode_multi",
    "bpsf_sync", "bpsf_get_tuning", "bpsf_set_tuning", "bpsf_autotune", "bpsf_serve_start", "bpsf_serve_submit",
    "bpsf_serve_poll", "bpsf_serve_stop", "bpsf_bb_code", "bpsf_phenom_code", "bpsf_syndrome", "bpsf_decode_debug",
    "bpsf_num_trials", "bpsf_last_work", "bpsf_status_str", "bpsf_last_error", "bpsf_decode_noalloc",
    "bpsf_noalloc_max_shots", "bpsf_selftest_wait", "bpsf_serve_replay", "bpsf_set_trials",
    "bpsf_decode_multi_host", "bpsf_plain_replay",
)


class BpsfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("bpsf status %d: %s" % (status, message))
        self.status = status


class bpsf_params(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("alpha", C.c_float), ("w", C.c_int32), ("w_max", C.c_int32),
                ("short_iter", C.c_int32), ("select", C.c_int32), ("flags", C.c_uint32)]


class bpsf_tuning(C.Structure):
    _fields_ = [("warps_per_team", C.c_int32), ("slots_per_team", C.c_int32), ("warps_per_block", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("iter_chunk", C.c_int32)]

    def as_tuple(self):
        return (self.warps_per_team, self.slots_per_team, self.warps_per_block, self.blocks_per_sm, self.iter_chunk)


class bpsf_job(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("n_shots", C.c_int64), ("d_synd", C.c_void_p), ("synd_stride_words", C.c_int32),
                ("d_corr", C.c_void_p), ("corr_stride_words", C.c_int32), ("d_converged", C.c_void_p),
                ("d_iters", C.c_void_p), ("d_stage", C.c_void_p)]


class bpsf_work(C.Structure):
    _fields_ = [("initial_runs", C.c_int64), ("failed_shots", C.c_int64), ("trial_runs", C.c_int64),
                ("iterations", C.c_int64), ("edge_updates", C.c_int64), ("slot_capacity", C.c_int64),
                ("trials_cancelled", C.c_int64)]


class bpsf_serve_cfg(C.Structure):
    _fields_ = [("max_inflight_shots", C.c_int64), ("blocks", C.c_int32), ("idle_exit_us", C.c_int32),
                ("max_requests", C.c_int32), ("flags", C.c_uint32)]


_lib = None


def lib():
    """Load libbpsf (built in-tree by ``paper_2507_00254_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbpsf is not built (%s missing); run paper_2507_00254_gb300.build.build()" % LIB_PATH)
    try:  # let the CUDA runtime that torch already loaded serve the library
        import torch  # noqa: F401
    except Exception:
        pass
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
    st = C.c_int
    sig = {
        "bpsf_create": ([C.POINTER(vp), i32, i32, i64, i32, vp, vp, vp, C.POINTER(bpsf_params)], st),
        "bpsf_destroy": ([vp], None),
        "bpsf_decode": ([vp, i64, vp, i32, vp, i32, vp, vp, vp, vp], st),
        "bpsf_decode_plain": ([vp, i64, vp, i32, vp, i32, vp, vp, vp, vp], st),
        "bpsf_decode_noalloc": ([vp, i64, vp, i32, vp, i32, vp, vp, vp, vp], st),
        "bpsf_noalloc_max_shots": ([vp], i64),
        "bpsf_decode_host": ([vp, i64, vp, i32, vp, i32, vp, vp, vp, vp], st),
        "bpsf_decode_multi": ([i32, C.POINTER(bpsf_job), vp], st),
        "bpsf_decode_multi_host": ([i32, C.POINTER(bpsf_job), vp], st),
        "bpsf_sync": ([vp, vp], st),
        "bpsf_get_tuning": ([vp, C.POINTER(bpsf_tuning)], st),
        "bpsf_set_tuning": ([vp, C.POINTER(bpsf_tuning)], st),
        "bpsf_autotune": ([vp, C.c_double, i64, vp, C.POINTER(bpsf_tuning)], st),
        "bpsf_serve_start": ([C.POINTER(vp), C.POINTER(vp), i32, C.POINTER(bpsf_serve_cfg)], st),
        "bpsf_serve_submit": ([vp, i32, i64, vp, i64, C.POINTER(C.c_uint64)], st),
        "bpsf_serve_poll": ([vp, C.c_uint64, i64, vp, vp, vp, vp], st),
        "bpsf_serve_stop": ([vp], st),
        "bpsf_serve_replay": ([vp, i64, vp, vp, vp, vp, vp, C.POINTER(C.c_double)], st),
        "bpsf_plain_replay": ([C.POINTER(vp), i32, i64, vp, vp, vp, vp, vp, C.POINTER(C.c_double)], st),
        "bpsf_bb_code": ([i32, i32, i32, vp, vp, i32, vp, vp, i32, vp, vp, i64, C.POINTER(i64)], st),
        "bpsf_phenom_code": ([i32, i32, vp, vp, i32, vp, vp, i64, C.POINTER(i64)], st),
        "bpsf_syndrome": ([vp, i64, vp, i32, vp, i32, vp], st),
        "bpsf_decode_debug": ([vp, i64, vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp], st),
        "bpsf_num_trials": ([vp], i32),
        "bpsf_set_trials": ([vp, i32, vp], st),
        "bpsf_selftest_wait": ([vp, i64, vp], st),
        "bpsf_last_work": ([vp, C.POINTER(bpsf_work)], st),
        "bpsf_status_str": ([st], C.c_char_p),
        "bpsf_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _ = u32
    _lib = L
    return L


def check(status: int) -> None:
    if status != BPSF_OK:
        msg = lib().bpsf_last_error()
        raise BpsfError(status, msg.decode() if msg else "")


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# C-named entry points
# --------------------------------------------------------------------------

def bpsf_create(M: int, N: int, layout: int, ptr: np.ndarray, idx: np.ndarray, priors: np.ndarray,
                params: "bpsf_params") -> int:
    ptr = np.ascontiguousarray(ptr, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    priors = np.ascontiguousarray(np.broadcast_to(np.asarray(priors, dtype=np.float64), (N,)))
    h = C.c_void_p()
    check(lib().bpsf_create(C.byref(h), M, N, int(idx.shape[0]), layout, _np_ptr(ptr), _np_ptr(idx),
                            _np_ptr(priors), C.byref(params)))
    return h.value


def bpsf_destroy(h: int) -> None:
    lib().bpsf_destroy(h)


def bpsf_decode(h, n, d_synd, ss, d_corr, cs, d_conv, d_iters, d_stage, stream):
    check(lib().bpsf_decode(h, n, d_synd, ss, d_corr, cs, d_conv, d_iters, d_stage, stream))


def bpsf_decode_plain(h, n, d_synd, ss, d_corr, cs, d_conv, d_iters, d_stage, stream):
    check(lib().bpsf_decode_plain(h, n, d_synd, ss, d_corr, cs, d_conv, d_iters, d_stage, stream))


def bpsf_decode_noalloc(h, n, d_synd, ss, d_corr, cs, d_conv, d_iters, d_stage, stream):
    check(lib().bpsf_decode_noalloc(h, n, d_synd, ss, d_corr, cs, d_conv, d_iters, d_stage, stream))


def bpsf_noalloc_max_shots(h) -> int:
    return int(lib().bpsf_noalloc_max_shots(h))


def bpsf_decode_host(h, n, h_synd, ss, h_corr, cs, h_conv, h_iters, h_stage, stream):
    check(lib().bpsf_decode_host(h, n, h_synd, ss, h_corr, cs, h_conv, h_iters, h_stage, stream))


def bpsf_decode_multi(jobs, stream):
    arr = (bpsf_job * len(jobs))(*jobs)
    check(lib().bpsf_decode_multi(len(jobs), arr, stream))


def bpsf_decode_multi_host(jobs, stream):
    arr = (bpsf_job * len(jobs))(*jobs)
    check(lib().bpsf_decode_multi_host(len(jobs), arr, stream))


def bpsf_decode_debug(h, n, d_synd, ss, d_corr, cs, d_conv, d_iters, d_stage, d_lout, d_flips, d_phi, d_tsynd,
                      d_tconv, d_titers, stream):
    check(lib().bpsf_decode_debug(h, n, d_synd, ss, d_corr, cs, d_conv, d_iters, d_stage, d_lout, d_flips, d_phi,
                                  d_tsynd, d_tconv, d_titers, stream))


def bpsf_sync(h, stream):
    check(lib().bpsf_sync(h, stream))


def bpsf_get_tuning(h) -> bpsf_tuning:
    t = bpsf_tuning()
    check(lib().bpsf_get_tuning(h, C.byref(t)))
    return t


def bpsf_set_tuning(h, t: bpsf_tuning) -> None:
    check(lib().bpsf_set_tuning(h, C.byref(t)))


def bpsf_autotune(h, p_sample: float, n_sample: int, stream) -> bpsf_tuning:
    t = bpsf_tuning()
    check(lib().bpsf_autotune(h, p_sample, n_sample, stream, C.byref(t)))
    return t


def bpsf_syndrome(h, n, d_err, es, d_synd, ss, stream):
    check(lib().bpsf_syndrome(h, n, d_err, es, d_synd, ss, stream))


def bpsf_num_trials(h) -> int:
    return int(lib().bpsf_num_trials(h))


def bpsf_set_trials(h, masks) -> None:
    """Trial list as subset masks over Phi (bit j selects Phi[j]); empty restores the default."""
    m = np.ascontiguousarray(np.asarray(masks, dtype=np.uint64).reshape(-1))
    check(lib().bpsf_set_trials(h, int(m.shape[0]), m.ctypes.data_as(C.c_void_p) if m.shape[0] else None))


def bpsf_last_work(h) -> bpsf_work:
    w = bpsf_work()
    check(lib().bpsf_last_work(h, C.byref(w)))
    return w


def bpsf_selftest_wait(h, wait_us: int, stream) -> int:
    """Run the bounded-wait self test; returns the raw status (BPSF_ETIMEOUT expected)."""
    return int(lib().bpsf_selftest_wait(h, wait_us, stream))


def bpsf_serve_start(handles, cfg: "bpsf_serve_cfg") -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    s = C.c_void_p()
    check(lib().bpsf_serve_start(C.byref(s), arr, len(handles), C.byref(cfg)))
    return s.value


def bpsf_serve_submit(s, code: int, n: int, h_synd, timeout_us: int) -> int:
    t = C.c_uint64(0)
    check(lib().bpsf_serve_submit(s, code, n, h_synd, timeout_us, C.byref(t)))
    return t.value


def bpsf_serve_poll(s, ticket: int, timeout_us: int, h_corr, h_conv, h_iters, h_stage) -> int:
    """Returns the raw status so callers can tell BPSF_ETIMEOUT from errors."""
    st = int(lib().bpsf_serve_poll(s, ticket, timeout_us, h_corr, h_conv, h_iters, h_stage))
    if st not in (BPSF_OK, BPSF_ETIMEOUT):
        check(st)
    return st


def bpsf_serve_stop(s) -> None:
    check(lib().bpsf_serve_stop(s))


def bpsf_bb_code(l: int, m: int, a_terms, b_terms, which: int = 0):
    """CSR (ptr, idx) of H_X (which=0) or H_Z (which=1) of a BB code."""
    ax = np.array([t[0] for t in a_terms], dtype=np.int32)
    ay = np.array([t[1] for t in a_terms], dtype=np.int32)
    bx = np.array([t[0] for t in b_terms], dtype=np.int32)
    by = np.array([t[1] for t in b_terms], dtype=np.int32)
    n = l * m
    ptr = np.zeros(n + 1, dtype=np.int32)
    cap = n * (len(ax) + len(bx)) + 1
    idx = np.zeros(cap, dtype=np.int32)
    nnz = C.c_int64(0)
    check(lib().bpsf_bb_code(l, m, len(ax), _np_ptr(ax), _np_ptr(ay), len(bx), _np_ptr(bx), _np_ptr(by), which,
                             _np_ptr(ptr), _np_ptr(idx), cap, C.byref(nnz)))
    return ptr, idx[: nnz.value].copy()


def bpsf_phenom_code(M0: int, N0: int, ptr0: np.ndarray, idx0: np.ndarray, rounds: int):
    ptr0 = np.ascontiguousarray(ptr0, dtype=np.int32)
    idx0 = np.ascontiguousarray(idx0, dtype=np.int32)
    ptr = np.zeros(rounds * M0 + 1, dtype=np.int32)
    cap = rounds * (int(idx0.shape[0]) + 2 * M0) + 1
    idx = np.zeros(cap, dtype=np.int32)
    nnz = C.c_int64(0)
    check(lib().bpsf_phenom_code(M0, N0, _np_ptr(ptr0), _np_ptr(idx0), rounds, _np_ptr(ptr), _np_ptr(idx), cap,
                                 C.byref(nnz)))
    return ptr, idx[: nnz.value].copy()


# --------------------------------------------------------------------------
# Torch-facing wrapper
# --------------------------------------------------------------------------

@dataclass
class Params:
    max_iter: int = 50
    alpha: float = 0.625
    w: int = 4
    w_max: int = 0
    short_iter: int = 10
    select: int = BPSF_SELECT_MIN_WEIGHT
    layered: bool = False

    def c(self) -> bpsf_params:
        return bpsf_params(self.max_iter, self.alpha, self.w, self.w_max, self.short_iter, self.select,
                           BPSF_FLAG_LAYERED if self.layered else 0)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


class Decoder:
    """One code + priors + parameters on the current CUDA device."""

    def __init__(self, ptr, idx, M: int, N: int, priors, params: Params, layout: int = BPSF_CSR):
        self.M, self.N = int(M), int(N)
        self.Ws, self.Wn = (self.M + 31) // 32, (self.N + 31) // 32
        self.params = params
        self.handle = bpsf_create(self.M, self.N, layout, ptr, idx, priors, params.c())
        self.n_trials = bpsf_num_trials(self.handle)

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            bpsf_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, n: int, device="cuda"):
        import torch
        return dict(corr=torch.zeros((n, self.Wn), dtype=torch.int32, device=device),
                    conv=torch.zeros(n, dtype=torch.uint8, device=device),
                    iters=torch.zeros(n, dtype=torch.int16, device=device),
                    stage=torch.zeros(n, dtype=torch.uint8, device=device))

    def decode(self, synd, out=None, stream=None, plain=False, sync=True):
        """Decode an (n, Ws) int32 CUDA tensor of packed syndromes."""
        n = int(synd.shape[0])
        out = out or self.outputs(n, synd.device)
        sh = _stream_handle(stream)
        fn = bpsf_decode_plain if plain else bpsf_decode
        fn(self.handle, n, _dptr(synd), int(synd.shape[1]), _dptr(out["corr"]), int(out["corr"].shape[1]),
           _dptr(out["conv"]), _dptr(out["iters"]), _dptr(out.get("stage")), sh)
        if sync:
            bpsf_sync(self.handle, sh)
        return out

    def decode_debug(self, synd, stream=None):
        import torch
        n = int(synd.shape[0])
        dev = synd.device
        out = self.outputs(n, dev)
        T = max(self.n_trials, 1)
        w = max(self.params.w, 1)
        out.update(lout=torch.zeros((n, self.N), dtype=torch.float32, device=dev),
                   flips=torch.zeros((n, self.N), dtype=torch.int16, device=dev),
                   phi=torch.full((n, w), -1, dtype=torch.int32, device=dev),
                   trial_synd=torch.zeros((n, T, self.Ws), dtype=torch.int32, device=dev),
                   trial_conv=torch.full((n, T), 255, dtype=torch.uint8, device=dev),
                   trial_iters=torch.full((n, T), -1, dtype=torch.int16, device=dev))
        sh = _stream_handle(stream)
        bpsf_decode_debug(self.handle, n, _dptr(synd), int(synd.shape[1]), _dptr(out["corr"]), self.Wn,
                          _dptr(out["conv"]), _dptr(out["iters"]), _dptr(out["stage"]), _dptr(out["lout"]),
                          _dptr(out["flips"]), _dptr(out["phi"]), _dptr(out["trial_synd"]),
                          _dptr(out["trial_conv"]), _dptr(out["trial_iters"]), sh)
        bpsf_sync(self.handle, sh)
        return out

    def decode_host(self, synd_np: np.ndarray, stream=None):
        """End-to-end decode of host (numpy uint32/int32) syndromes; returns numpy outputs."""
        synd_np = np.ascontiguousarray(synd_np)
        n = int(synd_np.shape[0])
        corr = np.zeros((n, self.Wn), dtype=np.uint32)
        conv = np.zeros(n, dtype=np.uint8)
        iters = np.zeros(n, dtype=np.int16)
        stage = np.zeros(n, dtype=np.uint8)
        bpsf_decode_host(self.handle, n, _np_ptr(synd_np), int(synd_np.shape[1]), _np_ptr(corr), self.Wn,
                         _np_ptr(conv), _np_ptr(iters), _np_ptr(stage), _stream_handle(stream))
        return dict(corr=corr, conv=conv, iters=iters, stage=stage)

    def syndrome(self, err, stream=None):
        import torch
        n = int(err.shape[0])
        synd = torch.zeros((n, self.Ws), dtype=torch.int32, device=err.device)
        bpsf_syndrome(self.handle, n, _dptr(err), int(err.shape[1]), _dptr(synd), self.Ws, _stream_handle(stream))
        return synd

    @property
    def tuning(self):
        return bpsf_get_tuning(self.handle).as_tuple()

    @tuning.setter
    def tuning(self, t):
        bpsf_set_tuning(self.handle, bpsf_tuning(*t))

    def autotune(self, p_sample=0.05, n_sample=1 << 16, stream=None):
        return bpsf_autotune(self.handle, p_sample, n_sample, _stream_handle(stream)).as_tuple()

    def set_trials(self, masks) -> None:
        """Replace the trial set (see bpsf_set_trials); () restores the default."""
        bpsf_set_trials(self.handle, masks)

    def last_work(self):
        w = bpsf_last_work(self.handle)
        return dict(initial_runs=w.initial_runs, failed_shots=w.failed_shots, trial_runs=w.trial_runs,
                    iterations=w.iterations, edge_updates=w.edge_updates, slot_capacity=w.slot_capacity,
                    trials_cancelled=w.trials_cancelled)


class Server:
    """Continuous-batching server over several decoders (one code each)."""

    def __init__(self, decoders, max_inflight_shots=1 << 16, blocks=0, idle_exit_us=20000, max_requests=4096):
        self.decoders = list(decoders)
        cfg = bpsf_serve_cfg(max_inflight_shots, blocks, idle_exit_us, max_requests, 0)
        self.handle = bpsf_serve_start([d.handle for d in self.decoders], cfg)

    def submit(self, code: int, synd: np.ndarray, timeout_us: int = 10_000_000) -> int:
        synd = np.ascontiguousarray(synd).view(np.uint32)
        d = self.decoders[code]
        if synd.ndim != 2 or synd.shape[1] != d.Ws:
            raise ValueError("expected (n, %d) packed syndromes" % d.Ws)
        return bpsf_serve_submit(self.handle, code, int(synd.shape[0]), _np_ptr(synd), timeout_us)

    def poll(self, ticket: int, n: int, code: int, timeout_us: int = 10_000_000):
        """Results of a request, or None if it is not done within timeout_us."""
        d = self.decoders[code]
        corr = np.zeros((n, d.Wn), dtype=np.uint32)
        conv = np.zeros(n, dtype=np.uint8)
        iters = np.zeros(n, dtype=np.int16)
        stage = np.zeros(n, dtype=np.uint8)
        st = bpsf_serve_poll(self.handle, ticket, timeout_us, _np_ptr(corr), _np_ptr(conv), _np_ptr(iters),
                             _np_ptr(stage))
        if st == BPSF_ETIMEOUT:
            return None
        return dict(corr=corr, conv=conv, iters=iters, stage=stage)

    def replay(self, arrival_s, codes, synds):
        """Open-loop replay (arrival_s None: closed loop); returns (per-request latency in s, span in s)."""
        return _replay(lambda *a: lib().bpsf_serve_replay(self.handle, *a), arrival_s, codes, synds)

    def stop(self):
        h, self.handle = self.handle, None
        if h:
            bpsf_serve_stop(h)

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def _trace_args(arrival_s, codes, synds):
    n = len(codes)
    arr = None if arrival_s is None else np.ascontiguousarray(arrival_s, dtype=np.float64)
    cd = np.ascontiguousarray(codes, dtype=np.int32)
    synds = [np.ascontiguousarray(x).view(np.uint32) for x in synds]
    ns = np.array([x.shape[0] for x in synds], dtype=np.int64)
    ptrs = (C.c_void_p * n)(*[x.ctypes.data for x in synds])
    return n, arr, cd, synds, ns, ptrs


def _replay(fn, arrival_s, codes, synds):
    n, arr, cd, synds, ns, ptrs = _trace_args(arrival_s, codes, synds)
    lat = np.zeros(n, dtype=np.float64)
    span = C.c_double(0.0)
    check(fn(n, None if arr is None else _np_ptr(arr), _np_ptr(cd), _np_ptr(ns), ptrs, _np_ptr(lat), C.byref(span)))
    return lat, span.value


def plain_replay(decoders, arrival_s, codes, synds):
    """bpsf_plain_replay: the plain per-shot form serving a trace (arrival_s None: closed
    loop); returns (per-request latency in s, span in s)."""
    hs = (C.c_void_p * len(decoders))(*[d.handle for d in decoders])
    return _replay(lambda *a: lib().bpsf_plain_replay(hs, len(decoders), *a), arrival_s, codes, synds)


def decode_multi_host(decoders, synds, stream=None):
    """End-to-end form of decode_multi: host (numpy) syndromes in, numpy outputs out, one launch."""
    synds = [np.ascontiguousarray(s) for s in synds]
    outs, jobs = [], []
    for d, s in zip(decoders, synds):
        n = int(s.shape[0])
        o = dict(corr=np.zeros((n, d.Wn), dtype=np.uint32), conv=np.zeros(n, dtype=np.uint8),
                 iters=np.zeros(n, dtype=np.int16), stage=np.zeros(n, dtype=np.uint8))
        outs.append(o)
        jobs.append(bpsf_job(d.handle, n, _np_ptr(s), int(s.shape[1]), _np_ptr(o["corr"]), d.Wn, _np_ptr(o["conv"]),
                             _np_ptr(o["iters"]), _np_ptr(o["stage"])))
    bpsf_decode_multi_host(jobs, _stream_handle(stream))
    return outs


def decode_multi(decoders, synds, outs=None, stream=None, sync=True):
    """One launch over several (decoder, syndromes) pairs of different codes."""
    outs = outs or [d.outputs(int(s.shape[0]), s.device) for d, s in zip(decoders, synds)]
    jobs = []
    for d, s, o in zip(decoders, synds, outs):
        jobs.append(bpsf_job(d.handle, int(s.shape[0]), _dptr(s), int(s.shape[1]), _dptr(o["corr"]),
                             int(o["corr"].shape[1]), _dptr(o["conv"]), _dptr(o["iters"]), _dptr(o["stage"])))
    sh = _stream_handle(stream)
    bpsf_decode_multi(jobs, sh)
    if sync:
        for d in decoders:
            bpsf_sync(d.handle, sh)
    return outs
