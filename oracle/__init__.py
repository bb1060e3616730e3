"""BP-SF oracle (CPU, plain C in FP64 and canonical-FP32 modes).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg use it to check and time the CUDA decoder.  The
decoder package never imports it, and it imports nothing from the decoder.

Each function cites the part of "Fully Parallelized BP Decoding for Quantum
LDPC Codes Can Outperform BP-OSD" (arXiv 2507.00254) it follows; the C source
``bpsf_oracle.c`` lists how points the paper leaves open are read.  Every
function here is pinned by a ``-m "not gpu"`` test against something other
than itself (worked example, closed forms, brute force, code parameters);
none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "bpsf_oracle.c"), os.path.join(_HERE, "bp_body.inc")]

_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-o", _LIB_PATH + ".tmp", _SRC[0], "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        vp = C.c_void_p
        L.oracle_shift_matrix.argtypes = [C.c_int, _u8p]
        L.oracle_bb_code.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _i32p, _i32p, _u8p, _u8p]
        L.oracle_phenom_code.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _u8p]
        L.oracle_gf2_rank.argtypes = [_u8p, C.c_int, C.c_int]
        L.oracle_gf2_rank.restype = C.c_int
        L.oracle_logicals.argtypes = [_u8p, C.c_int, _u8p, C.c_int, C.c_int, _u8p, C.c_int]
        L.oracle_logicals.restype = C.c_int
        L.oracle_code_new.argtypes = [_u8p, C.c_int, C.c_int]
        L.oracle_code_new.restype = vp
        L.oracle_code_free.argtypes = [vp]
        L.oracle_code_nnz.argtypes = [vp]
        L.oracle_code_set_layered.argtypes = [vp, C.c_int]
        L.oracle_code_layer.argtypes = [vp, C.c_int]
        L.oracle_code_layer.restype = C.c_int
        L.oracle_code_nnz.restype = C.c_int
        L.oracle_syndrome.argtypes = [vp, _u8p, _u8p]
        L.oracle_llr_f64.argtypes = [_f64p, C.c_int, _f64p]
        L.oracle_llr_f32.argtypes = [_f64p, C.c_int, _f32p]
        L.oracle_top.argtypes = [_u16p, C.c_int, C.c_int, _i32p]
        for sfx, rp, rt in (("f64", _f64p, C.c_double), ("f32", _f32p, C.c_float)):
            fn = getattr(L, "oracle_bp_" + sfx)
            fn.argtypes = [vp, rp, _u8p, C.c_int, rt, C.c_int, _u8p, vp, vp, C.POINTER(C.c_int)]
            fn.restype = C.c_int
            fn = getattr(L, "oracle_trials_" + sfx)
            fn.argtypes = [vp, rp, _u8p, _i32p, C.c_int, C.c_int, vp, C.c_int, C.c_int, rt, vp, vp, vp, vp]
            fn.restype = C.c_int
            fn = getattr(L, "oracle_bpsf_" + sfx)
            fn.argtypes = [vp, rp, _u8p, C.c_int, rt, C.c_int, C.c_int, vp, C.c_int, C.c_int, C.c_int, _u8p,
                           C.POINTER(C.c_int), C.POINTER(C.c_int), vp, vp]
            fn.restype = C.c_int
            fn = getattr(L, "oracle_bpsf_batch_" + sfx)
            fn.argtypes = [vp, rp, C.c_int64, _u8p, C.c_int, rt, C.c_int, C.c_int, vp, C.c_int, C.c_int, C.c_int,
                           _u8p, _u8p, _i32p, _u8p, C.c_int, vp]
        L.oracle_bp_sumproduct.argtypes = [vp, _f64p, _u8p, C.c_int, _f64p]
        L.oracle_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# Code construction (Appendix "Code Construction")
# --------------------------------------------------------------------------

def shift_matrix(l: int) -> np.ndarray:
    """S_l = I_l >> 1 (Appendix, GB codes)."""
    out = np.zeros((l, l), dtype=np.uint8)
    lib().oracle_shift_matrix(l, out)
    return out


def bb_code(l: int, m: int, a_terms, b_terms):
    """(H_X, H_Z) of the BB code with A = a(x, y), B = b(x, y) (Appendix, BB codes).

    Terms are (i, j) for the monomial x^i y^j; H_X = [A|B], H_Z = [B^T|A^T].
    """
    ax = np.array([t[0] for t in a_terms], dtype=np.int32)
    ay = np.array([t[1] for t in a_terms], dtype=np.int32)
    bx = np.array([t[0] for t in b_terms], dtype=np.int32)
    by = np.array([t[1] for t in b_terms], dtype=np.int32)
    n = l * m
    hx = np.zeros((n, 2 * n), dtype=np.uint8)
    hz = np.zeros((n, 2 * n), dtype=np.uint8)
    lib().oracle_bb_code(l, m, len(ax), ax, ay, len(bx), bx, by, hx, hz)
    return hx, hz


def phenom_code(h0: np.ndarray, rounds: int) -> np.ndarray:
    """R-round phenomenological detector matrix [I_R (x) H0 | B_R (x) I_m0]."""
    h0 = np.ascontiguousarray(h0, dtype=np.uint8)
    m0, n0 = h0.shape
    out = np.zeros((rounds * m0, rounds * n0 + rounds * m0), dtype=np.uint8)
    lib().oracle_phenom_code(h0, m0, n0, rounds, out)
    return out


def gf2_rank(a: np.ndarray) -> int:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return int(lib().oracle_gf2_rank(a, a.shape[0], a.shape[1]))


def logicals(hx: np.ndarray, hz: np.ndarray) -> np.ndarray:
    """L_X: basis of ker(H_Z) modulo rowspace(H_X) (Eq. MLD_quantum, degeneracy)."""
    hx = np.ascontiguousarray(hx, dtype=np.uint8)
    hz = np.ascontiguousarray(hz, dtype=np.uint8)
    n = hx.shape[1]
    lx = np.zeros((n, n), dtype=np.uint8)
    k = lib().oracle_logicals(hx, hx.shape[0], hz, hz.shape[0], n, lx, n)
    return lx[:k].copy()


# Named workloads (Appendix Table bbcodes, plus the two extra BB codes of the
# mixed-size batch).  Terms are (power of x, power of y).
BB_CODES = {
    "bb72": (6, 6, [(3, 0), (0, 1), (0, 2)], [(0, 3), (1, 0), (2, 0)]),
    "bb90": (15, 3, [(9, 0), (0, 1), (0, 2)], [(0, 0), (2, 0), (7, 0)]),
    "bb108": (9, 6, [(3, 0), (0, 1), (0, 2)], [(0, 3), (1, 0), (2, 0)]),
    "bb144": (12, 6, [(3, 0), (0, 1), (0, 2)], [(0, 3), (1, 0), (2, 0)]),
    "bb288": (12, 12, [(3, 0), (0, 2), (0, 7)], [(0, 3), (1, 0), (2, 0)]),
    # Appendix "GB codes": [[254,28]], l = 127, m = 1 (polynomials in x only).
    "gb254": (127, 1, [(0, 0), (15, 0), (20, 0), (28, 0), (66, 0)], [(0, 0), (58, 0), (59, 0), (100, 0), (121, 0)]),
    # Appendix "Coprime-BB codes" (Table cbbcodes): polynomials in pi = x y.
    "cbb126": (7, 9, [(0, 0), (1, 1), (58, 58)], [(0, 0), (13, 13), (41, 41)]),
    "cbb154": (7, 11, [(0, 0), (1, 1), (31, 31)], [(0, 0), (19, 19), (53, 53)]),
}


def named_code(name: str):
    l, m, a, b = BB_CODES[name]
    return bb_code(l, m, a, b)


# --------------------------------------------------------------------------
# Decoder (Section II-B and Algorithm 1)
# --------------------------------------------------------------------------

@dataclass
class Params:
    max_iter: int = 50
    alpha: float = 0.625
    w: int = 4
    w_max: int = 0          # 0 -> w
    short_iter: int = 10
    select: int = 0         # 0 min weight, 1 earliest converged trial of the list
    trials: tuple = ()      # explicit trial list (subset masks over Phi); () -> weight <= w_max
    layered: bool = False   # layered schedule (rows by greedy layer) instead of flooding


class Code:
    """Tanner graph of a dense H (Section II-B) plus the oracle decoder on it."""

    def __init__(self, H: np.ndarray):
        self.H = np.ascontiguousarray(H, dtype=np.uint8)
        self.M, self.N = self.H.shape
        self._h = lib().oracle_code_new(self.H, self.M, self.N)
        self.nnz = int(lib().oracle_code_nnz(self._h))

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.oracle_code_free(h)

    # s = H e (mod 2) (Section II-B, e H^T = s): the dense GF(2) mat-vec of the C
    # oracle, one shot at a time.
    def syndrome_matvec(self, e: np.ndarray) -> np.ndarray:
        e = np.ascontiguousarray(np.atleast_2d(e), dtype=np.uint8)
        out = np.zeros((e.shape[0], self.M), dtype=np.uint8)
        for k in range(e.shape[0]):
            row = np.ascontiguousarray(e[k])
            tmp = np.zeros(self.M, dtype=np.uint8)
            lib().oracle_syndrome(self._h, row, tmp)
            out[k] = tmp
        return out

    # The same s = H e (mod 2) for a batch, as one library matrix product: the
    # integer counts (at most the row weight) are exact in float32, and their
    # parity is the syndrome bit.
    def syndrome(self, e: np.ndarray) -> np.ndarray:
        e = np.atleast_2d(np.asarray(e))
        if e.shape[0] <= 8:
            return self.syndrome_matvec(e)
        if not hasattr(self, "_hT32"):
            self._hT32 = np.ascontiguousarray(self.H.T, dtype=np.float32)
        cnt = e.astype(np.float32) @ self._hT32
        return (cnt.astype(np.int64) & 1).astype(np.uint8)

    @staticmethod
    def llr(priors, fp32: bool):
        p = np.ascontiguousarray(priors, dtype=np.float64)
        if fp32:
            out = np.zeros(p.shape[0], dtype=np.float32)
            lib().oracle_llr_f32(p, p.shape[0], out)
        else:
            out = np.zeros(p.shape[0], dtype=np.float64)
            lib().oracle_llr_f64(p, p.shape[0], out)
        return out

    def _lch(self, priors, fp32):
        pri = np.broadcast_to(np.asarray(priors, dtype=np.float64), (self.N,))
        return self.llr(np.ascontiguousarray(pri), fp32)

    def schedule(self, layered: bool):
        """Select the flooding (default) or the layered schedule for the runs that follow."""
        lib().oracle_code_set_layered(self._h, int(bool(layered)))

    def layers(self):
        """Layer of every row under the layered schedule."""
        self.schedule(True)
        return np.array([lib().oracle_code_layer(self._h, j) for j in range(self.M)], dtype=np.int64)

    def bp(self, s, priors, max_iter, alpha, fp32=True, stop_on_converge=True, track=False, layered=False):
        """One min-sum BP run; returns dict(e, converged, iters, lout, flips)."""
        self.schedule(layered)
        lch = self._lch(priors, fp32)
        s = np.ascontiguousarray(s, dtype=np.uint8)
        e = np.zeros(self.N, dtype=np.uint8)
        lout = np.zeros(self.N, dtype=np.float32 if fp32 else np.float64)
        flips = np.zeros(self.N, dtype=np.uint16) if track else None
        it = C.c_int(0)
        fn = lib().oracle_bp_f32 if fp32 else lib().oracle_bp_f64
        alpha_t = np.float32(alpha) if fp32 else float(alpha)
        conv = fn(self._h, lch, s, int(max_iter), alpha_t, int(stop_on_converge), e, _ptr(flips), _ptr(lout),
                  C.byref(it))
        return dict(e=e, converged=bool(conv), iters=it.value, lout=lout, flips=flips)

    def trials(self, s, priors, phi, params: Params, fp32=True):
        """Every trial of one failed shot: (s', converged, iters, e' xor t), in list order."""
        self.schedule(params.layered)
        lch = self._lch(priors, fp32)
        w = len(phi)
        wm = w if params.w_max <= 0 or params.w_max > w else params.w_max
        masks, nm = _masks(params)
        cap = max(1, nm if nm else sum(1 for m in range(1, 1 << w) if bin(m).count("1") <= wm))
        synd = np.zeros((cap, self.M), dtype=np.uint8)
        conv = np.zeros(cap, dtype=np.uint8)
        iters = np.zeros(cap, dtype=np.int32)
        es = np.zeros((cap, self.N), dtype=np.uint8)
        fn = lib().oracle_trials_f32 if fp32 else lib().oracle_trials_f64
        alpha_t = np.float32(params.alpha) if fp32 else float(params.alpha)
        n = fn(self._h, lch, np.ascontiguousarray(s, dtype=np.uint8), np.asarray(phi, dtype=np.int32), w, wm,
               _ptr(masks), nm, params.short_iter, alpha_t, _ptr(synd), _ptr(conv), _ptr(iters), _ptr(es))
        return synd[:n], conv[:n].astype(bool), iters[:n], es[:n]

    def bpsf(self, s, priors, params: Params, fp32=True):
        """BP-SF of one syndrome (Algorithm 1); dict(e, converged, iters, stage, phi, flips)."""
        self.schedule(params.layered)
        lch = self._lch(priors, fp32)
        e = np.zeros(self.N, dtype=np.uint8)
        it, st = C.c_int(0), C.c_int(0)
        phi = np.full(max(params.w, 1), -1, dtype=np.int32)
        flips = np.zeros(self.N, dtype=np.uint16)
        fn = lib().oracle_bpsf_f32 if fp32 else lib().oracle_bpsf_f64
        alpha_t = np.float32(params.alpha) if fp32 else float(params.alpha)
        masks, nm = _masks(params)
        conv = fn(self._h, lch, np.ascontiguousarray(s, dtype=np.uint8), params.max_iter, alpha_t, params.w,
                  params.w_max, _ptr(masks), nm, params.short_iter, params.select, e, C.byref(it), C.byref(st),
                  _ptr(phi), _ptr(flips))
        return dict(e=e, converged=bool(conv), iters=it.value, stage=st.value,
                    phi=phi[: params.w] if params.w > 0 else phi[:0], flips=flips)

    def bpsf_batch(self, synd, priors, params: Params, fp32=True, threads=1, shot_s=None):
        """BP-SF over a batch of syndromes (n, M) -> (e (n, N), converged, iters, stage).
        shot_s: optional float64 array of n, filled with each shot's wall time in seconds."""
        synd = np.ascontiguousarray(synd, dtype=np.uint8)
        n = synd.shape[0]
        self.schedule(params.layered)
        lch = self._lch(priors, fp32)
        e = np.zeros((n, self.N), dtype=np.uint8)
        conv = np.zeros(n, dtype=np.uint8)
        iters = np.zeros(n, dtype=np.int32)
        stage = np.zeros(n, dtype=np.uint8)
        fn = lib().oracle_bpsf_batch_f32 if fp32 else lib().oracle_bpsf_batch_f64
        alpha_t = np.float32(params.alpha) if fp32 else float(params.alpha)
        masks, nm = _masks(params)
        if shot_s is not None:
            assert shot_s.dtype == np.float64 and shot_s.shape == (n,) and shot_s.flags["C_CONTIGUOUS"]
        fn(self._h, lch, n, synd, params.max_iter, alpha_t, params.w, params.w_max, _ptr(masks), nm,
           params.short_iter, params.select, e, conv, iters, stage, int(threads), _ptr(shot_s))
        return e, conv.astype(bool), iters, stage

    def sumproduct(self, s, priors, iters):
        """Sum-product BP (FP64) for a fixed number of iterations; posterior LLRs."""
        lch = self._lch(priors, False)
        out = np.zeros(self.N, dtype=np.float64)
        lib().oracle_bp_sumproduct(self._h, lch, np.ascontiguousarray(s, dtype=np.uint8), int(iters), out)
        return out


def _masks(params: Params):
    """The explicit trial list of params as a uint64 array (None and 0 if default)."""
    if not params.trials:
        return None, 0
    m = np.ascontiguousarray(np.asarray(params.trials, dtype=np.uint64))
    return m, int(m.shape[0])


def top(flips: np.ndarray, w: int) -> np.ndarray:
    """Phi = top(flip_count, w) (Algorithm 1)."""
    f = np.ascontiguousarray(flips, dtype=np.uint16)
    out = np.zeros(w, dtype=np.int32)
    lib().oracle_top(f, f.shape[0], w, out)
    return out


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def logical_failures(H, lx, e, e_hat, converged, fold=None):
    """Harness check (Eq. MLD_quantum): a shot fails iff it did not converge, or the
    residual r = fold(e xor e_hat) has H r != 0 or L_X r != 0.  ``fold`` maps the
    phenomenological columns to the data qubits (XOR over rounds); None = identity.
    Dense integer arithmetic, written out per shot."""
    r = (np.asarray(e, dtype=np.uint8) ^ np.asarray(e_hat, dtype=np.uint8))
    if fold is not None:
        r = fold(r)
    hs = (r.astype(np.int64) @ np.asarray(H, dtype=np.int64).T) % 2
    ls = (r.astype(np.int64) @ np.asarray(lx, dtype=np.int64).T) % 2
    return (~np.asarray(converged, dtype=bool)) | hs.any(axis=1) | ls.any(axis=1)


def phenom_fold(n_data: int, rounds: int):
    """Residual on the data qubits: XOR of the data blocks of all rounds."""
    def f(r):
        r = np.asarray(r, dtype=np.uint8)
        out = np.zeros((r.shape[0], n_data), dtype=np.uint8)
        for t in range(rounds):
            out ^= r[:, t * n_data:(t + 1) * n_data]
        return out
    return f
