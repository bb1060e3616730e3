"""Evaluation harness: bit packing, X logicals and logical-failure counting.

A decoded shot fails when it did not converge or when the residual
r = e xor e_hat (folded over rounds for the phenomenological model) is not
a stabiliser: H_X r != 0 or L_X r != 0, with L_X a basis of ker(H_Z) modulo
rowspace(H_X) (Section II-A, degeneracy).  Host-side numpy; not on the
decoding path.
"""
from __future__ import annotations

import numpy as np


def pack_rows(bits: np.ndarray) -> np.ndarray:
    """(n, nb) 0/1 -> (n, ceil(nb/32)) uint32, least significant bit first."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    n, nb = bits.shape
    w = (nb + 31) // 32
    pad = np.zeros((n, 32 * w), dtype=np.uint8)
    pad[:, :nb] = bits
    b = np.packbits(pad.reshape(n, w, 4, 8), axis=-1, bitorder="little").reshape(n, w, 4)
    return b.view(np.uint32).reshape(n, w)


def unpack_rows(words: np.ndarray, nb: int) -> np.ndarray:
    words = np.ascontiguousarray(words).view(np.uint32)
    n, w = words.shape
    b = np.unpackbits(words.view(np.uint8).reshape(n, w * 4), axis=-1, bitorder="little")
    return b[:, :nb]


def _rref(a: np.ndarray):
    a = (np.asarray(a, dtype=np.uint8) & 1).copy()
    rows, cols = a.shape
    piv, r = [], 0
    for c in range(cols):
        if r == rows:
            break
        nz = np.nonzero(a[r:, c])[0]
        if nz.size == 0:
            continue
        p = r + nz[0]
        a[[r, p]] = a[[p, r]]
        hit = np.nonzero(a[:, c])[0]
        hit = hit[hit != r]
        a[hit] ^= a[r]
        piv.append(c)
        r += 1
    return a[:r], piv


def gf2_rank(a) -> int:
    return len(_rref(a)[1])


def x_logicals(hx: np.ndarray, hz: np.ndarray) -> np.ndarray:
    """Basis of ker(H_Z) modulo rowspace(H_X)."""
    R, piv = _rref(hz)
    n = hz.shape[1]
    free = [c for c in range(n) if c not in set(piv)]
    base_rank = gf2_rank(hx)
    stack = np.array(hx, dtype=np.uint8)
    out = []
    for f in free:
        v = np.zeros(n, dtype=np.uint8)
        v[f] = 1
        for i, pc in enumerate(piv):
            v[pc] = R[i, f]
        cand = np.vstack([stack, v])
        rk = gf2_rank(cand)
        if rk > base_rank:
            stack, base_rank = cand, rk
            out.append(v)
    return np.array(out, dtype=np.uint8)


def failures(hx: np.ndarray, lx: np.ndarray, err_bits: np.ndarray, corr_bits: np.ndarray, converged: np.ndarray,
             n_data: int = 0, rounds: int = 1) -> np.ndarray:
    r = (np.asarray(err_bits, dtype=np.uint8) ^ np.asarray(corr_bits, dtype=np.uint8))
    if rounds > 1:
        folded = np.zeros((r.shape[0], n_data), dtype=np.uint8)
        for t in range(rounds):
            folded ^= r[:, t * n_data:(t + 1) * n_data]
        r = folded
    hs = (r.astype(np.int32) @ hx.T.astype(np.int32)) & 1
    ls = (r.astype(np.int32) @ lx.T.astype(np.int32)) & 1
    return (~np.asarray(converged, dtype=bool)) | hs.any(axis=1) | ls.any(axis=1)
