"""Codes the decoder is exercised on, built through libbpsf's own builders.

Bivariate bicycle codes (Appendix "Code Construction", Table bbcodes), the
two extra BB codes of the mixed-size batch, the [[254,28]] generalised
bicycle code (Appendix "GB codes": m = 1, polynomials in x) and the
coprime-BB codes [[126,12,10]] and [[154,6,16]] (Appendix "Coprime-BB
codes": polynomials in pi = x y, so pi^e is the term (e, e)), and the
12-round phenomenological detector matrix of the [[144,12,12]] code.  Terms
are (power of x, power of y).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import bpsf as _b

BB = {
    "bb72": (6, 6, ((3, 0), (0, 1), (0, 2)), ((0, 3), (1, 0), (2, 0))),
    "bb90": (15, 3, ((9, 0), (0, 1), (0, 2)), ((0, 0), (2, 0), (7, 0))),
    "bb108": (9, 6, ((3, 0), (0, 1), (0, 2)), ((0, 3), (1, 0), (2, 0))),
    "bb144": (12, 6, ((3, 0), (0, 1), (0, 2)), ((0, 3), (1, 0), (2, 0))),
    "bb288": (12, 12, ((3, 0), (0, 2), (0, 7)), ((0, 3), (1, 0), (2, 0))),
    "gb254": (127, 1, ((0, 0), (15, 0), (20, 0), (28, 0), (66, 0)), ((0, 0), (58, 0), (59, 0), (100, 0), (121, 0))),
    "cbb126": (7, 9, ((0, 0), (1, 1), (58, 58)), ((0, 0), (13, 13), (41, 41))),
    "cbb154": (7, 11, ((0, 0), (1, 1), (31, 31)), ((0, 0), (19, 19), (53, 53))),
}

PHENOM_ROUNDS = 12


@dataclass
class CodeCSR:
    name: str
    M: int
    N: int
    ptr: np.ndarray
    idx: np.ndarray
    n_data: int = 0      # data qubits (phenomenological: per round)
    rounds: int = 1

    def dense(self) -> np.ndarray:
        H = np.zeros((self.M, self.N), dtype=np.uint8)
        for j in range(self.M):
            H[j, self.idx[self.ptr[j]:self.ptr[j + 1]]] = 1
        return H


def bb(name: str, which: int = 0) -> CodeCSR:
    l, m, a, b = BB[name]
    ptr, idx = _b.bpsf_bb_code(l, m, a, b, which)
    n = l * m
    return CodeCSR(name, n, 2 * n, ptr, idx, n_data=2 * n)


def phenom(name: str = "bb144", rounds: int = PHENOM_ROUNDS) -> CodeCSR:
    h0 = bb(name)
    ptr, idx = _b.bpsf_phenom_code(h0.M, h0.N, h0.ptr, h0.idx, rounds)
    return CodeCSR(name + "_phenom%d" % rounds, rounds * h0.M, rounds * h0.N + rounds * h0.M, ptr, idx,
                   n_data=h0.N, rounds=rounds)
