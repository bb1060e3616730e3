"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random inputs: error vectors, shot counts and arrival
times.  It holds none of the decoder's arithmetic (no check matrix, no
syndrome, no message update), so both the CPU oracle and the CUDA path can
consume its output without sharing any code with each other.

Generator: a counter-based form of SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014; the 64-bit
finaliser constants are the ones published with Vigna's ``splitmix64.c``).
Draw number ``c`` of a stream with key ``k`` is ``mix64(k + (c + 1) * GAMMA)``
in wrapping uint64 arithmetic, so any shot range can be regenerated on its
own (no state to checkpoint).  A Bernoulli(p) draw is ``(u >> 11) < P`` with
``P = round(p * 2**53)``.

Column convention for the 12-round phenomenological model (used by both
builders): columns ``[t*n, (t+1)*n)`` hold the data errors of round ``t``
(``t = 0..R-1``), then columns ``R*n + [t*m0, (t+1)*m0)`` hold the
measurement errors of round ``t``.  The sampler draws no measurement error in
the last round (the final round is perfect).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30, _S27, _S31 = np.uint64(30), np.uint64(27), np.uint64(31)

# Fixed seeds per workload (one stream per physical error rate).
SEEDS = {
    "bb72_cc": 1001,
    "bb144_cc": (2001, 2002, 2003, 2004),
    "bb144_phenom": (3001, 3002),
    "mixed_counts": 4000,
    "mixed": (4001, 4002, 4003, 4004, 4005),
    "serve": 5001,
    "families": (6001, 6002, 6003),
}


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _S30)) * _M1
        z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def stream_key(seed: int, stream: int = 0) -> np.uint64:
    """Key of one independent stream, derived from (seed, stream)."""
    with np.errstate(over="ignore"):
        a = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(1))
        b = mix64(np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(2))
        return np.uint64(a ^ (b * np.uint64(3)))


def draws(key: np.uint64, ctr: np.ndarray) -> np.ndarray:
    """Raw 64-bit draws for counters ``ctr`` of the stream ``key``."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + (ctr + np.uint64(1)) * GAMMA)


def threshold53(p: float) -> np.uint64:
    """Integer threshold so that Bernoulli(p) is ``(u >> 11) < threshold``."""
    if not (0.0 <= p <= 1.0):
        raise ValueError("p must lie in [0, 1]")
    return np.uint64(int(round(p * float(1 << 53))))


def bernoulli_bits(seed: int, stream: int, shot0: int, n_shots: int, n_bits: int,
                   p, chunk_shots: int = 1 << 16) -> np.ndarray:
    """i.i.d. Bernoulli error bits, shape (n_shots, n_bits), dtype uint8.

    Bit ``i`` of shot ``s`` uses counter ``s * n_bits + i`` of the stream, so
    shots ``[shot0, shot0 + n_shots)`` do not depend on any other shot.
    ``p`` is a scalar or a length-``n_bits`` array of per-bit rates.
    """
    key = stream_key(seed, stream)
    p_arr = np.broadcast_to(np.asarray(p, dtype=np.float64), (n_bits,))
    thr = np.array([threshold53(float(x)) for x in p_arr], dtype=np.uint64)
    out = np.empty((n_shots, n_bits), dtype=np.uint8)
    cols = np.arange(n_bits, dtype=np.uint64)
    for a in range(0, n_shots, chunk_shots):
        b = min(n_shots, a + chunk_shots)
        shots = np.arange(shot0 + a, shot0 + b, dtype=np.uint64)
        ctr = shots[:, None] * np.uint64(n_bits) + cols[None, :]
        u = draws(key, ctr) >> np.uint64(11)
        out[a:b] = (u < thr[None, :]).astype(np.uint8)
    return out


def phenom_error_bits(seed: int, stream: int, shot0: int, n_shots: int, n: int, m0: int,
                      rounds: int, p: float, q: float) -> np.ndarray:
    """Errors of the R-round phenomenological model in the column convention above.

    Data errors at rate ``p`` in every round, measurement errors at rate
    ``q`` in rounds ``0..R-2``, none in the last (perfect) round.
    """
    n_cols = rounds * n + rounds * m0
    rates = np.empty(n_cols, dtype=np.float64)
    rates[: rounds * n] = p
    rates[rounds * n:] = q
    rates[rounds * n + (rounds - 1) * m0:] = 0.0
    return bernoulli_bits(seed, stream, shot0, n_shots, n_cols, rates)


def uniform_ints(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """``count`` integers uniform on [lo, hi] (inclusive), by rejection-free scaling."""
    key = stream_key(seed, stream)
    u = draws(key, np.arange(count, dtype=np.uint64)) >> np.uint64(11)
    span = hi - lo + 1
    return lo + ((u.astype(np.float64) / float(1 << 53)) * span).astype(np.int64)


def poisson_arrivals(seed: int, stream: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds, ascending) of a Poisson process of the given rate."""
    key = stream_key(seed, stream)
    u = (draws(key, np.arange(count, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64)
    u = (u + 0.5) / float(1 << 53)
    return np.cumsum(-np.log(u) / rate_per_s)


def uniform_choice(seed: int, stream: int, count: int, n_choices: int,
                   weights=None) -> np.ndarray:
    """``count`` indices in [0, n_choices) drawn with the given weights."""
    key = stream_key(seed, stream)
    u = (draws(key, np.arange(count, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64)
    u = u / float(1 << 53)
    w = np.ones(n_choices) if weights is None else np.asarray(weights, dtype=np.float64)
    cdf = np.cumsum(w) / np.sum(w)
    return np.minimum(np.searchsorted(cdf, u, side="right"), n_choices - 1)


def sample_trial_masks(seed: int, w: int, w_max: int, n_s: int) -> np.ndarray:
    """Sampled trial set of BP-SF: for each weight k = 1..w_max, n_s distinct
    k-subsets of the w oscillating bits (partial Fisher-Yates: position r
    takes index r + (u mod (w - r)) of a counter-based draw u; a duplicate
    subset is drawn again).  Returned as subset masks
    over Phi (bit j selects Phi[j]), weight by weight, in draw order; a weight
    with fewer than n_s subsets contributes all of them in ascending order."""
    if not (1 <= w <= 64 and 1 <= w_max <= w and n_s >= 1):
        raise ValueError("need 1 <= w_max <= w <= 64 and n_s >= 1")
    from itertools import combinations
    from math import comb
    out = []
    for k in range(1, w_max + 1):
        if comb(w, k) <= n_s:
            out.extend(sorted(sum(1 << b for b in c) for c in combinations(range(w), k)))
            continue
        key = stream_key(seed, k)
        seen, ctr = set(), 0
        while len(seen) < n_s:
            u = draws(key, np.arange(ctr, ctr + k, dtype=np.uint64))
            ctr += k
            idx = list(range(w))
            for r in range(k):  # partial Fisher-Yates: position r takes a uniform pick of the rest
                j = r + int(u[r] % np.uint64(w - r))
                idx[r], idx[j] = idx[j], idx[r]
            m = 0
            for b in idx[:k]:
                m |= 1 << b
            if m not in seen:
                seen.add(m)
                out.append(m)
    return np.array(out, dtype=np.uint64)
