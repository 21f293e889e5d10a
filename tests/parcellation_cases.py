"""Connectivity rows whose fractions C[r][t] / sum_t C[r][t] lie at, or within
2^-55 relative of, the midpoint between two neighbouring binary32 values, with
the binary32 each rounds to (ties to even) known from the construction.

A midpoint in the binade [2^-k-1, 2^-k) is K 2^-s with K odd in
[2^24, 2^25) and s = k + 25; it lies between the binary32 values m 2^-(s-1)
and (m + 1) 2^-(s-1), m = (K - 1) / 2.  Taking b with K b = -1 (mod 2^s)
and a = (K b + 1) / 2^s gives a / b = K 2^-s + 1 / (b 2^s): just above the
midpoint, so the nearest is the upper value; K b = +1 (mod 2^s) and
a = (K b - 1) / 2^s lie just below it (the lower value); b = c 2^s and
a = K c hit it exactly (the even one of m and m + 1).  Rows hold a, and
b - a split into int32-sized entries, so b is their sum.
"""
from __future__ import annotations

import numpy as np

I32_MAX = 2 ** 31 - 1


def _split(rest: int) -> list:
    out = []
    while rest > 0:
        v = min(rest, I32_MAX)
        out.append(v)
        rest -= v
    return out


def midpoint_rows(seed: int, n_rows: int, k_max: int = 6):
    """(rows, want): rows a list of int lists (entries < 2^31, sums >= 2^25),
    want[i] = (column of a, the binary32 nearest to a / sum as np.float32)."""
    rng = np.random.default_rng(seed)
    rows, want = [], []
    for i in range(n_rows):
        k = int(rng.integers(0, k_max + 1))
        s = k + 25
        K = int(rng.integers(2 ** 23, 2 ** 24)) * 2 + 1          # odd, in [2^24, 2^25)
        m = (K - 1) // 2
        kind = i % 3
        if kind == 2:                                              # exactly on the midpoint
            c = int(rng.integers(1, 2 ** 31 // K + 1))
            b, a = c << s, K * c
            q = m if m % 2 == 0 else m + 1
        else:
            sign = -1 if kind == 0 else 1                          # K b = sign (mod 2^s)
            b0 = (sign * pow(K, -1, 2 ** s)) % (2 ** s)
            j_max = max(1, (I32_MAX * 2 ** s // K - b0) >> s)      # keep a below 2^31
            b = b0 + (int(rng.integers(1, min(j_max, 63) + 1)) << s)
            a = (K * b - sign) >> s
            assert a * 2 ** s == K * b - sign and a <= I32_MAX
            q = m + 1 if kind == 0 else m
        row = [a] + _split(b - a)
        pos = int(rng.integers(0, len(row)))
        row[0], row[pos] = row[pos], row[0]
        rows.append(row)
        want.append((pos, np.float32(np.ldexp(np.float64(q), -(s - 1)))))
    return rows, want


def as_matrix(rows, M: int) -> np.ndarray:
    """Rows padded with zeros to M entries, int64 [len(rows), M]."""
    C = np.zeros((len(rows), M), dtype=np.int64)
    for i, r in enumerate(rows):
        assert len(r) <= M
        C[i, :len(r)] = r
    return C


# Rows whose binary64 quotient, rounded again to binary32, is one unit off
# the nearest binary32 (found by exact rational search).
DOUBLE_ROUNDING_ROWS = [[540202477, 118111586], [383832729, 335299414], [687800308, 624435623]]
