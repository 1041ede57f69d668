"""Pauli strings in X^x Z^z form and exact per-string accumulation.

A string X^x Z^z (Z applied first) maps |b> -> (-1)**popc(b & z) |b ^ x>.
Product rule: (X^x1 Z^z1)(X^x2 Z^z2) = (-1)**popc(z1 & x2) X^(x1^x2) Z^(z1^z2),
because moving Z^z1 through X^x2 picks one sign per shared qubit.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


def popcount(a: np.ndarray) -> np.ndarray:
    """Bit count of a non-negative integer array."""
    a = np.asarray(a, dtype=np.uint64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    out = np.zeros(a.shape, dtype=np.int64)
    v = a.copy()
    while np.any(v):
        out += (v & np.uint64(1)).astype(np.int64)
        v >>= np.uint64(1)
    return out


def parity(a: np.ndarray) -> np.ndarray:
    return popcount(a) & 1


@dataclasses.dataclass
class PauliTable:
    """A Pauli sum  sum_t coeff[t] * i**phase[t] * X^x[t] Z^z[t]  on n qubits."""

    n: int
    x: np.ndarray       # int64 masks
    z: np.ndarray       # int64 masks
    phase: np.ndarray   # int64 in 0..3
    coeff: np.ndarray   # float64

    def __len__(self) -> int:
        return int(self.x.shape[0])

    def weights(self) -> np.ndarray:
        """Complex coefficient c * i**phase of each term."""
        return self.coeff * (1j ** self.phase)


def accumulate_exact(x: np.ndarray, z: np.ndarray, val: np.ndarray, n: int,
                     term_drop: float = 0.0) -> PauliTable:
    """Sum real contributions per (x, z) exactly, then round once.

    Every contribution handed in here is an integral times a power of two, so
    it is exact; ``math.fsum`` returns the correctly rounded value of the exact
    sum, which makes the table independent of accumulation order.  Exact
    zeros are dropped, then terms with |c| < term_drop.  Output is sorted by
    (x, z) ascending with phase 0 (all coefficients of a real operator are
    real in X^x Z^z form).
    """
    x = np.asarray(x, dtype=np.int64)
    z = np.asarray(z, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    if x.size == 0:
        e = np.zeros(0, dtype=np.int64)
        return PauliTable(n, e, e.copy(), e.copy(), np.zeros(0))
    order = np.lexsort((z, x))
    xs, zs, vs = x[order], z[order], val[order]
    brk = np.flatnonzero((np.diff(xs) != 0) | (np.diff(zs) != 0)) + 1
    starts = np.concatenate(([0], brk))
    ends = np.concatenate((brk, [xs.size]))
    ox, oz, oc = [], [], []
    for s, e in zip(starts, ends):
        c = math.fsum(vs[s:e].tolist())
        if c == 0.0 or abs(c) < term_drop:
            continue
        ox.append(int(xs[s]))
        oz.append(int(zs[s]))
        oc.append(c)
    ox = np.array(ox, dtype=np.int64)
    return PauliTable(n, ox, np.array(oz, dtype=np.int64),
                      np.zeros(ox.shape, dtype=np.int64), np.array(oc, dtype=np.float64))


def string_product(xa, za, xb, zb):
    """(X^xa Z^za)(X^xb Z^zb) -> (sign, x, z), elementwise over arrays."""
    sign = 1 - 2 * parity(np.asarray(za, dtype=np.int64) & np.asarray(xb, dtype=np.int64))
    return sign, np.bitwise_xor(xa, xb), np.bitwise_xor(za, zb)


def label(x: int, z: int, n: int) -> str:
    """Qubit-0-first I/X/Y/Z label of X^x Z^z, ignoring the i's that Y = iXZ carries."""
    out = []
    for j in range(n):
        xb, zb = (x >> j) & 1, (z >> j) & 1
        out.append("IZXY"[xb * 2 + zb])
    return "".join(out)
