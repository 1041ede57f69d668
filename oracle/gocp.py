"""Greedy Operator Commutativity Partitioning (Sec. III.A, Algorithm 1).

The non-commutativity graph has one vertex per pool operator and an edge
(i, j) iff [A_i, A_j] != 0 as operators.  The commutator of two Pauli sums is
evaluated exactly: for strings s of A_i and t of A_j,

    P_s P_t - P_t P_s = ((-1)**(z_s.x_t) - (-1)**(z_t.x_s)) X^(x_s^x_t) Z^(z_s^z_t),

so the commutator is a sum over the product strings with integer weights once
every coefficient is scaled to an integer; it is zero iff every product
string's summed weight is zero.  Coefficients carry i**phase, so weights are
Gaussian integers (re, im).

Colouring: vertices sorted by descending degree (Largest-First; ties keep pool
order), each placed in the lowest-index family holding none of its
neighbours, a new family being opened when every existing one does.
"""

from __future__ import annotations

import numpy as np

from .pauli import PauliTable, parity

_SCALE = 8.0   # generator coefficients are multiples of 1/8


def _int_weights(t: PauliTable):
    c = t.coeff * _SCALE
    ci = np.rint(c).astype(np.int64)
    if not np.array_equal(ci.astype(np.float64), c):
        raise ValueError("coefficients are not multiples of 1/8")
    ph = t.phase % 4
    # c * i**phase as a Gaussian integer
    re = np.where(ph == 0, ci, np.where(ph == 2, -ci, 0))
    im = np.where(ph == 1, ci, np.where(ph == 3, -ci, 0))
    return re, im


def commutes(a: PauliTable, b: PauliTable) -> bool:
    """Exact test of [A, B] == 0."""
    ra, ia = _int_weights(a)
    rb, ib = _int_weights(b)
    xs, zs = a.x[:, None], a.z[:, None]
    xt, zt = b.x[None, :], b.z[None, :]
    d = (1 - 2 * parity(zs & xt)) - (1 - 2 * parity(zt & xs))      # in {-2, 0, 2}
    wr = (ra[:, None] * rb[None, :] - ia[:, None] * ib[None, :]) * d
    wi = (ra[:, None] * ib[None, :] + ia[:, None] * rb[None, :]) * d
    kx = (xs ^ xt).ravel()
    kz = (zs ^ zt).ravel()
    keys = kx * (1 << 32) + kz
    _, inv = np.unique(keys, return_inverse=True)
    sr = np.zeros(inv.max() + 1, dtype=np.int64)
    si = np.zeros_like(sr)
    np.add.at(sr, inv, wr.ravel())
    np.add.at(si, inv, wi.ravel())
    return not (np.any(sr != 0) or np.any(si != 0))


def conflict_graph(pool: list[PauliTable]) -> list[set]:
    """Adjacency sets of the non-commutativity graph."""
    m = len(pool)
    adj = [set() for _ in range(m)]
    for i in range(m):
        for j in range(i + 1, m):
            if not commutes(pool[i], pool[j]):
                adj[i].add(j)
                adj[j].add(i)
    return adj


def largest_first_colouring(adj: list[set]) -> np.ndarray:
    """Algorithm 1 on a given graph: family index of every vertex."""
    m = len(adj)
    order = sorted(range(m), key=lambda v: (-len(adj[v]), v))
    family = np.full(m, -1, dtype=np.int64)
    n_fam = 0
    for v in order:
        taken = {int(family[u]) for u in adj[v] if family[u] >= 0}
        k = 0
        while k < n_fam and k in taken:
            k += 1
        if k == n_fam:
            n_fam += 1
        family[v] = k
    return family


def gocp(pool: list[PauliTable]) -> np.ndarray:
    return largest_first_colouring(conflict_graph(pool))
