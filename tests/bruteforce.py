"""Brute-force constructions that pin the oracle to definitions other than its own.

Nothing here uses the X^x Z^z bit formulas of the oracle:
  * ladder operators come from their action on occupation-number states,
    a_j |m> = (-1)**(sum_{k<j} m_k) m_j |m - e_j>, as sparse matrices;
  * Pauli strings are Kronecker products of the 2x2 matrices I, X, Y, Z;
  * the Bravyi-Kitaev matrix comes from the recursive Seeley-Richard-Love
    block construction, not from the Fenwick-tree rule.
Sizes are kept to n <= 10 qubits.
"""

from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


@functools.lru_cache(maxsize=None)
def ladder(n: int, j: int) -> sp.csr_matrix:
    """Annihilation operator of mode j on n modes (basis index bit k = n_k)."""
    dim = 1 << n
    rows, cols, vals = [], [], []
    for m in range(dim):
        if (m >> j) & 1:
            below = bin(m & ((1 << j) - 1)).count("1")
            rows.append(m ^ (1 << j))
            cols.append(m)
            vals.append((-1.0) ** below)
    return sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(dim, dim))


def create(n: int, j: int) -> sp.csr_matrix:
    return ladder(n, j).conj().T.tocsr()


def hamiltonian_dense(ints, int_drop: float = 0.0) -> np.ndarray:
    """E0 + sum h_pq a+ a + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs from matrices."""
    h = np.where(np.abs(ints.h) < int_drop, 0.0, ints.h)
    g = np.where(np.abs(ints.g) < int_drop, 0.0, ints.g)
    n_orb = h.shape[0]
    n = 2 * n_orb
    dim = 1 << n
    out = sp.identity(dim, dtype=np.complex128, format="csr") * ints.e0
    for p in range(n_orb):
        for q in range(n_orb):
            if h[p, q] == 0:
                continue
            for s in (0, 1):
                out = out + h[p, q] * (create(n, 2 * p + s) @ ladder(n, 2 * q + s))
    for p in range(n_orb):
        for q in range(n_orb):
            for r in range(n_orb):
                for s_ in range(n_orb):
                    v = g[p, q, r, s_]
                    if v == 0:
                        continue
                    for a in (0, 1):
                        for b in (0, 1):
                            op = (create(n, 2 * p + a) @ create(n, 2 * r + b)
                                  @ ladder(n, 2 * s_ + b) @ ladder(n, 2 * q + a))
                            out = out + 0.5 * v * op
    return out.toarray()


def excitation_dense(n: int, occ, virt) -> np.ndarray:
    """tau = a+_a a_i - h.c. or a+_a a+_b a_j a_i - h.c. from matrices."""
    if len(occ) == 1:
        e = create(n, virt[0]) @ ladder(n, occ[0])
    else:
        (i, j), (a, b) = occ, virt
        e = create(n, a) @ create(n, b) @ ladder(n, j) @ ladder(n, i)
    e = e.toarray()
    return e - e.conj().T


def pauli_matrix(x: int, z: int, n: int) -> np.ndarray:
    """X^x Z^z as a Kronecker product, qubit 0 the least significant index bit."""
    out = np.ones((1, 1), dtype=np.complex128)
    for j in reversed(range(n)):
        xb, zb = (x >> j) & 1, (z >> j) & 1
        if xb and zb:
            m = PX @ PZ
        elif xb:
            m = PX
        elif zb:
            m = PZ
        else:
            m = I2
        out = np.kron(out, m)
    return out


def table_dense(t) -> np.ndarray:
    dim = 1 << t.n
    out = np.zeros((dim, dim), dtype=np.complex128)
    for x, z, ph, c in zip(t.x.tolist(), t.z.tolist(), t.phase.tolist(), t.coeff.tolist()):
        out += c * (1j ** ph) * pauli_matrix(x, z, t.n)
    return out


def srl_beta(n: int) -> np.ndarray:
    """Seeley-Richard-Love BK matrix: beta_1 = [1], beta_2m = [[beta_m, 0],
    [A_m, beta_m]] with A_m zero except a last row of ones; other sizes take
    the top-left block of the next power of two."""
    b = np.ones((1, 1), dtype=np.uint8)
    while b.shape[0] < n:
        m = b.shape[0]
        a = np.zeros((m, m), dtype=np.uint8)
        a[-1, :] = 1
        b = np.block([[b, np.zeros((m, m), dtype=np.uint8)], [a, b]])
    return b[:n, :n].copy()


def permutation_from_gf2(beta: np.ndarray) -> np.ndarray:
    """Matrix of |m> -> |beta m> on 2**n basis states."""
    n = beta.shape[0]
    dim = 1 << n
    perm = np.zeros((dim, dim))
    for m in range(dim):
        bits = np.array([(m >> j) & 1 for j in range(n)])
        img = (beta.astype(np.int64) @ bits) % 2
        mi = int(sum(int(v) << j for j, v in enumerate(img)))
        perm[mi, m] = 1.0
    return perm


def number_ops(n: int):
    """Total number N and 2*S_z = N_alpha - N_beta as diagonal arrays."""
    idx = np.arange(1 << n)
    na = sum(((idx >> j) & 1) for j in range(0, n, 2))
    nb = sum(((idx >> j) & 1) for j in range(1, n, 2))
    return na + nb, na - nb


def slater_condon_hf(ints, n_elec: int) -> float:
    """<HF|H|HF> = E0 + sum_i h_ii + 1/2 sum_ij [(ii|jj) - delta_spin (ij|ji)]."""
    occ = list(range(n_elec))
    e = ints.e0
    for i in occ:
        e += ints.h[i // 2, i // 2]
    for i in occ:
        for j in occ:
            p, q = i // 2, j // 2
            e += 0.5 * ints.g[p, p, q, q]
            if i % 2 == j % 2:
                e -= 0.5 * ints.g[p, q, q, p]
    return float(e)
