"""Fermionic Hamiltonian (Eq. 2) mapped to a Pauli sum (Eq. 3) under the
Jordan-Wigner and Bravyi-Kitaev transformations (Sec. II.A).

Spin-orbital i = 2p + sigma (sigma 0 = alpha, 1 = beta); qubit i carries it.
Eq. (2) with h_ijkl read as the physicist integral <ij|kl> = (ik|jl) gives

    H = E0 + sum_{pq,s} h_pq a+_{ps} a_{qs}
           + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}.

Both mappings write every ladder operator as two X^x Z^z strings,

    a_j  = 1/2 X^x Z^zp - 1/2 X^x Z^(zp ^ ze)
    a+_j = 1/2 X^x Z^zp + 1/2 X^x Z^(zp ^ ze)

where, for the basis relabelling |n> -> |beta n> over GF(2) that defines the
encoding, x = beta e_j flips the encoded bits touched by occupation j,
zp = beta^-T m_j reads the parity of occupations below j (m_j = 2**j - 1) and
ze = beta^-T e_j reads occupation j itself.  Jordan-Wigner is beta = I (local
occupation, Z strings of length O(N)); Bravyi-Kitaev is the Fenwick-tree
matrix whose row j sums occupations j+1-lowbit(j+1) .. j (parity stored on a
binary tree, string weight O(log N)).
"""

from __future__ import annotations

import dataclasses

import numpy as np

from .pauli import PauliTable, accumulate_exact, parity


# ---------------------------------------------------------------- GF(2) helpers

def bk_matrix(n: int) -> np.ndarray:
    """Fenwick-tree Bravyi-Kitaev matrix: row j has ones in columns
    j+1-lowbit(j+1) .. j."""
    b = np.zeros((n, n), dtype=np.uint8)
    for j in range(n):
        low = (j + 1) & -(j + 1)
        b[j, j + 1 - low: j + 1] = 1
    return b


def gf2_inverse(m: np.ndarray) -> np.ndarray:
    """Inverse of a square 0/1 matrix over GF(2) by Gauss-Jordan elimination."""
    n = m.shape[0]
    a = np.concatenate([m.astype(np.uint8) % 2, np.eye(n, dtype=np.uint8)], axis=1)
    for col in range(n):
        piv = next((r for r in range(col, n) if a[r, col]), None)
        if piv is None:
            raise ValueError("matrix is singular over GF(2)")
        if piv != col:
            a[[col, piv]] = a[[piv, col]]
        for r in range(n):
            if r != col and a[r, col]:
                a[r] ^= a[col]
    return a[:, n:].copy()


def matvec_mask(m: np.ndarray, v: int) -> int:
    """GF(2) product of matrix m with the bit vector v (bit j = component j)."""
    n = m.shape[0]
    bits = np.array([(v >> j) & 1 for j in range(n)], dtype=np.int64)
    out_bits = (m.astype(np.int64) @ bits) % 2
    return int(sum(int(b) << j for j, b in enumerate(out_bits)))


# ---------------------------------------------------------------- mappings

@dataclasses.dataclass(frozen=True)
class Encoding:
    """A GF(2) encoding |n> -> |beta n> with its ladder-operator strings."""

    name: str
    n: int
    beta: np.ndarray

    @property
    def beta_inv_t(self) -> np.ndarray:
        return gf2_inverse(self.beta).T.copy()

    def ladder(self, j: int):
        """(x, zp, ze) of mode j."""
        bit = self.beta_inv_t
        x = matvec_mask(self.beta, 1 << j)
        zp = matvec_mask(bit, (1 << j) - 1)
        ze = matvec_mask(bit, 1 << j)
        return x, zp, ze

    def encode_occupation(self, occ_mask: int) -> int:
        return matvec_mask(self.beta, occ_mask)


def jordan_wigner(n: int) -> Encoding:
    return Encoding("jw", n, np.eye(n, dtype=np.uint8))


def bravyi_kitaev(n: int) -> Encoding:
    return Encoding("bk", n, bk_matrix(n))


def encoding(name: str, n: int) -> Encoding:
    if name == "jw":
        return jordan_wigner(n)
    if name == "bk":
        return bravyi_kitaev(n)
    raise ValueError(f"unknown mapping {name!r}")


def _ladder_tables(enc: Encoding):
    n = enc.n
    lx = np.zeros(n, dtype=np.int64)
    lzp = np.zeros(n, dtype=np.int64)
    lze = np.zeros(n, dtype=np.int64)
    for j in range(n):
        lx[j], lzp[j], lze[j] = enc.ladder(j)
    return lx, lzp, lze


def expand_products(enc: Encoding, modes: np.ndarray, daggers, coeff: np.ndarray):
    """All X^x Z^z contributions of  coeff[r] * L_1 L_2 ... L_K  (operator
    product, L_1 leftmost) with L_m = a+_{modes[r,m]} if daggers[m] else
    a_{modes[r,m]}.  Returns flat arrays (x, z, value), 2**K per row."""
    modes = np.asarray(modes, dtype=np.int64)
    coeff = np.asarray(coeff, dtype=np.float64)
    rows, k = modes.shape
    lx, lzp, lze = _ladder_tables(enc)
    xs, zs, vs = [], [], []
    for choice in range(1 << k):
        x = np.zeros(rows, dtype=np.int64)
        z = np.zeros(rows, dtype=np.int64)
        val = coeff.copy()
        for m in range(k):
            j = modes[:, m]
            pick = (choice >> m) & 1
            zm = lzp[j] ^ (lze[j] if pick else 0)
            s = 0.5 if (daggers[m] or not pick) else -0.5
            sign = 1 - 2 * parity(z & lx[j])
            val = val * s * sign
            x = x ^ lx[j]
            z = z ^ zm
        xs.append(x)
        zs.append(z)
        vs.append(val)
    return np.concatenate(xs), np.concatenate(zs), np.concatenate(vs)


def hamiltonian_table(ints, mapping: str = "jw", int_drop: float = 0.0,
                      term_drop: float = 0.0) -> PauliTable:
    """Eq. (2) -> Eq. (3): the qubit Hamiltonian of spatial integrals ``ints``.

    Integrals with |v| < int_drop are zeroed before mapping; mapped terms are
    accumulated exactly per (x, z) and those with |c| < term_drop dropped.
    """
    h = np.where(np.abs(ints.h) < int_drop, 0.0, ints.h)
    g = np.where(np.abs(ints.g) < int_drop, 0.0, ints.g)
    n_orb = h.shape[0]
    n = 2 * n_orb
    enc = encoding(mapping, n)
    xs, zs, vs = [np.zeros(1, dtype=np.int64)], [np.zeros(1, dtype=np.int64)], [np.array([ints.e0])]

    # one-body: h_pq a+_{p s} a_{q s}
    p, q = np.nonzero(h)
    for s in (0, 1):
        modes = np.stack([2 * p + s, 2 * q + s], axis=1)
        x, z, v = expand_products(enc, modes, (True, False), h[p, q])
        xs.append(x); zs.append(z); vs.append(v)

    # two-body: 1/2 (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}
    p, q, r, s_ = np.nonzero(g)
    vals = 0.5 * g[p, q, r, s_]
    for sig in (0, 1):
        for tau in (0, 1):
            modes = np.stack([2 * p + sig, 2 * r + tau, 2 * s_ + tau, 2 * q + sig], axis=1)
            x, z, v = expand_products(enc, modes, (True, True, False, False), vals)
            xs.append(x); zs.append(z); vs.append(v)

    return accumulate_exact(np.concatenate(xs), np.concatenate(zs), np.concatenate(vs),
                            n, term_drop=term_drop)


def hf_index(mapping: str, n: int, n_elec: int) -> int:
    """Basis index of the closed-shell reference: spin-orbitals 0..N_e-1
    occupied, encoded by the mapping (JW: 2**N_e - 1)."""
    return encoding(mapping, n).encode_occupation((1 << n_elec) - 1)
