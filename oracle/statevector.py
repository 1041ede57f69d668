"""Statevector side of the method, complex128, term by term.

  apply_terms     out[b ^ x] += c i**phase (-1)**popc(b & z) psi[b] per term (Eq. 3)
  taylor5         psi' = sum_{m=0..5} theta**m / m! v_m, v_m = A v_{m-1}  (Eq. 5, 6)
  prepare_state   psi_P = T_P ... T_1 |ref>  (operator selected first acts first)
  energy          Rayleigh quotient <psi|H|psi> / <psi|psi>  (Eq. 1)
  pool_gradients  g_k = <psi^|[H, A_k]|psi^> = 2 Re <H psi^|A_k psi^>  (Eq. 4)
  energy_grad     E and dE/dtheta_j by forward mode: T_j replaced by
                  T'_j = d T_j / d theta_j = sum_{m=1..5} theta**(m-1)/(m-1)! A**m

No intermediate renormalisation: the Taylor propagator is not exactly unitary,
and Eq. (1) divides by <psi|psi>.  The paper's remark that A_k**2 = I is not
used: for an anti-Hermitian fermionic excitation A**2 is minus a projector, so
the literal chain of Eq. (6) is evaluated as written.
"""

from __future__ import annotations

import math

import numpy as np

from .pauli import PauliTable, parity


def basis_state(n: int, index: int) -> np.ndarray:
    v = np.zeros(1 << n, dtype=np.complex128)
    v[index] = 1.0
    return v


def apply_terms(t: PauliTable, psi: np.ndarray) -> np.ndarray:
    """Pauli sum times state, one term at a time over all basis indices."""
    dim = psi.shape[0]
    idx = np.arange(dim, dtype=np.int64)
    out = np.zeros(dim, dtype=np.complex128)
    for x, z, ph, c in zip(t.x.tolist(), t.z.tolist(), t.phase.tolist(), t.coeff.tolist()):
        sign = 1 - 2 * parity(idx & z)
        out[idx ^ x] += (c * (1j ** ph)) * sign * psi
    return out


def apply_terms_at(t: PauliTable, psi: np.ndarray, rows, block: int = 1) -> np.ndarray:
    """Selected entries (H psi)[k] = sum_t c_t i**ph_t (-1)**popc((k^x_t) & z_t) psi[k ^ x_t]
    (`block` rows at a time; each row is still one sum over all terms)."""
    rows = np.asarray(rows, dtype=np.int64)
    w = t.weights()
    out = np.zeros(rows.shape[0], dtype=np.complex128)
    if block <= 1:
        for r, k in enumerate(rows.tolist()):
            src = k ^ t.x
            sign = 1 - 2 * parity(src & t.z)
            out[r] = np.sum(w * sign * psi[src])
        return out
    for r0 in range(0, rows.shape[0], block):
        src = rows[r0:r0 + block, None] ^ t.x[None, :]
        sign = 1 - 2 * parity(src & t.z[None, :])
        out[r0:r0 + block] = np.sum(w[None, :] * sign * psi[src], axis=1)
    return out


def taylor5(a: PauliTable, theta: float, psi: np.ndarray) -> np.ndarray:
    """Eq. (5) evaluated as the chain of Eq. (6), summed in order m = 0..5."""
    out = psi.copy()
    v = psi
    for m in range(1, 6):
        v = apply_terms(a, v)
        out = out + (theta ** m / math.factorial(m)) * v
    return out


def taylor5_derivative(a: PauliTable, theta: float, psi: np.ndarray) -> np.ndarray:
    """d/dtheta of the truncated series: sum_{m=1..5} theta**(m-1)/(m-1)! A**m psi."""
    out = np.zeros_like(psi)
    v = psi
    for m in range(1, 6):
        v = apply_terms(a, v)
        out = out + (theta ** (m - 1) / math.factorial(m - 1)) * v
    return out


def prepare_state(ref: np.ndarray, pool: list[PauliTable], ops, thetas) -> np.ndarray:
    psi = ref.copy()
    for k, th in zip(list(ops), list(thetas)):
        psi = taylor5(pool[int(k)], float(th), psi)
    return psi


def energy(h: PauliTable, psi: np.ndarray) -> float:
    hpsi = apply_terms(h, psi)
    return float(np.vdot(psi, hpsi).real / np.vdot(psi, psi).real)


def fidelity(a: np.ndarray, b: np.ndarray) -> float:
    """|<a|b>|**2 / (<a|a><b|b>)."""
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def pool_gradients(h: PauliTable, pool: list[PauliTable], psi: np.ndarray) -> np.ndarray:
    """Eq. (4) on the normalised state, for every pool operator."""
    psi_n = psi / np.sqrt(np.vdot(psi, psi).real)
    hpsi = apply_terms(h, psi_n)
    return np.array([2.0 * np.vdot(hpsi, apply_terms(a, psi_n)).real for a in pool])


def energy_grad(h: PauliTable, ref: np.ndarray, pool: list[PauliTable], ops, thetas):
    """E(theta) and dE/dtheta_j, j = 1..P, by forward-mode propagation.

    dE/dtheta_j = 2 Re <(H - E) psi | d_j psi> / <psi|psi>, with d_j psi the
    state prepared with T_j replaced by its derivative.
    """
    ops = [int(k) for k in ops]
    thetas = [float(t) for t in thetas]
    psi = prepare_state(ref, pool, ops, thetas)
    nrm = np.vdot(psi, psi).real
    hpsi = apply_terms(h, psi)
    e = float(np.vdot(psi, hpsi).real / nrm)
    resid = hpsi - e * psi
    grads = np.zeros(len(ops))
    for j in range(len(ops)):
        d = ref.copy()
        for i, (k, th) in enumerate(zip(ops, thetas)):
            if i == j:
                d = taylor5_derivative(pool[k], th, d)
            else:
                d = taylor5(pool[k], th, d)
        grads[j] = 2.0 * np.vdot(resid, d).real / nrm
    return e, grads


# ---------------------------------------------------------------- sparse states
#
# The same per-term formula restricted to the nonzero entries of a state held
# as (indices, values).  It lets full-size (24-qubit) cases with a sparse
# input (a basis state evolved by operators of the pool) be checked exactly.
# Entries whose sum is exactly zero (strings of one generator cancelling at a
# basis state the excitation cannot act on) are dropped: a zero amplitude
# contributes nothing to any later product or sum, so every result is the
# same as with the zeros kept, and the held support stays that of the state.

def apply_terms_sparse(t: PauliTable, idx: np.ndarray, vals: np.ndarray, chunk: int = 512):
    idx = np.asarray(idx, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.complex128)
    w = t.weights()
    outs_i, outs_v = [], []
    for s in range(0, len(t), chunk):
        xs, zs, ws = t.x[s:s + chunk, None], t.z[s:s + chunk, None], w[s:s + chunk, None]
        sign = 1 - 2 * parity(idx[None, :] & zs)
        outs_i.append((idx[None, :] ^ xs).ravel())
        outs_v.append((ws * sign * vals[None, :]).ravel())
    if not outs_i:
        return np.zeros(0, np.int64), np.zeros(0, np.complex128)
    ai = np.concatenate(outs_i)
    av = np.concatenate(outs_v)
    keys, inv = np.unique(ai, return_inverse=True)
    acc = np.zeros(keys.shape[0], dtype=np.complex128)
    np.add.at(acc, inv, av)
    keep = acc != 0
    return keys[keep], acc[keep]


def apply_group_sparse(a: PauliTable, idx: np.ndarray, vals: np.ndarray):
    """A psi for a generator whose strings share one x mask (every pool
    operator): (A psi)[b ^ x] = D(b) psi[b] with D(b) = sum_t w_t
    (-1)**popc(b & z_t) -- Eq. (3) with the terms of one x-group summed per
    basis state before the product.  A fermionic excitation's string weights
    are multiples of 1/8, so D(b) is exact and is exactly zero where the
    excitation cannot act (there the term-by-term products leave rounding
    residue of order 1e-16 |psi[b]|)."""
    x = int(a.x[0])
    assert np.all(a.x == x), "strings of one generator share their x mask"
    idx = np.asarray(idx, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.complex128)
    w = a.weights()
    d = np.zeros(idx.shape[0], dtype=np.complex128)
    for zt, wt in zip(a.z.tolist(), w.tolist()):
        d += wt * (1 - 2 * parity(idx & zt))
    keep = d != 0
    oi = idx[keep] ^ x
    ov = d[keep] * vals[keep]
    order = np.argsort(oi)
    return oi[order], ov[order]


def _sparse_axpy(ai, av, bi, bv, scale):
    keys, inv = np.unique(np.concatenate([ai, bi]), return_inverse=True)
    acc = np.zeros(keys.shape[0], dtype=np.complex128)
    np.add.at(acc, inv, np.concatenate([av, scale * bv]))
    keep = acc != 0
    return keys[keep], acc[keep]


def taylor5_sparse(a: PauliTable, theta: float, idx, vals):
    """taylor5 on a sparse state (the chain v_m = A v_{m-1} of Eq. 6)."""
    oi, ov = np.asarray(idx, np.int64), np.asarray(vals, np.complex128)
    vi, vv = oi, ov
    for m in range(1, 6):
        vi, vv = apply_group_sparse(a, vi, vv)
        oi, ov = _sparse_axpy(oi, ov, vi, vv, theta ** m / math.factorial(m))
    return oi, ov


def taylor5_derivative_sparse(a: PauliTable, theta: float, idx, vals):
    """taylor5_derivative on a sparse state."""
    oi, ov = np.zeros(0, np.int64), np.zeros(0, np.complex128)
    vi, vv = np.asarray(idx, np.int64), np.asarray(vals, np.complex128)
    for m in range(1, 6):
        vi, vv = apply_group_sparse(a, vi, vv)
        oi, ov = _sparse_axpy(oi, ov, vi, vv, theta ** (m - 1) / math.factorial(m - 1))
    return oi, ov


def prepare_state_sparse(ref_index: int, pool: list[PauliTable], ops, thetas, keep_at=None):
    """psi_P = T_P ... T_1 |ref> on a sparse state.  With keep_at (operator
    positions j) also returns {j: psi_j}, psi_j the state before operator j
    acts, for forward-mode derivatives (derivative_state_sparse)."""
    idx, vals = np.array([ref_index], np.int64), np.array([1.0 + 0j])
    want = set() if keep_at is None else {int(j) for j in keep_at}
    kept = {}
    for j, (k, th) in enumerate(zip(list(ops), list(thetas))):
        if j in want:
            kept[j] = (idx, vals)
        idx, vals = taylor5_sparse(pool[int(k)], float(th), idx, vals)
    if keep_at is None:
        return idx, vals
    return idx, vals, kept


def derivative_state_sparse(pool: list[PauliTable], ops, thetas, j: int, psi_j):
    """d psi_P / d theta_j (forward mode, as in energy_grad) from psi_j, the
    state before operator j acts: T'_j, then T_{j+1} .. T_P."""
    idx, vals = taylor5_derivative_sparse(pool[int(ops[j])], float(thetas[j]), *psi_j)
    for k, th in zip(list(ops)[j + 1:], list(thetas)[j + 1:]):
        idx, vals = taylor5_sparse(pool[int(k)], float(th), idx, vals)
    return idx, vals


def sparse_dot(ai, av, bi, bv) -> complex:
    """<a|b> of two sparse states."""
    common, ia, ib = np.intersect1d(ai, bi, return_indices=True)
    return complex(np.sum(np.conj(av[ia]) * bv[ib]))
