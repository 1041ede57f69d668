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


def apply_terms_at(t: PauliTable, psi: np.ndarray, rows) -> np.ndarray:
    """Selected entries (H psi)[k] = sum_t c_t i**ph_t (-1)**popc((k^x_t) & z_t) psi[k ^ x_t]."""
    rows = np.asarray(rows, dtype=np.int64)
    w = t.weights()
    out = np.zeros(rows.shape[0], dtype=np.complex128)
    for r, k in enumerate(rows.tolist()):
        src = k ^ t.x
        sign = 1 - 2 * parity(src & t.z)
        out[r] = np.sum(w * sign * psi[src])
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
# input (a basis state evolved by a few operators) be checked exactly.

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
    return keys, acc


def _sparse_axpy(ai, av, bi, bv, scale):
    keys, inv = np.unique(np.concatenate([ai, bi]), return_inverse=True)
    acc = np.zeros(keys.shape[0], dtype=np.complex128)
    np.add.at(acc, inv, np.concatenate([av, scale * bv]))
    return keys, acc


def taylor5_sparse(a: PauliTable, theta: float, idx, vals):
    oi, ov = np.asarray(idx, np.int64), np.asarray(vals, np.complex128)
    vi, vv = oi, ov
    for m in range(1, 6):
        vi, vv = apply_terms_sparse(a, vi, vv)
        oi, ov = _sparse_axpy(oi, ov, vi, vv, theta ** m / math.factorial(m))
    return oi, ov


def prepare_state_sparse(ref_index: int, pool: list[PauliTable], ops, thetas):
    idx, vals = np.array([ref_index], np.int64), np.array([1.0 + 0j])
    for k, th in zip(list(ops), list(thetas)):
        idx, vals = taylor5_sparse(pool[int(k)], float(th), idx, vals)
    return idx, vals


def sparse_dot(ai, av, bi, bv) -> complex:
    """<a|b> of two sparse states."""
    common, ia, ib = np.intersect1d(ai, bi, return_indices=True)
    return complex(np.sum(np.conj(av[ia]) * bv[ib]))
