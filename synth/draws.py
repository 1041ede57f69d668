"""Seeded random states, ansatz draws and the serving request stream."""

from __future__ import annotations

import dataclasses

import numpy as np


def random_state(n_qubits: int, seed: int, normalize: bool = True) -> np.ndarray:
    """A complex128 vector of length 2**n with i.i.d. complex-normal entries."""
    rng = np.random.default_rng(seed)
    dim = 1 << n_qubits
    v = rng.normal(size=dim) + 1j * rng.normal(size=dim)
    if normalize:
        v = v / np.linalg.norm(v)
    return v.astype(np.complex128)


def draw_ansatz(pool_size: int, n_ops: int, seed: int = 0,
                theta_sigma: float = 0.05) -> tuple[np.ndarray, np.ndarray]:
    """Ansatz of ``n_ops`` operators drawn uniformly (with replacement) from a
    pool of ``pool_size`` with rng(seed+1), angles N(0, theta_sigma) with
    rng(seed+2)."""
    ops = np.random.default_rng(seed + 1).integers(0, pool_size, size=n_ops).astype(np.int32)
    theta = np.random.default_rng(seed + 2).normal(0.0, theta_sigma, size=n_ops)
    return ops, theta.astype(np.float64)


@dataclasses.dataclass(frozen=True)
class ServingRequest:
    index: int
    arrival_s: float
    n_qubits: int
    n_orb: int
    n_elec: int
    seed: int
    n_ops: int
    op_draw: np.ndarray      # uniform [0,1) draws; op index = floor(u * pool_size)
    theta: np.ndarray


def serving_requests(n_requests: int, rate_per_s: float, seed: int = 7,
                     qubit_choices=(10, 12, 14, 16, 18, 20, 22),
                     ops_range=(10, 80), theta_sigma: float = 0.05):
    """Poisson-arriving energy+gradient requests of mixed qubit counts.

    Request i uses Hamiltonian seed 1000+i, n qubits uniform over
    ``qubit_choices``, 2*floor(n/4) electrons (closed shell), between
    ops_range[0] and ops_range[1] operators and N(0, theta_sigma) angles.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests) if rate_per_s > 0 else np.zeros(n_requests)
    arrivals = np.cumsum(gaps)
    out = []
    for i in range(n_requests):
        n = int(rng.choice(qubit_choices))
        n_ops = int(rng.integers(ops_range[0], ops_range[1] + 1))
        u = rng.random(n_ops)
        th = rng.normal(0.0, theta_sigma, size=n_ops)
        out.append(ServingRequest(index=i, arrival_s=float(arrivals[i]), n_qubits=n,
                                  n_orb=n // 2, n_elec=2 * (n // 4), seed=1000 + i,
                                  n_ops=n_ops, op_draw=u, theta=th))
    return out
