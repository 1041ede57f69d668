"""The ADAPT-VQE loop (Sec. II.B; Eq. 4 for selection, Eq. 1 as objective).

Each iteration computes every pool gradient on the current state, stops when
the gradient norm falls below ``gtol`` or the ansatz reaches ``max_ops``,
otherwise appends the operator of largest |g| with angle 0 and re-optimises
all angles with BFGS (analytic gradient, warm start).  Gradients within a
relative ``tie_rel`` of the largest count as ties, broken by lowest pool
index (alpha/beta mirror operators have equal |g| in exact arithmetic).
The commuting families only schedule the gradient evaluation; selection is
over the whole pool.

With ``families`` given (the GOCP family of each pool operator, Algorithm 1)
an iteration adds a whole commuting family instead of one operator (the
"reduced search space" reading of Sec. III.A and IV.B): the family of the
selected operator, restricted to its members with |g| >= family_rel * max|g|,
appended in pool-index order, each with angle 0.
"""

from __future__ import annotations

import dataclasses

import numpy as np
from scipy.optimize import minimize

from . import statevector as sv


@dataclasses.dataclass
class AdaptResult:
    ops: list
    thetas: np.ndarray
    energies: list
    grad_norms: list
    converged: bool


def select(grads: np.ndarray, tie_rel: float) -> int:
    mag = np.abs(grads)
    top = mag.max()
    cand = np.flatnonzero(mag >= top * (1.0 - tie_rel))
    return int(cand.min())


def family_batch(grads: np.ndarray, families, k: int, family_rel: float) -> list:
    """Members of operator k's family with |g| >= family_rel * max|g|, by index."""
    mag = np.abs(grads)
    fam = np.asarray(families)
    cand = np.flatnonzero((fam == fam[k]) & (mag >= family_rel * mag.max()))
    return [int(c) for c in cand]


def adapt(h, pool, ref, max_ops: int = 30, gtol: float = 1e-4,
          tie_rel: float = 1e-8, bfgs_gtol: float = 1e-8, maxiter: int = 200,
          families=None, family_rel: float = 0.5) -> AdaptResult:
    ops: list[int] = []
    thetas = np.zeros(0)
    energies, norms = [], []
    converged = False
    while True:
        psi = sv.prepare_state(ref, pool, ops, thetas)
        energies.append(sv.energy(h, psi))
        g = sv.pool_gradients(h, pool, psi)
        gn = float(np.linalg.norm(g))
        norms.append(gn)
        if gn < gtol:
            converged = True
            break
        if len(ops) >= max_ops:
            break
        k = select(g, tie_rel)
        new = [k] if families is None else family_batch(g, families, k, family_rel)
        new = new[:max_ops - len(ops)]
        ops.extend(new)
        x0 = np.concatenate([thetas, np.zeros(len(new))])

        def fun(th, _ops=list(ops)):
            e, dg = sv.energy_grad(h, ref, pool, _ops, th)
            return e, dg

        res = minimize(fun, x0, jac=True, method="BFGS",
                       options=dict(gtol=bfgs_gtol, maxiter=maxiter))
        thetas = np.asarray(res.x, dtype=np.float64)
    return AdaptResult(ops=ops, thetas=thetas, energies=energies, grad_norms=norms,
                       converged=converged)
