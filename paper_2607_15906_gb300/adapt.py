"""ADAPT-VQE driver over the C ABI (Sec. II.B).

Each iteration runs one device selection step (prepare psi(theta), H psi, E,
every pool gradient g_k = 2 Re <H psi|A_k psi> (Eq. 4) in GOCP family
order, argmax with a relative tie window), stops when ||g||_2 < gtol or the
ansatz holds max_ops operators, else appends the selected operator with
angle 0 and re-optimises all angles with BFGS, the energy and dE/dtheta of
each evaluation coming from the adjoint sweep (gocp_energy_grad).

family=True adds a whole commuting family per iteration (the "reduced search
space" reading of GOCP, Sec. III.A and IV.B): the GOCP family of the
selected operator, restricted to members with |g| >= family_rel * max|g|,
appended in pool-index order with angle 0.
"""

from __future__ import annotations

import dataclasses

import numpy as np

try:
    from scipy.optimize import minimize
except Exception:  # pragma: no cover
    minimize = None


@dataclasses.dataclass
class AdaptRun:
    ops: list
    thetas: np.ndarray
    energies: list
    grad_norms: list
    converged: bool
    evaluations: int
    gradients: list = dataclasses.field(default_factory=list)   # pool gradients of each iteration


def adapt(problem, max_ops: int = 30, gtol: float = 1e-4, tie_rel: float | None = None,
          bfgs_gtol: float = 1e-8, maxiter: int = 200, eval_budget: int | None = None,
          family: bool = False, family_rel: float = 0.5) -> AdaptRun:
    """Run ADAPT-VQE on a built problem.  tie_rel defaults to 1e-8 (c128) or
    1e-4 (c64); eval_budget caps the energy+gradient evaluations of each
    re-optimisation (None: run BFGS to bfgs_gtol / maxiter)."""
    if minimize is None:
        raise RuntimeError("scipy is needed for the re-optimisation")
    if tie_rel is None:
        tie_rel = 1e-8 if problem.precision == "c128" else 1e-4
    ws = problem.workspace()
    fam = problem.pool()[5] if family else None
    if family and np.any(fam < 0):
        raise ValueError("family=True needs a problem built with GOCP colouring")
    ops: list[int] = []
    thetas = np.zeros(0)
    energies, norms, grads = [], [], []
    evals = 0
    converged = False
    while True:
        e, _, g, sel = problem.adapt_step(np.asarray(ops, np.int32), thetas, ws=ws, tie_rel=tie_rel)
        energies.append(e)
        grads.append(np.asarray(g).copy())
        gn = float(np.linalg.norm(g))
        norms.append(gn)
        if gn < gtol:
            converged = True
            break
        if len(ops) >= max_ops:
            break
        if family:
            mag = np.abs(g)
            new = [int(c) for c in np.flatnonzero((fam == fam[int(sel)]) & (mag >= family_rel * mag.max()))]
        else:
            new = [int(sel)]
        new = new[:max_ops - len(ops)]
        ops.extend(new)
        x0 = np.concatenate([thetas, np.zeros(len(new))])
        op_arr = np.asarray(ops, np.int32)

        def fun(th):
            nonlocal evals
            evals += 1
            return problem.energy_grad(op_arr, th, ws=ws)

        opts = dict(gtol=bfgs_gtol, maxiter=maxiter)
        if eval_budget is not None:
            opts["maxiter"] = max(1, eval_budget)
        res = minimize(fun, x0, jac=True, method="BFGS", options=opts)
        thetas = np.asarray(res.x, dtype=np.float64)
    return AdaptRun(ops=ops, thetas=thetas, energies=energies, grad_norms=norms,
                    converged=converged, evaluations=evals, gradients=grads)
