"""Oracle work spread over the host cores.

Test infrastructure only (see the package docstring): used by the full-size
parity tests and by the oracle timing of bench.py.  Every worker runs
functions of ``oracle.statevector`` on a slice of rows or of pool operators;
this module adds no arithmetic of its own beyond gathering the slices and
one dot product per operator (Eq. 4).  Workers are started with the 'spawn'
method, so none is forked from a process that has touched the GPU, and they
import only numpy and the oracle.
"""

from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from . import statevector as sv
from .pauli import PauliTable


def _pack(t: PauliTable):
    return (t.n, np.asarray(t.x), np.asarray(t.z), np.asarray(t.phase), np.asarray(t.coeff))


def _unpack(a) -> PauliTable:
    return PauliTable(*a)


def procs() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def start(n_procs: int):
    """A pool of n_procs spawned workers (None for n_procs <= 1: in-process)."""
    return mp.get_context("spawn").Pool(n_procs) if n_procs > 1 else None


def _map(fn, jobs, n_procs, pool=None):
    if pool is not None:
        return pool.map(fn, jobs)
    if n_procs <= 1 or len(jobs) <= 1:
        return [fn(j) for j in jobs]
    with start(min(n_procs, len(jobs))) as p:
        return p.map(fn, jobs)


_DENSE: dict = {}


def _dense(n, si, svals):
    """psi as a dense 2^n array (the lookup apply_terms_at indexes), kept for
    the next job on the same state in this process."""
    key = (n, si.size, int(si[0]) if si.size else -1, int(si[-1]) if si.size else -1,
           complex(svals[0]) if si.size else 0j, complex(svals[-1]) if si.size else 0j)
    if key not in _DENSE:
        _DENSE.clear()
        psi = np.zeros(1 << n, np.complex128)
        psi[si] = svals
        _DENSE[key] = psi
    return _DENSE[key]


def _rows_job(args):
    h, n, si, svals, rows = args
    return sv.apply_terms_at(_unpack(h), _dense(n, si, svals), rows, block=8)


def hpsi_rows(h: PauliTable, si, svals, rows, n_procs: int | None = None, pool=None) -> np.ndarray:
    """(H psi)[rows] for a sparse psi, by oracle.statevector.apply_terms_at."""
    n_procs = procs() if n_procs is None else n_procs
    rows = np.asarray(rows, np.int64)
    parts = np.array_split(rows, max(1, 4 * n_procs))
    jobs = [(_pack(h), h.n, si, svals, p) for p in parts if p.size]
    return np.concatenate(_map(_rows_job, jobs, n_procs, pool)) if jobs else np.zeros(0, np.complex128)


def _support_job(args):
    gens, n, si, svals = args
    mask = np.zeros(1 << n, bool)
    for g in gens:
        ai, _ = sv.apply_group_sparse(_unpack(g), si, svals)
        mask[ai] = True
    return mask


def generator_support(pool: list[PauliTable], si, svals, n_procs: int | None = None) -> np.ndarray:
    """Boolean mask of the union of supp(A_k psi) over the pool."""
    n_procs = procs() if n_procs is None else n_procs
    n = pool[0].n
    chunks = np.array_split(np.arange(len(pool)), max(1, 2 * n_procs))
    jobs = [([_pack(pool[k]) for k in c], n, si, svals) for c in chunks if c.size]
    mask = np.zeros(1 << n, bool)
    for m in _map(_support_job, jobs, n_procs):
        mask |= m
    return mask


def _grad_job(args):
    gens, si, svals, rows, hrows = args
    out = np.zeros(len(gens))
    for i, g in enumerate(gens):
        ai, av = sv.apply_group_sparse(_unpack(g), si, svals)
        pos = np.searchsorted(rows, ai)
        if ai.size and (np.any(pos >= rows.size) or np.any(rows[np.minimum(pos, rows.size - 1)] != ai)):
            raise AssertionError("H psi was not evaluated on the support of A_k psi")
        out[i] = 2.0 * np.sum(np.conj(hrows[pos]) * av).real
    return out


def pool_gradients(pool: list[PauliTable], si, svals, rows, hrows, nrm: float,
                   n_procs: int | None = None) -> np.ndarray:
    """g_k = 2 Re <H psi|A_k psi> / <psi|psi> (Eq. 4) for every k, with H psi
    given on `rows` (sorted), which must cover every supp(A_k psi)."""
    n_procs = procs() if n_procs is None else n_procs
    chunks = np.array_split(np.arange(len(pool)), max(1, 2 * n_procs))
    jobs = [([_pack(pool[k]) for k in c], si, svals, rows, hrows) for c in chunks if c.size]
    return np.concatenate(_map(_grad_job, jobs, n_procs)) / nrm


def _dots_job(args):
    gens, si, svals, vi, vv = args
    out = np.zeros(len(gens))
    for i, g in enumerate(gens):
        ai, av = sv.apply_group_sparse(_unpack(g), si, svals)
        out[i] = 2.0 * sv.sparse_dot(vi, vv, ai, av).real
    return out


def generator_dots(gens: list[PauliTable], si, svals, vi, vv, n_procs: int | None = None,
                   pool=None) -> np.ndarray:
    """2 Re <v|A_k psi> for each generator (Eq. 4 with v = H psi), psi and v
    sparse (v zero outside vi)."""
    n_procs = procs() if n_procs is None else n_procs
    chunks = np.array_split(np.arange(len(gens)), max(1, min(len(gens), 2 * n_procs)))
    jobs = [([_pack(gens[k]) for k in c], si, svals, vi, vv) for c in chunks if c.size]
    return np.concatenate(_map(_dots_job, jobs, n_procs, pool))


def _deriv_job(args):
    tabs, ops, thetas, j, psi_j = args
    pool = {k: _unpack(t) for k, t in tabs.items()}
    return sv.derivative_state_sparse(pool, ops, thetas, j, psi_j)


def derivative_states(pool: list[PauliTable], ops, thetas, kept: dict, n_procs: int | None = None,
                      workers=None) -> dict:
    """{j: d psi_P / d theta_j} (derivative_state_sparse) for every j in
    kept = {j: psi_j}, one j per job."""
    n_procs = procs() if n_procs is None else n_procs
    ops = [int(k) for k in ops]
    jobs = []
    for j, psi_j in kept.items():
        tabs = {k: _pack(pool[k]) for k in set(ops[j:])}
        jobs.append((tabs, ops, list(thetas), j, psi_j))
    return dict(zip(kept.keys(), _map(_deriv_job, jobs, n_procs, workers)))
