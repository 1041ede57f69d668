"""Molecular-shaped synthetic integrals.

The paper benchmarks real molecules (BeH2, H2O, LiH; Sec. IV) whose integrals
and geometries are not available here.  These seeded draws stand in for them
with the same shapes: a diagonal-dominant, symmetric one-electron matrix h_pq
and a Coulomb-dominant two-electron tensor (pq|rs) in chemist notation with
the 8-fold permutational symmetry of real orbitals, plus a constant energy
offset.  Off-diagonal elements optionally decay as exp(-|p-q|/3).

Draw order (fixed, so that any implementation reproduces the same numbers):
  1. h_pp = -U(0.5, 1.5) for p = 0..n-1, then sorted ascending, so that the
     lowest orbitals are the occupied ones of an aufbau reference.
  2. h_pq for p < q in row-major order: N(0, 0.1) * w(q - p).
  3. (pq|rs) over canonical quadruples p >= q, r >= s, pair(rs) <= pair(pq)
     with pair(pq) = p(p+1)/2 + q, iterated pq-major:
     U(0.3, 0.7) when p == q and r == s, else N(0, 0.05) * w(|p-q| + |r-s|).
     All 8 symmetric copies are filled.
  w(d) = exp(-d/3) when ``decay`` is set, else 1.  The constant is 0.7.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Integrals:
    """Spatial-orbital integrals: h (n,n), g (n,n,n,n) chemist (pq|rs), e0."""

    h: np.ndarray
    g: np.ndarray
    e0: float

    @property
    def n_orb(self) -> int:
        return int(self.h.shape[0])


def _w(d: int, decay: bool) -> float:
    return math.exp(-d / 3.0) if decay else 1.0


def molecular_integrals(n_orb: int, seed: int = 0, decay: bool = False,
                        e0: float = 0.7) -> Integrals:
    """Draw seeded integrals for ``n_orb`` spatial orbitals (see module doc)."""
    if n_orb < 1:
        raise ValueError("n_orb must be >= 1")
    rng = np.random.default_rng(seed)
    h = np.zeros((n_orb, n_orb), dtype=np.float64)
    diag = -rng.uniform(0.5, 1.5, size=n_orb)
    diag.sort()
    for p in range(n_orb):
        h[p, p] = diag[p]
    for p in range(n_orb):
        for q in range(p + 1, n_orb):
            v = float(rng.normal(0.0, 0.1)) * _w(q - p, decay)
            h[p, q] = v
            h[q, p] = v
    g = np.zeros((n_orb,) * 4, dtype=np.float64)
    pairs = [(p, q) for p in range(n_orb) for q in range(p + 1)]
    for ipq, (p, q) in enumerate(pairs):
        for irs in range(ipq + 1):
            r, s = pairs[irs]
            if p == q and r == s:
                v = float(rng.uniform(0.3, 0.7))
            else:
                v = float(rng.normal(0.0, 0.05)) * _w(abs(p - q) + abs(r - s), decay)
            for (a, b, c, d) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                                 (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
                g[a, b, c, d] = v
    return Integrals(h=h, g=g, e0=float(e0))


# Workload presets.  n_orb spatial orbitals -> 2*n_orb qubits; n_elec electrons
# in a closed-shell aufbau reference.  int_drop zeroes integrals with
# |value| < int_drop before mapping; term_drop removes mapped Pauli terms with
# |coeff| < term_drop.
CONFIGS = {
    "c1_4q": dict(n_orb=2, n_elec=2, decay=False, int_drop=0.0, term_drop=0.0, seed=0),
    "c2_14q": dict(n_orb=7, n_elec=6, decay=True, int_drop=0.0, term_drop=0.0, seed=0),
    "c3_20q": dict(n_orb=10, n_elec=10, decay=True, int_drop=0.0, term_drop=1e-6, seed=0),
    "c5_24q": dict(n_orb=12, n_elec=8, decay=True, int_drop=1e-3, term_drop=0.0, seed=0),
}


def config_integrals(name: str) -> tuple[Integrals, dict]:
    """Integrals and build parameters of a named preset."""
    cfg = dict(CONFIGS[name])
    ints = molecular_integrals(cfg["n_orb"], seed=cfg["seed"], decay=cfg["decay"])
    return ints, cfg
