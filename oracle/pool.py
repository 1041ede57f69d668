"""Spin-conserving singles + doubles excitation pool (Sec. II.B, Table II).

Occupied spin-orbitals are 0..N_e-1 (closed-shell aufbau reference), virtual
ones N_e..n-1; spin-orbital i has spin i % 2.  Generators are anti-Hermitian
with unit coefficient:

    singles  tau = a+_a a_i - a+_i a_a,            i occ, a virt, same spin,
    doubles  tau = a+_a a+_b a_j a_i - h.c.,       i<j occ, a<b virt,
                                                   spin(i)+spin(j) = spin(a)+spin(b).

Order: all singles by (i, a), then all doubles by (i, j, a, b).  The counts
reproduce Table II: 92 operators at 12 qubits / 8 electrons and 204 at
14 qubits / 6 electrons.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from .mapping import encoding, expand_products
from .pauli import PauliTable, accumulate_exact


@dataclasses.dataclass
class Excitation:
    kind: str              # "single" | "double"
    occ: tuple             # (i,) or (i, j)
    virt: tuple            # (a,) or (a, b)


def excitations(n_qubits: int, n_elec: int) -> list[Excitation]:
    occ = list(range(n_elec))
    virt = list(range(n_elec, n_qubits))
    out = []
    for i in occ:
        for a in virt:
            if i % 2 == a % 2:
                out.append(Excitation("single", (i,), (a,)))
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for ia, a in enumerate(virt):
                for b in virt[ia + 1:]:
                    if (i % 2) + (j % 2) == (a % 2) + (b % 2):
                        out.append(Excitation("double", (i, j), (a, b)))
    return out


def generator_table(exc: Excitation, mapping: str, n_qubits: int) -> PauliTable:
    """Pauli strings of tau = E - E^dagger for one excitation."""
    enc = encoding(mapping, n_qubits)
    if exc.kind == "single":
        (i,), (a,) = exc.occ, exc.virt
        fwd = np.array([[a, i]])
        bwd = np.array([[i, a]])
        dag = (True, False)
    else:
        (i, j), (a, b) = exc.occ, exc.virt
        fwd = np.array([[a, b, j, i]])           # a+_a a+_b a_j a_i
        bwd = np.array([[i, j, b, a]])           # its adjoint a+_i a+_j a_b a_a
        dag = (True, True, False, False)
    x1, z1, v1 = expand_products(enc, fwd, dag, np.array([1.0]))
    x2, z2, v2 = expand_products(enc, bwd, dag, np.array([-1.0]))
    return accumulate_exact(np.concatenate([x1, x2]), np.concatenate([z1, z2]),
                            np.concatenate([v1, v2]), n_qubits)


def pool_tables(n_qubits: int, n_elec: int, mapping: str) -> list[PauliTable]:
    return [generator_table(e, mapping, n_qubits) for e in excitations(n_qubits, n_elec)]
