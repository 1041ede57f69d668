"""Pins of the ADAPT loop (Sec. II.B) on the 4-qubit case."""

import numpy as np

import bruteforce as bf
from oracle import adapt, mapping, pool, statevector as sv
from synth import config_integrals


def _run(mp):
    ints, c = config_integrals("c1_4q")
    h = mapping.hamiltonian_table(ints, mp)
    tabs = pool.pool_tables(4, 2, mp)
    ref = sv.basis_state(4, mapping.hf_index(mp, 4, 2))
    return ints, h, adapt.adapt(h, tabs, ref, max_ops=10, gtol=1e-4)


def test_adapt_4q_reaches_sector_ground_state():
    ints, h, res = _run("jw")
    assert res.converged
    # the N=2, S_z=0 sector of 4 spin-orbitals is 4-dimensional and the pool
    # (2 singles + 1 double) spans it, so ADAPT reaches the sector minimum
    hd = bf.hamiltonian_dense(ints)
    nn, sz = bf.number_ops(4)
    sel = np.flatnonzero((nn == 2) & (sz == 0))
    e0 = np.linalg.eigvalsh(hd[np.ix_(sel, sel)])[0]
    assert res.energies[-1] >= e0 - 1e-12                 # variational
    assert res.energies[-1] - e0 < 1e-7
    assert all(b <= a + 1e-12 for a, b in zip(res.energies, res.energies[1:]))


def test_adapt_trajectory_mapping_invariant():
    _, _, jw = _run("jw")
    _, _, bk = _run("bk")
    assert jw.ops == bk.ops
    assert np.max(np.abs(np.array(jw.energies) - np.array(bk.energies))) < 1e-10


def test_selection_tie_rule():
    g = np.array([0.1, -0.3, 0.3 * (1 - 1e-10), 0.29])
    assert adapt.select(g, 1e-8) == 1
    g = np.array([0.1, 0.3 * (1 - 1e-10), -0.3, 0.29])
    assert adapt.select(g, 1e-8) == 1
    assert adapt.select(np.array([0.2, 0.29, -0.3]), 0.1) == 1
