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


def _family_run(n_orb, n_elec, mp, seed, max_ops):
    from oracle import gocp
    ints = config_integrals("c1_4q")[0] if n_orb == 2 else __import__("synth").molecular_integrals(n_orb, seed=seed)
    n = 2 * n_orb
    h = mapping.hamiltonian_table(ints, mp)
    tabs = pool.pool_tables(n, n_elec, mp)
    fam = gocp.gocp(tabs)
    ref = sv.basis_state(n, mapping.hf_index(mp, n, n_elec))
    return ints, tabs, fam, adapt.adapt(h, tabs, ref, max_ops=max_ops, gtol=1e-4, families=fam)


def test_family_adapt_batches_commute_and_converge():
    """Family-batched ADAPT (the GOCP 'reduced search space' reading): every
    batch lies in one family and its generators commute as matrices (built
    from ladder operators, not from the oracle's tables); energies never
    rise; at 4 qubits the run reaches the N=2, S_z=0 ground state."""
    for n_orb, n_elec, mp, seed, max_ops in ((2, 2, "jw", 0, 10), (3, 2, "bk", 1, 12), (4, 4, "jw", 2, 12)):
        ints, tabs, fam, res = _family_run(n_orb, n_elec, mp, seed, max_ops)
        n = 2 * n_orb
        exc = pool.excitations(n, n_elec)
        assert len(res.energies) >= 2
        assert all(b <= a + 1e-12 for a, b in zip(res.energies, res.energies[1:]))
        # rebuild the batches: consecutive ops of one family added in one iteration
        batches, cur = [], []
        for k in res.ops:
            if cur and (fam[k] != fam[cur[-1]] or k <= cur[-1]):
                batches.append(cur)
                cur = []
            cur.append(k)
        batches.append(cur)
        for b in batches:
            mats = [bf.excitation_dense(n, exc[k].occ, exc[k].virt) for k in b]
            for i in range(len(mats)):
                for j in range(i + 1, len(mats)):
                    assert np.max(np.abs(mats[i] @ mats[j] - mats[j] @ mats[i])) < 1e-12
        if n_orb == 2:
            hd = bf.hamiltonian_dense(ints)
            nn, sz = bf.number_ops(4)
            sel = np.flatnonzero((nn == 2) & (sz == 0))
            e0 = np.linalg.eigvalsh(hd[np.ix_(sel, sel)])[0]
            assert res.converged and res.energies[-1] - e0 < 1e-7


def test_family_batch_rule():
    g = np.array([0.5, -0.3, 0.1, -0.45, 0.26])
    fam = np.array([0, 0, 1, 0, 0])
    assert adapt.family_batch(g, fam, 0, 0.5) == [0, 1, 3, 4]
    assert adapt.family_batch(g, fam, 0, 0.7) == [0, 3]
    assert adapt.family_batch(g, fam, 2, 0.5) == []      # the batch is that family's members above the bar
