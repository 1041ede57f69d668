"""Pins of the oracle's statevector functions (Eq. 1, 3, 4, 5, 6)."""

import math

import numpy as np
import pytest
import scipy.linalg as sla

import bruteforce as bf
from oracle import mapping, pool, statevector as sv
from oracle.pauli import PauliTable
from synth import molecular_integrals, random_state, config_integrals


def _random_table(n, t, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 1 << n, size=t)
    z = rng.integers(0, 1 << n, size=t)
    ph = rng.integers(0, 4, size=t)
    c = rng.normal(size=t)
    return PauliTable(n, x.astype(np.int64), z.astype(np.int64), ph.astype(np.int64), c)


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_apply_matches_kronecker_matrices(n):
    t = _random_table(n, 40, seed=n)
    psi = random_state(n, seed=100 + n)
    assert np.max(np.abs(sv.apply_terms(t, psi) - bf.table_dense(t) @ psi)) < 1e-12
    rows = np.arange(0, 1 << n, 3)
    assert np.max(np.abs(sv.apply_terms_at(t, psi, rows) - (bf.table_dense(t) @ psi)[rows])) < 1e-12


@pytest.mark.parametrize("mp", ["jw", "bk"])
def test_hamiltonian_apply_matches_ladder_matrix(mp):
    ints = molecular_integrals(4, seed=11, decay=True)
    t = mapping.hamiltonian_table(ints, mp)
    perm = bf.permutation_from_gf2(bf.srl_beta(8)) if mp == "bk" else np.eye(256)
    hd = perm @ bf.hamiltonian_dense(ints) @ perm.T
    psi = random_state(8, seed=5)
    assert np.max(np.abs(sv.apply_terms(t, psi) - hd @ psi)) < 1e-12
    e = sv.energy(t, psi)
    assert abs(e - np.vdot(psi, hd @ psi).real) < 1e-12


def test_taylor_chain_vs_expm_and_truncation_bound():
    nq, ne = 6, 2
    tabs = pool.pool_tables(nq, ne, "jw")
    psi = random_state(nq, seed=1)
    for t in tabs[:6]:
        a = bf.table_dense(t)
        for th in (0.05, -0.2, 0.7):
            exact = sla.expm(th * a) @ psi
            got = sv.taylor5(t, th, psi)
            # per active pair T5 - exp = (c5 - cos) I + (s5 - sin) A, ||A|| = 1
            bound = abs(th) ** 6 / 720 + abs(th) ** 7 / 5040 + 1e-14
            assert np.linalg.norm(got - exact) <= bound * 1.0001
            # closed form of the truncated series on each pair
            c5 = 1 - th ** 2 / 2 + th ** 4 / 24
            s5 = th - th ** 3 / 6 + th ** 5 / 120
            a2 = a @ a
            closed = psi + s5 * (a @ psi) + (1 - c5) * (a2 @ psi)
            assert np.max(np.abs(got - closed)) < 1e-14


def test_taylor_derivative_is_series_derivative():
    nq, ne = 6, 2
    tabs = pool.pool_tables(nq, ne, "jw")
    psi = random_state(nq, seed=2)
    h = 1e-6
    for t in tabs[::4]:
        for th in (0.1, -0.6):
            fd = (sv.taylor5(t, th + h, psi) - sv.taylor5(t, th - h, psi)) / (2 * h)
            assert np.max(np.abs(sv.taylor5_derivative(t, th, psi) - fd)) < 1e-9


def test_gradients_equal_commutator_and_append_derivative():
    ints = molecular_integrals(3, seed=4, decay=True)
    h = mapping.hamiltonian_table(ints, "jw")
    tabs = pool.pool_tables(6, 2, "jw")
    psi = random_state(6, seed=8)
    g = sv.pool_gradients(h, tabs, psi)
    hd = bf.table_dense(h)
    pn = psi / np.linalg.norm(psi)
    for k, t in enumerate(tabs):
        a = bf.table_dense(t)
        comm = np.vdot(pn, (hd @ a - a @ hd) @ pn)
        assert abs(comm.imag) < 1e-13
        assert abs(g[k] - comm.real) < 1e-12
        eps = 1e-5
        ep = sv.energy(h, sv.taylor5(t, eps, psi))
        em = sv.energy(h, sv.taylor5(t, -eps, psi))
        assert abs(g[k] - (ep - em) / (2 * eps)) < 1e-8


def test_energy_grad_forward_mode_vs_central_differences():
    ints = molecular_integrals(3, seed=2, decay=True)
    h = mapping.hamiltonian_table(ints, "jw")
    tabs = pool.pool_tables(6, 2, "jw")
    ref = sv.basis_state(6, mapping.hf_index("jw", 6, 2))
    rng = np.random.default_rng(3)
    ops = rng.integers(0, len(tabs), size=6)
    th = rng.normal(0, 0.3, size=6)
    e, grad = sv.energy_grad(h, ref, tabs, ops, th)
    assert abs(e - sv.energy(h, sv.prepare_state(ref, tabs, ops, th))) < 1e-14
    hstep = 1e-5
    for j in range(len(ops)):
        tp, tm = th.copy(), th.copy()
        tp[j] += hstep
        tm[j] -= hstep
        fd = (sv.energy(h, sv.prepare_state(ref, tabs, ops, tp))
              - sv.energy(h, sv.prepare_state(ref, tabs, ops, tm))) / (2 * hstep)
        assert abs(fd - grad[j]) < 1e-8


def test_rayleigh_quotient_scale_invariant_and_fidelity():
    ints, c = config_integrals("c1_4q")
    h = mapping.hamiltonian_table(ints, "jw")
    psi = random_state(4, seed=0, normalize=False)
    assert abs(sv.energy(h, psi) - sv.energy(h, 3.7 * psi)) < 1e-13
    assert abs(sv.fidelity(psi, (0.5 - 2j) * psi) - 1.0) < 1e-14
    other = random_state(4, seed=1)
    assert sv.fidelity(psi, other) < 1.0


def test_sector_preserved_by_taylor():
    nq, ne = 8, 4
    tabs = pool.pool_tables(nq, ne, "jw")
    ref = sv.basis_state(nq, mapping.hf_index("jw", nq, ne))
    rng = np.random.default_rng(0)
    psi = sv.prepare_state(ref, tabs, rng.integers(0, len(tabs), 12), rng.normal(0, 0.3, 12))
    nn, sz = bf.number_ops(nq)
    outside = (nn != ne) | (sz != 0)
    # exact arithmetic keeps the sector; string-by-string float sums leave
    # only rounding residue outside it
    assert np.max(np.abs(psi[outside])) < 1e-15
    assert np.linalg.norm(psi[~outside]) > 0.9


def test_sparse_paths_equal_dense():
    ints = molecular_integrals(4, seed=7, decay=True)
    h = mapping.hamiltonian_table(ints, "jw")
    tabs = pool.pool_tables(8, 4, "jw")
    hf = mapping.hf_index("jw", 8, 4)
    rng = np.random.default_rng(1)
    ops, th = rng.integers(0, len(tabs), 9), rng.normal(0, 0.3, 9)
    dense = sv.prepare_state(sv.basis_state(8, hf), tabs, ops, th)
    si, svals = sv.prepare_state_sparse(hf, tabs, ops, th)
    rebuilt = np.zeros(256, np.complex128)
    rebuilt[si] = svals
    assert np.max(np.abs(rebuilt - dense)) < 1e-14
    hi, hv = sv.apply_terms_sparse(h, si, svals)
    hd = np.zeros(256, np.complex128)
    hd[hi] = hv
    assert np.max(np.abs(hd - sv.apply_terms(h, dense))) < 1e-13
    assert abs(sv.sparse_dot(si, svals, hi, hv) - np.vdot(dense, hd)) < 1e-13


def test_sparse_group_apply_derivative_and_intermediates_equal_dense():
    """apply_group_sparse (a generator's strings summed per basis state
    before the product) equals the term-by-term dense apply; the sparse
    derivative state and the kept intermediate states equal their dense
    forward-mode counterparts; exact zeros are not held."""
    nq, ne = 8, 4
    tabs = pool.pool_tables(nq, ne, "bk")
    hf = mapping.hf_index("bk", nq, ne)
    rng = np.random.default_rng(5)
    ops, th = rng.integers(0, len(tabs), 7), rng.normal(0, 0.3, 7)
    ref = sv.basis_state(nq, hf)
    si, svals, kept = sv.prepare_state_sparse(hf, tabs, ops, th, keep_at=[0, 3, 6])
    assert np.all(svals != 0)
    dense = sv.prepare_state(ref, tabs, ops, th)
    for k in (0, len(tabs) // 2, len(tabs) - 1):
        ai, av = sv.apply_group_sparse(tabs[k], si, svals)
        assert np.all(av != 0) and np.all(np.diff(ai) > 0)
        back = np.zeros(1 << nq, np.complex128)
        back[ai] = av
        assert np.max(np.abs(back - sv.apply_terms(tabs[k], dense))) < 1e-14
    for j in (0, 3, 6):
        pre = np.zeros(1 << nq, np.complex128)
        pre[kept[j][0]] = kept[j][1]
        assert np.max(np.abs(pre - sv.prepare_state(ref, tabs, ops[:j], th[:j]))) < 1e-14
        di, dv = sv.derivative_state_sparse(tabs, ops, th, j, kept[j])
        d = ref.copy()
        for i, (k, t) in enumerate(zip(ops, th)):
            d = sv.taylor5_derivative(tabs[k], t, d) if i == j else sv.taylor5(tabs[k], t, d)
        got = np.zeros(1 << nq, np.complex128)
        got[di] = dv
        assert np.max(np.abs(got - d)) < 1e-14


def test_parallel_oracle_equals_serial():
    """oracle.parallel (spawned workers over slices) gives the serial oracle's
    H psi rows and pool gradients."""
    from oracle import parallel
    ints = molecular_integrals(4, seed=3, decay=True)
    h = mapping.hamiltonian_table(ints, "jw")
    tabs = pool.pool_tables(8, 4, "jw")
    hf = mapping.hf_index("jw", 8, 4)
    rng = np.random.default_rng(2)
    ops, th = rng.integers(0, len(tabs), 6), rng.normal(0, 0.3, 6)
    si, svals = sv.prepare_state_sparse(hf, tabs, ops, th)
    dense = np.zeros(256, np.complex128)
    dense[si] = svals
    rows = np.flatnonzero(parallel.generator_support(tabs, si, svals, n_procs=2) | (dense != 0))
    hrows = parallel.hpsi_rows(h, si, svals, rows, n_procs=2)
    assert np.max(np.abs(hrows - sv.apply_terms(h, dense)[rows])) < 1e-13
    nrm = float(np.vdot(dense, dense).real)
    g = parallel.pool_gradients(tabs, si, svals, rows, hrows, nrm, n_procs=2)
    assert np.max(np.abs(g - sv.pool_gradients(h, tabs, dense))) < 1e-13
    hi = rows[hrows != 0]
    dots = parallel.generator_dots(tabs, si, svals, hi, hrows[hrows != 0], n_procs=2)
    assert np.max(np.abs(dots / nrm - g)) < 1e-13
    _, _, kept = sv.prepare_state_sparse(hf, tabs, ops, th, keep_at=[1, 4])
    ds = parallel.derivative_states(tabs, ops, th, kept, n_procs=2)
    for j in (1, 4):
        di, dv = sv.derivative_state_sparse(tabs, ops, th, j, kept[j])
        assert np.array_equal(ds[j][0], di) and np.array_equal(ds[j][1], dv)
