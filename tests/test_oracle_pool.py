"""Pins of the excitation pool (Sec. II.B, Table II, Sec. III.B)."""

import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import bruteforce as bf
from oracle import mapping, pool
from oracle.pauli import parity

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("row", GOLDEN["table2_pool_sizes"])
def test_pool_sizes_match_table2(row):
    assert len(pool.excitations(row["qubits"], row["electrons"])) == row["pool"]


@pytest.mark.parametrize("nq,ne,count", [(4, 2, 3), (20, 10, 875), (24, 8, 1424)])
def test_pool_sizes_closed_form(nq, ne, count):
    # singles 2*o*v, doubles 2*C(o,2)*C(v,2) + o^2 v^2 with o, v occupied/virtual spatial orbitals
    o, v = ne // 2, (nq - ne) // 2
    closed = 2 * o * v + 2 * (o * (o - 1) // 2) * (v * (v - 1) // 2) + o * o * v * v
    assert closed == count
    assert len(pool.excitations(nq, ne)) == count


@pytest.mark.parametrize("nq,ne", [(4, 2), (6, 2), (8, 4)])
@pytest.mark.parametrize("mp", ["jw", "bk"])
def test_generators_equal_ladder_matrices(nq, ne, mp):
    perm = bf.permutation_from_gf2(bf.srl_beta(nq)) if mp == "bk" else np.eye(1 << nq)
    for exc in pool.excitations(nq, ne):
        t = pool.generator_table(exc, mp, nq)
        ref = perm @ bf.excitation_dense(nq, exc.occ, exc.virt) @ perm.T
        assert np.max(np.abs(bf.table_dense(t) - ref)) < 1e-14


@pytest.mark.parametrize("mp", ["jw", "bk"])
def test_generator_structure(mp):
    nq, ne = 8, 4
    for exc in pool.excitations(nq, ne):
        t = pool.generator_table(exc, mp, nq)
        assert len(np.unique(t.x)) == 1 and t.x[0] != 0          # one x-group
        assert len(t) == (2 if exc.kind == "single" else 8)
        assert np.all(parity(t.x & t.z) == 1)                    # anti-Hermitian strings
        assert set(np.abs(t.coeff).tolist()) == ({0.5} if exc.kind == "single" else {0.125})


def test_generators_anti_hermitian_cube_and_closed_form_exponential():
    nq, ne = 6, 2
    for exc in pool.excitations(nq, ne):
        a = bf.table_dense(pool.generator_table(exc, "jw", nq))
        assert np.max(np.abs(a + a.conj().T)) == 0.0
        a2 = a @ a
        assert np.max(np.abs(a2 @ a + a)) < 1e-14                 # A^3 = -A (A^2 = -projector)
        assert np.max(np.abs(a2 @ a2 + a2)) < 1e-14
        for th in (0.3, -1.1):
            closed = np.eye(1 << nq) + np.sin(th) * a + (1 - np.cos(th)) * a2
            assert np.max(np.abs(sla.expm(th * a) - closed)) < 1e-12


def test_pool_generators_clifford_image_between_mappings():
    nq, ne = 10, 4
    beta = mapping.bk_matrix(nq)
    bit = mapping.gf2_inverse(beta).T
    for exc in pool.excitations(nq, ne):
        jw = pool.generator_table(exc, "jw", nq)
        bk = pool.generator_table(exc, "bk", nq)
        ix = np.array([mapping.matvec_mask(beta, int(v)) for v in jw.x])
        iz = np.array([mapping.matvec_mask(bit, int(v)) for v in jw.z])
        o = np.lexsort((iz, ix))
        assert np.array_equal(ix[o], bk.x) and np.array_equal(iz[o], bk.z)
        assert np.array_equal(jw.coeff[o], bk.coeff)
