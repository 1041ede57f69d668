"""Pins of the oracle's qubit mappings (Eq. 2 -> Eq. 3, Sec. II.A).

Each check compares against a construction that does not reuse the oracle's
bit formulas: sparse ladder matrices built from occupation-number action,
Kronecker-product Pauli matrices, the recursive SRL Bravyi-Kitaev matrix, the
Slater-Condon closed form, and exact algebraic invariants.
"""

import json
import os

import numpy as np
import pytest

import bruteforce as bf
from oracle import mapping
from oracle.pauli import parity, popcount
from synth import molecular_integrals, config_integrals

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("n_orb,seed,decay", [(2, 0, False), (3, 1, True), (4, 2, True)])
def test_jw_table_equals_ladder_hamiltonian(n_orb, seed, decay):
    ints = molecular_integrals(n_orb, seed=seed, decay=decay)
    t = mapping.hamiltonian_table(ints, "jw")
    dense = bf.hamiltonian_dense(ints)
    assert np.max(np.abs(bf.table_dense(t) - dense)) < 1e-12


@pytest.mark.parametrize("n_orb,seed", [(2, 0), (3, 3), (4, 4)])
def test_bk_table_equals_permuted_ladder_hamiltonian(n_orb, seed):
    ints = molecular_integrals(n_orb, seed=seed, decay=True)
    n = 2 * n_orb
    t = mapping.hamiltonian_table(ints, "bk")
    perm = bf.permutation_from_gf2(bf.srl_beta(n))
    dense = perm @ bf.hamiltonian_dense(ints) @ perm.T
    assert np.max(np.abs(bf.table_dense(t) - dense)) < 1e-12


@pytest.mark.parametrize("n", list(range(1, 25)))
def test_fenwick_bk_matrix_equals_srl_recursion(n):
    assert np.array_equal(mapping.bk_matrix(n), bf.srl_beta(n))


def test_bk_weight_is_logarithmic():
    for n in (8, 16, 24, 32):
        enc = mapping.bravyi_kitaev(n)
        worst = 0
        for j in range(n):
            x, zp, ze = enc.ladder(j)
            worst = max(worst, bin(x | zp | ze).count("1"))
        assert worst <= 2 * int(np.ceil(np.log2(n))) + 1


@pytest.mark.parametrize("cfg", ["c1_4q", "c2_14q", "c3_20q"])
def test_bk_table_is_clifford_image_of_jw(cfg):
    ints, c = config_integrals(cfg)
    jw = mapping.hamiltonian_table(ints, "jw", c["int_drop"], c["term_drop"])
    bk = mapping.hamiltonian_table(ints, "bk", c["int_drop"], c["term_drop"])
    n = jw.n
    beta = mapping.bk_matrix(n)
    bit = mapping.gf2_inverse(beta).T
    img_x = np.array([mapping.matvec_mask(beta, int(v)) for v in jw.x])
    img_z = np.array([mapping.matvec_mask(bit, int(v)) for v in jw.z])
    order = np.lexsort((img_z, img_x))
    assert np.array_equal(img_x[order], bk.x)
    assert np.array_equal(img_z[order], bk.z)
    # bit-exact coefficients: the same exact sums, rounded once
    assert np.array_equal(jw.coeff[order].view(np.int64), bk.coeff.view(np.int64))
    assert len(np.unique(jw.x)) == len(np.unique(bk.x))


@pytest.mark.parametrize("cfg", ["c1_4q", "c2_14q", "c5_24q"])
def test_terms_hermitian_and_sorted(cfg):
    ints, c = config_integrals(cfg)
    for mp in ("jw", "bk"):
        t = mapping.hamiltonian_table(ints, mp, c["int_drop"], c["term_drop"])
        # c X^x Z^z is Hermitian with real c iff popc(x & z) is even
        assert np.all(parity(t.x & t.z) == 0)
        assert np.all(t.phase == 0)
        keys = t.x * (1 << 32) + t.z
        assert np.all(np.diff(keys) > 0)
        assert np.all(t.coeff != 0)


@pytest.mark.parametrize("cfg,n_elec", [("c1_4q", 2), ("c2_14q", 6), ("c3_20q", 10)])
def test_hf_energy_is_slater_condon(cfg, n_elec):
    ints, c = config_integrals(cfg)
    for mp in ("jw", "bk"):
        t = mapping.hamiltonian_table(ints, mp, c["int_drop"], 0.0)
        hf = mapping.hf_index(mp, t.n, n_elec)
        diag = t.x == 0
        e = np.sum(t.coeff[diag] * (1 - 2 * parity(np.int64(hf) & t.z[diag])))
        assert abs(e - bf.slater_condon_hf(ints, n_elec)) < 1e-12


def test_hf_reference_indices():
    assert mapping.hf_index("jw", 4, 2) == 0b0011
    assert mapping.hf_index("bk", 4, 2) == 0b0001


@pytest.mark.parametrize("n_orb,seed", [(2, 0), (3, 5), (4, 6)])
def test_jw_bk_spectra_equal(n_orb, seed):
    ints = molecular_integrals(n_orb, seed=seed, decay=True)
    ejw = np.linalg.eigvalsh(bf.table_dense(mapping.hamiltonian_table(ints, "jw")))
    ebk = np.linalg.eigvalsh(bf.table_dense(mapping.hamiltonian_table(ints, "bk")))
    assert np.max(np.abs(ejw - ebk)) < 1e-11


def test_number_and_spin_conserved():
    ints = molecular_integrals(3, seed=9, decay=False)
    hd = bf.table_dense(mapping.hamiltonian_table(ints, "jw"))
    nn, sz = bf.number_ops(6)
    assert np.max(np.abs(hd * (nn[:, None] - nn[None, :]))) < 1e-14
    assert np.max(np.abs(hd * (sz[:, None] - sz[None, :]))) < 1e-14


def test_drops_are_strict_thresholds():
    ints, c = config_integrals("c3_20q")
    t = mapping.hamiltonian_table(ints, "jw", 0.0, 1e-6)
    assert np.all(np.abs(t.coeff) >= 1e-6)
    full = mapping.hamiltonian_table(ints, "jw", 0.0, 0.0)
    assert len(full) > len(t)


def test_table1_manifold_constant():
    g = GOLDEN["table1_manifold"]
    assert (1 << g["qubits"]) ** 2 == g["elements"]
    assert abs(g["elements"] - g["printed"]) / g["printed"] < 0.005
    d = GOLDEN["dense_bytes_complex128_14q"]
    assert g["elements"] * 16 == d["bytes"]
    assert abs(d["bytes"] / 1e9 - d["printed_gb"]) < 0.05


def test_popcount_matches_python():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 1 << 32, size=1000)
    assert np.array_equal(popcount(a), np.array([bin(int(v)).count("1") for v in a]))
