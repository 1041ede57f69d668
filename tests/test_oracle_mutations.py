"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
notice them: a dropped sign, a transposed operand, a dropped term, a wrong
factor, a reversed order."""

import math

import numpy as np
import pytest
import scipy.linalg as sla

import bruteforce as bf
from oracle import gocp, mapping, pool, statevector as sv
from synth import molecular_integrals, random_state


def _ham_error(ints):
    t = mapping.hamiltonian_table(ints, "jw")
    return np.max(np.abs(bf.table_dense(t) - bf.hamiltonian_dense(ints)))


def test_dropped_jordan_wigner_sign_is_caught(monkeypatch):
    ints = molecular_integrals(3, seed=1, decay=True)
    assert _ham_error(ints) < 1e-12
    monkeypatch.setattr(mapping, "parity", lambda a: np.zeros_like(np.asarray(a)))
    assert _ham_error(ints) > 1e-3


def test_transposed_bk_operand_is_caught(monkeypatch):
    ints = molecular_integrals(3, seed=2, decay=True)
    perm = bf.permutation_from_gf2(bf.srl_beta(6))
    ref = perm @ bf.hamiltonian_dense(ints) @ perm.T
    monkeypatch.setattr(mapping.Encoding, "beta_inv_t", property(lambda self: self.beta.T.copy()))
    t = mapping.hamiltonian_table(ints, "bk")
    assert np.max(np.abs(bf.table_dense(t) - ref)) > 1e-3


def test_dropped_fifth_order_is_caught(monkeypatch):
    tabs = pool.pool_tables(6, 2, "jw")
    psi = random_state(6, seed=1)
    a = bf.table_dense(tabs[0])
    th = 0.7

    def truncated(t, theta, p):
        out, v = p.copy(), p
        for m in range(1, 5):
            v = sv.apply_terms(t, v)
            out = out + theta ** m / math.factorial(m) * v
        return out

    monkeypatch.setattr(sv, "taylor5", truncated)
    got = sv.taylor5(tabs[0], th, psi)
    bound = abs(th) ** 6 / 720 + abs(th) ** 7 / 5040
    assert np.linalg.norm(got - sla.expm(th * a) @ psi) > bound


def test_missing_gradient_factor_is_caught(monkeypatch):
    ints = molecular_integrals(3, seed=4, decay=True)
    h = mapping.hamiltonian_table(ints, "jw")
    tabs = pool.pool_tables(6, 2, "jw")
    psi = random_state(6, seed=8)
    orig = sv.pool_gradients

    monkeypatch.setattr(sv, "pool_gradients", lambda h_, p_, s_: 0.5 * orig(h_, p_, s_))
    g = sv.pool_gradients(h, tabs, psi)
    eps = 1e-5
    fd = [(sv.energy(h, sv.taylor5(t, eps, psi)) - sv.energy(h, sv.taylor5(t, -eps, psi))) / (2 * eps)
          for t in tabs]
    assert np.max(np.abs(g - np.array(fd))) > 1e-4


def test_reversed_degree_order_is_caught():
    adj = [{4, 1}, {4, 0}, {4}, {4}, {0, 1, 2, 3}]
    good = gocp.largest_first_colouring(adj).tolist()
    # smallest-first order gives a different colouring of the same graph
    m = len(adj)
    order = sorted(range(m), key=lambda v: (len(adj[v]), v))
    fam = [-1] * m
    for v in order:
        taken = {fam[u] for u in adj[v] if fam[u] >= 0}
        k = 0
        while k in taken:
            k += 1
        fam[v] = k
    assert fam != good == [1, 2, 1, 1, 0]
