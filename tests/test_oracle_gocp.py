"""Pins of GOCP (Sec. III.A, Algorithm 1)."""

import numpy as np
import pytest

import bruteforce as bf
from oracle import gocp, pool


@pytest.mark.parametrize("nq,ne,mp", [(6, 2, "jw"), (8, 4, "jw"), (8, 4, "bk")])
def test_exact_commutator_matches_dense(nq, ne, mp):
    tabs = pool.pool_tables(nq, ne, mp)
    dense = [bf.table_dense(t) for t in tabs]
    for i in range(len(tabs)):
        for j in range(len(tabs)):
            c = dense[i] @ dense[j] - dense[j] @ dense[i]
            assert gocp.commutes(tabs[i], tabs[j]) == (np.max(np.abs(c)) < 1e-12)


def test_largest_first_by_hand():
    # path 0-1-2-3: degrees 1,2,2,1 -> order 1,2,0,3 -> families 1:F0 2:F1 0:F1 3:F0
    adj = [{1}, {0, 2}, {1, 3}, {2}]
    assert gocp.largest_first_colouring(adj).tolist() == [1, 0, 1, 0]
    # star centre 4 with leaves 0..3 plus edge 0-1: order 4,0,1,2,3
    adj = [{4, 1}, {4, 0}, {4}, {4}, {0, 1, 2, 3}]
    assert gocp.largest_first_colouring(adj).tolist() == [1, 2, 1, 1, 0]
    # no edges: one family
    assert gocp.largest_first_colouring([set(), set(), set()]).tolist() == [0, 0, 0]
    # complete graph K4: four families, ties broken by index
    adj = [{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}]
    assert gocp.largest_first_colouring(adj).tolist() == [0, 1, 2, 3]


@pytest.mark.parametrize("nq,ne", [(8, 4), (12, 8)])
def test_colouring_valid_bounded_and_mapping_invariant(nq, ne):
    fam = {}
    for mp in ("jw", "bk"):
        tabs = pool.pool_tables(nq, ne, mp)
        adj = gocp.conflict_graph(tabs)
        f = gocp.largest_first_colouring(adj)
        for v in range(len(adj)):
            assert all(f[u] != f[v] for u in adj[v])            # families commute internally
        assert f.max() + 1 <= max(len(a) for a in adj) + 1      # K <= max degree + 1
        fam[mp] = (adj, f)
    assert fam["jw"][0] == fam["bk"][0]
    assert np.array_equal(fam["jw"][1], fam["bk"][1])


def test_disjoint_excitations_commute():
    nq, ne = 12, 4
    exc = pool.excitations(nq, ne)
    tabs = pool.pool_tables(nq, ne, "jw")
    for i in range(0, len(exc), 7):
        for j in range(0, len(exc), 5):
            si = set(exc[i].occ) | set(exc[i].virt)
            sj = set(exc[j].occ) | set(exc[j].virt)
            if not (si & sj):
                assert gocp.commutes(tabs[i], tabs[j])
