"""The C++ host builder behind the C ABI, bit-exact against the oracle.

Runs without a GPU: problems are built with device = -1 (host tables only).
"""

import math
import re
import os

import numpy as np
import pytest

from oracle import gocp as ogocp, mapping, pool as opool
from oracle.pauli import PauliTable, accumulate_exact
from synth import config_integrals, molecular_integrals

gb = pytest.importorskip("paper_2607_15906_gb300")


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2607_15906_gb300 import build
    build.build()
    gb.load()


def _host(ints, n_elec, mp, int_drop=0.0, term_drop=0.0, colour=True):
    return gb.Problem.build(ints, n_elec, mapping=mp, int_drop=int_drop, term_drop=term_drop,
                            device=-1, colour=colour)


@pytest.mark.parametrize("cfg,n_elec", [("c1_4q", 2), ("c2_14q", 6), ("c3_20q", 10), ("c5_24q", 8)])
@pytest.mark.parametrize("mp", ["jw", "bk"])
def test_hamiltonian_table_bit_exact(cfg, n_elec, mp):
    ints, c = config_integrals(cfg)
    ref = mapping.hamiltonian_table(ints, mp, c["int_drop"], c["term_drop"])
    p = _host(ints, n_elec, mp, c["int_drop"], c["term_drop"], colour=False)
    x, z, ph, co = p.terms()
    assert np.array_equal(x.astype(np.int64), ref.x)
    assert np.array_equal(z.astype(np.int64), ref.z)
    assert np.array_equal(ph.astype(np.int64), ref.phase)
    assert np.array_equal(co.view(np.int64), ref.coeff.view(np.int64))
    assert p.info["n_groups"] == len(np.unique(ref.x))
    assert p.info["ref_index"] == mapping.hf_index(mp, ref.n, n_elec)


@pytest.mark.parametrize("mp", ["jw", "bk"])
def test_hamiltonian_table_bit_exact_32_qubits(mp):
    """16 spatial orbitals, the largest problem: the top qubit (bit 31 of
    the masks) is in use, and the tables still match the oracle bit for
    bit; 17 orbitals and 33 table qubits are refused."""
    ints = molecular_integrals(16, seed=0, decay=True)
    ref = mapping.hamiltonian_table(ints, mp, 1e-3, 0.0)
    p = _host(ints, 8, mp, 1e-3, 0.0, colour=False)
    x, z, ph, co = p.terms()
    assert p.info["n_qubits"] == 32 and (int(np.max(ref.x | ref.z)) >> 31) == 1
    assert np.array_equal(x.astype(np.int64), ref.x)
    assert np.array_equal(z.astype(np.int64), ref.z)
    assert np.array_equal(ph.astype(np.int64), ref.phase)
    assert np.array_equal(co.view(np.int64), ref.coeff.view(np.int64))
    assert p.info["ref_index"] == mapping.hf_index(mp, 32, 8)
    with pytest.raises(gb.GocpError):
        _host(molecular_integrals(17, seed=0, decay=True), 8, mp, 1e-3, 0.0, colour=False)
    with pytest.raises(gb.GocpError):
        gb.Problem.from_tables(33, ([1], [0], [0], [1.0]), [], ref_index=0, device=-1)


@pytest.mark.parametrize("nq,ne", [(4, 2), (12, 8), (14, 6)])
@pytest.mark.parametrize("mp", ["jw", "bk"])
def test_pool_and_gocp_bit_exact(nq, ne, mp):
    ints = molecular_integrals(nq // 2, seed=3, decay=True)
    p = _host(ints, ne, mp)
    off, x, z, ph, co, fam = p.pool()
    tabs = opool.pool_tables(nq, ne, mp)
    assert p.pool_size == len(tabs)
    for k, t in enumerate(tabs):
        s = slice(off[k], off[k + 1])
        assert np.array_equal(x[s].astype(np.int64), t.x)
        assert np.array_equal(z[s].astype(np.int64), t.z)
        assert np.array_equal(co[s], t.coeff)
        assert np.all(ph[s] == 0)
    ref_fam = ogocp.gocp(tabs)
    assert np.array_equal(fam.astype(np.int64), ref_fam)
    assert p.info["n_families"] == ref_fam.max() + 1


def test_pool_sizes_large():
    for nq, ne, m in [(20, 10, 875), (24, 8, 1424)]:
        ints = molecular_integrals(nq // 2, seed=0, decay=True)
        p = _host(ints, ne, "jw", colour=False)
        assert p.pool_size == m


def test_exact_sum_matches_fsum():
    rng = np.random.default_rng(0)
    for trial in range(200):
        n = int(rng.integers(1, 60))
        v = rng.normal(size=n) * 10.0 ** rng.integers(-30, 30, size=n)
        if trial % 3 == 0:                           # heavy cancellation
            v = np.concatenate([v, -v[: n // 2], [1e-300, -1e-300, 5e-324]])
        got = gb.exact_sum(v)
        assert got == math.fsum(v.tolist()) or (got == 0 and math.fsum(v.tolist()) == 0)
    assert gb.exact_sum([1e308, 1e308, -1e308]) == 1e308
    assert gb.exact_sum([0.1] * 10) == math.fsum([0.1] * 10)
    assert gb.exact_sum([]) == 0.0
    # ties round to even
    assert gb.exact_sum([1.0, 2.0 ** -53]) == 1.0
    assert gb.exact_sum([1.0 + 2.0 ** -52, 2.0 ** -53]) == 1.0 + 2.0 ** -51


def test_tables_are_canonicalised_exactly():
    rng = np.random.default_rng(5)
    n, t = 6, 300
    x = rng.integers(0, 1 << n, size=t).astype(np.uint32)
    z = rng.integers(0, 1 << n, size=t).astype(np.uint32)
    x[100:200] = x[:100]; z[100:200] = z[:100]            # duplicates
    ph = np.zeros(t, np.uint8)
    ph[::2] = 2                                           # sign flips only: real
    c = rng.normal(size=t)
    p = gb.Problem.from_tables(n, (x, z, ph, c), [], ref_index=0, device=-1)
    gx, gz, gph, gc = p.terms()
    ref = accumulate_exact(x.astype(np.int64), z.astype(np.int64),
                           np.where(ph == 2, -c, c), n)
    assert np.array_equal(gx.astype(np.int64), ref.x) and np.array_equal(gz.astype(np.int64), ref.z)
    assert np.array_equal(gc.view(np.int64), ref.coeff.view(np.int64))


def test_bad_arguments_are_rejected():
    ints = molecular_integrals(2, seed=0)
    with pytest.raises(gb.GocpError):
        gb.Problem.build(ints, 7, device=-1)                      # too many electrons
    with pytest.raises(gb.GocpError):
        gb.Problem.from_tables(3, ([1], [0], [0], [1.0]), [([1, 2], [0, 0], [0, 0], [1.0, 1.0])],
                               ref_index=0, device=-1)            # generator with two x masks
    with pytest.raises(gb.GocpError):
        gb.Problem.from_tables(3, ([9], [0], [0], [1.0]), [], ref_index=0, device=-1)  # mask > n
    p = gb.Problem.build(ints, 2, device=-1)
    import ctypes
    with pytest.raises(gb.GocpError) as e:
        from paper_2607_15906_gb300._lib import check, load
        check(load().gocp_apply_h(p.handle, ctypes.c_void_p(1), ctypes.c_void_p(2), None))
    assert e.value.code == -7                                     # ENODEV: host-only problem


def test_sector_layout_dimensions_host_only():
    """GOCP_BUILD_SECTOR: D = C(n_orb, ceil(N/2)) C(n_orb, floor(N/2)) amplitudes
    per state; table-built problems and host-only compute calls are refused."""
    import ctypes
    import math
    for n_orb, n_elec in ((2, 2), (5, 3), (7, 6), (12, 8)):
        ints = molecular_integrals(n_orb, seed=1)
        p = gb.Problem.build(ints, n_elec, device=-1, sector=True, colour=False)
        d = math.comb(n_orb, (n_elec + 1) // 2) * math.comb(n_orb, n_elec // 2)
        assert p.info["sector"] == 1 and p.info["state_dim"] == d == p.dim
        assert (p.info["n_alpha"], p.info["n_beta"]) == ((n_elec + 1) // 2, n_elec // 2)
        assert p.state_bytes() == 8 * d
        f = gb.Problem.build(ints, n_elec, device=-1, colour=False)
        assert f.info["sector"] == 0 and f.dim == 1 << (2 * n_orb)
    with pytest.raises(gb.GocpError) as e:
        from paper_2607_15906_gb300._lib import check, load
        check(load().gocp_sector_expand(p.handle, ctypes.c_void_p(1), ctypes.c_void_p(2), None))
    assert e.value.code == -7
    from paper_2607_15906_gb300 import _lib
    x = np.array([1], np.uint32)
    z = np.array([0], np.uint32)
    ph = np.array([0], np.uint8)
    c = np.array([1.0])
    args = _lib.TableArgs(n_qubits=2, precision=0, device=-1, flags=0, n_terms=1,
                          x=x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                          z=z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                          phase=ph.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                          coeff=c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    out = ctypes.c_void_p()
    assert load().gocp_build_from_tables(ctypes.byref(args), ctypes.byref(out)) == 0
    load().gocp_problem_free(out)
    args.flags = _lib.GOCP_BUILD_SECTOR                           # the same tables, sector layout
    assert load().gocp_build_from_tables(ctypes.byref(args), ctypes.byref(out)) == -1
    assert b"integrals" in load().gocp_last_error()


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "gocp.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(gocp_[a-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 25
    lib = gb.load()
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_server_needs_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2607_15906_gb300.serving import Server
    with pytest.raises(gb.GocpError) as e:
        Server(hbm_budget_bytes=1 << 20)
    assert e.value.code in (-7, -1)
