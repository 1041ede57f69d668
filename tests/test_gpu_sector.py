"""Sector layout (GOCP_BUILD_SECTOR) against the oracle and the full layout.

A sector-layout state holds the D determinants with the reference state's
alpha and beta electron counts.  Since H and the pool conserve both counts,
every result must equal the full-layout result restricted to those rows:

  * 4 and 14 qubits, complex128, JW and BK: the prepared state (expanded to
    2^n) equals the oracle's, and E, H psi, the pool gradients and dE/dtheta
    equal the oracle's / finite differences within 1e-10.
  * 14-24 qubits: sector and full layout agree (complex128 1e-10; complex64
    within the complex64 tolerances), the ADAPT selection is the same.
  * expand / compress round trips are exact; the server and the static energy
    entry point refuse sector problems.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15906_gb300 as gb  # noqa: E402
from oracle import mapping, pool as opool, statevector as sv  # noqa: E402
from synth import config_integrals, draw_ansatz, molecular_integrals, random_state  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2607_15906_gb300 import build
    build.build()
    gb.load()


def _host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.complex128).ravel()


def _pair(ints, n_elec, mp, prec, **kw):
    full = gb.Problem.build(ints, n_elec, mapping=mp, precision=prec, device=0, **kw)
    sec = gb.Problem.build(ints, n_elec, mapping=mp, precision=prec, device=0, sector=True, **kw)
    return full, sec


@pytest.mark.parametrize("n_orb,n_elec,mp", [(2, 2, "jw"), (2, 2, "bk"), (7, 6, "jw"), (7, 6, "bk"), (5, 3, "jw")])
def test_sector_matches_oracle_c128(n_orb, n_elec, mp):
    ints = molecular_integrals(n_orb, seed=n_orb + n_elec, decay=True)
    n = 2 * n_orb
    p = gb.Problem.build(ints, n_elec, mapping=mp, precision="c128", device=0, sector=True)
    na, nb = (n_elec + 1) // 2, n_elec // 2
    assert p.sector and p.dim == math.comb(n_orb, na) * math.comb(n_orb, nb)
    assert p.state_bytes() == 16 * p.dim
    h = mapping.hamiltonian_table(ints, mp)
    tabs = opool.pool_tables(n, n_elec, mp)
    ops, th = draw_ansatz(len(tabs), min(12, 3 * len(tabs)), seed=n, theta_sigma=0.3)
    ref0 = sv.basis_state(n, mapping.hf_index(mp, n, n_elec))
    ref = sv.prepare_state(ref0, tabs, ops, th)
    psi = p.new_states(1)[0]
    p.prepare_state(ops, th, psi)
    got = _host(p.expand(psi))
    assert np.max(np.abs(got - ref)) <= 1e-10
    # H psi and the energy
    hpsi = p.new_states(1)[0]
    e, nrm = p.energy(psi, hpsi)
    hr = sv.apply_terms(h, ref)
    assert abs(e - sv.energy(h, ref)) <= 1e-10 * max(1.0, abs(e))
    assert abs(nrm - np.vdot(ref, ref).real) <= 1e-10
    assert np.max(np.abs(_host(p.expand(hpsi)) - hr)) <= 1e-10 * max(1.0, np.max(np.abs(hr)))
    # pool gradients (Eq. 4)
    g = p.pool_gradients(psi, hpsi)
    assert np.max(np.abs(g - sv.pool_gradients(h, tabs, ref))) <= 1e-10
    # dE/dtheta by the adjoint sweep vs central differences of the oracle energy
    e2, de = p.energy_grad(ops, th)
    assert abs(e2 - e) <= 1e-12 * max(1.0, abs(e))
    for j in (0, len(ops) // 2, len(ops) - 1):
        tp, tm = th.copy(), th.copy()
        tp[j] += 1e-5
        tm[j] -= 1e-5
        hi = sv.energy(h, sv.prepare_state(ref0, tabs, ops, tp))
        lo = sv.energy(h, sv.prepare_state(ref0, tabs, ops, tm))
        assert abs((hi - lo) / 2e-5 - de[j]) <= 1e-7


def test_sector_round_trip_and_taylor_step():
    ints, c = config_integrals("c2_14q")
    full, sec = _pair(ints, 6, "jw", "c128")
    ops, th = draw_ansatz(full.pool_size, 20, seed=5, theta_sigma=0.2)
    pf = full.new_states(1)[0]
    full.prepare_state(ops, th, pf)
    ps = sec.compress(pf)
    back = sec.expand(ps)
    # the prepared state lives in the sector: compress/expand returns it exactly
    assert torch.equal(back, pf)
    assert torch.equal(sec.compress(back), ps)
    # one more Taylor step on the caller's state, both layouts
    full.taylor_step(int(ops[3]), 0.7, pf)
    sec.taylor_step(int(ops[3]), 0.7, ps)
    assert np.max(np.abs(_host(sec.expand(ps)) - _host(pf))) <= 1e-12


@pytest.mark.parametrize("cfg,n_elec,mp,prec,n_ops", [
    ("c2_14q", 6, "bk", "c128", 30),
    ("c3_20q", 10, "jw", "c128", 60),
    ("c3_20q", 10, "jw", "c64", 60),
    ("c5_24q", 8, "jw", "c64", 100),
])
def test_sector_matches_full_layout(cfg, n_elec, mp, prec, n_ops):
    ints, c = config_integrals(cfg)
    kw = dict(int_drop=c.get("int_drop", 0.0), term_drop=c.get("term_drop", 0.0))
    full, sec = _pair(ints, n_elec, mp, prec, **kw)
    ops, th = draw_ansatz(full.pool_size, n_ops, seed=0)
    tol = dict(c128=dict(s=1e-10, e=1e-10, g=1e-10), c64=dict(s=2e-5, e=1e-6, g=2e-6))[prec]
    # adapt step: energy, gradients, selection
    ef, nf, gf, sf = full.adapt_step(ops, th, tie_rel=1e-4)
    es, ns, gs, ss = sec.adapt_step(ops, th, tie_rel=1e-4)
    assert abs(es - ef) <= tol["e"] * max(1.0, abs(ef))
    assert abs(ns - nf) <= tol["e"]
    assert np.max(np.abs(gs - gf)) <= tol["g"] * max(1.0, np.max(np.abs(gf)))
    assert ss == sf
    # energy and dE/dtheta by the adjoint sweep
    e1, d1 = full.energy_grad(ops, th)
    e2, d2 = sec.energy_grad(ops, th)
    assert abs(e2 - e1) <= tol["e"] * max(1.0, abs(e1))
    assert np.max(np.abs(d2 - d1)) <= tol["g"] * max(1.0, np.max(np.abs(d1)))
    # prepared states and H psi agree on every row
    pf, hf = full.new_states(2)
    full.prepare_state(ops, th, pf)
    full.apply_h(pf, hf)
    ps, hs = sec.new_states(2)
    sec.prepare_state(ops, th, ps)
    sec.apply_h(ps, hs)
    a, b = _host(sec.expand(ps)), _host(pf)
    assert np.max(np.abs(a - b)) <= tol["s"]
    # H psi on the sector rows.  (Outside them the full-layout H psi is zero
    # only if H conserves the electron counts exactly; dropping Pauli terms
    # below term_drop (20 qubits) can leave ~1e-8 there, which the sector
    # layout does not hold and which no energy or gradient sees.)
    a, b = _host(hs), _host(sec.compress(hf))
    assert np.max(np.abs(a - b)) <= tol["s"] * max(1.0, np.max(np.abs(b)))
    if c.get("term_drop", 0.0) == 0.0:
        a, b = _host(sec.expand(hs)), _host(hf)
        assert np.max(np.abs(a - b)) <= tol["s"] * max(1.0, np.max(np.abs(b)))


def test_sector_dense_input_is_the_restriction():
    # H psi of a random (dense) sector state equals the full-layout H psi of
    # its expansion, restricted to the sector rows
    ints, c = config_integrals("c2_14q")
    full, sec = _pair(ints, 6, "jw", "c128")
    ps = sec.new_states(1)[0]
    rnd = random_state(14, seed=9)
    ps.copy_(sec.compress(torch.from_numpy(rnd).to("cuda:0")))
    hs = sec.new_states(1)[0]
    sec.apply_h(ps, hs)
    pf = sec.expand(ps)
    hf = full.new_states(1)[0]
    full.apply_h(pf, hf)
    want = _host(sec.compress(hf))
    assert np.max(np.abs(_host(hs) - want)) <= 1e-10 * np.max(np.abs(want))


def test_sector_rejections():
    ints, c = config_integrals("c1_4q")
    sec = gb.Problem.build(ints, 2, precision="c64", device=0, sector=True)
    psi, hpsi = sec.new_states(2)
    out = np.zeros(2)
    lib = gb.load()
    import ctypes as C
    rc = lib.gocp_energy_static(sec.handle, C.c_void_p(psi.data_ptr()), C.c_void_p(hpsi.data_ptr()),
                                out.ctypes.data_as(C.POINTER(C.c_double)), gb._lib.GOCP_MEM_HOST, None)
    assert rc == gb._lib.GOCP_EINVAL
    from paper_2607_15906_gb300.serving import Server
    srv = Server(hbm_budget_bytes=64 << 20, max_slots=4, device=0)
    try:
        with pytest.raises(gb._lib.GocpError) as e:
            srv.submit(sec, [0], [0.1])
        assert e.value.code == gb._lib.GOCP_EINVAL
    finally:
        srv.close()
    full = gb.Problem.build(ints, 2, precision="c64", device=0)
    with pytest.raises(gb._lib.GocpError):
        full.expand(full.new_states(1)[0])


def test_sector_28_qubits_vs_sparse_oracle():
    """28 qubits (14 orbitals, 8 electrons, integrals < 1e-3 dropped) in the
    sector layout: D = C(14,4)^2 = 1,002,001 rows.  E, a sample of pool
    gradients and dE/dtheta (central differences of the oracle energy)
    against the sparse oracle, complex64 tolerances."""
    ints = molecular_integrals(14, seed=0, decay=True)
    p = gb.Problem.build(ints, 8, precision="c64", int_drop=1e-3, device=0, sector=True)
    assert p.n_qubits == 28 and p.dim == math.comb(14, 4) ** 2
    h = mapping.hamiltonian_table(ints, "jw", 1e-3, 0.0)
    tabs = opool.pool_tables(28, 8, "jw")
    assert p.pool_size == len(tabs)
    ops, th = draw_ansatz(len(tabs), 6, seed=3, theta_sigma=0.3)
    ref = mapping.hf_index("jw", 28, 8)

    def sparse_energy(theta):
        si, sv_ = sv.prepare_state_sparse(ref, tabs, ops, theta)
        hi, hv = sv.apply_terms_sparse(h, si, sv_)
        return (sv.sparse_dot(si, sv_, hi, hv) / sv.sparse_dot(si, sv_, si, sv_)).real, si, sv_, hi, hv

    e_ref, si, svals, hi, hv = sparse_energy(th)
    nn = sv.sparse_dot(si, svals, si, svals).real
    e, nrm, g, sel = p.adapt_step(ops, th, tie_rel=1e-4)
    assert abs(e - e_ref) <= 1e-6
    rng = np.random.default_rng(0)
    for k in list(rng.integers(0, len(tabs), size=6)) + [sel]:
        ai, av = sv.apply_terms_sparse(tabs[int(k)], si, svals)
        gk = 2.0 * sv.sparse_dot(hi, hv, ai, av).real / nn
        assert abs(g[int(k)] - gk) <= 2e-6 * max(1.0, abs(gk))
    e2, de = p.energy_grad(ops, th)
    assert abs(e2 - e_ref) <= 1e-6
    for j in (0, 5):
        tp, tm = th.copy(), th.copy()
        tp[j] += 1e-4
        tm[j] -= 1e-4
        fd = (sparse_energy(tp)[0] - sparse_energy(tm)[0]) / 2e-4
        assert abs(de[j] - fd) <= 2e-5 * max(1.0, abs(fd))
