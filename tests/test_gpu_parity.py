"""CUDA path vs the oracle, element by element, through the C ABI.

Tolerances, the same in every test, with no per-test multipliers:
  complex128: 1e-10 relative on every quantity (states and H psi relative to
              their largest entry, E to max(1, |E|), gradients and
              dE/dtheta to max(1, their largest magnitude)).
  complex64 : |E - E_oracle| <= 1e-6 Ha relative to max(1, |E|) and
              fidelity >= 1 - 1e-6 (the precision targets); states and H psi
              within 2e-5 of their largest entry; gradients and dE/dtheta
              within 2e-6 of max(1, their largest magnitude).  The last two
              follow from FP32 rounding: an entry of H psi sums about G
              products of |D| <= 5 in FP32 (relative error 6e-8 each), so its
              error is about sqrt(G) 6e-8 5 ~ 1e-5 |psi| at G ~ 4000 groups;
              a gradient is a sum of such entries times amplitudes of a
              normalised state, so its error stays below ~1e-6.
Each comparison prints its error over its tolerance (`pytest -s`).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15906_gb300 as gb  # noqa: E402
from oracle import mapping, pool as opool, statevector as sv  # noqa: E402
from oracle.pauli import PauliTable, parity  # noqa: E402
from synth import config_integrals, draw_ansatz, molecular_integrals, random_state  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL = {"c128": dict(state=1e-10, energy=1e-10, grad=1e-10),
       "c64": dict(state=2e-5, energy=1e-6, grad=2e-6)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2607_15906_gb300 import build
    build.build()
    gb.load()


def _within(what, err, tol):
    """err <= tol, with the ratio printed for the record."""
    print(f"TOLCHECK {what}: err {err:.3e} tol {tol:.3e} ratio {err / tol if tol else float('inf'):.3f}")
    assert err <= tol, (what, err, tol)


def _to_dev(p, psi):
    dt = np.complex64 if p.precision == "c64" else np.complex128
    return torch.from_numpy(psi.astype(dt)).to(f"cuda:{p.device}")


def _host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.complex128).ravel()


def _case(n_orb, n_elec, mp, seed=0, decay=True, int_drop=0.0, term_drop=0.0):
    ints = molecular_integrals(n_orb, seed=seed, decay=decay)
    h = mapping.hamiltonian_table(ints, mp, int_drop, term_drop)
    tabs = opool.pool_tables(2 * n_orb, n_elec, mp)
    return ints, h, tabs


SMALL = [(2, 2, "jw", 0), (3, 2, "bk", 1), (4, 4, "jw", 2), (5, 4, "bk", 3), (5, 6, "jw", 4), (7, 6, "jw", 0)]


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n_orb,n_elec,mp,seed", SMALL)
def test_apply_h_and_energy(prec, n_orb, n_elec, mp, seed):
    ints, h, _ = _case(n_orb, n_elec, mp, seed)
    p = gb.Problem.build(ints, n_elec, mapping=mp, precision=prec, device=0)
    n = 2 * n_orb
    psi = random_state(n, seed=10 + seed)
    d = _to_dev(p, psi)
    psi_in = _host(d)                          # the rounded input the kernel saw
    hd = torch.empty_like(d)
    e, nrm = p.energy(d, hd)
    ref = sv.apply_terms(h, psi_in)
    got = _host(hd)
    scale = np.max(np.abs(ref))
    _within(f"apply_h {prec} {n_orb}o hpsi", np.max(np.abs(got - ref)), TOL[prec]["state"] * scale)
    e_ref = sv.energy(h, psi_in)
    _within(f"apply_h {prec} {n_orb}o E", abs(e - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))
    assert abs(nrm - np.vdot(psi_in, psi_in).real) <= 1e-12
    # apply without the energy epilogue gives the same vector
    h2 = torch.empty_like(d)
    p.apply_h(d, h2)
    assert np.array_equal(_host(h2), got)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n_orb,n_elec,mp,seed", SMALL[:5])
def test_prepare_state_and_fidelity(prec, n_orb, n_elec, mp, seed):
    ints, h, tabs = _case(n_orb, n_elec, mp, seed)
    p = gb.Problem.build(ints, n_elec, mapping=mp, precision=prec, device=0)
    n = 2 * n_orb
    ops, th = draw_ansatz(len(tabs), 12, seed=seed, theta_sigma=0.3)
    ref = sv.prepare_state(sv.basis_state(n, p.info["ref_index"]), tabs, ops, th)
    d = p.new_states(1)[0]
    p.prepare_state(ops, th, d)
    got = _host(d)
    _within(f"prepare {prec} {n_orb}o psi", np.max(np.abs(got - ref)), TOL[prec]["state"] * np.max(np.abs(ref)))
    _within(f"prepare {prec} {n_orb}o 1-F", 1.0 - sv.fidelity(got, ref), 1e-12 if prec == "c128" else 1e-6)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_single_taylor_step_on_random_state(prec):
    ints, h, tabs = _case(5, 4, "jw", 6)
    p = gb.Problem.build(ints, 4, precision=prec, device=0)
    psi = random_state(10, seed=1)
    for k in (0, 7, len(tabs) - 1):
        d = _to_dev(p, psi)
        psi_in = _host(d)
        p.taylor_step(k, 0.37, d)
        ref = sv.taylor5(tabs[k], 0.37, psi_in)
        _within(f"taylor_step {prec} op {k}", np.max(np.abs(_host(d) - ref)), TOL[prec]["state"] * np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n_orb,n_elec,mp,seed", [(3, 2, "jw", 0), (5, 4, "bk", 1), (7, 6, "jw", 0)])
def test_pool_gradients(prec, n_orb, n_elec, mp, seed):
    ints, h, tabs = _case(n_orb, n_elec, mp, seed)
    p = gb.Problem.build(ints, n_elec, mapping=mp, precision=prec, device=0)
    n = 2 * n_orb
    ops, th = draw_ansatz(len(tabs), 6, seed=seed, theta_sigma=0.3)
    ws = p.workspace()
    p.prepare_state(ops, th, ws[0])
    p.energy(ws[0], ws[1])
    g = p.pool_gradients(ws[0], ws[1])
    psi_in = _host(ws[0])
    g_ref = sv.pool_gradients(h, tabs, psi_in)
    _within(f"pool_gradients {prec} {n_orb}o", np.max(np.abs(g - g_ref)),
            TOL[prec]["grad"] * max(1.0, np.max(np.abs(g_ref))))


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n_orb,n_elec,mp,seed", [(2, 2, "jw", 0), (3, 2, "bk", 2), (4, 4, "jw", 3)])
def test_energy_grad_adjoint(prec, n_orb, n_elec, mp, seed):
    ints, h, tabs = _case(n_orb, n_elec, mp, seed)
    p = gb.Problem.build(ints, n_elec, mapping=mp, precision=prec, device=0)
    n = 2 * n_orb
    ops, th = draw_ansatz(len(tabs), 8, seed=seed, theta_sigma=0.3)
    e, de = p.energy_grad(ops, th)
    ref = sv.basis_state(n, p.info["ref_index"])
    e_ref, de_ref = sv.energy_grad(h, ref, tabs, ops, th)
    _within(f"energy_grad {prec} {n_orb}o E", abs(e - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))
    _within(f"energy_grad {prec} {n_orb}o dE", np.max(np.abs(de - de_ref)),
            TOL[prec]["grad"] * max(1.0, np.max(np.abs(de_ref))))
    if prec == "c128":
        hs = 1e-5
        for j in range(len(ops)):
            tp, tm = th.copy(), th.copy()
            tp[j] += hs
            tm[j] -= hs
            fd = (sv.energy(h, sv.prepare_state(ref, tabs, ops, tp))
                  - sv.energy(h, sv.prepare_state(ref, tabs, ops, tm))) / (2 * hs)
            assert abs(de[j] - fd) < 1e-8


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_adapt_step_selection(prec):
    ints, h, tabs = _case(4, 4, "jw", 5)
    p = gb.Problem.build(ints, 4, precision=prec, device=0)
    ops, th = draw_ansatz(len(tabs), 3, seed=5, theta_sigma=0.2)
    e, nrm, g, sel = p.adapt_step(ops, th, tie_rel=1e-8 if prec == "c128" else 1e-4)
    psi = sv.prepare_state(sv.basis_state(8, p.info["ref_index"]), tabs, ops, th)
    g_ref = sv.pool_gradients(h, tabs, psi)
    mag = np.abs(g_ref)
    allowed = np.flatnonzero(mag >= mag.max() * (1 - 1e-3))
    assert sel == allowed.min()
    e_ref = sv.energy(h, psi)
    _within(f"adapt_step {prec} E", abs(e - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))


def _hermitian_random_table(n, t, rng, anti=False):
    x = rng.integers(0, 1 << n, size=t)
    z = rng.integers(0, 1 << n, size=t)
    base = parity(x & z) ^ (1 if anti else 0)
    ph = base + 2 * rng.integers(0, 2, size=t)       # c i^ph X^x Z^z (anti-)Hermitian
    c = rng.integers(-8, 9, size=t) / 8.0 if anti else rng.normal(size=t)
    c[c == 0] = 0.125
    return PauliTable(n, x.astype(np.int64), z.astype(np.int64), ph.astype(np.int64), c)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 11])
def test_random_tables_with_phases(prec, n):
    rng = np.random.default_rng(n)
    H = _hermitian_random_table(n, 5 * n + 3, rng)
    gens = []
    for _ in range(4):
        x = int(rng.integers(1, 1 << n))
        z = rng.integers(0, 1 << n, size=3).astype(np.int64)
        ph = (parity(x & z) ^ 1) + 2 * rng.integers(0, 2, size=3)    # anti-Hermitian strings
        c = rng.integers(1, 9, size=3) / 8.0
        gens.append(PauliTable(n, np.full(3, x, np.int64), z, ph.astype(np.int64), c))
    to_t = lambda t: (t.x.astype(np.uint32), t.z.astype(np.uint32), (t.phase % 4).astype(np.uint8), t.coeff)
    try:
        p = gb.Problem.from_tables(n, to_t(H), [to_t(g) for g in gens], ref_index=0, precision=prec, device=0)
    except gb.GocpError:
        pytest.skip("random generator summed to zero")
    psi = random_state(n, seed=3 * n)
    d = _to_dev(p, psi)
    psi_in = _host(d)
    hd = torch.empty_like(d)
    e, _ = p.energy(d, hd)
    ref = sv.apply_terms(H, psi_in)
    _within(f"random table {prec} {n}q hpsi", np.max(np.abs(_host(hd) - ref)), TOL[prec]["state"] * np.max(np.abs(ref)))
    # generator tables as the library canonicalised them
    off, gx, gz, gph, gc, fam = p.pool()
    tabs = [PauliTable(n, gx[off[k]:off[k + 1]].astype(np.int64), gz[off[k]:off[k + 1]].astype(np.int64),
                       gph[off[k]:off[k + 1]].astype(np.int64), gc[off[k]:off[k + 1]]) for k in range(len(gens))]
    ops, th = np.array([0, 1, 2, 3, 1], np.int32), np.array([0.3, -0.2, 0.5, 0.1, -0.4])
    d2 = p.new_states(1)[0]
    p.prepare_state(ops, th, d2)
    sref = sv.prepare_state(sv.basis_state(n, 0), tabs, ops, th)
    _within(f"random table {prec} {n}q psi", np.max(np.abs(_host(d2) - sref)), TOL[prec]["state"] * np.max(np.abs(sref)))
    e2, de = p.energy_grad(ops, th)
    e_ref, de_ref = sv.energy_grad(H, sv.basis_state(n, 0), tabs, ops, th)
    _within(f"random table {prec} {n}q E", abs(e2 - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))
    _within(f"random table {prec} {n}q dE", np.max(np.abs(de - de_ref)),
            TOL[prec]["grad"] * max(1.0, np.max(np.abs(de_ref))))


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [8, 10])
def test_chain_list_overflow_falls_back(prec, n):
    """Tracked Taylor and adjoint chains follow a list of the state's nonzero
    amplitudes, with room for a quarter of them; generators with one-qubit x
    masks spread |0> over all 2^n amplitudes, so the list overflows part-way
    through the forward chain (and before the adjoint sweep) and the steps
    enumerate pairs from there on.  States, E and dE/dtheta against the oracle."""
    rng = np.random.default_rng(40 + n)
    H = _hermitian_random_table(n, 6 * n, rng)
    gens = []
    for q in range(n):
        x = 1 << q
        z = rng.integers(0, 1 << n, size=2).astype(np.int64)
        ph = (parity(x & z) ^ 1) + 2 * rng.integers(0, 2, size=2)    # anti-Hermitian strings
        c = rng.integers(1, 9, size=2) / 8.0
        gens.append(PauliTable(n, np.full(2, x, np.int64), z, ph.astype(np.int64), c))
    to_t = lambda t: (t.x.astype(np.uint32), t.z.astype(np.uint32), (t.phase % 4).astype(np.uint8), t.coeff)
    try:
        p = gb.Problem.from_tables(n, to_t(H), [to_t(g) for g in gens], ref_index=0, precision=prec, device=0)
    except gb.GocpError:
        pytest.skip("random generator summed to zero")
    off, gx, gz, gph, gc, fam = p.pool()
    tabs = [PauliTable(n, gx[off[k]:off[k + 1]].astype(np.int64), gz[off[k]:off[k + 1]].astype(np.int64),
                       gph[off[k]:off[k + 1]].astype(np.int64), gc[off[k]:off[k + 1]]) for k in range(len(gens))]
    ops = np.concatenate([np.arange(len(tabs)), rng.permutation(len(tabs))[:4]]).astype(np.int32)
    th = rng.uniform(0.2, 0.7, size=len(ops)) * rng.choice([-1.0, 1.0], size=len(ops))
    d = p.new_states(1)[0]
    p.prepare_state(ops, th, d)
    sref = sv.prepare_state(sv.basis_state(n, 0), tabs, ops, th)
    assert np.count_nonzero(sref) > (1 << n) // 4
    _within(f"overflow {prec} {n}q psi", np.max(np.abs(_host(d) - sref)), TOL[prec]["state"] * np.max(np.abs(sref)))
    e2, de = p.energy_grad(ops, th)
    e_ref, de_ref = sv.energy_grad(H, sv.basis_state(n, 0), tabs, ops, th)
    _within(f"overflow {prec} {n}q E", abs(e2 - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))
    _within(f"overflow {prec} {n}q dE", np.max(np.abs(de - de_ref)),
            TOL[prec]["grad"] * max(1.0, np.max(np.abs(de_ref))))


def _grouped_random_table(n, rng):
    """A Hermitian table with x-groups of 1..40 terms (z-ranks from 0 to
    beyond the LUT limit), real and imaginary weights, a diagonal group, one
    exactly paired group (z, w), (z ^ x, -w) of the one-body form (x of
    even weight, as e_p ^ e_q: then both partners are Hermitian with weights
    on the same axis), and one group whose masks lie within one bit of a
    centre (the one-body-with-spectators shape, with real and imaginary
    weights)."""
    xs, zs = [], []
    for size in [1, 2, 3, 4, 6, 8, 9, 12, 17, 25, 40, 5, 7]:
        x = int(rng.integers(1, 1 << n))
        xs += [x] * size
        zs += list(rng.integers(0, 1 << n, size=size))
    xs += [0] * 20                                     # diagonal group
    zs += list(rng.integers(0, 1 << n, size=20))
    x, z = np.array(xs, np.int64), np.array(zs, np.int64)
    ph = parity(x & z) + 2 * rng.integers(0, 2, size=len(x))     # c i^ph X^x Z^z Hermitian
    c = rng.normal(size=len(x))
    q = rng.choice(n, size=2, replace=False)           # paired group: x = e_q0 ^ e_q1
    xp = (1 << int(q[0])) | (1 << int(q[1]))
    zp = rng.integers(0, 1 << n, size=10)
    zp = zp[(zp & xp) != xp]                           # one of each pair {z, z ^ x}
    zp = np.unique(np.where((zp >> int(q.min())) & 1, zp ^ xp, zp))
    php = parity(xp & zp) + 2 * rng.integers(0, 2, size=len(zp))
    cp = rng.normal(size=len(zp))
    x = np.concatenate([x, np.full(2 * len(zp), xp, np.int64)])
    z = np.concatenate([z, zp, zp ^ xp])
    ph = np.concatenate([ph, php, php ^ 2])            # partner: same c, opposite sign
    c = np.concatenate([c, cp, cp])
    # a group whose masks lie within one bit of a centre, the flipped bits
    # partly inside x (so its weights are real and imaginary)
    xl = int(rng.integers(1, 1 << n))
    zc = int(rng.integers(0, 1 << n))
    zl = np.array([zc] + [zc ^ (1 << int(r)) for r in rng.choice(n, size=min(n, 11), replace=False)], np.int64)
    phl = parity(xl & zl) + 2 * rng.integers(0, 2, size=len(zl))
    x = np.concatenate([x, np.full(len(zl), xl, np.int64)])
    z = np.concatenate([z, zl])
    ph = np.concatenate([ph, phl])
    c = np.concatenate([c, rng.normal(size=len(zl))])
    return PauliTable(n, x, z, ph.astype(np.int64), c)


@pytest.fixture(params=["auto", "staged", "scatter"])
def hpsi_path(request, monkeypatch):
    """Which tiled H psi kernel runs: chosen from the live-octet count (auto),
    the staged kernel for every state, or the scatter kernel for every state."""
    frac = {"auto": None, "staged": "0", "scatter": "1"}[request.param]
    if frac is None:
        monkeypatch.delenv("GOCP_SPARSE_FRAC", raising=False)
    else:
        monkeypatch.setenv("GOCP_SPARSE_FRAC", frac)
    return request.param


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [12, 13, 15, 16])
def test_tiled_h_random_grouped_tables(prec, n, hpsi_path):
    """H psi through the tiled kernels (one tile at n = 12 complex128 / 13
    complex64, several above): LUT groups, term lists with imaginary weights,
    a paired group, x masks over all bits; a dense random state (no octet is
    skipped) and a sparse one (most octets skipped), each through the staged
    kernel, the scatter kernel and the automatic choice."""
    rng = np.random.default_rng(100 + n)
    H = _grouped_random_table(n, rng)
    to_t = lambda t: (t.x.astype(np.uint32), t.z.astype(np.uint32), (t.phase % 4).astype(np.uint8), t.coeff)
    p = gb.Problem.from_tables(n, to_t(H), [], ref_index=0, precision=prec, device=0)
    for kind in ("dense", "sparse"):
        psi = random_state(n, seed=7 * n)
        if kind == "sparse":
            keep = np.zeros(1 << n, bool)
            keep[np.random.default_rng(n).integers(0, 1 << n, size=40)] = True
            psi = np.where(keep, psi, 0)
        d = _to_dev(p, psi)
        psi_in = _host(d)
        hd = torch.empty_like(d)
        e, nrm = p.energy(d, hd)
        ref = sv.apply_terms(H, psi_in)
        _within(f"grouped {prec} {n}q {kind} {hpsi_path} hpsi", np.max(np.abs(_host(hd) - ref)),
                TOL[prec]["state"] * np.max(np.abs(ref)))
        e_ref = np.vdot(psi_in, ref).real / np.vdot(psi_in, psi_in).real
        _within(f"grouped {prec} {n}q {kind} {hpsi_path} E", abs(e - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("path", ["staged", "scatter"])
def test_tiled_h_on_sector_states(prec, path, monkeypatch):
    """Prepared ADAPT states (16 qubits, 8 electrons: only the N = 8, S_z = 0
    determinants are nonzero, a quarter of the octets at most) through the
    staged and the scatter H psi kernel: every entry of H psi and the energy
    against the oracle, and the pool gradients that read H psi."""
    monkeypatch.setenv("GOCP_SPARSE_FRAC", "0" if path == "staged" else "1")
    ints, h, tabs = _case(8, 8, "jw", 5)
    p = gb.Problem.build(ints, 8, precision=prec, device=0)
    ops, th = draw_ansatz(len(tabs), 24, seed=5, theta_sigma=0.3)
    ws = p.workspace()
    p.prepare_state(ops, th, ws[0])
    psi_in = _host(ws[0])
    live = np.any(psi_in.reshape(-1, 8) != 0, axis=1).mean()
    assert 0 < live <= 0.25
    e, nrm = p.energy(ws[0], ws[1])
    ref = sv.apply_terms(h, psi_in)
    _within(f"sector state {prec} {path} hpsi", np.max(np.abs(_host(ws[1]) - ref)), TOL[prec]["state"] * np.max(np.abs(ref)))
    e_ref = np.vdot(psi_in, ref).real / np.vdot(psi_in, psi_in).real
    _within(f"sector state {prec} {path} E", abs(e - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))
    e2, _, g, sel = p.adapt_step(ops, th, ws=ws, tie_rel=1e-4)
    g_ref = sv.pool_gradients(h, tabs, psi_in)
    _within(f"sector state {prec} {path} E2", abs(e2 - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))
    _within(f"sector state {prec} {path} grads", np.max(np.abs(g - g_ref)),
            TOL[prec]["grad"] * max(1.0, np.max(np.abs(g_ref))))


@pytest.mark.parametrize("prec,scale", [("c128", 1e-150), ("c128", 1e150), ("c64", 1e-30), ("c64", 1e30)])
def test_scatter_h_at_extreme_scales(prec, scale, monkeypatch):
    """The scatter kernel's fixed-point scale 2^F follows the largest
    amplitude, and complex128 forms its products as integers (weights at
    2^Fd, amplitudes at 2^(F + 63 - Fd)): a sector state with random phases
    (complex amplitudes), scaled by 1e+-150 (complex128) or 1e+-30
    (complex64), gives scale x the oracle's H psi entry by entry and the
    same energy, with no device error."""
    monkeypatch.setenv("GOCP_SPARSE_FRAC", "1")
    ints, h, tabs = _case(8, 8, "jw", 5)
    p = gb.Problem.build(ints, 8, precision=prec, device=0)
    ops, th = draw_ansatz(len(tabs), 24, seed=5, theta_sigma=0.3)
    ws = p.workspace()
    p.prepare_state(ops, th, ws[0])
    base = _host(ws[0])
    phase = np.exp(2j * np.pi * np.random.default_rng(11).random(base.size))
    psi_in = base * phase * scale
    d = _to_dev(p, psi_in)
    hd = torch.empty_like(d)
    e, nrm = p.energy(d, hd)
    assert p.device_errors() == 0
    ref = sv.apply_terms(h, psi_in)
    _within(f"scaled {prec} {scale:g} hpsi", np.max(np.abs(_host(hd) - ref)), TOL[prec]["state"] * np.max(np.abs(ref)))
    e_ref = np.vdot(psi_in, ref).real / np.vdot(psi_in, psi_in).real
    _within(f"scaled {prec} {scale:g} E", abs(e - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n_orb,n_elec", [(7, 6), (8, 8), (9, 8)])
def test_scatter_tile_split_is_bit_identical(prec, n_orb, n_elec, monkeypatch):
    """With few output tiles the scatter kernel lets several blocks share a
    tile and adds their 64-bit fixed-point accumulators in global memory:
    H psi and E equal, bit for bit, the one-block-per-tile result
    (GOCP_SCATTER_PARTS=1), and E the oracle's."""
    ints = molecular_integrals(n_orb, seed=0, decay=True)
    h = mapping.hamiltonian_table(ints, "jw", 1e-3, 0.0)
    p = gb.Problem.build(ints, n_elec, precision=prec, int_drop=1e-3, device=0, colour=False)
    ops, th = draw_ansatz(p.pool_size, 40, seed=2, theta_sigma=0.3)
    ws = p.workspace()
    p.prepare_state(ops, th, ws[0])
    out = {}
    for parts in ("1", "64"):
        monkeypatch.setenv("GOCP_SCATTER_PARTS", parts)
        hd = torch.empty_like(ws[0])
        e, nrm = p.energy(ws[0], hd)
        out[parts] = (hd, e, nrm)
    assert torch.equal(out["1"][0], out["64"][0])
    assert out["1"][1] == out["64"][1] and out["1"][2] == out["64"][2]
    if prec == "c64":   # split accumulator words against the carry form, both tile splits
        for parts in ("1", "64"):
            monkeypatch.setenv("GOCP_SCATTER_PARTS", parts)
            monkeypatch.setenv("GOCP_SCATTER_SPLIT", "0")
            hd = torch.empty_like(ws[0])
            e, nrm = p.energy(ws[0], hd)
            monkeypatch.delenv("GOCP_SCATTER_SPLIT")
            assert torch.equal(out["1"][0], hd) and out["1"][1] == e and out["1"][2] == nrm
    assert p.device_errors() == 0
    psi_in = _host(ws[0])
    ref = sv.apply_terms(h, psi_in)
    e_ref = np.vdot(psi_in, ref).real / np.vdot(psi_in, psi_in).real
    _within(f"split {prec} {2 * n_orb}q E", abs(out["64"][1] - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))
    _within(f"split {prec} {2 * n_orb}q hpsi", np.max(np.abs(_host(out["64"][0]) - ref)),
            TOL[prec]["state"] * np.max(np.abs(ref)))
    p.close()


def test_empty_ansatz_gives_reference_energy():
    ints, h, tabs = _case(4, 4, "bk", 1)
    p = gb.Problem.build(ints, 4, mapping="bk", precision="c128", device=0)
    e, de = p.energy_grad(np.zeros(0, np.int32), np.zeros(0))
    assert de.size == 0
    hf = sv.basis_state(8, mapping.hf_index("bk", 8, 4))
    assert abs(e - sv.energy(h, hf)) < 1e-12


def test_device_ansatz_out_of_range_is_flagged_not_faulted():
    ints, h, tabs = _case(3, 2, "jw", 0)
    p = gb.Problem.build(ints, 2, precision="c128", device=0)
    ops = torch.tensor([0, 99, 1], dtype=torch.int32, device="cuda:0")
    th = torch.tensor([0.1, 0.2, 0.3], dtype=torch.float64, device="cuda:0")
    d = p.new_states(1)[0]
    p.prepare_state(ops, th, d)
    assert p.device_errors() == 1
    ref = sv.prepare_state(sv.basis_state(6, p.info["ref_index"]), tabs, [0, 1], [0.1, 0.3])
    assert np.max(np.abs(_host(d) - ref)) < 1e-12   # the bad operator acted as identity
    assert p.device_errors() == 0
    with pytest.raises(gb.GocpError):
        p.prepare_state(np.array([0, 99]), np.array([0.1, 0.2]), d)   # host arrays are checked up front


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_full_size_20q_sampled_rows(prec):
    ints, c = config_integrals("c3_20q")
    h = mapping.hamiltonian_table(ints, "jw", c["int_drop"], c["term_drop"])
    p = gb.Problem.build(ints, 10, precision=prec, term_drop=c["term_drop"], device=0)
    psi = random_state(20, seed=77)
    d = _to_dev(p, psi)
    psi_in = _host(d)
    hd = torch.empty_like(d)
    e, nrm = p.energy(d, hd)
    rows = np.random.default_rng(0).integers(0, 1 << 20, size=48)
    rows = np.concatenate([rows, [0, (1 << 20) - 1, p.info["ref_index"]]])
    ref = sv.apply_terms_at(h, psi_in, rows)
    got = _host(hd)[rows]
    scale = np.max(np.abs(ref))
    _within(f"20q rows {prec}", np.max(np.abs(got - ref)), TOL[prec]["state"] * scale)


@pytest.mark.parametrize("path", ["auto", "staged"])
def test_full_size_24q_sparse_prepare_energy_gradients(path, monkeypatch):
    """The 24-qubit ADAPT step (the automatic choice takes the scatter H psi
    kernel for these states) against the sparse oracle."""
    if path == "staged":
        monkeypatch.setenv("GOCP_SPARSE_FRAC", "0")
    else:
        monkeypatch.delenv("GOCP_SPARSE_FRAC", raising=False)
    ints, c = config_integrals("c5_24q")
    h = mapping.hamiltonian_table(ints, "jw", c["int_drop"], c["term_drop"])
    tabs = opool.pool_tables(24, 8, "jw")
    p = gb.Problem.build(ints, 8, precision="c64", int_drop=c["int_drop"], device=0)
    ops, th = draw_ansatz(len(tabs), 6, seed=0, theta_sigma=0.3)
    ws = p.workspace()
    e2, nrm, g, sel = p.adapt_step(ops, th, ws=ws, tie_rel=1e-4)
    si, svals = sv.prepare_state_sparse(p.info["ref_index"], tabs, ops, th)
    got = _host(ws[0])
    ref = np.zeros(1 << 24, np.complex128)
    ref[si] = svals
    _within(f"24q 6-op {path} psi", np.max(np.abs(got - ref)), TOL["c64"]["state"] * np.max(np.abs(ref)))
    _within(f"24q 6-op {path} 1-F", 1.0 - sv.fidelity(got, ref), 1e-6)
    hi, hv = sv.apply_terms_sparse(h, si, svals)
    nn = sv.sparse_dot(si, svals, si, svals).real
    e_ref = sv.sparse_dot(si, svals, hi, hv).real / nn
    _within(f"24q 6-op {path} E", abs(e2 - e_ref), TOL["c64"]["energy"] * max(1.0, abs(e_ref)))
    gs = {}
    for k in list(range(0, len(tabs), 97)) + [int(np.argmax(np.abs(g)))]:
        ai, av = sv.apply_terms_sparse(tabs[k], si, svals)
        gs[k] = 2 * sv.sparse_dot(hi, hv, ai, av).real / nn
    gscale = max(1.0, max(abs(v) for v in gs.values()))
    _within(f"24q 6-op {path} grads", max(abs(g[k] - v) for k, v in gs.items()), TOL["c64"]["grad"] * gscale)


def test_larger_n_26q_c64():
    """26 qubits (13 orbitals, 12 electrons, integrals < 1e-3 dropped): a
    512 MiB complex64 state.  Sampled rows of H psi for a random state, and a
    sparse prepared state's energy, against the oracle."""
    ints = molecular_integrals(13, seed=0, decay=True)
    h = mapping.hamiltonian_table(ints, "jw", 1e-3, 0.0)
    p = gb.Problem.build(ints, 12, precision="c64", int_drop=1e-3, device=0, colour=False)
    assert p.n_qubits == 26 and p.info["n_terms"] == len(h)
    psi = random_state(26, seed=26)
    d = _to_dev(p, psi)
    del psi
    psi_in = _host(d)
    hd = torch.empty_like(d)
    p.energy(d, hd)
    rows = np.concatenate([np.random.default_rng(1).integers(0, 1 << 26, size=24), [0, (1 << 26) - 1]])
    ref = sv.apply_terms_at(h, psi_in, rows)
    got = _host(hd)[rows]
    _within("26q rows", np.max(np.abs(got - ref)), TOL["c64"]["state"] * np.max(np.abs(ref)))
    del d, hd, psi_in
    torch.cuda.empty_cache()
    tabs = opool.pool_tables(26, 12, "jw")
    ops, th = draw_ansatz(len(tabs), 4, seed=3, theta_sigma=0.3)
    ws = p.workspace()
    p.prepare_state(ops, th, ws[0])
    e, nrm = p.energy(ws[0], ws[1])
    si, svals = sv.prepare_state_sparse(p.info["ref_index"], tabs, ops, th)
    hi, hv = sv.apply_terms_sparse(h, si, svals)
    nn = sv.sparse_dot(si, svals, si, svals).real
    e_ref = sv.sparse_dot(si, svals, hi, hv).real / nn
    _within("26q E", abs(e - e_ref), TOL["c64"]["energy"] * max(1.0, abs(e_ref)))


def _sparse_prepared_check(n_orb, n_elec, label, n_ops=6, seed=3, grads=8):
    """A full-layout (2^n) complex64 problem at n = 2 n_orb: a prepared sparse
    state compared with the oracle on the oracle's support (and no other
    amplitude nonzero), E, and a sample of pool gradients."""
    ints = molecular_integrals(n_orb, seed=0, decay=True)
    h = mapping.hamiltonian_table(ints, "jw", 1e-3, 0.0)
    tabs = opool.pool_tables(2 * n_orb, n_elec, "jw")
    p = gb.Problem.build(ints, n_elec, precision="c64", int_drop=1e-3, device=0, colour=False)
    assert p.n_qubits == 2 * n_orb and p.dim == 1 << (2 * n_orb) and p.info["n_terms"] == len(h)
    ops, th = draw_ansatz(len(tabs), n_ops, seed=seed, theta_sigma=0.3)
    ws = p.workspace()
    e, nrm, g, sel = p.adapt_step(ops, th, ws=ws, tie_rel=1e-4)
    si, svals = sv.prepare_state_sparse(p.info["ref_index"], tabs, ops, th)
    at = torch.from_numpy(si).to("cuda:0")
    got = ws[0][at].cpu().numpy().astype(np.complex128)
    assert int(torch.view_as_real(ws[0]).ne(0).any(-1).sum().item()) == len(si)
    _within(f"{label} psi", np.max(np.abs(got - svals)), TOL["c64"]["state"] * np.max(np.abs(svals)))
    hi, hv = sv.apply_terms_sparse(h, si, svals)
    nn = sv.sparse_dot(si, svals, si, svals).real
    e_ref = sv.sparse_dot(si, svals, hi, hv).real / nn
    _within(f"{label} E", abs(e - e_ref), TOL["c64"]["energy"] * max(1.0, abs(e_ref)))
    ks = sorted(set(np.linspace(0, len(tabs) - 1, grads).astype(int).tolist() + [sel]))
    gs = {}
    for k in ks:
        ai, av = sv.apply_group_sparse(tabs[k], si, svals)
        gs[k] = 2 * sv.sparse_dot(hi, hv, ai, av).real / nn
    gscale = max(1.0, max(abs(v) for v in gs.values()))
    _within(f"{label} grads", max(abs(g[k] - v) for k, v in gs.items()), TOL["c64"]["grad"] * gscale)
    assert p.device_errors() == 0
    del ws
    p.close()
    torch.cuda.empty_cache()


def test_larger_n_28q_c64():
    """28 qubits in the full layout (14 orbitals, 8 electrons; a 2 GiB
    complex64 state): sampled H psi rows of a dense random state (the
    staged kernel), then a prepared sparse state (the scatter kernel,
    list-driven chains and gradients) against the oracle."""
    ints = molecular_integrals(14, seed=0, decay=True)
    h = mapping.hamiltonian_table(ints, "jw", 1e-3, 0.0)
    p = gb.Problem.build(ints, 8, precision="c64", int_drop=1e-3, device=0, colour=False)
    rng = np.random.default_rng(28)
    gen = torch.Generator(device="cuda:0").manual_seed(28)
    d = torch.randn(1 << 28, dtype=torch.complex64, device="cuda:0", generator=gen)
    d /= torch.linalg.vector_norm(d)
    hd = torch.empty_like(d)
    e, nrm = p.energy(d, hd)
    rows = np.concatenate([rng.integers(0, 1 << 28, size=12), [0, (1 << 28) - 1]]).astype(np.int64)
    # only the source amplitudes the sampled rows need (rows ^ x of every
    # term) come back to the host; the oracle indexes them through a lookup
    src = np.unique((rows[:, None] ^ h.x[None, :]).ravel())
    vals = d[torch.from_numpy(src).to("cuda:0")].cpu().numpy().astype(np.complex128)

    class _Gathered:
        def __getitem__(self, idx):
            return vals[np.searchsorted(src, idx)]

    ref = sv.apply_terms_at(h, _Gathered(), rows)
    got = hd[torch.from_numpy(rows).to("cuda:0")].cpu().numpy().astype(np.complex128)
    _within("28q dense rows", np.max(np.abs(got - ref)), TOL["c64"]["state"] * np.max(np.abs(ref)))
    del d, hd
    p.close()
    torch.cuda.empty_cache()
    _sparse_prepared_check(14, 8, "28q sparse")


def test_larger_n_30q_c64():
    """30 qubits in the full layout (15 orbitals, 8 electrons; an 8 GiB
    complex64 state): a prepared sparse state, E and sampled pool gradients
    against the oracle."""
    _sparse_prepared_check(15, 8, "30q sparse", n_ops=5)


def test_larger_n_32q_c64():
    """32 qubits in the full layout (16 orbitals, 8 electrons; a 32 GiB
    complex64 state, amplitude indices up to 2^32 - 1 in the uint32 index
    types): a prepared sparse state, E and sampled pool gradients against
    the oracle."""
    _sparse_prepared_check(16, 8, "32q sparse", n_ops=4)


@pytest.mark.parametrize("n_orb,n_elec,prec", [(5, 4, "c128"), (6, 6, "c64"), (6, 6, "c128"), (7, 6, "c64"),
                                               (7, 6, "c128"), (8, 8, "c64"), (8, 8, "c128")])
def test_onchip_chains_match_oracle(n_orb, n_elec, prec, monkeypatch):
    """Forward chains of states up to 128 KiB (14 qubits complex64, 13
    complex128) and backward sweeps whose psi and lambda together fit 128 KiB
    (13 / 12 qubits) run as one block over shared memory; larger ones, up to
    2 MiB, in the distributed shared memory of one cluster of 2..16 blocks
    (here: 14 qubits complex64 backward on 2 blocks, 14 complex128 forward /
    backward on 2 / 4, 16 complex64 on 4 / 8, 16 complex128 on 8 / 16).
    States, E and dE/dtheta against the oracle (Eq. 5, 6; the adjoint of
    Eq. 1).  Every form is enabled here (GOCP_ONCHIP_CHAINS=all); by default
    complex64 takes the one-block form and complex128 the grid kernels."""
    monkeypatch.setenv("GOCP_ONCHIP_CHAINS", "all")
    ints, h, tabs = _case(n_orb, n_elec, "jw", n_orb)
    p = gb.Problem.build(ints, n_elec, precision=prec, device=0)
    n = 2 * n_orb
    ops, th = draw_ansatz(len(tabs), 16, seed=n_orb, theta_sigma=0.3)
    ref = sv.basis_state(n, p.info["ref_index"])
    d = p.new_states(1)[0]
    p.prepare_state(ops, th, d)
    want = sv.prepare_state(ref, tabs, ops, th)
    _within(f"onchip {prec} {n}q psi", np.max(np.abs(_host(d) - want)), TOL[prec]["state"] * np.max(np.abs(want)))
    e, de = p.energy_grad(ops, th)
    e_ref, de_ref = sv.energy_grad(h, ref, tabs, ops, th)
    _within(f"onchip {prec} {n}q E", abs(e - e_ref), TOL[prec]["energy"] * max(1.0, abs(e_ref)))
    _within(f"onchip {prec} {n}q dE", np.max(np.abs(de - de_ref)), TOL[prec]["grad"] * max(1.0, np.max(np.abs(de_ref))))
    bad = np.array([0, 10 ** 6, 1], np.int32)      # an out-of-range operator acts as the identity, flagged
    p.prepare_state(torch.from_numpy(bad).cuda(), torch.tensor([0.2, 0.3, -0.1], dtype=torch.float64).cuda(), d)
    assert p.device_errors() == 1
    _within(f"onchip {prec} {n}q flagged", np.max(np.abs(_host(d) - sv.prepare_state(ref, tabs, [0, 1], [0.2, -0.1]))),
            TOL[prec]["state"])
    p.close()


@pytest.mark.parametrize("mode", ["default", "all"])
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_tracked_chain_matches_step_by_step(prec, mode, monkeypatch):
    """Above the on-chip sizes a prepared state's chain walks the list of its
    nonzero amplitudes (one launch per step, replayed as a graph); applying
    the same operators one gocp_taylor_step at a time to the reference state
    (each step enumerating the operator's pairs) gives the same state bit for
    bit (the per-pair arithmetic is the same), and both match the oracle.
    mode "all": the prepared chain runs in one cluster (4 blocks complex64,
    8 complex128)."""
    if mode == "all":
        monkeypatch.setenv("GOCP_ONCHIP_CHAINS", "all")
    else:
        monkeypatch.delenv("GOCP_ONCHIP_CHAINS", raising=False)
    ints, h, tabs = _case(8, 8, "jw", 3)                  # 16 qubits
    p = gb.Problem.build(ints, 8, precision=prec, device=0)
    ops, th = draw_ansatz(len(tabs), 20, seed=4, theta_sigma=0.3)
    a = p.new_states(1)[0]
    p.prepare_state(ops, th, a)
    b = p.new_states(1)[0]
    p.reference_state(b)
    for k, t in zip(ops, th):
        p.taylor_step(int(k), float(t), b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    want = sv.prepare_state(sv.basis_state(16, p.info["ref_index"]), tabs, ops, th)
    _within(f"tracked chain {prec} psi", np.max(np.abs(_host(a) - want)), TOL[prec]["state"] * np.max(np.abs(want)))
    assert p.device_errors() == 0
    p.close()


def test_cluster_chain_16_blocks_18q_c64(monkeypatch):
    """An 18-qubit complex64 forward chain (2 MiB) runs in one cluster of 16
    blocks: the prepared state against the oracle on its support (and no
    other amplitude nonzero), and the same state as the step-by-step path."""
    monkeypatch.setenv("GOCP_ONCHIP_CHAINS", "all")
    ints, h, tabs = _case(9, 8, "jw", 2)
    p = gb.Problem.build(ints, 8, precision="c64", device=0)
    ops, th = draw_ansatz(len(tabs), 24, seed=6, theta_sigma=0.3)
    a = p.new_states(1)[0]
    p.prepare_state(ops, th, a)
    b = p.new_states(1)[0]
    p.reference_state(b)
    for k, t in zip(ops, th):
        p.taylor_step(int(k), float(t), b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    si, svals = sv.prepare_state_sparse(p.info["ref_index"], tabs, ops, th)
    got = _host(a)
    assert np.count_nonzero(got) == len(si)
    _within("cluster 18q psi", np.max(np.abs(got[si] - svals)), TOL["c64"]["state"] * np.max(np.abs(svals)))
    assert p.device_errors() == 0
    p.close()
