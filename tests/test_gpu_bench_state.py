"""The timed 24-qubit ADAPT step, on its exact inputs, against the oracle.

Workload: 12 orbitals, 8 electrons, Jordan-Wigner, integrals below 1e-3
dropped, the 1424-operator pool and the 100-operator ansatz
draw_ansatz(1424, 100, seed=0) (theta ~ N(0, 0.05)) -- the state that
bench.py times.  For complex64 and complex128, through gocp_adapt_step and
gocp_energy_grad of the grown 101-operator ansatz (the selected operator
appended at theta = 0):

  * every amplitude of psi (Eq. 5, 6) and the fidelity,
  * E (Eq. 1),
  * all 1424 pool gradients (Eq. 4) and the selected operator,
  * dE/dtheta_j of the adjoint sweep at j = 0, 1, 50, 96..100 against the
    oracle's forward mode (T_j replaced by its derivative).

The oracle prepares the state in sparse form (prepare_state_sparse) and
evaluates H psi (apply_terms_at) on every row that a product needs: the
union of the supports of psi, of every A_k psi and of every derivative state.

Tolerances (the benchmark spec's): complex128 1e-10 relative on every quantity;
complex64 |E - E_oracle| <= 1e-6 Ha and fidelity >= 1 - 1e-6, amplitudes
within 2e-5 of max|psi|, gradients and dE/dtheta within 2e-6 of
max(1, max|g|).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15906_gb300 as gb  # noqa: E402
from oracle import adapt as oadapt, mapping, parallel as oracle_jobs, pool as opool, statevector as sv  # noqa: E402
from synth import config_integrals, draw_ansatz  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

N_OPS = 100
J = [0, 1, 50, 96, 97, 98, 99]
TIE = {"c64": 1e-4, "c128": 1e-8}
TOL = {"c128": dict(state=1e-10, energy=1e-10, grad=1e-10, fid=1e-12),
       "c64": dict(state=2e-5, energy=1e-6, grad=2e-6, fid=1e-6)}


@pytest.fixture(scope="module")
def oracle24():
    ints, c = config_integrals("c5_24q")
    h = mapping.hamiltonian_table(ints, "jw", c["int_drop"], c["term_drop"])
    tabs = opool.pool_tables(24, 8, "jw")
    ops, th = draw_ansatz(len(tabs), N_OPS, seed=0)
    hf = mapping.hf_index("jw", 24, 8)
    si, svals, kept = sv.prepare_state_sparse(hf, tabs, ops, th, keep_at=J)
    nrm = float(np.sum(np.abs(svals) ** 2))
    deriv = {j: sv.derivative_state_sparse(tabs, ops, th, j, kept[j]) for j in J}
    mask = oracle_jobs.generator_support(tabs, si, svals)
    mask[si] = True
    for di, _ in deriv.values():
        mask[di] = True
    rows = np.flatnonzero(mask).astype(np.int64)
    hrows = oracle_jobs.hpsi_rows(h, si, svals, rows)
    psi = np.zeros(1 << 24, np.complex128)
    psi[si] = svals
    e = float(np.sum(np.conj(psi[rows]) * hrows).real / nrm)
    g = oracle_jobs.pool_gradients(tabs, si, svals, rows, hrows, nrm)
    resid = hrows - e * psi[rows]

    def dtheta(di, dv):
        pos = np.searchsorted(rows, di)
        assert np.all(rows[pos] == di)
        return float(2.0 * np.sum(np.conj(resid[pos]) * dv).real / nrm)

    sel = {prec: oadapt.select(g, TIE[prec]) for prec in TIE}
    de = {prec: {j: dtheta(*deriv[j]) for j in J} for prec in TIE}
    for prec in TIE:   # the appended operator at theta = 0: T'(0) = A
        de[prec][N_OPS] = dtheta(*sv.apply_group_sparse(tabs[sel[prec]], si, svals))
    return dict(ints=ints, cfg=c, ops=ops, th=th, psi=psi, nnz=len(si), e=e, g=g, sel=sel, de=de)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2607_15906_gb300 import build
    build.build()
    gb.load()


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_bench_state_24q(prec, oracle24):
    o = oracle24
    tol = TOL[prec]
    p = gb.Problem.build(o["ints"], 8, precision=prec, int_drop=o["cfg"]["int_drop"],
                         term_drop=o["cfg"]["term_drop"], device=0)
    ws = p.workspace()
    e, nrm, g, sel = p.adapt_step(o["ops"], o["th"], ws=ws, tie_rel=TIE[prec])
    torch.cuda.synchronize()
    got = ws[0].cpu().numpy().astype(np.complex128)
    ref = o["psi"]
    amax = np.max(np.abs(ref))
    state_err = np.max(np.abs(got - ref)) / amax
    infid = 1.0 - sv.fidelity(got, ref)
    e_err = abs(e - o["e"])
    gscale = max(1.0, np.max(np.abs(o["g"])))
    g_err = np.max(np.abs(g - o["g"])) / gscale
    print(f"\n24q {prec}: nnz {np.count_nonzero(got)} (oracle {o['nnz']}), state {state_err:.3e} "
          f"(tol {tol['state']:.0e}), 1-F {infid:.3e}, |dE| {e_err:.3e}, grads {g_err:.3e}, "
          f"selected {sel} (oracle {o['sel'][prec]})")
    assert state_err <= tol["state"]
    assert infid <= tol["fid"]
    assert e_err <= tol["energy"] * max(1.0, abs(o["e"]))
    assert g_err <= tol["grad"]
    mag = np.abs(o["g"])
    assert mag[sel] >= mag.max() * (1.0 - TIE[prec]) - 2 * tol["grad"] * gscale
    # the grown ansatz through the adjoint sweep (the oracle's selection appended)
    k = o["sel"][prec]
    ops_g = np.append(o["ops"], np.int32(k)).astype(np.int32)
    th_g = np.append(o["th"], 0.0)
    e2, de = p.energy_grad(ops_g, th_g, ws=ws)
    ref_de = o["de"][prec]
    dscale = max(1.0, max(abs(v) for v in ref_de.values()))
    de_err = max(abs(de[j] - v) for j, v in ref_de.items()) / dscale
    print(f"24q {prec}: grown ansatz |dE| {abs(e2 - o['e']):.3e}, dE/dtheta {de_err:.3e}")
    assert abs(e2 - o["e"]) <= tol["energy"] * max(1.0, abs(o["e"]))
    assert de_err <= tol["grad"]
    assert p.device_errors() == 0
    p.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_bench_state_h_psi_reproducible(prec, oracle24):
    """H psi and E of the timed state are the same bit for bit from call to
    call (the scatter kernel sums in fixed point, the energy partials in tile
    order), and so are the pool gradients built on them."""
    o = oracle24
    p = gb.Problem.build(o["ints"], 8, precision=prec, int_drop=o["cfg"]["int_drop"],
                         term_drop=o["cfg"]["term_drop"], device=0)
    ws = p.workspace()
    p.prepare_state(o["ops"], o["th"], ws[0])
    first = None
    for _ in range(3):
        e, nrm = p.energy(ws[0], ws[1])
        g = p.pool_gradients(ws[0], ws[1])
        cur = (ws[1].clone(), e, nrm, g)
        if first is None:
            first = cur
        else:
            assert torch.equal(first[0], cur[0])
            assert first[1] == cur[1] and first[2] == cur[2]
            assert np.array_equal(first[3], cur[3])
    assert abs(first[1] - o["e"]) <= TOL[prec]["energy"] * max(1.0, abs(o["e"]))
    p.close()


def test_bench_state_split_accumulator_is_bit_identical(oracle24, monkeypatch):
    """complex64: the scatter kernel's split accumulator words (low 16 bits
    of each product and the product shifted right by 16, summed by
    independent atomics) give the same integers as the 64-bit words with a
    carry between their halves (GOCP_SCATTER_SPLIT=0): H psi, E and the pool
    gradients of the timed state are equal bit for bit."""
    o = oracle24
    p = gb.Problem.build(o["ints"], 8, precision="c64", int_drop=o["cfg"]["int_drop"],
                         term_drop=o["cfg"]["term_drop"], device=0)
    ws = p.workspace()
    p.prepare_state(o["ops"], o["th"], ws[0])
    out = {}
    for split in ("1", "0"):
        monkeypatch.setenv("GOCP_SCATTER_SPLIT", split)
        hd = torch.empty_like(ws[0])
        e, nrm = p.energy(ws[0], hd)
        out[split] = (hd, e, nrm, p.pool_gradients(ws[0], hd))
    assert torch.equal(out["1"][0], out["0"][0])
    assert out["1"][1] == out["0"][1] and out["1"][2] == out["0"][2]
    assert np.array_equal(out["1"][3], out["0"][3])
    assert abs(out["1"][1] - o["e"]) <= TOL["c64"]["energy"] * max(1.0, abs(o["e"]))
    assert p.device_errors() == 0
    p.close()
