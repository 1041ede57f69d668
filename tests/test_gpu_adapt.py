"""ADAPT driver and autograd Function over the GPU path.

  * 4 qubits: the GPU ADAPT run follows the oracle's trajectory (same
    operators, same energies) under JW and BK alike.
  * 20 qubits, 60-operator ansatz, theta ~ N(0, 0.05): dE/dtheta from the
    adjoint torch.autograd.Function equals central finite differences of
    the complex128 energy (h = 1e-5), and the complex64 path agrees with the
    complex128 one (energy, gradient, state fidelity).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15906_gb300 as gb  # noqa: E402
from paper_2607_15906_gb300.adapt import adapt as gpu_adapt  # noqa: E402
from paper_2607_15906_gb300.autograd import ansatz_energy  # noqa: E402
from oracle import adapt as oadapt, mapping, pool as opool, statevector as sv  # noqa: E402
from synth import config_integrals, draw_ansatz  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2607_15906_gb300 import build
    build.build()
    gb.load()


@pytest.mark.parametrize("mp", ["jw", "bk"])
def test_adapt_4q_follows_oracle(mp):
    ints, c = config_integrals("c1_4q")
    p = gb.Problem.build(ints, 2, mapping=mp, precision="c128", device=0)
    run = gpu_adapt(p, max_ops=10, gtol=1e-4)
    h = mapping.hamiltonian_table(ints, mp)
    tabs = opool.pool_tables(4, 2, mp)
    ref = oadapt.adapt(h, tabs, sv.basis_state(4, mapping.hf_index(mp, 4, 2)), max_ops=10, gtol=1e-4)
    assert run.converged and ref.converged
    assert run.ops == ref.ops
    assert np.max(np.abs(np.array(run.energies) - np.array(ref.energies))) < 1e-9


def test_adapt_4q_c64_reaches_same_energy():
    ints, c = config_integrals("c1_4q")
    p128 = gb.Problem.build(ints, 2, precision="c128", device=0)
    p64 = gb.Problem.build(ints, 2, precision="c64", device=0)
    r128 = gpu_adapt(p128, max_ops=10)
    r64 = gpu_adapt(p64, max_ops=10)
    assert r64.ops == r128.ops
    assert abs(r64.energies[-1] - r128.energies[-1]) < 1e-6


def test_autograd_adjoint_20q_vs_finite_differences_and_c64():
    ints, c = config_integrals("c3_20q")
    kw = dict(term_drop=c["term_drop"], device=0)
    p128 = gb.Problem.build(ints, 10, precision="c128", **kw)
    p64 = gb.Problem.build(ints, 10, precision="c64", **kw)
    ops, th = draw_ansatz(p128.pool_size, 60, seed=0)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    e = ansatz_energy(theta, p128, ops)
    e.backward()
    g128 = theta.grad.numpy().copy()
    # central differences of the complex128 energy, h = 1e-5, on a sample of parameters
    ws = p128.workspace()
    hs = 1e-5
    for j in list(range(0, 60, 7)) + [59]:
        tp, tm = th.copy(), th.copy()
        tp[j] += hs
        tm[j] -= hs
        ep, _ = p128.energy_grad(ops, tp, ws=ws)
        em, _ = p128.energy_grad(ops, tm, ws=ws)
        assert abs((ep - em) / (2 * hs) - g128[j]) < 1e-8
    # complex64 path against complex128 (device-resident theta this time)
    th_d = torch.tensor(th, dtype=torch.float64, device="cuda:0", requires_grad=True)
    e64 = ansatz_energy(th_d, p64, ops)
    e64.backward()
    assert abs(float(e64.detach()) - float(e.detach())) < 1e-6
    assert np.max(np.abs(th_d.grad.cpu().numpy() - g128)) < 2e-5
    s128 = p128.new_states(1)[0]
    s64 = p64.new_states(1)[0]
    p128.prepare_state(ops, th, s128)
    p64.prepare_state(ops, th, s64)
    torch.cuda.synchronize()
    a = s128.cpu().numpy()
    b = s64.cpu().numpy().astype(np.complex128)
    assert 1.0 - sv.fidelity(a, b) < 1e-6


def test_adapt_14q_mapping_invariant_30_operators():
    """The 14-qubit workload (7 orbitals, 6 electrons, 204-operator pool)
    grown to 30 operators under JW and BK, complex128: the same operator at
    every iteration and the same energies (Sec. IV.B; BK is a basis
    permutation of JW, so the method is exactly mapping invariant).

    The selection window is 1e-6 relative: the BFGS re-optimisation stops at
    a gradient norm of 1e-8, so the angles -- and with them the pool
    gradients -- of the two mappings agree only to about 1e-8 relative, and
    two operators whose |g| lie closer than that (alpha/beta mirror
    excitations of a nearly symmetric state) may otherwise be ordered
    differently."""
    ints, c = config_integrals("c2_14q")
    runs = {}
    for mp in ("jw", "bk"):
        p = gb.Problem.build(ints, 6, mapping=mp, precision="c128", device=0)
        runs[mp] = gpu_adapt(p, max_ops=30, gtol=1e-4, tie_rel=1e-6)
    assert len(runs["jw"].ops) == 30
    a, b = runs["jw"], runs["bk"]
    for i, (x, y) in enumerate(zip(a.ops, b.ops)):
        if x != y:
            ga, gb_ = np.abs(a.gradients[i]), np.abs(b.gradients[i])
            pytest.fail(f"iteration {i}: JW chose {x}, BK {y}; |g| JW {ga[x]:.15g} {ga[y]:.15g}, "
                        f"BK {gb_[x]:.15g} {gb_[y]:.15g}, max {ga.max():.15g}")
    assert np.max(np.abs(np.array(runs["jw"].energies) - np.array(runs["bk"].energies))) < 1e-9
    assert all(b <= a + 1e-12 for a, b in zip(runs["jw"].energies, runs["jw"].energies[1:]))


@pytest.mark.parametrize("n_orb,n_elec,mp,seed", [(2, 2, "jw", 0), (2, 2, "bk", 0), (4, 4, "jw", 2), (4, 4, "bk", 2)])
def test_family_adapt_follows_oracle(n_orb, n_elec, mp, seed):
    """Family-batched ADAPT: the GPU driver adds the same commuting batches as
    the oracle and reaches the same energies (complex128)."""
    from oracle import gocp
    from synth import molecular_integrals
    ints = config_integrals("c1_4q")[0] if n_orb == 2 else molecular_integrals(n_orb, seed=seed)
    n = 2 * n_orb
    p = gb.Problem.build(ints, n_elec, mapping=mp, precision="c128", device=0)
    run = gpu_adapt(p, max_ops=12, gtol=1e-4, family=True)
    h = mapping.hamiltonian_table(ints, mp)
    tabs = opool.pool_tables(n, n_elec, mp)
    fam = gocp.gocp(tabs)
    assert np.array_equal(p.pool()[5], fam)
    ref = oadapt.adapt(h, tabs, sv.basis_state(n, mapping.hf_index(mp, n, n_elec)), max_ops=12, gtol=1e-4,
                       families=fam)
    assert run.ops == ref.ops
    assert np.max(np.abs(np.array(run.energies) - np.array(ref.energies))) < 1e-9
