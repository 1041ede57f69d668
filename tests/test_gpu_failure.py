"""Failure detection on the GPU without a fault.

The staged H psi kernel bounds every wait on its shared-memory staging
barriers (2 s, or GOCP_STAGE_WAIT_NS nanoseconds from the environment).  A
limit of 0 ns makes every staging wait give up at once, as a wait that ran
out: the blocks record bit 1 of the device error flags, let the copies they
started land (always with the full limit), and return.  The
test checks that the call returns, that gocp_device_errors reports the flag,
and that the next call, at the default limit, is correct again -- the
context stays usable.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15906_gb300 as gb  # noqa: E402
from oracle import mapping, statevector as sv  # noqa: E402
from synth import molecular_integrals, random_state  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2607_15906_gb300 import build
    build.build()
    gb.load()


def test_staging_wait_runs_out_and_is_reported(monkeypatch):
    ints = molecular_integrals(10, seed=2, decay=True)        # 20 qubits
    h = mapping.hamiltonian_table(ints, "jw")
    p = gb.Problem.build(ints, 10, precision="c64", device=0, colour=False)
    monkeypatch.setenv("GOCP_SPARSE_FRAC", "0")               # a dense state: the staged kernel
    psi = torch.from_numpy(random_state(20, seed=9).astype(np.complex64)).to("cuda:0")
    hpsi = torch.empty_like(psi)
    assert p.device_errors() == 0
    monkeypatch.setenv("GOCP_STAGE_WAIT_NS", "0")
    p.energy(psi, hpsi)                                       # returns; results undefined
    assert p.device_errors() == 2                             # bit 1: a staging wait gave up
    monkeypatch.delenv("GOCP_STAGE_WAIT_NS")
    e, nrm = p.energy(psi, hpsi)
    assert p.device_errors() == 0
    psi_in = psi.cpu().numpy().astype(np.complex128)
    rows = np.concatenate([np.random.default_rng(3).integers(0, 1 << 20, size=24), [0, (1 << 20) - 1]])
    ref = sv.apply_terms_at(h, psi_in, rows)
    got = hpsi.cpu().numpy().astype(np.complex128)[rows]
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))
    assert abs(nrm - np.vdot(psi_in, psi_in).real) <= 1e-6
    p.close()
