"""gocp_energy_static, the allocation-free energy entry point.

It exists for callers that cannot call cudaMalloc where they compute (a host
loop with real-time or no-blocking guarantees, or a caller whose device
memory belongs to another allocator): its reduction scratch is a fixed
device array inside the library.  Through the C ABI, two calls in a row must
give the same H psi and energy as gocp_energy: bit for bit below the tile
size (where both run the untiled kernel), within the tolerances of the
parity tests above it (where gocp_energy runs the tiled kernels); states
beyond the array's 24-qubit limit must be refused.  The file name keeps
this module last in collection order.
"""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15906_gb300 as gb  # noqa: E402
from paper_2607_15906_gb300 import _lib  # noqa: E402
from synth import molecular_integrals, random_state  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL = {"c128": dict(state=1e-10, energy=1e-10), "c64": dict(state=2e-5, energy=1e-6)}


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    from paper_2607_15906_gb300 import build
    build.build()
    gb.load()


def _energy_static(p, psi, hpsi, mem):
    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)
    if mem == _lib.GOCP_MEM_HOST:
        out = np.zeros(2)
        rc = lib.gocp_energy_static(p.handle, C.c_void_p(psi.data_ptr()), C.c_void_p(hpsi.data_ptr()),
                                    out.ctypes.data_as(C.c_void_p), mem, stream)
        _lib.check(rc, "gocp_energy_static")
        return float(out[0]), float(out[1])
    out = torch.zeros(2, dtype=torch.float64, device=f"cuda:{p.device}")
    rc = lib.gocp_energy_static(p.handle, C.c_void_p(psi.data_ptr()), C.c_void_p(hpsi.data_ptr()),
                                C.c_void_p(out.data_ptr()), mem, stream)
    _lib.check(rc, "gocp_energy_static")
    torch.cuda.synchronize()
    return float(out[0]), float(out[1])


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n_orb,n_elec", [(2, 2), (5, 4), (7, 6), (10, 10)])
def test_static_energy_matches_gocp_energy_twice(prec, n_orb, n_elec):
    ints = molecular_integrals(n_orb, seed=21 + n_orb, decay=True)
    p = gb.Problem.build(ints, n_elec, precision=prec, device=0)
    n = 2 * n_orb
    dt = np.complex64 if prec == "c64" else np.complex128
    psi = torch.from_numpy(random_state(n, seed=5 + n).astype(dt)).to("cuda:0")
    h_ref = torch.empty_like(psi)
    e_ref, nrm_ref = p.energy(psi, h_ref)
    ref = h_ref.cpu().numpy().astype(np.complex128)
    scale = np.max(np.abs(ref))
    for call, mem in enumerate([_lib.GOCP_MEM_HOST, _lib.GOCP_MEM_DEVICE]):
        h = torch.full_like(psi, float("nan"))
        e, nrm = _energy_static(p, psi, h, mem)
        got = h.cpu().numpy().astype(np.complex128)
        if n < (13 if prec == "c64" else 12):      # the same kernel as gocp_energy
            assert np.array_equal(got, ref) and e == e_ref and nrm == nrm_ref, call
        assert np.max(np.abs(got - ref)) <= TOL[prec]["state"] * scale, call
        assert abs(e - e_ref) <= TOL[prec]["energy"] * max(1.0, abs(e_ref)), call
        assert abs(nrm - nrm_ref) <= 1e-12 * max(1.0, nrm_ref), call


def test_static_energy_rejects_states_beyond_its_array():
    ints = molecular_integrals(13, seed=1, decay=True)
    p = gb.Problem.build(ints, 2, precision="c64", device=0, colour=False)    # 26 qubits
    dummy = torch.zeros(4, dtype=torch.complex64, device="cuda:0")
    out = np.zeros(2)
    rc = _lib.load().gocp_energy_static(p.handle, C.c_void_p(dummy.data_ptr()),
                                        C.c_void_p(dummy[2:].data_ptr()), out.ctypes.data_as(C.c_void_p),
                                        _lib.GOCP_MEM_HOST, None)
    assert rc == _lib.GOCP_EINVAL
    msg = _lib.load().gocp_last_error().decode()
    assert "24 qubits" in msg and "32768" in msg
