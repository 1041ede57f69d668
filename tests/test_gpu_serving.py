"""The continuous-batching server: results equal the direct path and the
oracle, are bit-identical alone and in a mixed stream, and admission,
cancellation and polling behave as documented."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15906_gb300 as gb  # noqa: E402
from paper_2607_15906_gb300.serving import Server  # noqa: E402
from oracle import mapping, pool as opool, statevector as sv  # noqa: E402
from synth import draw_ansatz, molecular_integrals  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2607_15906_gb300 import build
    build.build()
    gb.load()


def _requests():
    out = []
    for i, (n, prec) in enumerate([(4, "c128"), (6, "c64"), (8, "c128"), (10, "c64"), (12, "c64"),
                                   (8, "c64"), (6, "c128"), (14, "c64"), (4, "c64")]):
        ints = molecular_integrals(n // 2, seed=1000 + i, decay=True)
        ne = 2 * (n // 4)
        p = gb.Problem.build(ints, ne, precision=prec, device=0)
        ops, th = draw_ansatz(p.pool_size, 5 + 3 * i, seed=i, theta_sigma=0.2)
        out.append((ints, ne, p, ops, th))
    return out


def test_mixed_stream_matches_direct_and_oracle():
    reqs = _requests()
    with Server(hbm_budget_bytes=64 << 20, max_slots=16) as srv:
        tickets = [srv.submit(p, ops, th) for (_, _, p, ops, th) in reqs]
        results = [srv.result(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["max_resident"] >= 2
    for (ints, ne, p, ops, th), (e, de) in zip(reqs, results):
        e_d, de_d = p.energy_grad(ops, th)
        tol = 1e-10 if p.precision == "c128" else 1e-6
        assert abs(e - e_d) <= tol * max(1.0, abs(e_d))
        assert np.max(np.abs(de - de_d)) <= (1e-10 if p.precision == "c128" else 2e-5)
        if p.n_qubits <= 8:
            h = mapping.hamiltonian_table(ints, "jw")
            tabs = opool.pool_tables(p.n_qubits, ne, "jw")
            e_o, de_o = sv.energy_grad(h, sv.basis_state(p.n_qubits, p.info["ref_index"]), tabs, ops, th)
            assert abs(e - e_o) <= tol * max(1.0, abs(e_o))
            assert np.max(np.abs(de - de_o)) <= (1e-10 if p.precision == "c128" else 2e-5)


def test_alone_and_in_the_mix_are_bit_identical():
    reqs = _requests()
    alone = []
    with Server(hbm_budget_bytes=64 << 20, max_slots=16) as srv:
        for (_, _, p, ops, th) in reqs:
            alone.append(srv.result(srv.submit(p, ops, th)))
    with Server(hbm_budget_bytes=64 << 20, max_slots=16) as srv:
        tickets = [srv.submit(p, ops, th) for (_, _, p, ops, th) in reqs]
        mixed = [srv.result(t) for t in tickets]
    for (ea, da), (em, dm) in zip(alone, mixed):
        assert ea == em
        assert np.array_equal(da, dm)


def test_admission_by_arena_memory():
    ints = molecular_integrals(6, seed=3, decay=True)
    p = gb.Problem.build(ints, 6, precision="c64", device=0)      # 12 qubits: 2 states = 64 KiB
    ops, th = draw_ansatz(p.pool_size, 20, seed=1)
    with Server(hbm_budget_bytes=2 * 65536, max_slots=16) as srv:  # room for two requests
        tickets = [srv.submit(p, ops, th) for _ in range(7)]
        res = [srv.result(t) for t in tickets]
        st = srv.stats()
    assert st["max_resident"] <= 2 and st["completed"] == 7
    assert all(r[0] == res[0][0] and np.array_equal(r[1], res[0][1]) for r in res)


def test_cancel_poll_and_rejections():
    ints = molecular_integrals(7, seed=4, decay=True)
    big = gb.Problem.build(ints, 6, precision="c64", device=0)     # 14 qubits
    ops, th = draw_ansatz(big.pool_size, 60, seed=2)
    with Server(hbm_budget_bytes=1 << 18, max_slots=2) as srv:     # 256 KiB arena
        ts = [srv.submit(big, ops, th) for _ in range(6)]
        srv.cancel(ts[-1])
        with pytest.raises(gb.GocpError) as e:
            srv.result(ts[-1])
        assert e.value.code == -6                                  # ECANCELED
        for t in ts[:-1]:
            assert srv.result(t) is not None
        with pytest.raises(gb.GocpError) as e:
            srv.poll(ts[0])                                        # already retired
        assert e.value.code == -1
        huge = gb.Problem.build(molecular_integrals(9, seed=5, decay=True), 8, precision="c128", device=0)
        hops, hth = draw_ansatz(huge.pool_size, 3, seed=3)
        with pytest.raises(gb.GocpError) as e:
            srv.submit(huge, hops, hth)                            # 18 qubits never fit 256 KiB
        assert e.value.code == -2
        with pytest.raises(gb.GocpError):
            srv.submit(big, np.array([big.pool_size]), np.array([0.1]))
    with Server(hbm_budget_bytes=1 << 20, max_slots=1) as srv:
        ts = [srv.submit(big, ops, th) for _ in range(4)]
        assert srv.poll(ts[-1], timeout_s=0.0) is None              # still queued
        assert srv.result(ts[-1]) is not None
        for t in ts[:-1]:
            srv.result(t)


def test_admission_by_free_device_memory():
    """hbm_budget_bytes = 0: states come from the server's memory pool as
    requests are admitted against free device memory; results equal the
    arena server's bit for bit (same kernels, same block counts)."""
    reqs = _requests()
    with Server(hbm_budget_bytes=64 << 20, max_slots=16) as srv:
        arena = [srv.result(srv.submit(p, ops, th)) for (_, _, p, ops, th) in reqs]
    with Server(hbm_budget_bytes=0, max_slots=16) as srv:
        tickets = [srv.submit(p, ops, th) for (_, _, p, ops, th) in reqs]
        pooled = [srv.result(t) for t in tickets]
        st = srv.stats()
    assert st["arena_bytes"] == 0 and st["completed"] == len(reqs)
    assert st["arena_in_use"] == 0 and st["arena_peak"] >= 2 * reqs[-2][2].state_bytes()
    for (ea, da), (ep, dp) in zip(arena, pooled):
        assert ea == ep and np.array_equal(da, dp)


@pytest.mark.parametrize("mode", ["default", "all"])
def test_cluster_stage_requests(mode, monkeypatch):
    """Requests of 16 and 18 qubits run their chains in one thread-block
    cluster each (16 qubits complex64: 4 / 8 blocks, complex128: 8 / 16; 18
    qubits complex64: a 16-block forward chain, per-step backward stages),
    mixed with a small one-block request: the same results alone and in the
    mix bit for bit, and the direct path's within the parity tolerances.
    mode "default": the on-chip forms the library picks by default (one
    block for complex64, none for complex128); "all": clusters too."""
    if mode == "all":
        monkeypatch.setenv("GOCP_ONCHIP_CHAINS", "all")
    else:
        monkeypatch.delenv("GOCP_ONCHIP_CHAINS", raising=False)
    reqs = []
    for i, (n, prec) in enumerate([(16, "c64"), (18, "c64"), (16, "c128"), (10, "c64")]):
        ints = molecular_integrals(n // 2, seed=2000 + i, decay=True)
        ne = 2 * (n // 4)
        p = gb.Problem.build(ints, ne, precision=prec, device=0, colour=False)
        ops, th = draw_ansatz(p.pool_size, 12 + 4 * i, seed=i, theta_sigma=0.2)
        reqs.append((p, ops, th))
    alone = []
    with Server(hbm_budget_bytes=0, max_slots=16) as srv:
        for (p, ops, th) in reqs:
            alone.append(srv.result(srv.submit(p, ops, th)))
    with Server(hbm_budget_bytes=0, max_slots=16) as srv:
        tickets = [srv.submit(p, ops, th) for (p, ops, th) in reqs]
        mixed = [srv.result(t) for t in tickets]
    for (p, ops, th), (ea, da), (em, dm) in zip(reqs, alone, mixed):
        assert ea == em and np.array_equal(da, dm)
        e_d, de_d = p.energy_grad(ops, th)
        tol = 1e-10 if p.precision == "c128" else 1e-6
        assert abs(ea - e_d) <= tol * max(1.0, abs(e_d))
        assert np.max(np.abs(da - de_d)) <= (1e-10 if p.precision == "c128" else 2e-6) * max(1.0, np.max(np.abs(de_d)))
        assert p.device_errors() == 0
