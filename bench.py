#!/usr/bin/env python
"""ADAPT-iteration benchmark of the GB300 GOCP ADAPT-VQE hot path.

Workload (one GPU): 24 qubits = 12 spatial orbitals, 8 electrons, seeded
molecular-shaped integrals with off-diagonal decay, integrals |v| < 1e-3
dropped, Jordan-Wigner, 1424-operator singles+doubles pool, complex64 state
(128 MiB), a 100-operator ansatz drawn from the pool with angles N(0, 0.05).

One step = one ADAPT iteration with a one-evaluation re-optimisation budget:
  1. prepare psi(theta) (100 fused O(5) Taylor steps), H psi, E, all 1424 pool
     gradients, argmax selection                         (gocp_adapt_step)
  2. E and dE/dtheta of the grown 101-operator ansatz by the adjoint sweep
                                                         (gocp_energy_grad)
`value` times steps with the ansatz, states and outputs resident on the
device; `e2e` times the same step through the host-array API (ansatz copied
in from pinned memory, E / gradients / dE copied out every step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gocp|reference]

With N > 1 (torchrun) every rank runs an independent replica (the path has
no exchange step): value = iterations of all ranks / max rank time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import config_integrals, draw_ansatz, molecular_integrals  # noqa: E402

WORKLOAD = "c5_24q"
N_OPS = 100
N_ELEC = 8
METRIC = "ADAPT iterations/s (24 qubits, complex64, 1424-op pool, 100-op ansatz + adjoint dE/dtheta)"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


# ---------------------------------------------------------------- GPU arm

def slowest_rank(times, device="cpu"):
    """Each rank's timings -> the maximum over ranks (all_reduce MAX)."""
    import torch
    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t]


def replica_throughput(steps: int, world: int, slowest_secs: float) -> float:
    """Whole-job value of independent replicas: iterations of all ranks over
    the slowest rank's time (weak scaling: work per rank is fixed)."""
    return world * steps / slowest_secs


def run_gpu(args, rank, world, device):
    import torch
    import paper_2607_15906_gb300 as gb
    from paper_2607_15906_gb300 import _lib

    torch.cuda.set_device(device)
    gb.load()
    ints, cfg = config_integrals(WORKLOAD)
    prob = gb.Problem.build(ints, N_ELEC, mapping="jw", precision=args.precision,
                            int_drop=cfg["int_drop"], term_drop=cfg["term_drop"], device=device)
    m = prob.pool_size
    ops, theta = draw_ansatz(m, N_OPS, seed=0)
    dev = f"cuda:{device}"
    ops_d = torch.from_numpy(ops).to(dev)
    th_d = torch.from_numpy(theta).to(dev)
    ops_g = torch.zeros(N_OPS + 1, dtype=torch.int32, device=dev)
    ops_g[:N_OPS] = ops_d
    th_g = torch.zeros(N_OPS + 1, dtype=torch.float64, device=dev)
    th_g[:N_OPS] = th_d
    ws = prob.workspace()
    e2 = torch.zeros(2, dtype=torch.float64, device=dev)
    grads = torch.zeros(m, dtype=torch.float64, device=dev)
    sel = torch.zeros(1, dtype=torch.int32, device=dev)
    e_out = torch.zeros(1, dtype=torch.float64, device=dev)
    de_out = torch.zeros(N_OPS + 1, dtype=torch.float64, device=dev)

    def step_device():
        prob.adapt_step(ops_d, th_d, ws=ws, tie_rel=1e-4, out=(e2, grads, sel))
        ops_g[N_OPS:].copy_(sel)                       # append the selected operator, theta = 0
        prob.energy_grad(ops_g, th_g, ws=ws, out_e=e_out, out_de=de_out)

    pin_ops = torch.from_numpy(ops).pin_memory().numpy()
    pin_th = torch.from_numpy(theta).pin_memory().numpy()
    pin_og = torch.zeros(N_OPS + 1, dtype=torch.int32).pin_memory().numpy()
    pin_tg = torch.zeros(N_OPS + 1, dtype=torch.float64).pin_memory().numpy()
    pin_og[:N_OPS] = ops
    pin_tg[:N_OPS] = theta
    h2d = pin_ops.nbytes + pin_th.nbytes + pin_og.nbytes + pin_tg.nbytes
    d2h = 16 + 8 * m + 4 + 8 + 8 * (N_OPS + 1)

    def step_host():
        e, nrm, g, s = prob.adapt_step(pin_ops, pin_th, ws=ws, tie_rel=1e-4)
        pin_og[N_OPS] = s
        prob.energy_grad(pin_og, pin_tg, ws=ws)

    stream = torch.cuda.current_stream(device)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        return a.elapsed_time(b) / 1e3

    # ---- device-resident timed region, with kernel timing and clock sampling
    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    _lib.profile_enable(True)
    for kind in range(4):
        _lib.profile_read(kind)
    launches0 = gb.launch_count()
    with ClockSampler(device) as clk:
        secs = timed(step_device, args.steps, 0)
    launches = gb.launch_count() - launches0
    _lib.profile_enable(False)
    kern = {name: _lib.profile_read(kind) for kind, name in
            enumerate(["apply_h", "taylor5", "pool_grad", "adjoint"])}
    clocks = clk.summary()
    # ---- end-to-end through the host-array API
    e2e_secs = timed(step_host, args.steps, 1)

    if world > 1:
        secs, e2e_secs = slowest_rank([secs, e2e_secs], device=dev)
    # nonzero amplitudes of the prepared state psi(theta), on which both H psi
    # calls of a step act (the appended operator has theta = 0); outside the
    # timed regions
    prob.adapt_step(ops_d, th_d, ws=ws, tie_rel=1e-4, out=(e2, grads, sel))
    nnz = int(torch.view_as_real(ws[0]).ne(0).any(-1).sum().item())
    info = prob.info
    return dict(prob=prob, secs=secs, e2e_secs=e2e_secs, kern=kern, clocks=clocks, launches=launches,
                h2d=h2d, d2h=d2h, info=info, e=float(e2[0]), sel=int(sel[0]), nnz=nnz)


def _adapt_step_timer(prob, device: int, n_ops: int = N_OPS, seed: int = 0):
    """step() = the bench step on `prob` (adapt_step of an n_ops-operator
    ansatz + energy_grad of the grown one), device-resident, and
    timed(steps, warmup) -> ms per step by CUDA events on the launch stream."""
    import torch

    ops, theta = draw_ansatz(prob.pool_size, n_ops, seed=seed)
    dev = f"cuda:{device}"
    ops_d = torch.from_numpy(ops).to(dev)
    th_d = torch.from_numpy(theta).to(dev)
    ops_g = torch.zeros(n_ops + 1, dtype=torch.int32, device=dev)
    ops_g[:n_ops] = ops_d
    th_g = torch.zeros(n_ops + 1, dtype=torch.float64, device=dev)
    th_g[:n_ops] = th_d
    ws = prob.workspace()
    e2 = torch.zeros(2, dtype=torch.float64, device=dev)
    g = torch.zeros(prob.pool_size, dtype=torch.float64, device=dev)
    sel = torch.zeros(1, dtype=torch.int32, device=dev)
    e_out = torch.zeros(1, dtype=torch.float64, device=dev)
    de_out = torch.zeros(n_ops + 1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(device)
    tie = 1e-4 if prob.precision == "c64" else 1e-8

    def step():
        prob.adapt_step(ops_d, th_d, ws=ws, tie_rel=tie, out=(e2, g, sel))
        ops_g[n_ops:].copy_(sel)
        prob.energy_grad(ops_g, th_g, ws=ws, out_e=e_out, out_de=de_out)

    def timed(steps: int, warmup: int) -> float:
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    return dict(step=step, timed=timed, ws=ws, e2=e2, g=g, sel=sel, e_out=e_out, de_out=de_out,
                ops=ops, theta=theta)


def full_layout_large(device: int, n_orb: int, n_elec: int = 8, steps: int = 3, warmup: int = 1):
    """The bench step in the full 2^n layout at n = 2 n_orb qubits (integrals
    < 1e-3 dropped, JW, a 100-operator ansatz drawn from the pool)."""
    import torch
    import paper_2607_15906_gb300 as gb

    ints = molecular_integrals(n_orb, seed=0, decay=True)
    t0 = time.time()
    prob = gb.Problem.build(ints, n_elec, mapping="jw", precision="c64", int_drop=1e-3, device=device,
                            colour=False)
    build_s = time.time() - t0
    t = _adapt_step_timer(prob, device)
    ms = t["timed"](steps, warmup)
    nnz = int(torch.view_as_real(t["ws"][0]).ne(0).any(-1).sum().item())
    info = prob.info
    out = {"qubits": 2 * n_orb, "electrons": n_elec, "state_bytes": prob.state_bytes(), "pool": prob.pool_size,
           "n_terms": info["n_terms"], "n_groups": info["n_groups"], "build_s": build_s,
           "device_bytes": info["device_bytes"], "nonzero_amplitudes": nnz,
           "iterations_per_s": 1e3 / ms, "ms_per_step": ms, "energy": float(t["e2"][0]),
           "selected": int(t["sel"][0]), "steps": steps, "warmup": warmup}
    del t
    prob.close()
    torch.cuda.empty_cache()
    return out


def sector_layout(device: int, full_e: float, full_sel: int, steps: int = 10, warmup: int = 3):
    """The same 24-qubit ADAPT step (adapt_step on the 100-operator ansatz +
    energy_grad of the grown one) on a sector-layout problem: states of the
    D = C(12,4)^2 = 245025 determinants with 4 alpha and 4 beta electrons
    instead of 2^24 amplitudes (GOCP_BUILD_SECTOR).  Device-resident, CUDA
    events; E and the selected operator are compared with the full layout."""
    import torch
    import paper_2607_15906_gb300 as gb
    from paper_2607_15906_gb300 import _lib

    ints, cfg = config_integrals(WORKLOAD)
    prob = gb.Problem.build(ints, N_ELEC, mapping="jw", precision="c64", int_drop=cfg["int_drop"],
                            term_drop=cfg["term_drop"], device=device, sector=True)
    ops, theta = draw_ansatz(prob.pool_size, N_OPS, seed=0)
    dev = f"cuda:{device}"
    ops_d = torch.from_numpy(ops).to(dev)
    th_d = torch.from_numpy(theta).to(dev)
    ops_g = torch.zeros(N_OPS + 1, dtype=torch.int32, device=dev)
    ops_g[:N_OPS] = ops_d
    th_g = torch.zeros(N_OPS + 1, dtype=torch.float64, device=dev)
    th_g[:N_OPS] = th_d
    ws = prob.workspace()
    e2 = torch.zeros(2, dtype=torch.float64, device=dev)
    g = torch.zeros(prob.pool_size, dtype=torch.float64, device=dev)
    sel = torch.zeros(1, dtype=torch.int32, device=dev)
    e_out = torch.zeros(1, dtype=torch.float64, device=dev)
    de_out = torch.zeros(N_OPS + 1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(device)

    def step():
        prob.adapt_step(ops_d, th_d, ws=ws, tie_rel=1e-4, out=(e2, g, sel))
        ops_g[N_OPS:].copy_(sel)
        prob.energy_grad(ops_g, th_g, ws=ws, out_e=e_out, out_de=de_out)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    _lib.profile_enable(True)
    for kind in range(4):
        _lib.profile_read(kind)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    _lib.profile_enable(False)
    kern = {name: {"launches_per_step": v[0] / steps, "ms_per_step": v[1] / steps}
            for name, v in ((name, _lib.profile_read(kind)) for kind, name in
                            enumerate(["apply_h", "taylor5", "pool_grad", "adjoint"]))}
    ms = a.elapsed_time(b) / steps
    return {"iterations_per_s": 1e3 / ms, "ms_per_step": ms, "state_dim": prob.dim,
            "energy": float(e2[0]), "energy_minus_full": float(e2[0]) - full_e,
            "selected": int(sel[0]), "selected_same_as_full": int(sel[0]) == full_sel,
            "kernels": kern, "steps": steps, "warmup": warmup,
            "note": "GOCP_BUILD_SECTOR: same ADAPT step on the N_a = N_b = 4 determinants only"}


def h_psi_by_n(device: int, peaks, how: str, reps: int = 20):
    """H psi (+E) at 14..24 qubits, complex64 and complex128: the call's
    CUDA-event time and 2S over it against the measured HBM peak (S = the
    state's bytes), for the prepared 100-operator ADAPT state (sector-confined;
    the scatter kernel from the tile size on) and for a dense random state
    (the staged kernel).  Integrals as the 24-qubit workload (decay, drop
    < 1e-3), 2 floor(n/4) electrons (8 at 24 qubits: the bench's state);
    below about 20 qubits both states sit in the 129 MB L2, so L2 rather than
    HBM bounds them."""
    import torch
    import paper_2607_15906_gb300 as gb

    out = {}
    dev = f"cuda:{device}"
    for n_orb in (7, 8, 9, 10, 11, 12):
        nq = 2 * n_orb
        ints = molecular_integrals(n_orb, seed=0, decay=True)
        for prec in ("c64", "c128"):
            n_elec = N_ELEC if nq == 24 else 2 * (nq // 4)
            prob = gb.Problem.build(ints, n_elec, mapping="jw", precision=prec, int_drop=1e-3,
                                    device=device, colour=False)
            ops, theta = draw_ansatz(prob.pool_size, N_OPS, seed=0)
            ws = prob.workspace()
            prob.prepare_state(ops, theta, ws[0])
            dense = torch.randn(1 << nq, dtype=ws[0].dtype, device=dev,
                                generator=torch.Generator(device=dev).manual_seed(nq))
            dense /= torch.linalg.vector_norm(dense)
            e_out = torch.zeros(2, dtype=torch.float64, device=dev)
            stream = torch.cuda.current_stream(device)
            rec = {}
            for label, psi in (("adapt_state", ws[0]), ("dense", dense)):
                for _ in range(3):
                    prob.energy(psi, ws[1], out=e_out)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(reps):
                    prob.energy(psi, ws[1], out=e_out)
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / reps
                alg = 2 * prob.state_bytes()
                rec[label] = {"ms": ms, "gb_s": alg / (ms * 1e-3) / 1e9,
                              "frac_hbm": alg / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
            nnz = int(torch.view_as_real(ws[0]).ne(0).any(-1).sum().item())
            rec["adapt_state"]["nonzero_amplitudes"] = nnz
            out[f"{nq}q_{prec}"] = rec
            del ws, dense
            prob.close()
            torch.cuda.empty_cache()
    return {"note": f"H psi call (kernels + listing), CUDA events, {reps} calls after 3 warm-up; 2S per call against "
                    f"{how} hbm_gbs {peaks['hbm_gbs']:.0f}; the 24-qubit ADAPT state is the bench's", "by_n": out}


def sector_30q(device: int, steps: int = 5, warmup: int = 2):
    """Larger n in the sector layout: the same ADAPT step at 30 qubits (15
    orbitals, 8 electrons, integrals < 1e-3 dropped, 100-operator ansatz
    from the 2684-operator pool): D = C(15,4)^2 = 1,863,225 rows (15 MB per
    complex64 state; the 2^30 layout holds 8.6 GB)."""
    import paper_2607_15906_gb300 as gb

    ints = molecular_integrals(15, seed=0, decay=True)
    t0 = time.time()
    prob = gb.Problem.build(ints, 8, mapping="jw", precision="c64", int_drop=1e-3, device=device, sector=True)
    build_s = time.time() - t0
    t = _adapt_step_timer(prob, device)
    ms = t["timed"](steps, warmup)
    info = prob.info
    out = {"qubits": 30, "state_dim": prob.dim, "pool": prob.pool_size, "n_terms": info["n_terms"],
           "n_groups": info["n_groups"], "build_s": build_s, "device_bytes": info["device_bytes"],
           "iterations_per_s": 1e3 / ms, "ms_per_step": ms, "energy": float(t["e2"][0]),
           "selected": int(t["sel"][0]), "steps": steps, "warmup": warmup}
    prob.close()
    return out


def serving_bench(device: int, n_requests: int = 2000, seed: int = 7, rates=(0.25, 0.5, 1.0, 2.0, 4.0)):
    """Mixed-size energy+gradient stream through the continuous-batching server.

    Requests follow synth.serving_requests (qubits uniform over 10..22,
    Hamiltonian seed 1000+i, 10-80 operators, theta ~ N(0, 0.05), complex64).
    Their Hamiltonians are built before the clock starts (host threads: the
    builder runs outside the GIL).  First every request is submitted at once
    to find the saturation throughput, then the same stream arrives as a
    Poisson process (seed `seed`) at each fraction of that rate; latency is
    completion minus arrival.
    """
    import concurrent.futures as cf

    import paper_2607_15906_gb300 as gb
    from paper_2607_15906_gb300.serving import Server
    from synth import molecular_integrals, serving_requests

    reqs = serving_requests(n_requests, rate_per_s=1.0, seed=seed)

    def build(r):
        ints = molecular_integrals(r.n_orb, seed=r.seed, decay=True)
        return r.index, gb.Problem.build(ints, r.n_elec, precision="c64", device=device, colour=False)

    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        probs = dict(ex.map(build, reqs))
    build_s = time.time() - t0
    ansatz = {r.index: (np.minimum((r.op_draw * probs[r.index].pool_size).astype(np.int32),
                                   probs[r.index].pool_size - 1), r.theta) for r in reqs}

    def run(arrivals):
        lat = []
        with Server(hbm_budget_bytes=0, max_slots=128, device=device) as srv:
            t0 = time.perf_counter()
            pending = {}
            order = sorted(range(len(reqs)), key=lambda i: arrivals[i])
            nxt = 0
            while nxt < len(order) or pending:
                now = time.perf_counter() - t0
                while nxt < len(order) and arrivals[order[nxt]] <= now:
                    i = order[nxt]
                    ops, th = ansatz[i]
                    pending[srv.submit(probs[i], ops, th)] = i
                    nxt += 1
                done = []
                for tk, i in pending.items():
                    if srv.poll(tk, timeout_s=0.0) is not None:
                        lat.append(time.perf_counter() - t0 - arrivals[i])
                        done.append(tk)
                for tk in done:
                    del pending[tk]
                if not done:
                    time.sleep(0.0002)
            total = time.perf_counter() - t0
            st = srv.stats()
        lat = np.array(lat)
        return {"requests": len(lat), "seconds": total, "throughput_rps": len(lat) / total,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_resident": int(st["max_resident"]), "batched_launches": int(st["launches"]),
                "ticks": int(st["ticks"]), "arena_bytes": int(st["arena_bytes"]),
                "arena_peak": int(st["arena_peak"])}

    run(np.zeros(len(reqs)))                                   # warm-up
    sat = run(np.zeros(len(reqs)))
    rate = sat["throughput_rps"]
    out = {"stream": f"{n_requests} requests, qubits uniform 10..22, 10-80 ops, complex64, "
                     f"Hamiltonian seed 1000+i, arrivals seed {seed}",
           "build_s": build_s, "saturation": sat, "saturation_rps": rate}
    for frac in rates:
        gaps = np.random.default_rng(seed).exponential(1.0 / (frac * rate), size=len(reqs))
        out[f"poisson_{frac}x"] = run(np.cumsum(gaps))
    for p in probs.values():
        p.close()
    return out


def c128_iterations(device: int, adjoint_steps: int = 5, plain_steps: int = 2):
    """complex128 on the same 24-qubit workload, both forms timed directly
    with CUDA events:
      adjoint: the bench step itself (adapt_step + energy_grad of the grown
               ansatz by the adjoint sweep) on a complex128 problem;
      plain:   one selection step plus a forward-difference gradient of the
               grown ansatz (the energy at theta and at theta + h e_j for the
               P + 1 = 101 angles: 102 prepare + H psi evaluations)."""
    import torch
    import paper_2607_15906_gb300 as gb

    ints, cfg = config_integrals(WORKLOAD)
    prob = gb.Problem.build(ints, N_ELEC, mapping="jw", precision="c128",
                            int_drop=cfg["int_drop"], term_drop=cfg["term_drop"], device=device)
    t = _adapt_step_timer(prob, device)
    adj_ms = t["timed"](adjoint_steps, 2)
    dev = f"cuda:{device}"
    ws = t["ws"]
    ops_d = torch.from_numpy(t["ops"]).to(dev)
    th_d = torch.from_numpy(t["theta"]).to(dev)
    ops_g = torch.zeros(N_OPS + 1, dtype=torch.int32, device=dev)
    ops_g[:N_OPS] = ops_d
    th_g = torch.zeros(N_OPS + 1, dtype=torch.float64, device=dev)
    th_g[:N_OPS] = th_d
    e2 = torch.zeros(2, dtype=torch.float64, device=dev)
    e_fd = torch.zeros((N_OPS + 2, 2), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(device)
    hstep = 1e-5

    def plain():
        prob.adapt_step(ops_d, th_d, ws=ws, tie_rel=1e-8, out=(e2, t["g"], t["sel"]))
        ops_g[N_OPS:].copy_(t["sel"])
        for j in range(N_OPS + 2):          # j = P + 1: the base point
            th = th_g.clone()
            if j <= N_OPS:
                th[j] += hstep
            prob.prepare_state(ops_g, th, ws[0])
            prob.energy(ws[0], ws[1], out=e_fd[j])

    plain()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(plain_steps):
        plain()
    b.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b) / plain_steps
    fd = ((e_fd[:N_OPS + 1, 0] - e_fd[N_OPS + 1, 0]) / hstep).cpu().numpy()
    prob.energy_grad(ops_g, th_g, ws=ws, out_e=t["e_out"], out_de=t["de_out"])
    adj = t["de_out"].cpu().numpy()
    out = {"adjoint_iterations_per_s": 1e3 / adj_ms, "adjoint_ms_per_step": adj_ms,
           "plain_iterations_per_s": 1e3 / plain_ms, "plain_ms_per_step": plain_ms,
           "plain_max_dE_dtheta_minus_adjoint": float(np.max(np.abs(fd - adj))),
           "steps": {"adjoint": adjoint_steps, "plain": plain_steps},
           "note": "both timed with CUDA events on the launch stream; plain = selection step + "
                   "forward differences (h = 1e-5) over all 101 angles"}
    prob.close()
    return out


def precision_block(device: int, res):
    """Precision of the headline (complex64) results against the complex128
    GPU path on the same inputs (the complex128 path matches the oracle to
    1e-10 relative: tests/test_gpu_bench_state.py), outside the timed region:
    E, fidelity of psi(theta), the pool gradients and dE/dtheta of the grown
    ansatz."""
    import torch
    import paper_2607_15906_gb300 as gb

    ints, cfg = config_integrals(WORKLOAD)
    out = {}
    states, vals = {}, {}
    for prec in ("c64", "c128"):
        prob = res["prob"] if prec == "c64" else gb.Problem.build(
            ints, N_ELEC, mapping="jw", precision="c128", int_drop=cfg["int_drop"],
            term_drop=cfg["term_drop"], device=device)
        ops, theta = draw_ansatz(prob.pool_size, N_OPS, seed=0)
        ws = prob.workspace()
        e, nrm, g, sel = prob.adapt_step(ops, theta, ws=ws, tie_rel=1e-4 if prec == "c64" else 1e-8)
        states[prec] = ws[0].to(torch.complex128, copy=True)   # the adjoint below overwrites ws
        e2, de = prob.energy_grad(np.append(ops, np.int32(sel)).astype(np.int32), np.append(theta, 0.0), ws=ws)
        vals[prec] = dict(e=e, g=g, sel=sel, de=de)
        if prec == "c128":
            prob.close()
    a, b = states["c64"], states["c128"]
    fid = float((torch.abs(torch.vdot(a, b)) ** 2 / (torch.vdot(a, a).real * torch.vdot(b, b).real)).item())
    v64, v128 = vals["c64"], vals["c128"]
    out = {"reference": "complex128 GPU path (matches the oracle to 1e-10 relative)",
           "energy_c64": v64["e"], "energy_c128": v128["e"],
           "abs_energy_error_ha": abs(v64["e"] - v128["e"]), "fidelity": fid, "infidelity": 1.0 - fid,
           "max_gradient_error": float(np.max(np.abs(v64["g"] - v128["g"]))),
           "max_dE_dtheta_error": float(np.max(np.abs(v64["de"] - v128["de"]))),
           "selected_c64": v64["sel"], "selected_c128": v128["sel"],
           "targets": {"abs_energy_error_ha": 1e-6, "infidelity": 1e-6}}
    return out


def adapt_14q(device: int, max_ops: int = 30):
    """Full ADAPT runs on the 14-qubit workload (7 orbitals, 6 electrons,
    204-operator pool) to 30 operators, complex128, under JW and BK: every
    iteration is a device selection step plus a BFGS re-optimisation whose
    energies and gradients come from the adjoint sweep.  Selection ties within
    1e-6 relative go to the lowest index (the BFGS stopping tolerance leaves
    the two mappings' gradients equal only to about 1e-8 relative)."""
    import paper_2607_15906_gb300 as gb
    from paper_2607_15906_gb300.adapt import adapt

    ints, cfg = config_integrals("c2_14q")
    out = {"workload": "14q ADAPT to 30 operators (7 orbitals, 6 electrons, 204-op pool), complex128"}
    runs = {}
    for mp in ("jw", "bk"):
        prob = gb.Problem.build(ints, 6, mapping=mp, precision="c128", device=device)
        t0 = time.perf_counter()
        run = adapt(prob, max_ops=max_ops, gtol=1e-4, tie_rel=1e-6)
        secs = time.perf_counter() - t0
        runs[mp] = run
        out[mp] = {"iterations": len(run.energies) - 1, "seconds": secs,
                   "iterations_per_s": (len(run.energies) - 1) / secs,
                   "energy_evaluations": run.evaluations, "final_energy": run.energies[-1],
                   "grad_norm": run.grad_norms[-1], "families": prob.info["n_families"]}
    same = 0
    while same < min(len(runs["jw"].ops), len(runs["bk"].ops)) and runs["jw"].ops[same] == runs["bk"].ops[same]:
        same += 1
    out["jw_bk_common_operator_prefix"] = same
    out["jw_bk_max_energy_diff"] = float(np.max(np.abs(np.array(runs["jw"].energies) -
                                                        np.array(runs["bk"].energies))))
    return out


def _counters(kernel: str, precision: str = "c64"):
    """ncu counters per launch recorded in profiles/kernel_counters.json
    for the kernel's instance of this precision (key "name<float>" or
    "name<double>"; DRAM bytes, warp instructions), only while the library
    reports the kernel revision they were captured on; else None."""
    try:
        import paper_2607_15906_gb300 as gb
        ver = gb.load().gocp_version().decode()
        key = f"{kernel}<{'float' if precision == 'c64' else 'double'}>"
        rec = json.load(open(os.path.join(ROOT, "profiles", "kernel_counters.json"))).get(key)
        if rec and f"{kernel}={rec['revision']}" in ver:
            return rec
    except Exception:
        pass
    return None


def roofline(res, peaks, how):
    """Dominant kernel class against its roof.

    H psi (Eq. 3) is graded against HBM: algorithmic bytes per launch = 2 S
    (read psi once, write H psi once; S = 2^n x amplitude bytes) over the
    call's CUDA-event duration, against the measured copy bandwidth.  Beside
    it: the FP32-equivalent arithmetic nnz(psi) (T + 4 G) against 152 SMs x
    128 lanes x 2 x clock ("alu"), the issue rate (ncu warp instructions per
    launch over 4 issue slots x 152 SMs x clock), the DRAM traffic (ncu) and
    its redundancy factor traffic / 2 S.  The Taylor, adjoint and gradient
    kernels are graded against HBM with the bytes of the nonzero amplitudes
    they read and write."""
    info = res["info"]
    n = info["n_qubits"]
    dim = 1 << n
    kern = res["kern"]
    tot = {k: v[1] for k, v in kern.items()}
    top = max(tot, key=tot.get)
    launches, ms = kern[top]
    per_launch_s = ms / 1e3 / max(launches, 1)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    amp = 8 if res["prob"].precision == "c64" else 16
    nnz = res.get("nnz", dim)
    if top == "apply_h":
        t, g = info["n_terms"], info["n_groups"]
        frac_env = min(0.25, max(0.0, float(os.environ.get("GOCP_SPARSE_FRAC", "") or 0.125)))
        name = "k_apply_h_sparse" if nnz <= int(frac_env * dim) else "k_apply_h_tiled"
        alg = 2 * dim * amp
        achieved = alg / per_launch_s / 1e9
        out = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{how} hbm_gbs",
               "algorithmic_bytes_per_launch": alg,
               "timed": "the H psi call (the kernel and its amplitude-listing kernels), CUDA events"}
        flops = nnz * (t + 4 * g)
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        out["alu"] = {"achieved": flops / per_launch_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                      "frac": flops / per_launch_s / 1e12 / fp32_peak, "flops_per_launch": flops,
                      "nonzero_amplitudes": nnz,
                      "peak_source": f"FP32 152 SM x 128 lanes x 2 x {sm_mhz:.0f} MHz (recipe unit counts)"}
        c = _counters(name, res["prob"].precision)
        out["traffic"] = c["dram_bytes_per_launch"] if c else None
        out["redundancy"] = (c["dram_bytes_per_launch"] / alg) if c else None
        out["traffic_note"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch: a lower bound "
                               "on the launch's own traffic (output lines still dirty in the 129 MB L2 when the "
                               "kernel ends are written back later)")
        if c and c.get("warp_instructions_per_launch"):
            inst = c["warp_instructions_per_launch"]
            ipeak = 4 * 152 * sm_mhz * 1e6 / 1e9
            out["issue"] = {"warp_instructions_per_launch": inst, "achieved": inst / per_launch_s / 1e9,
                            "peak": ipeak, "unit": "G warp instructions/s",
                            "frac": inst / per_launch_s / 1e9 / ipeak,
                            "peak_source": f"4 issue slots x 152 SMs x {sm_mhz:.0f} MHz"}
        else:
            out["issue"] = None
    else:
        per = {"taylor5": 2 * nnz * amp, "adjoint": 4 * nnz * amp, "pool_grad": 2 * nnz * amp}[top]
        achieved = per / per_launch_s / 1e9
        out = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
               "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{how} hbm_gbs"}
        c = _counters(top, res["prob"].precision)
        out["traffic"] = c["dram_bytes_per_launch"] if c else None
    out["launch_ms"] = per_launch_s * 1e3
    out["launches_per_step"] = launches / max(1, res.get("steps", 1))
    return out


class OracleIteration:
    """The oracle's ADAPT iteration on the bench workload, timed on the host
    cores from a bounded sample (test infrastructure: oracle/ is run only
    here and in tests/).

    One oracle iteration (oracle.statevector on the sparse state, the same
    work as the GPU step): prepare psi(theta) (100 Taylor steps), H psi on the
    rows the products need, E and all 1424 pool gradients, then E and
    dE/dtheta of the grown 101-operator ansatz by forward mode (prepare,
    H psi, one derivative state per angle).  The prepare is timed whole (the
    chain is sequential); H psi rows, gradient generators and derivative
    states are timed on samples and scaled by their counts:
        T = 2 t_prepare + 2 nnz t_row + M t_generator + (P + 1) t_derivative.
    With procs > 1 the sampled parts run on that many spawned workers
    (oracle.parallel), so t_row etc. are per-unit wall times at that width."""

    def __init__(self):
        from oracle import mapping, pool as opool, statevector as sv

        ints, cfg = config_integrals(WORKLOAD)
        self.h = mapping.hamiltonian_table(ints, "jw", cfg["int_drop"], cfg["term_drop"])
        self.tabs = opool.pool_tables(24, N_ELEC, "jw")
        self.ops, self.theta = draw_ansatz(len(self.tabs), N_OPS, seed=0)
        t0 = time.perf_counter()
        self.si, self.svals, self.kept = sv.prepare_state_sparse(
            mapping.hf_index("jw", 24, N_ELEC), self.tabs, self.ops, self.theta, keep_at=range(N_OPS))
        self.t_prepare = time.perf_counter() - t0
        self.rng = np.random.default_rng(11)

    def sample(self, procs: int, rows: int, gens: int, derivs: int, pool=None):
        from oracle import parallel

        nnz = len(self.si)
        r = np.sort(self.rng.choice(self.si, size=min(rows, nnz), replace=False))
        t0 = time.perf_counter()
        parallel.hpsi_rows(self.h, self.si, self.svals, r, n_procs=procs, pool=pool)
        t_row = (time.perf_counter() - t0) / len(r)
        ks = self.rng.choice(len(self.tabs), size=gens, replace=False)
        t0 = time.perf_counter()
        parallel.generator_dots([self.tabs[k] for k in ks], self.si, self.svals, self.si, self.svals,
                                n_procs=procs, pool=pool)
        t_gen = (time.perf_counter() - t0) / gens
        js = np.unique(np.linspace(0, N_OPS - 1, derivs).astype(int))
        t0 = time.perf_counter()
        parallel.derivative_states(self.tabs, self.ops, self.theta, {int(j): self.kept[int(j)] for j in js},
                                   n_procs=procs, workers=pool)
        t_der = (time.perf_counter() - t0) / len(js)
        m = len(self.tabs)
        secs = 2 * self.t_prepare + 2 * nnz * t_row + m * t_gen + (N_OPS + 1) * t_der
        desc = (f"oracle (sparse complex128) iteration: prepare timed whole ({self.t_prepare:.2f} s, serial); "
                f"H psi on {len(r)} of {nnz} rows, {gens} of {m} gradient generators and {len(js)} of "
                f"{N_OPS + 1} derivative states timed on {procs} process(es) and scaled by their counts")
        return secs, desc, {"t_prepare_s": self.t_prepare, "t_row_s": t_row, "t_generator_s": t_gen,
                            "t_derivative_s": t_der}


def cpu_baseline(procs_all: int):
    """The oracle on 1 core and on all cores (bounded samples, about 10 s each)."""
    from oracle import parallel

    it = OracleIteration()
    s1, d1, c1 = it.sample(1, rows=1024, gens=12, derivs=2)
    pool = parallel.start(procs_all)
    try:
        it.sample(procs_all, rows=4 * procs_all, gens=procs_all, derivs=procs_all, pool=pool)   # warm workers
        sn, dn, cn = it.sample(procs_all, rows=512 * procs_all, gens=4 * procs_all, derivs=procs_all,
                               pool=pool)
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    return {"value": 1.0 / sn, "unit": "iterations/s", "cores": procs_all, "kind": "oracle",
            "sample": dn, "components_s": cn, "nproc": os.cpu_count(),
            "one_core": {"value": 1.0 / s1, "cores": 1, "sample": d1, "components_s": c1}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gocp", choices=["gocp", "reference"])
    ap.add_argument("--precision", default="c64", choices=["c64", "c128"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the serving and complex128 sub-measurements")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    config = {"workload": "24q ADAPT iteration: 12 orbitals, 8 electrons, JW, int_drop 1e-3, "
                          "1424-op pool, 100-op ansatz, theta~N(0,0.05), seed 0",
              "qubits": 24, "ansatz_ops": N_OPS, "pool": 1424, "mapping": "jw",
              "l2": "working set 256 MiB (2 states) > 129 MB L2; no flush",
              "parallelism": f"replicas x{args.gpus}"}

    if args.impl == "reference":
        if rank != 0:
            return
        from oracle import parallel
        procs = parallel.procs()
        it = OracleIteration()
        pool = parallel.start(procs)
        vals = []
        try:
            for i in range(max(args.warmup, 0) + args.steps):
                secs, desc, comp = it.sample(procs, rows=512 * procs, gens=4 * procs, derivs=procs, pool=pool)
                if i >= args.warmup:
                    vals.append(secs)
        finally:
            if pool is not None:
                pool.close()
                pool.join()
        secs = float(np.mean(vals))
        value = 1.0 / secs
        line = {"metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic", "config": config, "impl": "reference",
                "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": procs, "kind": "oracle",
                                 "sample": desc, "nproc": os.cpu_count()},
                "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    res = run_gpu(args, rank, world, local)
    res["steps"] = args.steps
    peaks, how = _peaks()
    if rank == 0:
        secs = res["secs"]
        value = replica_throughput(args.steps, world, secs)
        e2e = replica_throughput(args.steps, world, res["e2e_secs"])
        roof = roofline(res, peaks, how)
        kern = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
                for k, v in res["kern"].items()}
        extras = {}
        if world == 1 and args.precision == "c64":
            extras["precision"] = precision_block(local, res)
            extras["sector_layout"] = sector_layout(local, res["e"], res["sel"])
        if not args.no_extras and world == 1:
            extras["c128"] = c128_iterations(local)
            extras["h_psi_by_n"] = h_psi_by_n(local, peaks, how)
            extras["full_layout_28q"] = full_layout_large(local, 14)
            extras["full_layout_30q"] = full_layout_large(local, 15)
            extras["full_layout_32q"] = full_layout_large(local, 16, steps=2)
            extras["sector_30q"] = sector_30q(local)
            extras["adapt_14q"] = adapt_14q(local)
            extras["serving"] = serving_bench(local)
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            from oracle import parallel
            cpu = cpu_baseline(parallel.procs())
        line = {"metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.precision, "data": "synthetic", "config": config,
                "e2e": {"value": e2e, "unit": "iterations/s", "h2d_bytes_per_step": res["h2d"],
                        "d2h_bytes_per_step": res["d2h"]},
                "gpu_launches": res["launches"], "roofline": roof, "cpu_baseline": cpu,
                "clocks": res["clocks"], "kernels": kern, "energy": res["e"], "selected": res["sel"],
                **extras}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
