"""bench.py's roofline accounting (host logic, no GPU).

H psi is graded against HBM with 2 S algorithmic bytes per launch (psi read
once, H psi written once, S = 2^n x amplitude bytes); beside it the
FP32-equivalent count nnz(psi) (T + 4G) FLOPs per launch (one signed add per
term and one complex x real multiply-add per group, per nonzero source
amplitude).  The chain and gradient kernels are counted as the bytes of the
nonzero amplitudes they read and write.  The kernel named is the one the
library chooses: the scatter kernel at or below GOCP_SPARSE_FRAC (default
1/8, at most 1/4) of 2^n nonzero amplitudes."""

import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.path.insert(0, ROOT)
    spec.loader.exec_module(mod)
    return mod


class _Prob:
    def __init__(self, precision):
        self.precision = precision


def _res(top_ms, top="apply_h", nnz=1000, n=20, precision="c64"):
    kern = {"apply_h": (2, 1.0), "taylor5": (201, 0.5), "pool_grad": (2, 0.2), "adjoint": (102, 0.3)}
    kern[top] = (kern[top][0], top_ms)
    return {"info": {"n_qubits": n, "n_terms": 500, "n_groups": 100}, "kern": kern, "nnz": nnz,
            "prob": _Prob(precision), "steps": 1}


PEAKS = {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}


@pytest.mark.parametrize("precision,amp", [("c64", 8), ("c128", 16)])
def test_h_psi_graded_on_hbm_with_alu_beside(monkeypatch, precision, amp):
    monkeypatch.delenv("GOCP_SPARSE_FRAC", raising=False)
    b = _bench()
    r = b.roofline(_res(10.0, nnz=1000, precision=precision), PEAKS, "measured")
    per_launch_s = 10.0 / 1e3 / 2
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["algorithmic_bytes_per_launch"] == 2 * (1 << 20) * amp
    assert r["achieved"] == pytest.approx(2 * (1 << 20) * amp / per_launch_s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])
    a = r["alu"]
    assert a["flops_per_launch"] == 1000 * (500 + 4 * 100)
    assert a["achieved"] == pytest.approx(1000 * 900 / per_launch_s / 1e12)
    assert a["frac"] == pytest.approx(a["achieved"] / (152 * 128 * 2 * 2070e6 / 1e12))
    assert a["nonzero_amplitudes"] == 1000


@pytest.mark.parametrize("frac_env,nnz,expect", [
    (None, (1 << 20) // 8, "k_apply_h_sparse"),
    (None, (1 << 20) // 8 + 1, "k_apply_h_tiled"),
    ("0", 10, "k_apply_h_tiled"),
    ("1", (1 << 20) // 4, "k_apply_h_sparse"),      # clamped to 1/4
    ("1", (1 << 20) // 4 + 1, "k_apply_h_tiled"),
])
def test_h_psi_kernel_named_as_the_library_chooses(monkeypatch, frac_env, nnz, expect):
    if frac_env is None:
        monkeypatch.delenv("GOCP_SPARSE_FRAC", raising=False)
    else:
        monkeypatch.setenv("GOCP_SPARSE_FRAC", frac_env)
    r = _bench().roofline(_res(10.0, nnz=nnz, n=20), PEAKS, "measured")
    assert r["kernel"] == expect


@pytest.mark.parametrize("top,factor", [("taylor5", 2), ("adjoint", 4), ("pool_grad", 2)])
@pytest.mark.parametrize("precision,amp", [("c64", 8), ("c128", 16)])
def test_chain_kernels_count_nonzero_bytes(top, factor, precision, amp):
    res = _res(50.0, top=top, nnz=4096, precision=precision)
    r = _bench().roofline(res, PEAKS, "measured")
    launches = res["kern"][top][0]
    per_launch_s = 50.0 / 1e3 / launches
    assert r["bound"] == "hbm" and r["kernel"] == top
    assert r["achieved"] == pytest.approx(factor * 4096 * amp / per_launch_s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])
