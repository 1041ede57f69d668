"""ctypes declarations of include/gocp.h and library loading.

The shared library is the only compute path: importing this module fails
loudly when it has not been built (there is no CPU fallback).
"""

from __future__ import annotations

import ctypes as C
import os

from . import build as _build

GOCP_OK, GOCP_EINVAL, GOCP_ENOMEM, GOCP_ECUDA = 0, -1, -2, -3
GOCP_EAGAIN, GOCP_ETIMEDOUT, GOCP_ECANCELED, GOCP_ENODEV = -4, -5, -6, -7
GOCP_JW, GOCP_BK = 0, 1
GOCP_C64, GOCP_C128 = 0, 1
GOCP_MEM_HOST, GOCP_MEM_DEVICE = 0, 1
GOCP_BUILD_NO_COLOURING, GOCP_BUILD_SECTOR = 1, 2
KERNEL_APPLY_H, KERNEL_TAYLOR, KERNEL_POOL_GRAD, KERNEL_ADJOINT = 0, 1, 2, 3

_NAMES = {GOCP_EINVAL: "EINVAL", GOCP_ENOMEM: "ENOMEM", GOCP_ECUDA: "ECUDA", GOCP_EAGAIN: "EAGAIN",
          GOCP_ETIMEDOUT: "ETIMEDOUT", GOCP_ECANCELED: "ECANCELED", GOCP_ENODEV: "ENODEV"}


class GocpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gocp {_NAMES.get(code, code)}: {msg}")
        self.code = code


class BuildArgs(C.Structure):
    _fields_ = [("n_orb", C.c_int), ("n_elec", C.c_int), ("mapping", C.c_int), ("precision", C.c_int),
                ("h", C.POINTER(C.c_double)), ("g", C.POINTER(C.c_double)), ("e0", C.c_double),
                ("int_drop", C.c_double), ("term_drop", C.c_double), ("device", C.c_int),
                ("flags", C.c_int)]


class TableArgs(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("precision", C.c_int), ("device", C.c_int), ("flags", C.c_int),
                ("n_terms", C.c_int64), ("x", C.POINTER(C.c_uint32)), ("z", C.POINTER(C.c_uint32)),
                ("phase", C.POINTER(C.c_uint8)), ("coeff", C.POINTER(C.c_double)),
                ("n_ops", C.c_int), ("op_offsets", C.POINTER(C.c_int64)),
                ("op_x", C.POINTER(C.c_uint32)), ("op_z", C.POINTER(C.c_uint32)),
                ("op_phase", C.POINTER(C.c_uint8)), ("op_coeff", C.POINTER(C.c_double)),
                ("ref_index", C.c_uint32)]


class Info(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("n_elec", C.c_int), ("mapping", C.c_int), ("precision", C.c_int),
                ("device", C.c_int), ("pool_size", C.c_int), ("n_families", C.c_int),
                ("ref_index", C.c_uint32), ("n_terms", C.c_int64), ("n_groups", C.c_int64),
                ("n_pool_strings", C.c_int64), ("device_bytes", C.c_size_t), ("state_dim", C.c_int64),
                ("sector", C.c_int), ("n_alpha", C.c_int), ("n_beta", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("cancelled", C.c_uint64),
                ("ticks", C.c_uint64), ("launches", C.c_uint64), ("max_resident", C.c_uint64),
                ("arena_bytes", C.c_size_t), ("arena_in_use", C.c_size_t), ("arena_peak", C.c_size_t),
                ("resident", C.c_int), ("queued", C.c_int)]


P = C.c_void_p
_SIGS = {
    "gocp_build": (C.c_int, [C.POINTER(BuildArgs), C.POINTER(P)]),
    "gocp_build_from_tables": (C.c_int, [C.POINTER(TableArgs), C.POINTER(P)]),
    "gocp_problem_info": (C.c_int, [P, C.POINTER(Info)]),
    "gocp_export_terms": (C.c_int, [P, P, P, P, P]),
    "gocp_export_pool": (C.c_int, [P, P, P, P, P, P, P]),
    "gocp_problem_free": (None, [P]),
    "gocp_exact_sum": (C.c_int, [P, C.c_int64, C.POINTER(C.c_double)]),
    "gocp_state_bytes": (C.c_size_t, [P]),
    "gocp_reference_state": (C.c_int, [P, P, P]),
    "gocp_prepare_state": (C.c_int, [P, P, P, C.c_int, C.c_int, P, P]),
    "gocp_taylor_step": (C.c_int, [P, C.c_int, C.c_double, P, P]),
    "gocp_apply_h": (C.c_int, [P, P, P, P]),
    "gocp_sector_expand": (C.c_int, [P, P, P, P]),
    "gocp_sector_compress": (C.c_int, [P, P, P, P]),
    "gocp_energy": (C.c_int, [P, P, P, P, C.c_int, P]),
    "gocp_energy_static": (C.c_int, [P, P, P, P, C.c_int, P]),
    "gocp_pool_gradients": (C.c_int, [P, P, P, P, C.c_int, P]),
    "gocp_energy_grad": (C.c_int, [P, P, P, C.c_int, C.c_int, P, P, P, P]),
    "gocp_adapt_step": (C.c_int, [P, P, P, C.c_int, C.c_int, P, C.c_double, P, P, P, P]),
    "gocp_device_errors": (C.c_int, [P, C.POINTER(C.c_int), P]),
    "gocp_server_create": (C.c_int, [C.c_size_t, C.c_int, C.c_int, C.POINTER(P)]),
    "gocp_server_destroy": (None, [P]),
    "gocp_submit": (C.c_int, [P, P, P, P, C.c_int, C.POINTER(C.c_uint64)]),
    "gocp_poll": (C.c_int, [P, C.c_uint64, P, P, C.c_int64]),
    "gocp_cancel": (C.c_int, [P, C.c_uint64]),
    "gocp_server_get_stats": (C.c_int, [P, C.POINTER(ServerStats)]),
    "gocp_profile_enable": (C.c_int, [C.c_int]),
    "gocp_profile_read": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "gocp_last_error": (C.c_char_p, []),
    "gocp_launch_count": (C.c_int64, []),
    "gocp_version": (C.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """The loaded library; raises if it is not built (unless asked to build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise GocpError(GOCP_ENODEV, f"CUDA library not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int, what: str = "") -> int:
    if rc != GOCP_OK:
        msg = load().gocp_last_error().decode(errors="replace")
        raise GocpError(rc, f"{what}: {msg}" if what else msg)
    return rc


def launch_count() -> int:
    return int(load().gocp_launch_count())


def profile_enable(on: bool) -> None:
    check(load().gocp_profile_enable(1 if on else 0), "profile_enable")


def profile_read(kind: int):
    """(launches, total_ms) of one kernel kind since the last read."""
    n = C.c_int64(0)
    ms = C.c_double(0.0)
    check(load().gocp_profile_read(kind, C.byref(n), C.byref(ms)), "profile_read")
    return int(n.value), float(ms.value)
