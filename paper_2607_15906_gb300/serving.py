"""Continuous-batching energy+gradient server (marshalling over the C ABI)."""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import GocpError, check, load


class Server:
    """Requests (problem, ansatz ops, angles) -> (E, dE/dtheta), batched on one GPU."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, device: int = 0):
        self._s = C.c_void_p()
        check(load().gocp_server_create(int(hbm_budget_bytes), int(max_slots), int(device),
                                        C.byref(self._s)), "server_create")
        self._n_ops = {}

    def submit(self, problem, ops, theta) -> int:
        o = np.ascontiguousarray(np.asarray(ops, dtype=np.int32))
        t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        if o.shape != t.shape:
            raise ValueError("ops and theta differ in length")
        tk = C.c_uint64(0)
        check(load().gocp_submit(self._s, problem.handle, o.ctypes.data_as(C.c_void_p),
                                 t.ctypes.data_as(C.c_void_p), int(o.size), C.byref(tk)), "submit")
        self._n_ops[tk.value] = int(o.size)
        return tk.value

    def poll(self, ticket: int, timeout_s: float | None = 0.0):
        """(E, dE) when finished; None if not finished within the timeout."""
        n = self._n_ops.get(ticket, 0)
        e = C.c_double(0.0)
        de = np.zeros(max(n, 1))
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        rc = load().gocp_poll(self._s, C.c_uint64(ticket), C.byref(e), de.ctypes.data_as(C.c_void_p), us)
        if rc in (_lib.GOCP_EAGAIN, _lib.GOCP_ETIMEDOUT):
            return None
        self._n_ops.pop(ticket, None)
        check(rc, "poll")
        return float(e.value), de[:n].copy()

    def result(self, ticket: int):
        return self.poll(ticket, timeout_s=None)

    def cancel(self, ticket: int) -> None:
        check(load().gocp_cancel(self._s, C.c_uint64(ticket)), "cancel")

    def stats(self) -> dict:
        st = _lib.ServerStats()
        check(load().gocp_server_get_stats(self._s, C.byref(st)), "server_stats")
        return {f: getattr(st, f) for f, _ in _lib.ServerStats._fields_}

    def close(self):
        if getattr(self, "_s", None) and self._s.value:
            load().gocp_server_destroy(self._s)
            self._s = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Server", "GocpError"]
