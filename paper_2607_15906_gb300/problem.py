"""Python face of a built problem: marshals numpy/torch arguments to the C ABI.

Device buffers are torch tensors (torch owns the memory and the streams);
every computation runs in the CUDA library.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import check, load

try:  # torch is plumbing (device memory, streams); host-only use works without a GPU
    import torch
except Exception:  # pragma: no cover
    torch = None

_MAPPINGS = {"jw": _lib.GOCP_JW, "bk": _lib.GOCP_BK}
_PRECISIONS = {"c64": _lib.GOCP_C64, "c128": _lib.GOCP_C128}


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream(device: int):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Problem:
    """A Hamiltonian + pool built by the library (host tables, optional device copy)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle
        info = _lib.Info()
        check(load().gocp_problem_info(self._h, C.byref(info)), "gocp_problem_info")
        self.info = {f: getattr(info, f) for f, _ in _lib.Info._fields_}

    # ------------------------------------------------------------ construction
    @classmethod
    def build(cls, ints, n_elec: int, mapping: str = "jw", precision: str = "c64",
              int_drop: float = 0.0, term_drop: float = 0.0, device: int = 0,
              colour: bool = True, sector: bool = False) -> "Problem":
        """sector=True: states hold only the determinants with the reference
        state's alpha and beta electron counts (gocp.h, GOCP_BUILD_SECTOR)."""
        h = np.ascontiguousarray(ints.h, dtype=np.float64)
        g = np.ascontiguousarray(ints.g, dtype=np.float64)
        a = _lib.BuildArgs(n_orb=h.shape[0], n_elec=n_elec, mapping=_MAPPINGS[mapping],
                           precision=_PRECISIONS[precision],
                           h=h.ctypes.data_as(C.POINTER(C.c_double)),
                           g=g.ctypes.data_as(C.POINTER(C.c_double)), e0=float(ints.e0),
                           int_drop=int_drop, term_drop=term_drop, device=device,
                           flags=(0 if colour else _lib.GOCP_BUILD_NO_COLOURING)
                           | (_lib.GOCP_BUILD_SECTOR if sector else 0))
        out = C.c_void_p()
        check(load().gocp_build(C.byref(a), C.byref(out)), "gocp_build")
        return cls(out)

    @classmethod
    def from_tables(cls, n_qubits: int, terms, generators, ref_index: int,
                    precision: str = "c64", device: int = 0, colour: bool = True) -> "Problem":
        """terms = (x, z, phase, coeff) arrays; generators = list of such tuples."""
        x, z, ph, c = (np.ascontiguousarray(terms[0], dtype=np.uint32),
                       np.ascontiguousarray(terms[1], dtype=np.uint32),
                       np.ascontiguousarray(terms[2], dtype=np.uint8),
                       np.ascontiguousarray(terms[3], dtype=np.float64))
        offs = np.zeros(len(generators) + 1, dtype=np.int64)
        for i, gen in enumerate(generators):
            offs[i + 1] = offs[i] + len(gen[0])
        cat = lambda k, dt: np.ascontiguousarray(
            np.concatenate([np.asarray(gn[k]) for gn in generators]) if generators else np.zeros(0), dtype=dt)
        ox, oz, oph, oc = cat(0, np.uint32), cat(1, np.uint32), cat(2, np.uint8), cat(3, np.float64)
        a = _lib.TableArgs(
            n_qubits=n_qubits, precision=_PRECISIONS[precision], device=device,
            flags=0 if colour else _lib.GOCP_BUILD_NO_COLOURING, n_terms=len(x),
            x=x.ctypes.data_as(C.POINTER(C.c_uint32)), z=z.ctypes.data_as(C.POINTER(C.c_uint32)),
            phase=ph.ctypes.data_as(C.POINTER(C.c_uint8)), coeff=c.ctypes.data_as(C.POINTER(C.c_double)),
            n_ops=len(generators), op_offsets=offs.ctypes.data_as(C.POINTER(C.c_int64)),
            op_x=ox.ctypes.data_as(C.POINTER(C.c_uint32)), op_z=oz.ctypes.data_as(C.POINTER(C.c_uint32)),
            op_phase=oph.ctypes.data_as(C.POINTER(C.c_uint8)),
            op_coeff=oc.ctypes.data_as(C.POINTER(C.c_double)), ref_index=ref_index)
        out = C.c_void_p()
        check(load().gocp_build_from_tables(C.byref(a), C.byref(out)), "gocp_build_from_tables")
        return cls(out)

    def close(self):
        if getattr(self, "_h", None):
            load().gocp_problem_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ properties
    @property
    def handle(self):
        return self._h

    @property
    def n_qubits(self) -> int:
        return self.info["n_qubits"]

    @property
    def dim(self) -> int:
        """Amplitudes per state: 2^n, or D in the sector layout."""
        return self.info["state_dim"]

    @property
    def sector(self) -> bool:
        return bool(self.info["sector"])

    def expand(self, psi):
        """Sector layout: the 2^n state with psi's amplitudes on the sector."""
        full = torch.empty(1 << self.n_qubits, dtype=self.torch_dtype, device=f"cuda:{self.device}")
        check(load().gocp_sector_expand(self._h, self._state(psi), C.c_void_p(full.data_ptr()),
                                        _stream(self.device)), "sector_expand")
        return full

    def compress(self, full):
        """Sector layout: the sector amplitudes of a 2^n state."""
        if not (isinstance(full, torch.Tensor) and full.is_cuda and full.is_contiguous()
                and full.dtype == self.torch_dtype and full.numel() >= 1 << self.n_qubits):
            raise TypeError("full must be a contiguous CUDA state of 2^n amplitudes")
        psi = self.new_states(1)[0]
        check(load().gocp_sector_compress(self._h, C.c_void_p(full.data_ptr()), self._state(psi),
                                          _stream(self.device)), "sector_compress")
        return psi

    @property
    def pool_size(self) -> int:
        return self.info["pool_size"]

    @property
    def device(self) -> int:
        return self.info["device"]

    @property
    def precision(self) -> str:
        return "c64" if self.info["precision"] == _lib.GOCP_C64 else "c128"

    @property
    def torch_dtype(self):
        return torch.complex64 if self.precision == "c64" else torch.complex128

    def state_bytes(self) -> int:
        return int(load().gocp_state_bytes(self._h))

    # ------------------------------------------------------------ export
    def terms(self):
        t = self.info["n_terms"]
        x = np.zeros(t, np.uint32); z = np.zeros(t, np.uint32)
        ph = np.zeros(t, np.uint8); c = np.zeros(t, np.float64)
        check(load().gocp_export_terms(self._h, _ptr(x), _ptr(z), _ptr(ph), _ptr(c)), "export_terms")
        return x, z, ph, c

    def pool(self):
        m, s = self.info["pool_size"], self.info["n_pool_strings"]
        off = np.zeros(m + 1, np.int64)
        x = np.zeros(s, np.uint32); z = np.zeros(s, np.uint32)
        ph = np.zeros(s, np.uint8); c = np.zeros(s, np.float64); fam = np.zeros(m, np.int32)
        check(load().gocp_export_pool(self._h, _ptr(off), _ptr(x), _ptr(z), _ptr(ph), _ptr(c),
                                      _ptr(fam)), "export_pool")
        return off, x, z, ph, c, fam

    # ------------------------------------------------------------ compute
    def new_states(self, count: int = 1):
        return torch.empty((count, self.dim), dtype=self.torch_dtype, device=f"cuda:{self.device}")

    def _state(self, t, count: int = 1):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise TypeError("states must be contiguous CUDA tensors")
        if t.dtype != self.torch_dtype or t.device.index != self.device:
            raise TypeError(f"state must be {self.torch_dtype} on cuda:{self.device}")
        if t.numel() < count * self.dim:
            raise ValueError("state buffer too small")
        return C.c_void_p(t.data_ptr())

    def _ansatz(self, ops, theta):
        """(ops_ptr, theta_ptr, n, mem, keepalive) for host arrays or CUDA tensors."""
        if torch is not None and isinstance(ops, torch.Tensor) and ops.is_cuda:
            if ops.dtype != torch.int32 or theta.dtype != torch.float64 or not theta.is_cuda:
                raise TypeError("device ansatz needs int32 ops and float64 theta on the GPU")
            ops, theta = ops.contiguous(), theta.contiguous()
            return (C.c_void_p(ops.data_ptr()), C.c_void_p(theta.data_ptr()), int(ops.numel()),
                    _lib.GOCP_MEM_DEVICE, (ops, theta))
        o = np.ascontiguousarray(np.asarray(ops, dtype=np.int32))
        t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        if o.shape != t.shape:
            raise ValueError("ops and theta differ in length")
        return _ptr(o), _ptr(t), int(o.size), _lib.GOCP_MEM_HOST, (o, t)

    def reference_state(self, psi):
        check(load().gocp_reference_state(self._h, self._state(psi), _stream(self.device)), "reference_state")
        return psi

    def prepare_state(self, ops, theta, psi):
        po, pt, n, mem, keep = self._ansatz(ops, theta)
        check(load().gocp_prepare_state(self._h, po, pt, n, mem, self._state(psi), _stream(self.device)),
              "prepare_state")
        return psi

    def taylor_step(self, op: int, theta: float, psi):
        check(load().gocp_taylor_step(self._h, int(op), float(theta), self._state(psi),
                                      _stream(self.device)), "taylor_step")
        return psi

    def apply_h(self, psi, hpsi):
        check(load().gocp_apply_h(self._h, self._state(psi), self._state(hpsi), _stream(self.device)), "apply_h")
        return hpsi

    def energy(self, psi, hpsi, out=None):
        """(E, <psi|psi>) as floats, or written into a CUDA float64 tensor `out` (no sync)."""
        if out is not None:
            check(load().gocp_energy(self._h, self._state(psi), self._state(hpsi),
                                     C.c_void_p(out.data_ptr()), _lib.GOCP_MEM_DEVICE,
                                     _stream(self.device)), "energy")
            return out
        res = np.zeros(2)
        check(load().gocp_energy(self._h, self._state(psi), self._state(hpsi), _ptr(res),
                                 _lib.GOCP_MEM_HOST, _stream(self.device)), "energy")
        return float(res[0]), float(res[1])

    def pool_gradients(self, psi, hpsi, out=None):
        if out is not None:
            check(load().gocp_pool_gradients(self._h, self._state(psi), self._state(hpsi),
                                             C.c_void_p(out.data_ptr()), _lib.GOCP_MEM_DEVICE,
                                             _stream(self.device)), "pool_gradients")
            return out
        g = np.zeros(self.pool_size)
        check(load().gocp_pool_gradients(self._h, self._state(psi), self._state(hpsi), _ptr(g),
                                         _lib.GOCP_MEM_HOST, _stream(self.device)), "pool_gradients")
        return g

    def workspace(self):
        return self.new_states(2)

    def energy_grad(self, ops, theta, ws=None, out_e=None, out_de=None):
        """E and dE/dtheta via the adjoint sweep.  Host arrays in -> floats/numpy out;
        CUDA ops/theta with out_e/out_de CUDA tensors -> device-resident, no sync."""
        ws = self.workspace() if ws is None else ws
        po, pt, n, mem, keep = self._ansatz(ops, theta)
        if mem == _lib.GOCP_MEM_DEVICE:
            check(load().gocp_energy_grad(self._h, po, pt, n, mem, self._state(ws, 2),
                                          C.c_void_p(out_e.data_ptr()), C.c_void_p(out_de.data_ptr()),
                                          _stream(self.device)), "energy_grad")
            return out_e, out_de
        e = np.zeros(1)
        de = np.zeros(max(n, 1))
        check(load().gocp_energy_grad(self._h, po, pt, n, mem, self._state(ws, 2), _ptr(e), _ptr(de),
                                      _stream(self.device)), "energy_grad")
        return float(e[0]), de[:n].copy()

    def adapt_step(self, ops, theta, ws=None, tie_rel: float = 1e-4, out=None):
        """Prepare psi(theta), H psi, E, all pool gradients and the selected operator.
        Host arrays -> (E, norm, grads, selected); with CUDA ansatz pass
        out=(e2, grads, sel) CUDA tensors for a device-resident step."""
        ws = self.workspace() if ws is None else ws
        po, pt, n, mem, keep = self._ansatz(ops, theta)
        if mem == _lib.GOCP_MEM_DEVICE:
            e2, g, sel = out
            check(load().gocp_adapt_step(self._h, po, pt, n, mem, self._state(ws, 2), float(tie_rel),
                                         C.c_void_p(e2.data_ptr()), C.c_void_p(g.data_ptr()),
                                         C.c_void_p(sel.data_ptr()), _stream(self.device)), "adapt_step")
            return out
        e2 = np.zeros(2)
        g = np.zeros(self.pool_size)
        sel = np.zeros(1, np.int32)
        check(load().gocp_adapt_step(self._h, po, pt, n, mem, self._state(ws, 2), float(tie_rel),
                                     _ptr(e2), _ptr(g), _ptr(sel), _stream(self.device)), "adapt_step")
        return float(e2[0]), float(e2[1]), g, int(sel[0])

    def device_errors(self) -> int:
        v = C.c_int(0)
        check(load().gocp_device_errors(self._h, C.byref(v), _stream(self.device)), "device_errors")
        return v.value


def exact_sum(values) -> float:
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
    out = C.c_double(0.0)
    check(load().gocp_exact_sum(_ptr(v), v.size, C.byref(out)), "exact_sum")
    return out.value
