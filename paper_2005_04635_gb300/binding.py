"""Thin ctypes binding of libgrover.so (C ABI in include/grover.h).

Argument marshalling only: torch supplies device memory (a complex64 or
complex128 CUDA tensor of 2^n elements) and the stream; every computation runs
in the library's CUDA kernels.  There is no fallback: if the library is not
built, or no CUDA device is usable, calls raise ``GroverError``.

The module-level functions carry the C names; ``State`` and ``Marked`` are
small owners of the opaque handles.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import library_path

GROVER_OK = 0
STATUS = {0: "GROVER_OK", 1: "GROVER_EINVAL", 2: "GROVER_ENOMEM", 3: "GROVER_ECUDA", 4: "GROVER_ETIMEOUT",
          5: "GROVER_EUNSORTED", 6: "GROVER_EDUP", 7: "GROVER_ERANGE", 8: "GROVER_EUNSUPPORTED"}
C64, C128 = 0, 1
ACC = {"default": 0, "fp32": 1, "kahan": 2, "fp64": 3, "exact": 4}

# every symbol include/grover.h declares, with its ctypes signature
_vp = ctypes.c_void_p
_SIGS = {
    "grover_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "grover_destroy": (ctypes.c_int, [_vp]),
    "grover_set_accum": (ctypes.c_int, [_vp, ctypes.c_int]),
    "grover_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64]),
    "grover_init_uniform": (ctypes.c_int, [_vp]),
    "grover_init_state": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "grover_marked_from_list": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.c_size_t]),
    "grover_marked_from_bitmask": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int]),
    "grover_marked_count": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "grover_marked_destroy": (ctypes.c_int, [_vp]),
    "grover_oracle": (ctypes.c_int, [_vp, _vp]),
    "grover_diffuse": (ctypes.c_int, [_vp]),
    "grover_iterate": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64]),
    "grover_iterate_gate": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64]),
    "grover_iterate_circuit": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.POINTER(ctypes.c_uint64)]),
    "grover_optimal_iterations": (ctypes.c_uint64, [ctypes.c_int, ctypes.c_uint64]),
    "grover_measure_probs": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "grover_measure_topm": (ctypes.c_int, [_vp, ctypes.c_size_t, _vp, _vp]),
    "grover_success_prob": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "grover_iterate_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_uint64, _vp]),
    "grover_batch_amps_needed": (ctypes.c_uint64, [ctypes.c_size_t, _vp]),
    "grover_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_size_t, _vp, _vp, _vp, _vp, _vp, ctypes.c_uint64, _vp]),
    "grover_batch_run": (ctypes.c_int, [_vp]),
    "grover_batch_tune": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint32)]),
    "grover_batch_set_packing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "grover_batch_set_packing_min_qubits": (ctypes.c_int, [_vp, ctypes.c_int]),
    "grover_batch_get_packing": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "grover_batch_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64]),
    "grover_batch_success": (ctypes.c_int, [_vp, _vp]),
    "grover_batch_destroy": (ctypes.c_int, [_vp]),
    "grover_phase_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_uint64, _vp]),
    "grover_phase_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_uint64, _vp, _vp, _vp]),
    "grover_sync": (ctypes.c_int, [_vp]),
    "grover_last_error": (ctypes.c_char_p, [_vp]),
    "grover_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


class GroverError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Loads libgrover.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise GroverError(3, f"{path} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int, handle=None):
    if st != GROVER_OK:
        msg = lib().grover_last_error(handle)
        raise GroverError(st, msg.decode() if msg else "")


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dptr(t):
    """Device pointer of a contiguous CUDA float64 tensor (None for an empty one)."""
    import torch
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float64 tensor")
    return t.data_ptr() if t.numel() else None


def grover_optimal_iterations(n: int, m: int) -> int:
    return int(lib().grover_optimal_iterations(n, m))


class Marked:
    """A validated marked set (the oracle's solution list) on the device."""

    def __init__(self, n: int, indices=None, bitmask=None):
        h = _vp()
        if bitmask is not None:
            if hasattr(bitmask, "data_ptr"):  # device tensor of int32/uint32 words
                st = lib().grover_marked_from_bitmask(ctypes.byref(h), n, bitmask.data_ptr(), bitmask.numel(), 1)
            else:
                w = np.ascontiguousarray(np.asarray(bitmask, dtype=np.uint32))
                st = lib().grover_marked_from_bitmask(ctypes.byref(h), n, w.ctypes.data, w.size, 0)
        else:
            idx = np.ascontiguousarray(np.asarray([] if indices is None else indices, dtype=np.uint64).reshape(-1))
            st = lib().grover_marked_from_list(ctypes.byref(h), n, idx.ctypes.data if idx.size else None, idx.size)
        _check(st)
        self.n = n
        self.handle = h

    @property
    def count(self) -> int:
        m = ctypes.c_uint64()
        _check(lib().grover_marked_count(self.handle, ctypes.byref(m)))
        return int(m.value)

    def close(self):
        if self.handle:
            _check(lib().grover_marked_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """A state handle bound to a caller-owned CUDA tensor of 2^n amplitudes."""

    def __init__(self, n: int, dtype: str = "c64", amps=None, stream=None, device=None):
        import torch
        tdt = {"c64": torch.complex64, "c128": torch.complex128}[dtype]
        if amps is None:
            amps = torch.empty(1 << n, dtype=tdt, device=device or "cuda")
        if amps.dtype != tdt or amps.numel() != (1 << n) or not amps.is_contiguous() or not amps.is_cuda:
            raise ValueError("amps must be a contiguous CUDA tensor of 2**n elements of the given dtype")
        self.n, self.dtype, self.amps = n, dtype, amps
        self.stream = stream
        h = _vp()
        _check(lib().grover_create(ctypes.byref(h), n, C64 if dtype == "c64" else C128, amps.data_ptr(),
                                   _stream_ptr(stream)))
        self.handle = h

    # -- calls with the C names -------------------------------------------------------
    def set_accum(self, mode: str):
        _check(lib().grover_set_accum(self.handle, ACC[mode]), self.handle)

    def set_resident(self, value: int):
        """-1 automatic, 0 one pass per iteration, 1 a persistent iterator
        (cluster, else grid), 2 the grid-wide persistent iterator."""
        _check(lib().grover_set_option(self.handle, 0, int(value)), self.handle)

    def set_gate_engine(self, value: int):
        """-1 automatic (complex64 from n = 26: tensor cores on every group of
        at most 7 bits), 0 CUDA-core butterflies, 1 tensor cores (complex64,
        n >= 13)."""
        _check(lib().grover_set_option(self.handle, 1, int(value)), self.handle)

    def set_staged(self, value: int):
        """-1 automatic (states larger than half the L2 staged through shared
        memory by bulk copies), 0 per-thread loads always, 1 staged whenever
        the state is a whole number of 16 KiB chunks."""
        _check(lib().grover_set_option(self.handle, 4, int(value)), self.handle)

    def set_option(self, opt: int, value: int):
        """grover_set_option: 0 resident, 1 gate engine, 2 wait limit, 3 test
        stall, 4 staged pass."""
        _check(lib().grover_set_option(self.handle, int(opt), int(value)), self.handle)

    def init_uniform(self):
        _check(lib().grover_init_uniform(self.handle), self.handle)

    def init_state(self, amps):
        """amps: a CUDA tensor (device copy) or a numpy array (host copy)."""
        if hasattr(amps, "data_ptr"):
            _check(lib().grover_init_state(self.handle, amps.data_ptr(), 1 if amps.is_cuda else 0), self.handle)
        else:
            npdt = np.complex64 if self.dtype == "c64" else np.complex128
            a = np.ascontiguousarray(np.asarray(amps, dtype=npdt))
            if a.size != (1 << self.n):
                raise ValueError("wrong number of amplitudes")
            _check(lib().grover_init_state(self.handle, a.ctypes.data, 0), self.handle)

    def oracle(self, marked: Marked):
        _check(lib().grover_oracle(self.handle, marked.handle), self.handle)

    def diffuse(self):
        _check(lib().grover_diffuse(self.handle), self.handle)

    def iterate(self, marked: Marked, k: int):
        _check(lib().grover_iterate(self.handle, marked.handle, int(k)), self.handle)

    def iterate_gate(self, marked: Marked, k: int):
        _check(lib().grover_iterate_gate(self.handle, marked.handle, int(k)), self.handle)

    def iterate_circuit(self, marked: Marked, k: int):
        """Conventional circuit gate by gate; returns (gates, full passes)."""
        g, p = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().grover_iterate_circuit(self.handle, marked.handle, int(k), ctypes.byref(g), ctypes.byref(p)),
               self.handle)
        return int(g.value), int(p.value)

    def measure_probs(self, out=None):
        """Returns p_i = |c_i|^2 (FP64): into a CUDA tensor if given, else a numpy array."""
        if out is not None:
            _check(lib().grover_measure_probs(self.handle, out.data_ptr(), 1), self.handle)
            return out
        p = np.empty(1 << self.n, dtype=np.float64)
        _check(lib().grover_measure_probs(self.handle, p.ctypes.data, 0), self.handle)
        return p

    def measure_topm(self, m: int):
        idx = np.zeros(m, dtype=np.uint64)
        p = np.zeros(m, dtype=np.float64)
        _check(lib().grover_measure_topm(self.handle, m, idx.ctypes.data, p.ctypes.data), self.handle)
        return idx, p

    def success_prob(self, marked: Marked):
        ps, nrm = ctypes.c_double(), ctypes.c_double()
        _check(lib().grover_success_prob(self.handle, marked.handle, ctypes.byref(ps), ctypes.byref(nrm)),
               self.handle)
        return ps.value, nrm.value

    def phase_forward(self, marked: Marked, phi, vphi, stats=None):
        """grover_phase_forward; phi, vphi: CUDA float64 tensors of K phases,
        stats: None or a CUDA float64 tensor of 2 (receives P and -log P)."""
        K = int(phi.numel())
        _check(lib().grover_phase_forward(self.handle, marked.handle, _dptr(phi), _dptr(vphi), K,
                                          _dptr(stats) if stats is not None else None), self.handle)

    def phase_backward(self, marked: Marked, phi, vphi, lam, grad_phi, grad_vphi):
        """grover_phase_backward; lam: CUDA complex64 tensor of 2^n (overwritten
        with lambda_0), grad_phi / grad_vphi: CUDA float64 tensors of K."""
        K = int(phi.numel())
        _check(lib().grover_phase_backward(self.handle, marked.handle, _dptr(phi), _dptr(vphi), K,
                                           lam.data_ptr(), _dptr(grad_phi), _dptr(grad_vphi)), self.handle)

    def sync(self):
        _check(lib().grover_sync(self.handle), self.handle)

    def close(self):
        if self.handle:
            _check(lib().grover_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent searches run in one persistent launch (complex64 states).

    n, k: sequences of qubit counts and iteration counts; marked: a sequence of
    sorted index lists.  The states live in one torch tensor (``amps``);
    instance i occupies ``offsets[i] : offsets[i] + 2**n[i]``."""

    def __init__(self, n, k, marked, stream=None, device=None):
        import torch
        count = len(n)
        n_arr = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
        k_arr = np.ascontiguousarray(np.asarray(k, dtype=np.uint64))
        lists = [np.asarray(mk, dtype=np.uint64).reshape(-1) for mk in marked]
        offs = np.zeros(count + 1, dtype=np.uint64)
        offs[1:] = np.cumsum([len(x) for x in lists])
        flat = np.ascontiguousarray(np.concatenate(lists) if offs[-1] else np.zeros(1, dtype=np.uint64))
        need = int(lib().grover_batch_amps_needed(count, n_arr.ctypes.data))
        if need == 0:
            raise GroverError(1, "instances need n in [1, 26]")
        self.amps = torch.empty(need, dtype=torch.complex64, device=device or "cuda")
        self.offsets = np.concatenate([[0], np.cumsum(1 << n_arr.astype(np.int64))])[:-1]
        self.n, self.k, self.marked = n_arr, k_arr, lists
        h = _vp()
        _check(lib().grover_batch_create(ctypes.byref(h), count, n_arr.ctypes.data, k_arr.ctypes.data,
                                         flat.ctypes.data, offs.ctypes.data, self.amps.data_ptr(), need,
                                         _stream_ptr(stream)))
        self.handle = h
        self.count = count

    def run(self):
        _check(lib().grover_batch_run(self.handle))

    def tune(self):
        th, oc = ctypes.c_int(), ctypes.c_uint32()
        _check(lib().grover_batch_tune(self.handle, ctypes.byref(th), ctypes.byref(oc)))
        return th.value, oc.value

    def set_packing(self, cluster_size: int, min_qubits: int | None = None):
        """16: clusters of 16 CTAs for instances with n >= min_qubits (17 by
        default, at least 17); 2: groups of CTAs holding the state in shared
        memory for instances with n >= min_qubits (at least 15); 0 or 1: one
        CTA each."""
        if min_qubits is not None:
            _check(lib().grover_batch_set_packing_min_qubits(self.handle, int(min_qubits)))
        _check(lib().grover_batch_set_packing(self.handle, int(cluster_size)))

    def set_option(self, opt: int, value: int):
        """grover_batch_set_option: 2 wait limit, 3 test stall."""
        _check(lib().grover_batch_set_option(self.handle, int(opt), int(value)))

    def packing(self):
        """(cluster size, threshold in qubits) in use."""
        cs, mq = ctypes.c_int(), ctypes.c_int()
        _check(lib().grover_batch_get_packing(self.handle, ctypes.byref(cs), ctypes.byref(mq)))
        return cs.value, mq.value

    def success(self):
        p = np.empty(self.count, dtype=np.float64)
        _check(lib().grover_batch_success(self.handle, p.ctypes.data))
        return p

    def state(self, i):
        return self.amps[int(self.offsets[i]): int(self.offsets[i]) + (1 << int(self.n[i]))]

    def close(self):
        if self.handle:
            _check(lib().grover_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
