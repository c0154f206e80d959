"""Plain FP64 CPU oracle for the Grover iterator -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``grover_oracle.c`` (plain C,
IEEE double, no FMA contraction) through ctypes and shares no code with the
CUDA path.  States are numpy ``complex128`` arrays of length N = 2^n.

Every function follows a named part of Chattopadhyay & Menon, "Fast simulation
of Grover's quantum search on classical computer" (arXiv 2005.04635):

* ``grover_operator``  -- proposed grover_search: Algorithm "n-qubit Oracle"
  then Algorithm "n-qubit Inversion about Mean", repeated k times.
* ``grover_gate``      -- conventional grover_search (section "Background"):
  oracle, H^{(x)n} (Eq. unitary, Algorithm "1-qubit Unitary Operation"),
  2|0><0| - I, H^{(x)n}.
* ``grover_circuit``   -- the same circuit gate by gate, the oracle built as in
  Fig. oracle1 (X-conjugated multi-controlled gate, phase kickback).
* ``closed_form_uniform`` / ``closed_form_general`` -- the rotation picture of
  G = (2|psi><psi| - I) O used as a pin and as the large-n reference.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle, library_path

_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        build_oracle()
    lib = ctypes.CDLL(path)
    sigs = {
        "or_init_zero": (None, [_dp, ctypes.c_int]),
        "or_init_uniform": (None, [_dp, ctypes.c_int]),
        "or_oracle_list": (None, [_dp, ctypes.c_int, _u64p, ctypes.c_size_t]),
        "or_oracle_bitmask": (None, [_dp, ctypes.c_int, _u32p]),
        "or_mean": (None, [_dp, ctypes.c_int, _dp, _dp]),
        "or_inversion_mean": (None, [_dp, ctypes.c_int]),
        "or_grover_operator": (None, [_dp, ctypes.c_int, _u64p, ctypes.c_size_t, ctypes.c_uint64]),
        "or_grover_operator_bitmask": (None, [_dp, ctypes.c_int, _u32p, ctypes.c_uint64]),
        "or_hadamard_qubit": (None, [_dp, ctypes.c_int, ctypes.c_int]),
        "or_hadamard_all": (None, [_dp, ctypes.c_int]),
        "or_phase_shift_zero": (None, [_dp, ctypes.c_int]),
        "or_grover_gate": (None, [_dp, ctypes.c_int, _u64p, ctypes.c_size_t, ctypes.c_uint64]),
        "or_x_qubit": (None, [_dp, ctypes.c_int, ctypes.c_int]),
        "or_mcz": (None, [_dp, ctypes.c_int, ctypes.c_int]),
        "or_grover_circuit": (ctypes.c_uint64, [_dp, ctypes.c_int, _u64p, ctypes.c_size_t, ctypes.c_uint64]),
        "or_optimal_iterations": (ctypes.c_uint64, [ctypes.c_int, ctypes.c_uint64]),
        "or_closed_form_uniform": (None, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _dp, _dp]),
        "or_closed_form_general": (None, [_dp, ctypes.c_int, _u64p, ctypes.c_size_t, ctypes.c_uint64]),
        "or_probs": (None, [_dp, ctypes.c_int, _dp]),
        "or_norm": (ctypes.c_double, [_dp, ctypes.c_int]),
        "or_success_prob": (ctypes.c_double, [_dp, ctypes.c_int, _u64p, ctypes.c_size_t]),
        "or_topm": (None, [_dp, ctypes.c_int, ctypes.c_size_t, _u64p, _dp]),
        "or_neumaier_sum": (ctypes.c_double, [_dp, ctypes.c_size_t, ctypes.c_size_t]),
        "or_set_mutation": (ctypes.c_int, [ctypes.c_int]),
        "or_phase_grover": (None, [_dp, ctypes.c_int, _u64p, ctypes.c_size_t, _dp, _dp, ctypes.c_uint64]),
        "or_phase_loss": (ctypes.c_double, [_dp, ctypes.c_int, _u64p, ctypes.c_size_t]),
        "or_phase_reduced": (ctypes.c_double, [ctypes.c_int, ctypes.c_uint64, _dp, _dp, ctypes.c_uint64,
                                               _dp, _dp, _dp, _dp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _state(psi: np.ndarray, n: int) -> np.ndarray:
    if psi.dtype != np.complex128 or psi.shape != (1 << n,) or not psi.flags.c_contiguous:
        raise ValueError("oracle state must be a contiguous complex128 array of length 2**n")
    return psi


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _marked(marked) -> np.ndarray:
    arr = np.ascontiguousarray(np.asarray(marked, dtype=np.uint64).reshape(-1))
    return arr


def _u64ptr(a: np.ndarray):
    return a.ctypes.data_as(_u64p)


# ---- state preparation -------------------------------------------------------
def init_zero(n: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().or_init_zero(_dptr(psi), n)
    return psi


def init_uniform(n: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().or_init_uniform(_dptr(psi), n)
    return psi


# ---- proposed method -------------------------------------------------------------
def oracle_list(psi, n, marked):
    m = _marked(marked)
    _load().or_oracle_list(_dptr(_state(psi, n)), n, _u64ptr(m), m.size)
    return psi


def oracle_bitmask(psi, n, words):
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    _load().or_oracle_bitmask(_dptr(_state(psi, n)), n, w.ctypes.data_as(_u32p))
    return psi


def mean(psi, n) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().or_mean(_dptr(_state(psi, n)), n, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def inversion_mean(psi, n):
    _load().or_inversion_mean(_dptr(_state(psi, n)), n)
    return psi


def grover_operator(psi, n, marked, k):
    m = _marked(marked)
    _load().or_grover_operator(_dptr(_state(psi, n)), n, _u64ptr(m), m.size, int(k))
    return psi


def grover_operator_bitmask(psi, n, words, k):
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    _load().or_grover_operator_bitmask(_dptr(_state(psi, n)), n, w.ctypes.data_as(_u32p), int(k))
    return psi


# ---- conventional circuit ------------------------------------------------------------
def hadamard_qubit(psi, n, q):
    _load().or_hadamard_qubit(_dptr(_state(psi, n)), n, q)
    return psi


def hadamard_all(psi, n):
    _load().or_hadamard_all(_dptr(_state(psi, n)), n)
    return psi


def phase_shift_zero(psi, n):
    _load().or_phase_shift_zero(_dptr(_state(psi, n)), n)
    return psi


def grover_gate(psi, n, marked, k):
    m = _marked(marked)
    _load().or_grover_gate(_dptr(_state(psi, n)), n, _u64ptr(m), m.size, int(k))
    return psi


def x_qubit(psi, n, q):
    _load().or_x_qubit(_dptr(_state(psi, n)), n, q)
    return psi


def mcz(psi, n, negate_all=False):
    _load().or_mcz(_dptr(_state(psi, n)), n, 1 if negate_all else 0)
    return psi


def grover_circuit(psi, n, marked, k):
    """Conventional circuit gate by gate (Fig. oracle1 oracle); returns (psi, gates)."""
    m = _marked(marked)
    g = _load().or_grover_circuit(_dptr(_state(psi, n)), n, _u64ptr(m), m.size, int(k))
    return psi, int(g)


# ---- iteration count, closed forms --------------------------------------------
def optimal_iterations(n: int, m: int) -> int:
    return int(_load().or_optimal_iterations(n, m))


def closed_form_uniform(n: int, m: int, k: int):
    a, b = ctypes.c_double(), ctypes.c_double()
    _load().or_closed_form_uniform(n, m, int(k), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def closed_form_general(psi, n, marked, k):
    m = _marked(marked)
    _load().or_closed_form_general(_dptr(_state(psi, n)), n, _u64ptr(m), m.size, int(k))
    return psi


# ---- measurement -------------------------------------------------------------------
def probs(psi, n) -> np.ndarray:
    p = np.empty(1 << n, dtype=np.float64)
    _load().or_probs(_dptr(_state(psi, n)), n, _dptr(p))
    return p


def norm(psi, n) -> float:
    return float(_load().or_norm(_dptr(_state(psi, n)), n))


def success_prob(psi, n, marked) -> float:
    m = _marked(marked)
    return float(_load().or_success_prob(_dptr(_state(psi, n)), n, _u64ptr(m), m.size))


def topm(psi, n, m: int):
    idx = np.zeros(m, dtype=np.uint64)
    p = np.zeros(m, dtype=np.float64)
    _load().or_topm(_dptr(_state(psi, n)), n, m, _u64ptr(idx), _dptr(p))
    return idx, p


def neumaier_sum(x) -> float:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return float(_load().or_neumaier_sum(_dptr(a), a.size, 1))


# ---- generalised phase iterator (differentiation) --------------------------------
def phase_grover(psi, n, marked, phi, vphi):
    m = _marked(marked)
    ph = np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    vp = np.ascontiguousarray(np.asarray(vphi, dtype=np.float64))
    assert ph.size == vp.size
    _load().or_phase_grover(_dptr(_state(psi, n)), n, _u64ptr(m), m.size, _dptr(ph), _dptr(vp), ph.size)
    return psi


def phase_loss(psi, n, marked) -> float:
    m = _marked(marked)
    return float(_load().or_phase_loss(_dptr(_state(psi, n)), n, _u64ptr(m), m.size))


def phase_reduced(n, m, phi, vphi):
    """(loss, alpha, beta) of the two-amplitude model for a uniform start."""
    ph = np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    vp = np.ascontiguousarray(np.asarray(vphi, dtype=np.float64))
    out = [ctypes.c_double() for _ in range(4)]
    loss = _load().or_phase_reduced(n, m, _dptr(ph), _dptr(vp), ph.size, *[ctypes.byref(o) for o in out])
    return float(loss), complex(out[0].value, out[1].value), complex(out[2].value, out[3].value)


def phase_grad_fd(loss_fn, phi, vphi, h=1e-6):
    """Central finite differences of loss_fn(phi, vphi) in FP64."""
    phi = np.asarray(phi, dtype=np.float64)
    vphi = np.asarray(vphi, dtype=np.float64)
    g1, g2 = np.zeros_like(phi), np.zeros_like(vphi)
    for t in range(phi.size):
        for arr, g in ((phi, g1), (vphi, g2)):
            a = arr.copy()
            a[t] += h
            up = loss_fn(a, vphi) if arr is phi else loss_fn(phi, a)
            a[t] -= 2 * h
            dn = loss_fn(a, vphi) if arr is phi else loss_fn(phi, a)
            g[t] = (up - dn) / (2 * h)
    return g1, g2


class mutation:
    """Context manager that plants one known mistake in the oracle (tests only)."""

    def __init__(self, which: int):
        self.which = which

    def __enter__(self):
        self.prev = _load().or_set_mutation(self.which)
        return self

    def __exit__(self, *exc):
        _load().or_set_mutation(self.prev)
        return False


MUTATIONS = {
    1: "inversion loops stop at N-1",
    2: "phase shift I - 2|0><0|",
    3: "update with <c> instead of 2<c>",
    4: "oracle flips index+1",
    5: "imaginary part updated with the wrong sign",
    6: "butterfly outputs swapped",
    7: "closed form rotates the wrong way",
    8: "mean divides by N-1",
}
