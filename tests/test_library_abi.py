"""The C-ABI library loads, exports every symbol include/grover.h declares, and
rejects bad arguments on the host before touching the GPU (CPU only)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2005_04635_gb300 import binding
from paper_2005_04635_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grover.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(gbuild.library_path()):
        gbuild.build()
    return binding.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grover_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("grover_create", "grover_init_uniform", "grover_init_state", "grover_marked_from_list",
                 "grover_marked_from_bitmask", "grover_oracle", "grover_diffuse", "grover_iterate",
                 "grover_iterate_gate", "grover_measure_probs", "grover_measure_topm", "grover_success_prob",
                 "grover_sync", "grover_last_error", "grover_optimal_iterations"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"libgrover.so does not export {name}"
        assert name in binding._SIGS, f"binding has no signature for {name}"


def test_status_strings(lib):
    for code, name in binding.STATUS.items():
        assert lib.grover_status_string(code).decode() == name


def test_optimal_iterations(lib):
    f = binding.grover_optimal_iterations
    assert f(3, 1) == 2 and f(12, 1) == 50
    assert [f(28, m) for m in (1, 4, 16)] == [12867, 6433, 3216]
    assert f(33, 1) == 72792 and f(26, 8) == 2274
    assert f(10, 0) == 0 and f(0, 1) == 0 and f(64, 1) == 0


def _marked(lib, n, idx):
    h = ctypes.c_void_p()
    a = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    st = lib.grover_marked_from_list(ctypes.byref(h), n, a.ctypes.data if a.size else None, a.size)
    return st, h


def test_marked_list_validation(lib):
    st, _ = _marked(lib, 4, [3, 1])
    assert binding.STATUS[st] == "GROVER_EUNSORTED"
    st, _ = _marked(lib, 4, [1, 1])
    assert binding.STATUS[st] == "GROVER_EDUP"
    st, _ = _marked(lib, 4, [1, 16])
    assert binding.STATUS[st] == "GROVER_ERANGE"
    assert b"16" in lib.grover_last_error(None)
    st, _ = _marked(lib, 0, [0])
    assert binding.STATUS[st] == "GROVER_EINVAL"
    st, _ = _marked(lib, 34, [0])
    assert binding.STATUS[st] == "GROVER_EINVAL"
    assert lib.grover_marked_from_list(None, 4, None, 0) == 1
    a = np.zeros(1, dtype=np.uint64)
    assert lib.grover_marked_from_list(ctypes.byref(ctypes.c_void_p()), 4, None, 1) == 1


def test_bitmask_validation(lib):
    h = ctypes.c_void_p()
    w = np.zeros(3, dtype=np.uint32)
    st = lib.grover_marked_from_bitmask(ctypes.byref(h), 6, w.ctypes.data, 3, 0)  # 2^6 needs 2 words
    assert binding.STATUS[st] == "GROVER_ERANGE"
    st = lib.grover_marked_from_bitmask(ctypes.byref(h), 6, None, 2, 0)
    assert binding.STATUS[st] == "GROVER_EINVAL"


def test_create_validation(lib):
    h = ctypes.c_void_p()
    assert lib.grover_create(None, 4, 0, 16, None) == 1
    assert lib.grover_create(ctypes.byref(h), 4, 0, None, None) == 1  # NULL buffer
    assert lib.grover_create(ctypes.byref(h), 4, 0, 8, None) == 1  # misaligned
    assert lib.grover_create(ctypes.byref(h), 34, 0, 16, None) == 1  # n too large for c64
    assert lib.grover_create(ctypes.byref(h), 33, 1, 16, None) == 1  # n too large for c128
    assert lib.grover_create(ctypes.byref(h), 4, 7, 16, None) == 1  # bad dtype
    assert h.value is None


def test_set_option_validation(lib):
    assert lib.grover_set_option(None, 0, -1) == 1


def test_null_handles(lib):
    for fn in ("grover_init_uniform", "grover_diffuse", "grover_sync"):
        assert getattr(lib, fn)(None) == 1
    assert lib.grover_iterate(None, None, 1) == 1
    assert lib.grover_destroy(None) == 0 and lib.grover_marked_destroy(None) == 0


def test_null_handles_of_the_extended_calls(lib):
    """Host-side validation of the phase, circuit, batch and allocation-free calls
    (no device work is reached)."""
    assert lib.grover_phase_forward(None, None, None, None, 0, None) == 1
    assert lib.grover_phase_backward(None, None, None, None, 0, None, None, None) == 1
    assert lib.grover_iterate_circuit(None, None, 1, None, None) == 1
    assert lib.grover_iterate_gate(None, None, 1) == 1
    assert lib.grover_batch_set_packing(None, 16) == 1
    assert lib.grover_batch_set_packing_min_qubits(None, 19) == 1
    assert lib.grover_batch_get_packing(None, None, None) == 1
    assert lib.grover_batch_set_option(None, 2, 1000) == 1
    assert lib.grover_batch_run(None) == 1
    assert lib.grover_batch_destroy(None) == 0
    assert lib.grover_batch_amps_needed(2, (ctypes.c_int * 2)(5, 27)) == 0  # n above 26
    assert lib.grover_batch_amps_needed(2, (ctypes.c_int * 2)(5, 6)) == 32 + 64
    assert lib.grover_iterate_noalloc(None, 10, 0, None, 0, 1, None) == 1


def header_enum(name_prefix):
    """(name, value) pairs of the header's enum constants starting with name_prefix."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + name_prefix + r"[A-Z_0-9]*)\s*=\s*(\d+)", text)}


def test_binding_option_ids_match_the_header():
    """The option ids the Python helpers pass to grover_set_option are the
    header's grover_option values (a renumbering would silently set the wrong
    option otherwise)."""
    opts = header_enum("GROVER_OPT_")
    assert opts == {"GROVER_OPT_RESIDENT": 0, "GROVER_OPT_GATE_ENGINE": 1, "GROVER_OPT_WAIT_LIMIT": 2,
                    "GROVER_OPT_TEST_STALL": 3, "GROVER_OPT_STAGED_PASS": 4}
    src = open(os.path.join(ROOT, "paper_2005_04635_gb300", "binding.py")).read()
    for helper, opt in (("set_resident", "GROVER_OPT_RESIDENT"), ("set_gate_engine", "GROVER_OPT_GATE_ENGINE"),
                        ("set_staged", "GROVER_OPT_STAGED_PASS")):
        body = src[src.index("def " + helper):]
        body = body[:body.index("\n    def ", 1)]
        m = re.search(r"grover_set_option\(self\.handle, (\d+),", body)
        assert m and int(m.group(1)) == opts[opt], helper
