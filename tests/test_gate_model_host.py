"""The host model behind the gate path's tolerances (CPU only).

tests/gate_model.py restates grover_iterate_gate's pass plan, emulates the
complex64 tensor-core passes with one, two or three bf16 slices per operand,
and bounds the error of a correct kernel.  These tests pin the model against
the oracle and show that the tolerances of tests/test_gpu_gate.py can fail:

* on the Gaussian inputs of test_gate_tensor_cores, a kernel that kept one
  bf16 slice would exceed the worst-case bound at every listed size;
* on the exact-arithmetic input of test_gate_exact_input, a kernel that kept
  one or two slices would not return -x bit for bit, while the correct
  three-slice split does, even under a pessimistic model of the tensor core's
  FP32 accumulator (addends aligned to the largest, truncated beyond 24 bits;
  checked here fibre by fibre).

No kernel is built for this: the faulty variants exist only as emulations.
"""
from __future__ import annotations

import numpy as np
import pytest

import gate_model as gm
import oracle
from paper_2005_04635_gb300 import inputs

# the sizes of test_gate_tensor_cores (n, M, k)
TC_CASES = [(13, 2, 2), (14, 1, 3), (15, 2, 1), (16, 3, 2), (18, 2, 1), (19, 2, 1), (20, 1, 2), (22, 4, 1), (23, 1, 1)]


def test_pass_plan_matches_bench_groups():
    import bench
    for n in range(1, 34):
        for tc in (False, True):
            assert gm.groups(n, tc) == bench.gate_groups(n, tc)
            assert sum(gm.groups(n, tc)) == n


def test_model_transform_is_the_oracle_hadamard():
    """The model's passes over all groups, scaled by 2^(-n/2), equal the
    oracle's H^{(x)n} (n butterflies with 1/sqrt(2))."""
    for n in (7, 9, 13, 15):
        x = inputs.gaussian_state(n, seed=90 + n)
        y = x.copy()
        for lo, kb, _tc, _s, _ph in gm.pass_plan(n, True)[: len(gm.groups(n, True))]:
            y = gm.apply_pass(y, n, lo, kb, 1.0)
        ref = oracle.hadamard_all(x.copy(), n)
        assert np.max(np.abs(y * 2.0 ** (-n / 2) - ref)) <= 1e-13


def test_model_iteration_is_the_oracle_circuit():
    """Three exact slices and FP32 stores: the emulation is the conventional
    circuit up to FP32 storage rounding, within the model's own bound."""
    for n, m, k in ((13, 2, 2), (15, 2, 1), (16, 3, 2)):
        marked = inputs.marked_indices(n, m, seed=600 + n)
        psi0 = inputs.gaussian_state(n, seed=601 + n).astype(np.complex64).astype(np.complex128)
        ref = oracle.grover_gate(psi0.copy(), n, marked, k)
        got = gm.emulate(psi0, n, marked, k, 3)
        assert np.linalg.norm(got - ref) <= gm.error_bound(psi0, n, marked, k)


def test_bf16_slices():
    g = np.random.default_rng(5)
    x = (g.standard_normal(1 << 16) * np.exp(g.uniform(-20, 20, 1 << 16))).astype(np.float32)
    three = gm.slices(x, 3)
    assert np.array_equal(three, x.astype(np.float64))  # b0 + b1 + b2 holds all 24 bits
    two = gm.slices(x, 2)
    rel = np.abs(two - x) / np.abs(x)
    assert np.max(rel) <= 2.0 ** -16 and np.mean(rel > 0) > 0.5
    # the constant of the exact-arithmetic input: 131583 = 131072 + 512 - 1
    c = np.array([gm.EXACT_C], dtype=np.float32)
    b0 = gm.bf16_rn(c)
    b1 = gm.bf16_rn(c - b0)
    b2 = gm.bf16_rn(c - b0 - b1)
    assert (float(b0[0]), float(b1[0]), float(b2[0])) == (131072.0, 512.0, -1.0)


@pytest.mark.parametrize("n,m,k", TC_CASES)
def test_one_slice_kernel_exceeds_the_bound(n, m, k):
    """The tolerance of test_gate_tensor_cores is tight enough to reject a
    kernel that kept only b0 (relative error 2^-9 per operand); the correct
    split's own storage rounding stays far inside it."""
    marked = inputs.marked_indices(n, m, seed=600 + n)
    psi0 = inputs.gaussian_state(n, seed=601 + n).astype(np.complex64).astype(np.complex128)
    ref = oracle.grover_gate(psi0.copy(), n, marked, k)
    E = gm.error_bound(psi0, n, marked, k)
    assert np.linalg.norm(gm.emulate(psi0, n, marked, k, 1) - ref) > 10 * E
    assert np.linalg.norm(gm.emulate(psi0, n, marked, k, 3) - ref) < 0.1 * E


@pytest.mark.parametrize("kb", [5, 6, 7])
def test_exact_fibres_under_the_accumulator_model(kb):
    """Premise of the exact-arithmetic test, fibre by fibre: both forms a
    fibre of exact_input takes (the factor, and its transform), at several
    powers of two, come out of the modelled tensor-core pass exactly with
    three slices, with zero guard bits; one or two slices do not."""
    f = gm.exact_factor(kb) * gm.EXACT_C
    W = gm.walsh(kb)
    for v in (f, W @ f):
        for a in (-60, -20, 0, 7):
            x = v * 2.0 ** a
            exact = W @ x
            assert np.array_equal(gm.tc_fibre(x, kb, 3), exact)
            assert not np.array_equal(gm.tc_fibre(x, kb, 2), exact)
            assert not np.array_equal(gm.tc_fibre(x, kb, 1), exact)


def test_exact_fibres_under_fp32_butterflies():
    """The CUDA-core engine's butterflies (FP32, one rounding per stage, any
    stage order) are exact on the same fibre forms, for its group sizes."""
    for kb in (4, 5, 6, 7, 8):
        f = gm.exact_factor(kb) * gm.EXACT_C
        W = gm.walsh(kb)
        for v in (f, W @ f):
            for order in (range(kb), reversed(range(kb))):
                y = v.astype(np.float32)
                for b in order:
                    t = y.reshape(-1, 2, 1 << b)
                    a0 = t[:, 0, :].copy()
                    t[:, 0, :] = a0 + t[:, 1, :]
                    t[:, 1, :] = a0 - t[:, 1, :]
                assert np.array_equal(y.astype(np.float64), W @ v)


@pytest.mark.parametrize("n", [13, 14, 15, 16, 18, 19, 20, 22, 23])
def test_exact_input_separates_the_slices(n):
    """On exact_input the gate path returns -x bit for bit after one
    iteration with three slices; with one or two it does not.  -x is the
    closed form (zero mean, no marked amplitude in the support), and the
    oracle's operator form agrees."""
    x = gm.exact_input(n)
    mk = gm.exact_marked(n)
    assert x[int(mk[0])] == 0 and np.sum(x) == 0
    assert np.array_equal(gm.emulate(x, n, mk, 1, 3), -x)
    for s in (1, 2):
        assert not np.array_equal(gm.emulate(x, n, mk, 1, s), -x)
    ref = oracle.grover_operator(x.copy(), n, mk, 1)
    assert np.max(np.abs(ref + x)) <= 1e-12 * np.max(np.abs(x))
    ref_gate = oracle.grover_gate(x.copy(), n, mk, 1)
    assert np.max(np.abs(ref_gate + x)) <= 1e-12 * np.max(np.abs(x))
