"""The conventional circuit gate by gate (grover_iterate_circuit) against the
FP64 oracle's gate-by-gate circuit (Fig. oracle1 oracle, X / MCZ phase shift,
per-qubit Hadamards) and against the operator path.

Tolerance: X gates and the multi-controlled Z are exact; each Hadamard pass
rounds a + b (or a - b) and the product with the rounded 1/sqrt(2), and the
rounded scale itself is off by at most one unit: an error vector of norm at
most 4 u per Hadamard pass for a unit-norm state, and unitary gates do not
amplify it.  k iterations hold 2 n k Hadamard passes: the error vector has
norm <= 8 n k u ||psi|| (checked as a norm), plus the FP64 oracle's own
rounding (three per butterfly stage, 6 n k 2^-53 ||psi||).
"""
from __future__ import annotations

import numpy as np
import pytest

import c64_bounds
import oracle
from paper_2005_04635_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = {"c64": 2.0 ** -24, "c128": 2.0 ** -53}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_04635_gb300 import binding
    binding.lib()
    return binding


def to_np(st):
    torch.cuda.synchronize()
    return st.amps.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,m,k", [(1, 1, 2), (2, 1, 1), (3, 2, 2), (5, 3, 2), (8, 1, 3), (12, 4, 2), (14, 2, 1)])
def test_circuit_matches_oracle(B, dtype, n, m, k):
    marked = inputs.marked_indices(n, m, seed=800 + n)
    psi0 = inputs.gaussian_state(n, seed=801 + n)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    st = B.State(n, dtype)
    st.init_state(psi0)
    gates, passes = st.iterate_circuit(B.Marked(n, marked), k)
    ref, ref_gates = oracle.grover_circuit(psi0.copy(), n, marked, k)
    assert gates == ref_gates
    zeros = sum(n - bin(int(x)).count("1") for x in marked)
    assert passes == k * (2 * zeros + 4 * n)
    bound = (8 * n * k * U[dtype] + 6 * n * k * U["c128"]) * np.linalg.norm(ref)
    assert np.linalg.norm(to_np(st) - ref) <= bound + 1e-300


def test_circuit_equals_operator_path_uniform(B):
    n, m, k = 20, 2, 3
    marked = inputs.marked_indices(n, m, seed=810)
    mk = B.Marked(n, marked)
    a = B.State(n, "c64")
    a.init_uniform()
    a.iterate_circuit(mk, k)
    b = B.State(n, "c64")
    b.init_uniform()
    b.set_resident(0)
    b.iterate(mk, k)
    # the circuit's error (8nku, gate by gate) plus the operator path's (c64_bounds)
    assert np.max(np.abs(to_np(a) - to_np(b))) <= 8 * n * k * U["c64"] + c64_bounds.norm_bound(k)


def test_circuit_empty_and_bitmask(B):
    n = 6
    psi0 = inputs.gaussian_state(n, seed=820)
    st = B.State(n, "c128")
    st.init_state(psi0)
    gates, passes = st.iterate_circuit(B.Marked(n, []), 2)
    assert gates == 2 * (2 * n + 2 * n + 1) and passes == 2 * 4 * n
    ref, _ = oracle.grover_circuit(psi0.copy(), n, [], 2)
    assert np.max(np.abs(to_np(st) - ref)) <= 1e-13
    with pytest.raises(B.GroverError) as ei:
        st.iterate_circuit(B.Marked(n, bitmask=inputs.bitmask(n, [3, 9])), 1)
    assert ei.value.status == 8
