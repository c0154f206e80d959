"""The conventional circuit (grover_iterate_gate) against the oracle.

Error bound: each butterfly stage of a Walsh-Hadamard pass rounds every output
once, adding an error vector of norm <= u * ||state|| (the normalised stage is
orthogonal; power-of-two scaling is exact; the oracle flip and 2|0><0| - I are
sign changes), and an iteration has 2n stages, so after k iterations
||error||_2 <= 2 n k u (u = 2^-24 for complex64, 2^-53 for complex128).  The
FP64 oracle's butterflies scale by a rounded 1/sqrt(2): three roundings per
stage, 6 n k 2^-53 more.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import c64_bounds
import gate_model
import oracle
from paper_2005_04635_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "three_qubit_101.txt")


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


def tol(dtype, n, k):
    """Bound on the 2-norm of GPU - oracle for a unit-norm state (module docstring)."""
    u = 2.0 ** -24 if dtype == "c64" else 2.0 ** -53
    return 2 * n * max(k, 1) * u + 6 * n * max(k, 1) * 2.0 ** -53 + 1e-15


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,m,k", [(1, 1, 1), (2, 1, 1), (3, 1, 2), (5, 2, 3), (8, 3, 5), (9, 1, 4), (12, 4, 6),
                                   (16, 1, 3), (17, 2, 2), (20, 1, 2)])
def test_gate_matches_oracle_circuit(B, dtype, n, m, k):
    marked = inputs.marked_indices(n, m, seed=500 + n)
    psi0 = inputs.gaussian_state(n, seed=501 + n)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    st = B.State(n, dtype)
    st.init_state(psi0)
    st.iterate_gate(B.Marked(n, marked), k)
    got = to_np(st)
    ref = oracle.grover_gate(psi0.copy(), n, marked, k)
    # the bound is on the error vector's norm (module docstring)
    assert np.linalg.norm(got - ref) <= tol(dtype, n, k)
    # the circuit and the equivalent operator agree (no global phase)
    ref_op = oracle.grover_operator(psi0.copy(), n, marked, k)
    assert np.linalg.norm(got - ref_op) <= tol(dtype, n, k) + 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_gate_equals_operator_path_uniform(B, dtype):
    n, m = 14, 3
    marked = inputs.marked_indices(n, m, seed=77)
    k = B.grover_optimal_iterations(n, m)
    mk = B.Marked(n, marked)
    a = B.State(n, dtype)
    a.init_uniform()
    a.iterate_gate(mk, k)
    b = B.State(n, dtype)
    b.init_uniform()
    b.iterate(mk, k)
    ga, gb = to_np(a), to_np(b)
    # both within their bounds of the exact result: the circuit's (tol, less the
    # oracle's part) and the operator path's (c64_bounds; complex128: 3u per iteration)
    op = c64_bounds.norm_bound(k) if dtype == "c64" else (3 * k + 1) * 2.0 ** -53
    assert np.linalg.norm(ga - gb) <= tol(dtype, n, k) + op
    ps_a, _ = a.success_prob(mk)
    ref = oracle.grover_operator(oracle.init_uniform(n), n, marked, k)
    assert abs(ps_a - oracle.success_prob(ref, n, marked)) <= (1e-10 if dtype == "c128" else 1e-4)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_gate_three_qubit_worked_example(B, dtype):
    """The paper's measurement outcome (|101>, 94.531 % / 0.781 %) through the circuit."""
    rows = []
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line and line.split()[0] not in ("n", "marked", "iterations"):
            a, b_ = line.split()
            rows.append((int(a, 2), float(b_)))
    st = B.State(3, dtype)
    st.init_uniform()
    st.iterate_gate(B.Marked(3, [5]), 2)
    p = st.measure_probs()
    for x, pct in rows:
        assert round(100 * p[x], 3) == pytest.approx(pct, abs=1e-9)
    idx, pp = st.measure_topm(1)
    assert int(idx[0]) == 5


def test_gate_bitmask_and_empty(B):
    n = 10
    marked = inputs.marked_indices(n, 300, seed=3)
    psi0 = inputs.gaussian_state(n, seed=4)
    for mk, mlist in ((B.Marked(n, bitmask=inputs.bitmask(n, marked)), marked), (B.Marked(n, []), [])):
        st = B.State(n, "c128")
        st.init_state(psi0)
        st.iterate_gate(mk, 3)
        ref = oracle.grover_gate(psi0.copy(), n, mlist, 3)
        assert np.max(np.abs(to_np(st) - ref)) <= tol("c128", n, 3)


# ---- tensor-core engine (complex64, n >= 13) ------------------------------------------
# The tolerance is a worst-case bound on the 2-norm of the error vector,
# computed from the state entering every pass (gate_model.error_bound: per
# output (K/16 + 3) u s sum_k |x_k| over the fibre that feeds it, chained
# through the later passes by their norms).  test_gate_model_host.py shows that
# a kernel keeping one bf16 slice of three exceeds it at every size below.  A
# two-slice kernel (2^-16 per operand) is within the worst case of 128 FP32
# accumulations; the exact-arithmetic test below is the one that rejects it.
@pytest.mark.parametrize("n,m,k", [(13, 2, 2), (14, 1, 3), (15, 2, 1), (16, 3, 2), (18, 2, 1), (19, 2, 1), (20, 1, 2),
                                   (22, 4, 1), (23, 1, 1)])
def test_gate_tensor_cores(B, n, m, k):
    marked = inputs.marked_indices(n, m, seed=600 + n)
    psi0 = inputs.gaussian_state(n, seed=601 + n).astype(np.complex64).astype(np.complex128)
    mk = B.Marked(n, marked)
    tc = B.State(n, "c64")
    tc.set_gate_engine(1)
    tc.init_state(psi0)
    tc.iterate_gate(mk, k)
    tc.sync()
    got = to_np(tc)
    ref = oracle.grover_gate(psi0.copy(), n, marked, k)
    bound = gate_model.error_bound(psi0, n, marked, k) + 1e-12
    assert np.linalg.norm(got - ref) <= bound


@pytest.mark.parametrize("engine", [1, 0])
@pytest.mark.parametrize("n", [13, 14, 15, 16, 18, 19, 20, 22, 23])
def test_gate_exact_input(B, engine, n):
    """gate_model.exact_input: C 2^-40 (1 + i/2), C = 2^17 + 511 (a nonzero
    third bf16 slice), times a tensor product over the engine's groups of a
    Walsh row on one block of 16 mids.  Every MMA step (and every butterfly) of
    every pass is exact in FP32 on it, so the iteration, which maps this
    zero-mean state with no marked amplitude in its support to -x, must give
    -x (then +x) bit for bit; a split that dropped the third slice computes
    with C + 1 (test_gate_model_host.py)."""
    x = gate_model.exact_input(n, tensor_cores=engine == 1)
    marked = gate_model.exact_marked(n)
    mk = B.Marked(n, marked)
    st = B.State(n, "c64")
    st.set_gate_engine(engine)
    st.init_state(x)
    for sign in (-1.0, 1.0):
        st.iterate_gate(mk, 1)
        st.sync()
        got = to_np(st)
        assert np.array_equal(got, sign * x), np.max(np.abs(got - sign * x))
    ref = oracle.grover_gate(x.copy(), n, marked, 2)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(x))


@pytest.mark.parametrize("n", [26, 29, 33])
def test_gate_default_engine_exact_input(B, n):
    """The default engine at sizes where it uses the tensor cores: n = 26 (the
    7-bit plan, all four groups on the tensor cores), n = 29 (the 8-bit plan
    has fewer groups: 8, 7, 7, 7, the 7-bit ones on the tensor cores, the
    8-bit one on CUDA cores) and n = 33 (the largest complex64 state, 64 GiB:
    7, 7, 7, 7, 5 on the tensor cores).  Same exact input and closed form (-x,
    then +x) as test_gate_exact_input; the input is built on the device."""
    free, _ = torch.cuda.mem_get_info()
    if free < (4 << 30) + 3 * (8 << n):
        pytest.skip("not enough free device memory")
    plan = gate_model.pass_plan(n, -1)
    assert any(tc for _lo, _kb, tc, _s, _p in plan)
    if n == 29:
        assert any(not tc for _lo, _kb, tc, _s, _p in plan)
    x = torch.ones(1, dtype=torch.complex64, device="cuda")
    for kb in gate_model.engine_groups(n, -1)[0]:
        f = torch.as_tensor(gate_model.exact_factor(kb), dtype=torch.complex64, device="cuda")
        x = torch.kron(f, x)
    x *= complex(gate_model.EXACT_C * gate_model.EXACT_SCALE) * (1.0 + 0.5j)
    mk = B.Marked(n, gate_model.exact_marked(n))
    st = B.State(n, "c64")
    st.init_state(x)
    for sign in (-1.0, 1.0):
        st.iterate_gate(mk, 1)
        st.sync()
        torch.cuda.synchronize()
        assert torch.equal(st.amps, sign * x)
    del st
    torch.cuda.empty_cache()


def test_gate_tensor_cores_uniform_success(B):
    n, m = 16, 1
    marked = inputs.marked_indices(n, m, seed=7)
    k = B.grover_optimal_iterations(n, m)
    mk = B.Marked(n, marked)
    st = B.State(n, "c64")
    st.set_gate_engine(1)
    st.init_uniform()
    st.iterate_gate(mk, k)
    ps, _ = st.success_prob(mk)
    st.sync()
    ref = oracle.grover_operator(oracle.init_uniform(n), n, marked, k)
    assert abs(ps - oracle.success_prob(ref, n, marked)) <= 1e-4
    idx, _ = st.measure_topm(1)
    assert int(idx[0]) == int(marked[0])


def test_gate_tensor_engine_refuses(B):
    st = B.State(12, "c64")
    st.set_gate_engine(1)
    with pytest.raises(B.GroverError):
        st.iterate_gate(B.Marked(12, [1]), 1)
    st2 = B.State(14, "c128")
    st2.set_gate_engine(1)
    with pytest.raises(B.GroverError):
        st2.iterate_gate(B.Marked(14, [1]), 1)


def test_tensor_core_wait_gives_up_and_recovers(B):
    """Failure detection without a GPU fault: the test hook withholds the MMA
    completion signal of one tensor-core pass, its bounded wait (short limit)
    runs out, grover_sync reports GROVER_ETIMEOUT, and the same handle then
    runs a correct search."""
    n = 14
    marked = inputs.marked_indices(n, 2, seed=31)
    mk = B.Marked(n, marked)
    st = B.State(n, "c64")
    st.set_gate_engine(1)
    st.set_option(2, 20000)  # about 2 ms per wait
    st.init_uniform()
    st.set_option(3, 1)
    st.iterate_gate(mk, 1)
    with pytest.raises(B.GroverError) as ei:
        st.sync()
    assert ei.value.status == 4  # GROVER_ETIMEOUT
    st.sync()  # the status word was cleared
    k = B.grover_optimal_iterations(n, 2)
    st.init_uniform()
    st.iterate_gate(mk, k)
    st.sync()
    ref = oracle.grover_operator(oracle.init_uniform(n), n, marked, k)
    bound = gate_model.error_bound(oracle.init_uniform(n), n, marked, k) + (k + 1) * 2.0 ** -22
    assert np.linalg.norm(to_np(st) - ref) <= bound
