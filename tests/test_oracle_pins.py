"""Pins for the FP64 CPU oracle (CPU only).

The oracle is checked against things other than itself: the paper's printed
three-qubit example, dense brute-force matrices built independently with numpy
Kronecker products (n <= 6), the textbook closed forms, exact special cases,
invariants (norm, involutions, reversibility) and library routines
(math.fsum, numpy sorting).  ``test_planted_mistakes_are_caught`` shows that
each plausible slip in the oracle fails at least one pin.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from paper_2005_04635_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "three_qubit_101.txt")


def read_golden(path=GOLDEN):
    meta, rows = {}, []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            a, b = line.split()
            if a in ("n", "marked", "iterations"):
                meta[a] = int(b)
            else:
                rows.append((int(a, 2), float(b)))
    return meta, rows


# --- dense brute force (independent of the oracle: numpy matrices) -------------
def dense_hadamard(n):
    h = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
    H = np.array([[1.0]])
    for _ in range(n):
        H = np.kron(H, h)
    return H


def dense_delta(n):
    """Section 'Inversion About Mean Operator': Delta_ii = 2/N - 1, Delta_ij = 2/N."""
    N = 1 << n
    return np.full((N, N), 2.0 / N) - np.eye(N)


def dense_oracle(n, marked):
    d = np.ones(1 << n)
    d[np.asarray(marked, dtype=np.int64)] = -1.0
    return np.diag(d)


def dense_phase_shift(n):
    """2|0><0| - I."""
    d = -np.ones(1 << n)
    d[0] = 1.0
    return np.diag(d)


# --- the paper's worked example --------------------------------------------------
@pytest.mark.parametrize("form", ["operator", "gate"])
def test_three_qubit_worked_example(form):
    meta, rows = read_golden()
    n, k = meta["n"], meta["iterations"]
    marked = [meta["marked"]]
    if form == "operator":
        psi = oracle.grover_operator(oracle.init_uniform(n), n, marked, k)
    else:  # |0>, H^{(x)n}, then the circuit
        psi = oracle.hadamard_all(oracle.init_zero(n), n)
        psi = oracle.grover_gate(psi, n, marked, k)
    p = oracle.probs(psi, n)
    for x, pct in rows:
        assert round(100.0 * p[x], 3) == pytest.approx(pct, abs=1e-9), (x, p[x])
    # exact dyadic values behind the rounded percentages: 121/128 and 1/128.
    # The operator form rounds only 1/sqrt(8); the circuit also rounds 1/sqrt(2)
    # in each of its (2k+1)n butterfly layers.
    tol = 4e-16 if form == "operator" else 8e-15
    assert abs(p[5] - 121.0 / 128.0) <= tol
    others = np.delete(p, 5)
    assert np.max(np.abs(others - 1.0 / 128.0)) <= tol / 8
    # amplitudes 11/(4 sqrt 8) and -1/(4 sqrt 8), signs included
    assert abs(psi[5].real - 11.0 / (4.0 * math.sqrt(8.0))) <= 2.5 * tol
    assert np.max(np.abs(np.delete(psi, 5) + 1.0 / (4.0 * math.sqrt(8.0)))) <= 2.5 * tol


def test_iteration_count_reading():
    """floor(pi/4 sqrt(N/M)) and not the literal loop count ceil(pi sqrt(N)/4)."""
    meta, rows = read_golden()
    n = meta["n"]
    assert oracle.optimal_iterations(n, 1) == meta["iterations"]
    psi = oracle.grover_operator(oracle.init_uniform(n), n, [5], 3)
    p = oracle.probs(psi, n)
    assert round(100 * p[5], 3) != pytest.approx(94.531)
    assert abs(p[5] - 0.3307) < 1e-3
    # configuration values: n=12 -> 50; n=28 -> 12867 / 6433 / 3216; n=33 -> 72792
    assert oracle.optimal_iterations(12, 1) == 50
    assert [oracle.optimal_iterations(28, m) for m in (1, 4, 16)] == [12867, 6433, 3216]
    assert oracle.optimal_iterations(33, 1) == 72792
    assert oracle.optimal_iterations(10, 0) == 0


# --- dense brute force ---------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_diffusion_equals_hadamard_phase_hadamard(n):
    H = dense_hadamard(n)
    lhs = H @ dense_phase_shift(n) @ H
    assert np.max(np.abs(lhs - dense_delta(n))) <= 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_primitives_match_dense_matrices(n):
    N = 1 << n
    psi0 = inputs.gaussian_state(n, seed=100 + n)
    marked = inputs.marked_indices(n, max(1, N // 5), seed=7 + n)
    # Hadamard on every qubit, one at a time
    for q in range(n):
        hq = np.kron(np.kron(np.eye(1 << (n - 1 - q)),
                             np.array([[1, 1], [1, -1]]) / math.sqrt(2)), np.eye(1 << q))
        got = oracle.hadamard_qubit(psi0.copy(), n, q)
        assert np.max(np.abs(got - hq @ psi0)) <= 1e-15
    got = oracle.hadamard_all(psi0.copy(), n)
    assert np.max(np.abs(got - dense_hadamard(n) @ psi0)) <= 1e-14
    got = oracle.inversion_mean(psi0.copy(), n)
    assert np.max(np.abs(got - dense_delta(n) @ psi0)) <= 1e-15
    got = oracle.oracle_list(psi0.copy(), n, marked)
    assert np.array_equal(got, dense_oracle(n, marked) @ psi0)
    got = oracle.phase_shift_zero(psi0.copy(), n)
    assert np.array_equal(got, dense_phase_shift(n) @ psi0)


@pytest.mark.parametrize("n,m,k", [(2, 1, 1), (3, 1, 2), (4, 2, 5), (5, 3, 9), (6, 1, 6), (6, 5, 11)])
def test_grover_matches_dense_product(n, m, k):
    marked = inputs.marked_indices(n, m, seed=n * 31 + m)
    G = dense_delta(n) @ dense_oracle(n, marked)
    for init in ("uniform", "gauss"):
        psi0 = oracle.init_uniform(n) if init == "uniform" else inputs.gaussian_state(n, seed=5)
        ref = psi0.copy()
        for _ in range(k):
            ref = G @ ref
        op = oracle.grover_operator(psi0.copy(), n, marked, k)
        assert np.max(np.abs(op - ref)) <= 1e-14
        gate = oracle.grover_gate(psi0.copy(), n, marked, k)
        assert np.max(np.abs(gate - ref)) <= 1e-13


# --- closed forms ---------------------------------------------------------------------
@pytest.mark.parametrize("n,m", [(3, 1), (4, 4), (6, 1), (8, 3), (10, 1), (12, 1), (12, 16)])
def test_closed_form_uniform_matches_operator(n, m):
    marked = inputs.marked_indices(n, m, seed=1000 + n)
    kopt = oracle.optimal_iterations(n, m)
    psi = oracle.init_uniform(n)
    done = 0
    for k in sorted({0, 1, 2, kopt // 2, kopt, kopt + 3}):
        oracle.grover_operator(psi, n, marked, k - done)
        done = k
        a, b = oracle.closed_form_uniform(n, m, k)
        mask = np.zeros(1 << n, dtype=bool)
        mask[marked.astype(np.int64)] = True
        assert np.max(np.abs(psi[mask] - a)) <= 1e-13
        assert np.max(np.abs(psi[~mask] - b)) <= 1e-13


def test_closed_form_uniform_special_cases():
    # M = N/4: theta = pi/6, one iteration reaches the marked set exactly
    for n in (2, 4, 8, 12):
        N = 1 << n
        marked = inputs.marked_indices(n, N // 4, seed=n)
        psi = oracle.grover_operator(oracle.init_uniform(n), n, marked, 1)
        assert abs(oracle.success_prob(psi, n, marked) - 1.0) <= 1e-14
        a, b = oracle.closed_form_uniform(n, N // 4, 1)
        assert abs(b) <= 1e-16 and abs(a - 1.0 / math.sqrt(N // 4)) <= 1e-15
    # M = 0: the uniform state is a fixed point of the diffusion
    psi = oracle.grover_operator(oracle.init_uniform(10), 10, [], 7)
    assert np.max(np.abs(psi - oracle.init_uniform(10))) <= 1e-16
    # M = N: every iteration multiplies the state by -1
    n = 4
    psi = oracle.grover_operator(oracle.init_uniform(n), n, np.arange(16), 3)
    assert np.max(np.abs(psi + oracle.init_uniform(n))) <= 1e-16
    a, _ = oracle.closed_form_uniform(n, 16, 3)
    assert abs(a + 0.25) <= 1e-15


@pytest.mark.parametrize("n,m,k", [(3, 1, 5), (5, 2, 7), (8, 1, 40), (9, 8, 3000), (10, 0, 4), (10, 1024, 3), (11, 7, 13)])
def test_closed_form_general_matches_operator(n, m, k):
    marked = inputs.marked_indices(n, m, seed=2000 + n)
    psi0 = inputs.gaussian_state(n, seed=3000 + n)
    op = oracle.grover_operator(psi0.copy(), n, marked, k)
    cf = oracle.closed_form_general(psi0.copy(), n, marked, k)
    assert np.max(np.abs(op - cf)) <= 1e-12 * max(1.0, k / 100)


# --- invariants -----------------------------------------------------------------------
def test_norm_preserved_and_involutions():
    n = 10
    marked = inputs.marked_indices(n, 3, seed=9)
    psi0 = inputs.gaussian_state(n, seed=11)
    psi = oracle.grover_operator(psi0.copy(), n, marked, 200)
    assert abs(1.0 - oracle.norm(psi, n)) <= 1e-12
    # O^2 = I exactly, D^2 = I to rounding
    o2 = oracle.oracle_list(oracle.oracle_list(psi0.copy(), n, marked), n, marked)
    assert np.array_equal(o2, psi0)
    d2 = oracle.inversion_mean(oracle.inversion_mean(psi0.copy(), n), n)
    assert np.max(np.abs(d2 - psi0)) <= 1e-16
    h2 = oracle.hadamard_all(oracle.hadamard_all(psi0.copy(), n), n)
    assert np.max(np.abs(h2 - psi0)) <= 1e-15
    # reversibility: G^{-1} = O D
    back = psi.copy()
    for _ in range(200):
        oracle.inversion_mean(back, n)
        oracle.oracle_list(back, n, marked)
    assert np.max(np.abs(back - psi0)) <= 1e-13
    # H^{(x)n}|0> is the uniform state
    u = oracle.hadamard_all(oracle.init_zero(n), n)
    assert np.max(np.abs(u - oracle.init_uniform(n))) <= 1e-16


def test_diffusion_preserves_sum():
    """<s|D = <s|: the amplitude sum is unchanged by the inversion about the mean."""
    n = 9
    psi0 = inputs.gaussian_state(n, seed=77)
    psi = oracle.inversion_mean(psi0.copy(), n)
    assert abs(psi.sum() - psi0.sum()) <= 1e-14


@pytest.mark.parametrize("n", [4, 9, 12])
def test_operator_equals_gate_circuit(n):
    m = 3 if n > 4 else 1
    marked = inputs.marked_indices(n, m, seed=n)
    k = oracle.optimal_iterations(n, m)
    for psi0 in (oracle.init_uniform(n), inputs.gaussian_state(n, seed=n + 1)):
        op = oracle.grover_operator(psi0.copy(), n, marked, k)
        gate = oracle.grover_gate(psi0.copy(), n, marked, k)
        assert np.max(np.abs(op - gate)) <= 1e-12


def test_bitmask_oracle_equals_list():
    n = 11
    marked = inputs.marked_indices(n, 37, seed=3)
    words = inputs.bitmask(n, marked)
    psi0 = inputs.gaussian_state(n, seed=4)
    a = oracle.grover_operator(psi0.copy(), n, marked, 9)
    b = oracle.grover_operator_bitmask(psi0.copy(), n, words, 9)
    assert np.array_equal(a, b)


# --- summation and measurement vs library routines -----------------------------------
def test_neumaier_sum():
    assert oracle.neumaier_sum([1e100, 1.0, -1e100]) == 1.0
    assert oracle.neumaier_sum([1.0, 1e100, 1.0, -1e100]) == 2.0
    g = np.random.default_rng(0)
    for scale in (1.0, 1e-8, 1e8):
        x = g.standard_normal(100_000) * scale * np.exp(g.uniform(-20, 20, 100_000))
        exact = math.fsum(x)
        assert abs(oracle.neumaier_sum(x) - exact) <= 2 * np.spacing(abs(exact)) + 1e-30


def test_measurement_helpers():
    n = 10
    psi = inputs.gaussian_state(n, seed=21)
    p = oracle.probs(psi, n)
    assert np.max(np.abs(p - np.abs(psi) ** 2) / (np.abs(psi) ** 2)) <= 1e-15
    assert abs(oracle.norm(psi, n) - math.fsum(np.abs(psi) ** 2)) <= 1e-15
    marked = inputs.marked_indices(n, 5, seed=2)
    assert abs(oracle.success_prob(psi, n, marked) - math.fsum(p[marked.astype(np.int64)])) <= 1e-16
    # top-m: (p desc, index asc), including ties
    q = np.round(p * 1e3) / 1e3
    for m in (1, 4, 16):
        idx, val = oracle.topm(np.sqrt(q).astype(np.complex128), n, m)
        qq = oracle.probs(np.sqrt(q).astype(np.complex128), n)
        order = np.lexsort((np.arange(1 << n), -qq))[:m]
        assert np.array_equal(idx.astype(np.int64), order)
        assert np.array_equal(val, qq[order])
    u = oracle.init_uniform(n)
    idx, _ = oracle.topm(u, n, 4)
    assert list(idx) == [0, 1, 2, 3]


# --- planted mistakes -------------------------------------------------------------------
def _pin_failures():
    """Runs a fast subset of the pins above; returns the names of those failing."""
    fails = []
    meta, rows = read_golden()
    n, k = meta["n"], meta["iterations"]
    psi = oracle.grover_operator(oracle.init_uniform(n), n, [meta["marked"]], k)
    p = oracle.probs(psi, n)
    if any(round(100 * p[x], 3) != pytest.approx(pct, abs=1e-9) for x, pct in rows):
        fails.append("golden-operator")
    g = oracle.grover_gate(oracle.hadamard_all(oracle.init_zero(n), n), n, [meta["marked"]], k)
    pg = oracle.probs(g, n)
    if any(round(100 * pg[x], 3) != pytest.approx(pct, abs=1e-9) for x, pct in rows):
        fails.append("golden-gate")
    n = 5
    marked = inputs.marked_indices(n, 3, seed=1)
    psi0 = inputs.gaussian_state(n, seed=2)
    G = dense_delta(n) @ dense_oracle(n, marked)
    ref = psi0.copy()
    for _ in range(3):  # odd: a global phase of -1 per iteration shows
        ref = G @ ref
    if np.max(np.abs(oracle.grover_operator(psi0.copy(), n, marked, 3) - ref)) > 1e-14:
        fails.append("dense-operator")
    if np.max(np.abs(oracle.grover_gate(psi0.copy(), n, marked, 3) - ref)) > 1e-13:
        fails.append("dense-gate")
    if np.max(np.abs(oracle.closed_form_general(psi0.copy(), n, marked, 3) - ref)) > 1e-13:
        fails.append("closed-form-general")
    a, b = oracle.closed_form_uniform(6, 1, 3)
    u = oracle.grover_operator(oracle.init_uniform(6), 6, [0], 3)
    if abs(u[0] - a) > 1e-13 or abs(u[1] - b) > 1e-13:
        fails.append("closed-form-uniform")
    return fails


def test_planted_mistakes_are_caught():
    assert _pin_failures() == []
    for which, what in oracle.MUTATIONS.items():
        with oracle.mutation(which):
            caught = _pin_failures()
        assert caught, f"planted mistake {which} ({what}) passes every pin"
    assert _pin_failures() == []


# --- generalised phase iterator (differentiation) --------------------------------------
def test_phase_iterator_at_pi_is_minus_grover():
    n, K = 8, 7
    marked = inputs.marked_indices(n, 3, seed=1)
    psi0 = inputs.gaussian_state(n, seed=2)
    ph = np.full(K, np.pi)
    a = oracle.phase_grover(psi0.copy(), n, marked, ph, ph)
    b = oracle.grover_operator(psi0.copy(), n, marked, K)
    assert np.max(np.abs(a - (-1) ** K * b)) <= 1e-13


def test_phase_iterator_dense_unitary_and_inverse():
    n, K = 5, 4
    N = 1 << n
    marked = inputs.marked_indices(n, 2, seed=3)
    g = np.random.default_rng(4)
    phi, vphi = g.uniform(0, 2 * np.pi, K), g.uniform(0, 2 * np.pi, K)
    psi0 = inputs.gaussian_state(n, seed=5)
    ref = psi0.copy()
    for t in range(K):  # dense matrices: O = I + (e^{i phi}-1) P_m, D = I + (e^{i vphi}-1) |s><s|
        P = np.zeros((N, N))
        P[marked.astype(np.int64), marked.astype(np.int64)] = 1.0
        S = np.full((N, N), 1.0 / N)
        O = np.eye(N) + (np.exp(1j * phi[t]) - 1) * P
        D = np.eye(N) + (np.exp(1j * vphi[t]) - 1) * S
        ref = D @ (O @ ref)
    got = oracle.phase_grover(psi0.copy(), n, marked, phi, vphi)
    assert np.max(np.abs(got - ref)) <= 1e-14
    assert abs(np.linalg.norm(got) - 1.0) <= 1e-14
    back = got.copy()  # inverse iterators: O(-phi), D(-vphi) in reverse order
    for t in reversed(range(K)):
        oracle.phase_grover(back, n, [], [0.0], [-vphi[t]])
        oracle.phase_grover(back, n, marked, [-phi[t]], [0.0])
    assert np.max(np.abs(back - psi0)) <= 1e-14


@pytest.mark.parametrize("n,m,K", [(4, 1, 3), (9, 3, 8), (12, 3, 32)])
def test_phase_reduced_model_matches_full_state(n, m, K):
    marked = inputs.marked_indices(n, m, seed=n)
    g = np.random.default_rng(n)
    phi, vphi = g.uniform(0, 2 * np.pi, K), g.uniform(0, 2 * np.pi, K)
    psi = oracle.phase_grover(oracle.init_uniform(n), n, marked, phi, vphi)
    loss, alpha, beta = oracle.phase_reduced(n, m, phi, vphi)
    mask = np.zeros(1 << n, dtype=bool)
    mask[marked.astype(np.int64)] = True
    assert np.max(np.abs(psi[mask] - alpha)) <= 1e-13 and np.max(np.abs(psi[~mask] - beta)) <= 1e-13
    assert abs(loss - oracle.phase_loss(psi, n, marked)) <= 1e-12
    # gradients by central differences agree between the two
    fd_full = oracle.phase_grad_fd(
        lambda a, b: oracle.phase_loss(oracle.phase_grover(oracle.init_uniform(n), n, marked, a, b), n, marked),
        phi[:4], vphi[:4], h=1e-6) if K <= 8 else None
    if fd_full is not None:
        fd_red = oracle.phase_grad_fd(lambda a, b: oracle.phase_reduced(n, m, a, b)[0], phi[:4], vphi[:4], h=1e-6)
        assert np.max(np.abs(fd_full[0] - fd_red[0])) <= 1e-7 and np.max(np.abs(fd_full[1] - fd_red[1])) <= 1e-7


@pytest.mark.parametrize("n,m,K", [(10, 1, 25), (20, 3, 32), (30, 5, 1000)])
def test_phase_reduced_model_at_pi_is_the_closed_form(n, m, K):
    """At phi = vphi = pi the reduced model is (-1)^K times the textbook rotation:
    alpha = sin((2K+1) theta) / sqrt(M), beta = cos((2K+1) theta) / sqrt(N - M)."""
    ph = np.full(K, np.pi)
    loss, alpha, beta = oracle.phase_reduced(n, m, ph, ph)
    theta = math.asin(math.sqrt(m / (1 << n)))
    a = (-1) ** K * math.sin((2 * K + 1) * theta) / math.sqrt(m)
    b = (-1) ** K * math.cos((2 * K + 1) * theta) / math.sqrt((1 << n) - m)
    assert abs(alpha - a) <= 1e-12 * max(1.0, abs(a)) * K and abs(beta - b) <= 1e-12 * K / math.sqrt(1 << n) + 1e-15
    assert abs(loss + math.log(m * a * a)) <= 1e-10


# --- the conventional circuit gate by gate (Fig. oracle1) ---------------------------------
def _dense_x(n, q):
    N = 1 << n
    X = np.zeros((N, N))
    for x in range(N):
        X[x ^ (1 << q), x] = 1.0
    return X


def test_x_and_mcz_against_dense():
    n = 4
    N = 1 << n
    psi0 = inputs.gaussian_state(n, seed=21)
    for q in range(n):
        got = oracle.x_qubit(psi0.copy(), n, q)
        assert np.array_equal(got, _dense_x(n, q) @ psi0)
    Z = np.eye(N)
    Z[N - 1, N - 1] = -1.0
    assert np.array_equal(oracle.mcz(psi0.copy(), n), Z @ psi0)
    assert np.array_equal(oracle.mcz(psi0.copy(), n, negate_all=True), -(Z @ psi0))


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_fig_oracle1_two_qubit_cases(s):
    """Fig. oracle1: for solution |s> of 2 qubits, X on the qubits where s has
    a 0, the multi-controlled gate, the same X: O = I - 2|s><s| on every basis
    state, with 2 zeros(s) X gates (|00>: 4, |01> and |10>: 2, |11>: 0)."""
    n = 2
    for x in range(4):
        e = np.zeros(4, dtype=np.complex128)
        e[x] = 1.0
        got, gates = oracle.grover_circuit(e.copy(), n, [s], 0)
        assert gates == 0
        # apply just the oracle part: X pattern, MCZ, X pattern
        for q in range(n):
            if not (s >> q) & 1:
                oracle.x_qubit(e, n, q)
        oracle.mcz(e, n)
        for q in range(n):
            if not (s >> q) & 1:
                oracle.x_qubit(e, n, q)
        want = np.zeros(4)
        want[x] = -1.0 if x == s else 1.0
        assert np.array_equal(e.real, want) and not np.any(e.imag)


@pytest.mark.parametrize("n,m,k", [(3, 1, 2), (5, 2, 3), (9, 3, 4), (12, 4, 5)])
def test_circuit_equals_operator_and_gate_form(n, m, k):
    marked = inputs.marked_indices(n, m, seed=30 + n)
    psi0 = inputs.gaussian_state(n, seed=31 + n)
    got, gates = oracle.grover_circuit(psi0.copy(), n, marked, k)
    ref = oracle.grover_operator(psi0.copy(), n, marked, k)
    assert np.max(np.abs(got - ref)) <= 1e-13
    zeros = sum(n - bin(int(x)).count("1") for x in marked)
    assert gates == k * ((2 * zeros + m) + 2 * n + (2 * n + 1))


def test_circuit_dense_product_n4():
    """One iteration equals the dense product of its gate list."""
    n, marked = 4, [5, 12]
    N = 1 << n
    Hs = [np.kron(np.kron(np.eye(1 << (n - 1 - q)), np.array([[1, 1], [1, -1]]) / math.sqrt(2)), np.eye(1 << q))
          for q in range(n)]
    Z = np.eye(N)
    Z[N - 1, N - 1] = -1.0
    U = np.eye(N)
    for s in marked:
        Xs = [_dense_x(n, q) for q in range(n) if not (s >> q) & 1]
        for X in Xs:
            U = X @ U
        U = Z @ U
        for X in Xs:
            U = X @ U
    for H in Hs:
        U = H @ U
    for q in range(n):
        U = _dense_x(n, q) @ U
    U = -Z @ U
    for q in range(n):
        U = _dense_x(n, q) @ U
    for H in Hs:
        U = H @ U
    psi0 = inputs.gaussian_state(n, seed=40)
    got, _ = oracle.grover_circuit(psi0.copy(), n, marked, 1)
    assert np.max(np.abs(got - U @ psi0)) <= 1e-14
