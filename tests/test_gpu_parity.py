"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances
  * complex128: max |gpu - oracle| <= 1e-11 after the full optimal run, and
    |1 - norm| <= 1e-12; top-m / argmax indices bit-exact.
  * complex64 (default accumulation): the worst-case bound of c64_bounds
    (u = 2^-24): per iteration the FP32 pairwise tile sums (8 or 16
    amplitudes) put an error vector of norm <= 2 gamma_4 ||c|| ~ 8u ||c|| into
    2 mu and the update c <- (2mu_hi - O c) + 2mu_lo rounds twice per stored
    amplitude (2u ||c||); the iteration is unitary, so after k iterations the
    error vector has norm <= ((1 + 10u + 64u^2)^k (1 + u) - 1) ||c||
    ~ (10k + 1) u ||c||.  The tests
    check that 2-norm; where every unmarked (marked) amplitude is one value,
    that value is within the bound over sqrt(N - M) (sqrt(M)).  The plain and
    compensated FP32 running sums have no useful worst-case bound at these
    sizes; their test keeps a per-amplitude margin of (k + 1) 2^-22 over the
    FP64 oracle (an observed margin, not a derived bound).  P_success within
    1e-4 of the oracle (the stated tolerance for FP32 results).
  * Under a uniform initial state every unmarked amplitude goes through the
    same operations on the same values, so all unmarked (and all marked)
    amplitudes must be bitwise equal: an exact check of indexing and tails.
"""
from __future__ import annotations

import numpy as np
import pytest

import c64_bounds
import oracle
from paper_2005_04635_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_04635_gb300 import binding
    binding.lib()
    return binding


def c64_tol(k):
    """Per-amplitude margin for the plain and compensated FP32 running sums
    (observed, not derived; module docstring)."""
    return (k + 1) * 2.0 ** -22


def c64_norm_bound(k, norm=1.0):
    """Bound on the 2-norm of the complex64 error vector after k iterations
    (default accumulation; c64_bounds)."""
    return c64_bounds.norm_bound(k, norm)


def assert_c64_close(got, ref, k):
    assert np.linalg.norm(got - ref) <= c64_norm_bound(k, np.linalg.norm(ref)), np.linalg.norm(got - ref)


def check_close(dtype, got, ref, k):
    if dtype == "c128":
        assert np.max(np.abs(got - ref)) <= 1e-12
    else:
        assert_c64_close(got, ref, k)


def check_group_values(got, ref, marked, k):
    """After check_groups: the one unmarked and the one marked value against
    the oracle's, each within the norm bound over the square root of its count."""
    mask = np.zeros(got.size, dtype=bool)
    mask[np.asarray(marked, dtype=np.int64)] = True
    E = c64_norm_bound(k)
    for sel in (mask, ~mask):
        cnt = int(np.count_nonzero(sel))
        if cnt:
            i = int(np.flatnonzero(sel)[0])
            assert abs(got[i] - ref[i]) <= E / np.sqrt(cnt), (cnt, abs(got[i] - ref[i]), E / np.sqrt(cnt))


def to_np(st):
    torch.cuda.synchronize()
    return st.amps.cpu().numpy().astype(np.complex128)


def check_groups(psi, marked):
    mask = np.zeros(psi.size, dtype=bool)
    mask[np.asarray(marked, dtype=np.int64)] = True
    for grp in (psi[mask], psi[~mask]):
        if grp.size:
            assert np.all(grp == grp[0]), "amplitudes of one group differ bitwise"


PATHS = {"auto": -1, "pass": 0}


@pytest.mark.parametrize("path", ["auto", "pass"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (3, 1), (5, 2), (6, 1), (9, 3), (12, 1), (12, 4), (16, 16), (17, 1), (18, 2), (20, 1)])
def test_uniform_full_run(B, dtype, n, m, path):
    marked = inputs.marked_indices(n, m, seed=n * 100 + m)
    k = B.grover_optimal_iterations(n, m)
    mk = B.Marked(n, marked)
    st = B.State(n, dtype)
    st.set_resident(PATHS[path])
    st.init_uniform()
    st.iterate(mk, k)
    ps, nrm = st.success_prob(mk)
    st.sync()
    got = to_np(st)
    ref = oracle.grover_operator(oracle.init_uniform(n), n, marked, k)
    err = np.max(np.abs(got - ref))
    if dtype == "c128":
        assert err <= 1e-11
        assert abs(1.0 - nrm) <= 1e-12
        assert abs(ps - oracle.success_prob(ref, n, marked)) <= 1e-12
    else:
        assert_c64_close(got, ref, k)
        assert abs(ps - oracle.success_prob(ref, n, marked)) <= 1e-4
    check_groups(got, marked)
    if dtype == "c64":
        check_group_values(got, ref, marked, k)
    if m <= 16 and m < (1 << n) // 4:
        idx, p = st.measure_topm(m)
        assert sorted(idx.tolist()) == marked.tolist()


@pytest.mark.parametrize("path", ["auto", "pass"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,m,k", [(4, 3, 7), (10, 8, 60), (14, 8, 200), (15, 5, 31)])
def test_gaussian_init(B, dtype, n, m, k, path):
    marked = inputs.marked_indices(n, m, seed=7 * n)
    psi0 = inputs.gaussian_state(n, seed=11 * n)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)  # the oracle starts from the stored values
    mk = B.Marked(n, marked)
    st = B.State(n, dtype)
    st.set_resident(PATHS[path])
    st.init_state(psi0)
    st.iterate(mk, k)
    st.sync()
    got = to_np(st)
    ref = oracle.grover_operator(psi0.copy(), n, marked, k)
    if dtype == "c128":
        assert np.max(np.abs(got - ref)) <= 1e-11
    else:
        assert_c64_close(got, ref, k)
    # top-m on the same final state: bit-exact against the oracle's selection
    idx, p = st.measure_topm(min(16, 1 << n))
    oidx, op = oracle.topm(got, n, min(16, 1 << n))
    assert np.array_equal(idx, oidx) and np.array_equal(p, op)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_large_marked_set_uses_bitmask(B, dtype):
    n, m = 13, 300  # more than 256 indices: the library adds a bitmask
    marked = inputs.marked_indices(n, m, seed=5)
    k = 5
    psi0 = inputs.gaussian_state(n, seed=6)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    ref = oracle.grover_operator(psi0.copy(), n, marked, k)
    for mk in (B.Marked(n, marked), B.Marked(n, bitmask=inputs.bitmask(n, marked))):
        assert mk.count == m
        st = B.State(n, dtype)
        st.init_state(psi0)
        st.iterate(mk, k)
        ps, _ = st.success_prob(mk)
        got = to_np(st)
        if dtype == "c128":
            assert np.max(np.abs(got - ref)) <= 1e-12
        else:
            assert_c64_close(got, ref, k)
        assert abs(ps - oracle.success_prob(ref, n, marked)) <= (1e-12 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_bitmask_small_list(B, dtype):
    n = 11
    marked = inputs.marked_indices(n, 6, seed=9)
    mk = B.Marked(n, bitmask=inputs.bitmask(n, marked))
    st = B.State(n, dtype)
    st.init_uniform()
    k = B.grover_optimal_iterations(n, 6)
    st.iterate(mk, k)
    got = to_np(st)
    ref = oracle.grover_operator(oracle.init_uniform(n), n, marked, k)
    if dtype == "c128":
        assert np.max(np.abs(got - ref)) <= 1e-11
    else:
        assert_c64_close(got, ref, k)
        check_groups(got, marked)
        check_group_values(got, ref, marked, k)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_separate_oracle_and_diffusion(B, dtype):
    """grover_oracle + grover_diffuse, alternately, equal grover_iterate."""
    n, k = 10, 9
    marked = inputs.marked_indices(n, 2, seed=3)
    psi0 = inputs.gaussian_state(n, seed=4)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    mk = B.Marked(n, marked)
    a = B.State(n, dtype)
    a.init_state(psi0)
    for _ in range(k):
        a.oracle(mk)
        a.diffuse()
    b = B.State(n, dtype)
    b.init_state(psi0)
    b.iterate(mk, k)
    ga, gb = to_np(a), to_np(b)
    ref = oracle.grover_operator(psi0.copy(), n, marked, k)
    if dtype == "c128":
        assert np.max(np.abs(ga - ref)) <= 1e-12 and np.max(np.abs(gb - ref)) <= 1e-12
    else:
        assert_c64_close(ga, ref, k)
        assert_c64_close(gb, ref, k)
    # the diffusion alone is the oracle's inversion about the mean
    c = B.State(n, dtype)
    c.init_state(psi0)
    c.diffuse()
    assert np.max(np.abs(to_np(c) - oracle.inversion_mean(psi0.copy(), n))) <= (1e-15 if dtype == "c128" else 1e-6)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_edge_marked_sets(B, dtype):
    n = 9
    N = 1 << n
    for marked in ([0], [N - 1], [0, N - 1], list(range(0, N, 4)), []):
        marked = np.asarray(marked, dtype=np.uint64)
        m = marked.size
        k = B.grover_optimal_iterations(n, m) if m else 5
        mk = B.Marked(n, marked)
        st = B.State(n, dtype)
        st.init_uniform()
        st.iterate(mk, k)
        got = to_np(st)
        ref = oracle.grover_operator(oracle.init_uniform(n), n, marked, k)
        if dtype == "c128":
            assert np.max(np.abs(got - ref)) <= 1e-12, marked
        else:
            assert_c64_close(got, ref, k)
        check_groups(got, marked)
        if dtype == "c64":
            check_group_values(got, ref, marked, k)


def test_measure_probs_bit_exact(B):
    n = 12
    marked = inputs.marked_indices(n, 3, seed=1)
    psi0 = inputs.gaussian_state(n, seed=2)
    for dtype in ("c128", "c64"):
        st = B.State(n, dtype)
        st.init_state(psi0 if dtype == "c128" else psi0.astype(np.complex64))
        st.iterate(B.Marked(n, marked), 17)
        got = to_np(st)
        p = st.measure_probs()
        assert np.array_equal(p, oracle.probs(got, n))
        pd = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        st.measure_probs(pd)
        torch.cuda.synchronize()
        assert np.array_equal(pd.cpu().numpy(), p)
        ps, nrm = st.success_prob(B.Marked(n, marked))
        assert abs(ps - oracle.success_prob(got, n, marked)) <= 1e-15
        assert abs(nrm - oracle.norm(got, n)) <= (1e-14 if dtype == "c128" else 1e-7)


def test_deterministic(B):
    n = 18
    marked = inputs.marked_indices(n, 4, seed=8)
    mk = B.Marked(n, marked)
    outs = []
    for _ in range(2):
        st = B.State(n, "c64")
        st.init_state(inputs.gaussian_state(n, seed=3).astype(np.complex64))
        st.iterate(mk, 33)
        outs.append(to_np(st))
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("mode", ["fp32", "kahan", "fp64", "exact"])
def test_accumulation_modes(B, mode):
    n, k = 16, 40
    marked = inputs.marked_indices(n, 8, seed=31)
    psi0 = inputs.gaussian_state(n, seed=32).astype(np.complex64).astype(np.complex128)
    st = B.State(n, "c64")
    st.set_accum(mode)
    st.init_state(psi0)
    mk = B.Marked(n, marked)
    st.iterate(mk, k)
    ps, _ = st.success_prob(mk)
    st.sync()
    ref = oracle.grover_operator(psi0.copy(), n, marked, k)
    got = to_np(st)
    assert abs(ps - oracle.success_prob(ref, n, marked)) <= 1e-4
    if mode in ("exact", "fp64"):  # derived worst-case bounds (c64_bounds)
        rho = c64_bounds.RHO["exact"] if mode == "exact" else c64_bounds.rho_fp64(n)
        assert np.linalg.norm(got - ref) <= c64_bounds.norm_bound(k, np.linalg.norm(ref), rho)
    else:
        assert np.max(np.abs(got - ref)) <= c64_tol(k)


def test_c128_fp64_accumulation(B):
    n, k = 15, 120
    marked = inputs.marked_indices(n, 2, seed=51)
    psi0 = inputs.gaussian_state(n, seed=52)
    st = B.State(n, "c128")
    st.set_accum("fp64")
    st.init_state(psi0)
    st.iterate(B.Marked(n, marked), k)
    ref = oracle.grover_operator(psi0.copy(), n, marked, k)
    assert np.max(np.abs(to_np(st) - ref)) <= 1e-12


@pytest.mark.parametrize("dtype,mode", [("c128", "exact"), ("c128", "fp64"), ("c64", "exact"), ("c64", "fp64")])
def test_mean_rounding(B, dtype, mode):
    """An amplitude that is exactly 0 becomes exactly 2<c> after one diffusion,
    which exposes the computed mean.  Exact mode: the correctly rounded mean, to
    one unit in the last place.  FP64 mode: the recursive-summation bound
    |S_hat - S| <= gamma_L * sum|x| (L additions per term, unit roundoff u), which
    holds for any summation order: complex128 L = N - 1, u = 2^-53; complex64
    L = 7 in FP32 (u = 2^-24, pairwise tile of 8) plus N/8 in FP64."""
    import math
    n = 16
    N = 1 << n
    psi0 = inputs.gaussian_state(n, seed=61) * 3.0
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    psi0[5] = 0.0
    st = B.State(n, dtype)
    st.set_accum(mode)
    st.init_state(psi0)
    st.diffuse()
    got = to_np(st)[5]
    for part, g in ((psi0.real, got.real), (psi0.imag, got.imag)):
        exact = 2.0 * math.fsum(part.tolist()) / N  # fsum: correctly rounded sum
        sum_abs = 2.0 * float(np.sum(np.abs(part))) / N
        if dtype == "c128":
            ulp = np.spacing(abs(exact))
            bound = ulp if mode == "exact" else ulp + (N - 1) * 2.0 ** -53 * sum_abs
        else:
            exact = float(np.float32(exact))
            ulp = float(np.spacing(np.float32(abs(exact))))
            bound = ulp if mode == "exact" else ulp + (7 * 2.0 ** -24 + (N / 8) * 2.0 ** -53) * sum_abs
        assert abs(g - exact) <= bound, (mode, abs(g - exact), bound)


def test_c128_rejects_fp32_accumulation(B):
    st = B.State(6, "c128")
    with pytest.raises(B.GroverError):
        st.set_accum("kahan")


def test_invalid_marked_for_state(B):
    st = B.State(6, "c64")
    with pytest.raises(B.GroverError):
        st.iterate(B.Marked(7, [1]), 1)
    with pytest.raises(B.GroverError):
        st.measure_topm(17)


# ---- persistent on-chip iterator ----------------------------------------------------
@pytest.mark.parametrize("dtype,n", [("c64", 1), ("c64", 3), ("c64", 11), ("c64", 18), ("c128", 1), ("c128", 2),
                                     ("c128", 12), ("c128", 17)])
def test_resident_forced(B, dtype, n):
    """The persistent iterator (forced on) against the oracle, Gaussian start,
    marked list and bitmask, then continued by the pass path (the mean it leaves
    behind must be the mean of O c)."""
    m = min(5, 1 << n)
    marked = inputs.marked_indices(n, m, seed=70 + n)
    psi0 = inputs.gaussian_state(n, seed=71 + n)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    k1, k2 = 23, 9
    ref1 = oracle.grover_operator(psi0.copy(), n, marked, k1)
    ref2 = oracle.grover_operator(ref1.copy(), n, marked, k2)
    for mk in (B.Marked(n, marked), B.Marked(n, bitmask=inputs.bitmask(n, marked))):
        st = B.State(n, dtype)
        st.set_resident(1)
        st.init_state(psi0)
        st.iterate(mk, k1)
        check_close(dtype, to_np(st), ref1, k1)
        st.set_resident(0)
        st.iterate(mk, k2)
        check_close(dtype, to_np(st), ref2, k1 + k2)


def test_resident_refuses_large_states(B):
    for opt in (1, 2):
        st = B.State(23, "c64")
        st.set_resident(opt)
        st.init_uniform()
        with pytest.raises(B.GroverError) as ei:
            st.iterate(B.Marked(23, [3]), 2)
        assert ei.value.status == 8  # GROVER_EUNSUPPORTED
    st2 = B.State(10, "c64")
    st2.set_resident(1)
    st2.set_accum("kahan")
    with pytest.raises(B.GroverError):
        st2.iterate(B.Marked(10, [3]), 2)


def test_resident_deterministic_and_equal_groups(B):
    n = 16
    marked = inputs.marked_indices(n, 3, seed=90)
    outs = []
    for _ in range(2):
        st = B.State(n, "c128")
        st.set_resident(1)
        st.init_uniform()
        st.iterate(B.Marked(n, marked), B.grover_optimal_iterations(n, 3))
        outs.append(to_np(st))
    assert np.array_equal(outs[0], outs[1])
    check_groups(outs[0], marked)


# ---- grid-wide persistent iterator ---------------------------------------------------------
@pytest.mark.parametrize("dtype,n", [("c64", 9), ("c64", 12), ("c64", 18), ("c64", 21), ("c64", 22), ("c128", 10),
                                     ("c128", 16), ("c128", 21)])
def test_resident_grid_forced(B, dtype, n):
    """The grid iterator (forced) against the oracle from a Gaussian start,
    with a marked list and a bitmask, then continued by the pass path."""
    m = min(7, 1 << n)
    marked = inputs.marked_indices(n, m, seed=170 + n)
    psi0 = inputs.gaussian_state(n, seed=171 + n)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    k1, k2 = (23, 9) if n <= 18 else (5, 3)
    ref1 = oracle.grover_operator(psi0.copy(), n, marked, k1)
    ref2 = oracle.grover_operator(ref1.copy(), n, marked, k2)
    marks = [B.Marked(n, marked)]
    if n <= 18:
        marks.append(B.Marked(n, bitmask=inputs.bitmask(n, marked)))
    for mk in marks:
        st = B.State(n, dtype)
        st.set_resident(2)
        st.init_state(psi0)
        st.iterate(mk, k1)
        st.sync()
        check_close(dtype, to_np(st), ref1, k1)
        st.set_resident(0)
        st.iterate(mk, k2)
        check_close(dtype, to_np(st), ref2, k1 + k2)


@pytest.mark.parametrize("dtype,n,m", [("c64", 20, 1), ("c64", 22, 4), ("c128", 19, 2)])
def test_resident_grid_full_run_uniform(B, dtype, n, m):
    """Full optimal run from the uniform state on the grid iterator: closed
    form, bitwise-equal groups, and the same result on a second run."""
    marked = inputs.marked_indices(n, m, seed=180 + n)
    k = B.grover_optimal_iterations(n, m)
    outs = []
    for _ in range(2):
        st = B.State(n, dtype)
        st.set_resident(2)
        st.init_uniform()
        st.iterate(B.Marked(n, marked), k)
        st.sync()
        outs.append(to_np(st))
    assert np.array_equal(outs[0], outs[1])
    check_groups(outs[0], marked)
    a_m, a_u = oracle.closed_form_uniform(n, m, k)
    E = c64_norm_bound(k)
    tol_m, tol_u = (1e-11, 1e-11) if dtype == "c128" else (E / np.sqrt(m), E / np.sqrt((1 << n) - m))
    idx = marked.astype(np.int64)
    assert abs(outs[0][idx[0]] - a_m) <= tol_m
    other = 0 if idx[0] != 0 else 1
    assert abs(outs[0][other] - a_u) <= tol_u


@pytest.mark.parametrize("n", [18, 21])
def test_resident_grid_wait_runs_out(B, n):
    """Failure detection without a GPU fault: CTA 0 withholds its first partial
    (test hook), every CTA's bounded wait runs out, the kernel returns and
    grover_sync reports GROVER_ETIMEOUT; the handle stays usable (n = 21: the
    kernel instance with 16-amplitude summation groups)."""
    marked = inputs.marked_indices(n, 2, seed=190)
    st = B.State(n, "c64")
    mk = B.Marked(n, marked)
    st.set_resident(2)
    st.set_option(2, 20000)  # wait limit: 20000 polls
    st.set_option(3, 1)      # stall hook
    st.init_uniform()
    st.iterate(mk, 10)
    with pytest.raises(B.GroverError) as ei:
        st.sync()
    assert ei.value.status == 4  # GROVER_ETIMEOUT
    st.set_option(2, 1 << 22)
    st.init_uniform()
    k = B.grover_optimal_iterations(n, 2)
    st.iterate(mk, k)
    st.sync()
    a_m, _ = oracle.closed_form_uniform(n, 2, k)
    assert abs(to_np(st)[int(marked[0])] - a_m) <= c64_bounds.group_bounds(n, 2, k)[0]


# ---- amplitudes outside the fixed-point window ----------------------------------------------
@pytest.mark.parametrize("path,n", [("pass", 14), ("cluster", 12), ("grid", 18), ("grid", 21)])
def test_out_of_window_amplitudes(B, path, n):
    """A state scaled by 64 (amplitudes above the 16 of the exact fixed-point
    window) takes the FP64 side sums in every reduction; the iterator is linear,
    so the result is 64 times the unit-norm one."""
    m, k = 3, 7
    marked = inputs.marked_indices(n, m, seed=900 + n)
    psi0 = inputs.gaussian_state(n, seed=901 + n)
    psi0[int(marked[0])] = 0.9  # one large amplitude, so the scaled state has values >= 16
    psi0 = psi0.astype(np.complex64).astype(np.complex128)
    scaled = (psi0 * 64.0).astype(np.complex64).astype(np.complex128)
    st = B.State(n, "c64")
    st.set_resident({"pass": 0, "cluster": 1, "grid": 2}[path])
    st.init_state(scaled)
    st.iterate(B.Marked(n, marked), k)
    st.sync()
    ref = oracle.grover_operator(scaled.copy(), n, marked, k)
    assert_c64_close(to_np(st), ref, k)
