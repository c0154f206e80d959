"""The staged iteration pass (k_pass_bulk: 16 KiB chunks moved by bulk copies
through two shared-memory buffers per CTA) against the per-thread
pass (k_pass): both treat every thread's vectors and summation groups alike,
so states and means must agree bit for bit, whatever the chunk count per CTA
(including counts that do not divide evenly), the marked-set form and the
accumulation mode; against the oracle where it can run; and its bounded wait
(GROVER_OPT_TEST_STALL withholds CTA 0's first copy, the wait runs out,
grover_sync reports GROVER_ETIMEOUT, the handle stays usable)."""
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


def run(B, n, dtype, mk, k, staged, psi0=None, accum=None):
    st = B.State(n, dtype)
    st.set_resident(0)
    st.set_staged(staged)
    if accum:
        st.set_accum(accum)
    if psi0 is None:
        st.init_uniform()
    else:
        st.init_state(psi0)
    st.iterate(mk, k)
    ps, nrm = st.success_prob(mk)
    st.sync()
    return st.amps.cpu().numpy().copy(), ps, nrm


# complex64 n = 11 is one chunk; n = 19 / 20 give 256 / 512 chunks over the
# SMs (uneven shares); complex128 n = 10 is one chunk
@pytest.mark.parametrize("dtype,n,m", [("c64", 11, 1), ("c64", 16, 3), ("c64", 19, 5), ("c64", 20, 2),
                                       ("c128", 10, 1), ("c128", 15, 4), ("c128", 19, 3)])
def test_staged_equals_per_thread_pass(B, dtype, n, m):
    marked = inputs.marked_indices(n, m, seed=900 + n)
    psi0 = inputs.gaussian_state(n, seed=901 + n)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64)
    for mk in (B.Marked(n, marked), B.Marked(n, bitmask=inputs.bitmask(n, marked))):
        a1, p1, n1 = run(B, n, dtype, mk, 9, staged=1, psi0=psi0)
        a0, p0, n0 = run(B, n, dtype, mk, 9, staged=0, psi0=psi0)
        assert np.array_equal(a1, a0)
        assert p1 == p0 and n1 == n0


@pytest.mark.parametrize("accum", ["fp32", "kahan", "fp64", "exact"])
def test_staged_equals_per_thread_pass_accum_modes(B, accum):
    n, m = 17, 2
    marked = inputs.marked_indices(n, m, seed=910)
    mk = B.Marked(n, marked)
    a1, _, _ = run(B, n, "c64", mk, 7, staged=1, accum=accum)
    a0, _, _ = run(B, n, "c64", mk, 7, staged=0, accum=accum)
    assert np.array_equal(a1, a0)


def test_staged_matches_oracle(B):
    n, m, k = 14, 3, 40
    marked = inputs.marked_indices(n, m, seed=920)
    psi0 = inputs.gaussian_state(n, seed=921).astype(np.complex64)
    got, _, _ = run(B, n, "c64", B.Marked(n, marked), k, staged=1, psi0=psi0)
    ref = oracle.grover_operator(psi0.astype(np.complex128), n, marked, k)
    # error vector of k complex64 iterations from the stored start (c64_bounds)
    assert np.linalg.norm(got.astype(np.complex128) - ref) <= c64_bounds.norm_bound(k, np.linalg.norm(ref))


def test_staged_default_above_l2(B):
    """n = 25 complex64 (256 MiB, above half the L2) takes the staged pass by
    default: equal to the forced per-thread pass bit for bit."""
    n, m, k = 25, 1, 3
    marked = inputs.marked_indices(n, m, seed=930)
    mk = B.Marked(n, marked)
    a1, _, _ = run(B, n, "c64", mk, k, staged=-1)
    a0, _, _ = run(B, n, "c64", mk, k, staged=0)
    assert np.array_equal(a1, a0)
    am, au = oracle.closed_form_uniform(n, m, k)
    # one marked value: the error-vector norm bound over sqrt(M) (c64_bounds)
    tol_m, tol_u = c64_bounds.group_bounds(n, m, k)
    assert abs(complex(a1[int(marked[0])]) - am) <= tol_m
    other = 0 if int(marked[0]) != 0 else 1
    assert np.all(np.delete(a1, marked.astype(np.int64)) == a1[other])  # the unmarked values are one number
    assert abs(complex(a1[other]) - au) <= tol_u


def test_staged_wait_runs_out(B):
    n = 16
    marked = inputs.marked_indices(n, 2, seed=940)
    mk = B.Marked(n, marked)
    st = B.State(n, "c64")
    st.set_resident(0)
    st.set_staged(1)
    st.set_option(2, 20000)  # wait limit
    st.set_option(3, 1)      # stall hook
    st.init_uniform()
    st.iterate(mk, 3)
    with pytest.raises(B.GroverError) as ei:
        st.sync()
    assert ei.value.status == 4  # GROVER_ETIMEOUT
    st.set_option(2, 1 << 22)
    st.init_uniform()
    k = B.grover_optimal_iterations(n, 2)
    st.iterate(mk, k)
    ps, _ = st.success_prob(mk)
    st.sync()
    am, _ = oracle.closed_form_uniform(n, 2, k)
    assert abs(ps - 2 * am * am) <= 1e-4


def test_staged_option_rejects_bad_value(B):
    st = B.State(12, "c64")
    with pytest.raises(B.GroverError) as ei:
        st.set_staged(2)
    assert ei.value.status == 1
