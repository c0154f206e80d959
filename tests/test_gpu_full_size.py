"""Full-size runs (the benchmark's launch configuration) against the oracle's
closed form for a uniform initial state:
  marked amplitude sin((2k+1)theta)/sqrt(M), unmarked cos((2k+1)theta)/sqrt(N-M).

The whole state is checked on the device (the group invariant: every unmarked
amplitude equals one value, every marked one another), then the two values are
compared with the closed form one by one.

complex64 bound (c64_bounds, u = 2^-24): the FP32 start 1/sqrt(N) is off by
an error vector of norm <= u, and each iteration adds one of norm
<= (10u + 64u^2) times the state's norm (the FP32 pairwise tile sums of the
mean, at most 8u, and two roundings per stored amplitude, 2u); the iteration
is unitary, so after k iterations ||error||_2 <= E = (1 + 10u + 64u^2)^k (1 + u) - 1.
Once the group check has shown that the N - M unmarked amplitudes are one
value v_u (and the M marked ones one value v_m), the error vector holds N - M
copies of v_u - a_u and M copies of v_m - a_m, so
  |v_u - a_u| <= E / sqrt(N - M),  |v_m - a_m| <= E / sqrt(M).
complex128: the same argument with u = 2^-53 gives far less than the 1e-11
the FP64 tolerance asks for.  P_success must be within 1e-4 of the FP64 value
(complex64).
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


def group_tolerances(dtype, n, m, k):
    """Per-element bounds on the marked and the unmarked value (module docstring)."""
    if dtype == "c128":
        return 1e-11, 1e-11
    return c64_bounds.group_bounds(n, m, k)


def run_and_check(B, n, m, dtype, k, seed):
    marked = inputs.marked_indices(n, m, seed)
    mk = B.Marked(n, marked)
    st = B.State(n, dtype)
    st.init_uniform()
    st.iterate(mk, k)
    ps, nrm = st.success_prob(mk)
    idx, p = st.measure_topm(m)
    st.sync()
    a = st.amps
    mi = torch.as_tensor(marked.astype(np.int64), device=a.device)
    mvals = a[mi]
    # one unmarked index: the smallest index not in the list
    u = next(x for x in range(m + 1) if x not in set(marked.tolist()))
    uval = a[u]
    n_diff_unmarked = int(torch.count_nonzero(a != uval).item())
    assert bool(torch.all(mvals == mvals[0]).item()), "marked amplitudes differ"
    assert n_diff_unmarked == m, "an unmarked amplitude differs from the others"
    am, au = oracle.closed_form_uniform(n, m, k)
    got_m = complex(mvals[0].item())
    got_u = complex(uval.item())
    tol_m, tol_u = group_tolerances(dtype, n, m, k)
    assert abs(got_m - am) <= tol_m and abs(got_u - au) <= tol_u, (got_m, am, tol_m, got_u, au, tol_u)
    p_ref = m * am * am
    assert abs(ps - p_ref) <= (1e-11 if dtype == "c128" else 1e-4)
    if dtype == "c128":
        assert abs(1.0 - nrm) <= 1e-12
    assert sorted(idx.tolist()) == marked.tolist()
    del st
    torch.cuda.empty_cache()


@pytest.mark.parametrize("m", [1, 4, 16])
def test_n28_c64_full_optimal(B, m):
    n = 28
    run_and_check(B, n, m, "c64", B.grover_optimal_iterations(n, m), seed=2800 + m)


@pytest.mark.parametrize("m", [1, 16])
def test_n28_c128_full_optimal(B, m):
    n = 28
    run_and_check(B, n, m, "c128", B.grover_optimal_iterations(n, m), seed=2810 + m)


def test_n33_c64_100_iterations(B):
    free, _ = torch.cuda.mem_get_info()
    if free < (80 << 30):
        pytest.skip("needs 80 GB of free device memory")
    run_and_check(B, 33, 1, "c64", 100, seed=3300)


def test_n32_c128_maximum_size(B):
    """The largest complex128 state the ABI accepts (2^32 amplitudes, 64 GiB)."""
    free, _ = torch.cuda.mem_get_info()
    if free < (80 << 30):
        pytest.skip("needs 80 GB of free device memory")
    run_and_check(B, 32, 4, "c128", 20, seed=3204)


def test_n33_c64_bitmask_marked_set(B):
    """n = 33 with M = 300 marked indices: above the list limit, so the oracle
    flip reads the 1 GiB bitmask in the same fused pass."""
    free, _ = torch.cuda.mem_get_info()
    if free < (80 << 30):
        pytest.skip("needs 80 GB of free device memory")
    n, m, k = 33, 300, 12
    marked = inputs.marked_indices(n, m, seed=3330)
    mk = B.Marked(n, marked)
    st = B.State(n, "c64")
    st.init_uniform()
    st.iterate(mk, k)
    ps, _ = st.success_prob(mk)
    st.sync()
    a = st.amps
    mvals = a[torch.as_tensor(marked.astype(np.int64), device=a.device)]
    assert bool(torch.all(mvals == mvals[0]).item())
    u = next(x for x in range(m + 1) if x not in set(marked.tolist()))
    uval = a[u]
    assert int(torch.count_nonzero(a != uval).item()) == m, "an unmarked amplitude differs from the others"
    am, au = oracle.closed_form_uniform(n, m, k)
    tol_m, tol_u = group_tolerances("c64", n, m, k)
    assert abs(complex(mvals[0].item()) - am) <= tol_m
    assert abs(complex(uval.item()) - au) <= tol_u
    assert abs(ps - m * am * am) <= 1e-4
    del st
    torch.cuda.empty_cache()
