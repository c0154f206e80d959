"""Batched searches (grover_batch_*): every instance against the oracle's
closed form for a uniform start (marked sin((2k+1)theta)/sqrt(M), unmarked
cos((2k+1)theta)/sqrt(N-M)), the exact group invariant, P_success within 1e-4
(complex64), bitwise determinism, and the autotuner."""
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


def make_instances(count, nlo, nhi, mmax, seed, kmode="optimal"):
    g = inputs.rng(seed)
    ns, ks, marks = [], [], []
    for i in range(count):
        n = int(g.integers(nlo, nhi + 1))
        m = int(g.integers(1, min(mmax, 1 << n) + 1))
        mk = inputs.marked_indices(n, m, seed * 1000 + i)
        k = oracle.optimal_iterations(n, m) if kmode == "optimal" else int(g.integers(0, 40))
        ns.append(n)
        ks.append(k)
        marks.append(mk)
    return ns, ks, marks


def check_instance(got, n, mk, k):
    N = 1 << n
    m = len(mk)
    mask = np.zeros(N, dtype=bool)
    mask[np.asarray(mk, dtype=np.int64)] = True
    am, au = oracle.closed_form_uniform(n, m, k)
    # the error vector of k complex64 iterations from the rounded uniform start
    # has norm <= c64_bounds.norm_bound(k); the group check makes the marked
    # (unmarked) values one number, so each is within that bound over sqrt(M)
    # (sqrt(N - M))
    e = c64_bounds.norm_bound(k)
    for grp, ref in ((got[mask], am), (got[~mask], au)):
        if grp.size:
            assert np.all(grp == grp[0]), (n, m, k)
            assert abs(complex(grp[0]) - ref) <= e / np.sqrt(grp.size) + 1e-12, (n, m, k, grp[0], ref)
    return m * am * am


@pytest.mark.parametrize("kmode", ["optimal", "random"])
def test_batch_matches_closed_form(B, kmode):
    ns, ks, marks = make_instances(96, 1, 17, 8, seed=11 if kmode == "optimal" else 12, kmode=kmode)
    b = B.Batch(ns, ks, marks)
    b.run()
    p = b.success()
    torch.cuda.synchronize()
    for i in range(len(ns)):
        got = b.state(i).cpu().numpy()
        pref = check_instance(got, ns[i], marks[i], ks[i])
        assert abs(p[i] - pref) <= 1e-4


def test_batch_deterministic_and_tuned(B):
    ns, ks, marks = make_instances(64, 6, 16, 8, seed=21)
    b = B.Batch(ns, ks, marks)
    b.run()
    s1 = b.amps.cpu().numpy().copy()
    p1 = b.success()
    threads, onchip = b.tune()
    assert threads in (256, 512, 1024) and onchip in (2048, 4096, 8192)
    b.run()
    p2 = b.success()
    s2 = b.amps.cpu().numpy()
    for i in range(len(ns)):
        pref = check_instance(s2[b.offsets[i]: b.offsets[i] + (1 << ns[i])], ns[i], marks[i], ks[i])
        # before and after tuning each P within its bound of the exact value
        assert abs(p1[i] - p2[i]) <= 2 * c64_bounds.p_bound(pref, c64_bounds.norm_bound(ks[i])) + 1e-15
    b.run()
    assert np.array_equal(b.success(), p2) and np.array_equal(b.amps.cpu().numpy(), s2)


def test_batch_rejects_bad_input(B):
    with pytest.raises(B.GroverError):
        B.Batch([5], [3], [[4, 2]])  # unsorted
    with pytest.raises(B.GroverError):
        B.Batch([5], [3], [[40]])  # out of range
    with pytest.raises(B.GroverError):
        B.Batch([27], [3], [[1]])  # n too large
    with pytest.raises(B.GroverError):
        B.Batch([10], [3], [list(range(65))])  # more than 64 marked


@pytest.mark.parametrize("packing,min_qubits", [(16, 17), (16, 19), (2, 15), (2, 19), (0, 17)])
def test_batch_large_instances_both_packings(B, packing, min_qubits):
    """Instances with n = 15..20 (clusters of 16 CTAs for n >= 17 or n >= 19:
    on chip up to n = 18, streamed through L2 above; groups of CTAs for n >= 15
    or n >= 19, on chip), mixed with small ones, against the closed form under
    each packing."""
    ns, ks, marks = make_instances(40, 15, 20, 8, seed=31)
    ns2, ks2, marks2 = make_instances(40, 3, 12, 8, seed=32)
    b = B.Batch(ns + ns2, ks + ks2, marks + marks2)
    b.set_packing(packing, min_qubits)
    assert b.packing() == (packing if packing > 1 else 1, min_qubits)
    b.run()
    p = b.success()
    torch.cuda.synchronize()
    all_n, all_k, all_m = ns + ns2, ks + ks2, marks + marks2
    for i in range(len(all_n)):
        got = b.state(i).cpu().numpy()
        pref = check_instance(got, all_n[i], all_m[i], all_k[i])
        assert abs(p[i] - pref) <= 1e-4
    b.run()
    assert np.array_equal(b.success(), p)  # deterministic


def test_batch_packing_rejects_bad_size(B):
    b = B.Batch([5], [2], [[3]])
    with pytest.raises(B.GroverError) as ei:
        b.set_packing(8)
    assert ei.value.status == 1
    with pytest.raises(B.GroverError) as ei:
        b.set_packing(16, 14)  # threshold below 15 qubits
    assert ei.value.status == 1


def test_batch_group_wait_gives_up_and_recovers(B):
    """Failure detection without a GPU fault: the test hook makes the first CTA
    of the first group withhold its first partial sums, the group's bounded
    waits (short limit) run out, grover_batch_success reports GROVER_ETIMEOUT,
    and the same batch then runs correctly."""
    ns, ks, marks = make_instances(12, 15, 17, 4, seed=41)
    ns2, ks2, marks2 = make_instances(12, 3, 10, 4, seed=42)
    b = B.Batch(ns + ns2, ks + ks2, marks + marks2)
    b.set_packing(2, 15)
    b.set_option(2, 20000)
    b.set_option(3, 1)
    b.run()
    with pytest.raises(B.GroverError) as ei:
        b.success()
    assert ei.value.status == 4  # GROVER_ETIMEOUT
    b.set_option(3, 0)
    b.run()
    p = b.success()
    torch.cuda.synchronize()
    all_n, all_k, all_m = ns + ns2, ks + ks2, marks + marks2
    for i in range(len(all_n)):
        pref = check_instance(b.state(i).cpu().numpy(), all_n[i], all_m[i], all_k[i])
        assert abs(p[i] - pref) <= 1e-4


def test_batch_group_edge_cases(B):
    """Groups of CTAs (n = 15..20) on the cases their loop treats apart: k = 0
    (the uniform start, written back after the first exchange), k = 1 and 2,
    random k, a size with a single instance, the marked amplitude in the last
    slot of the last CTA's slice; against the closed form, deterministic."""
    ns, ks, marks = make_instances(30, 15, 20, 8, seed=51, kmode="random")
    extra_n = [15, 15, 16, 20, 19]
    ns += extra_n
    ks += [0, 1, 2, 1, 0]
    marks += [inputs.marked_indices(n, 3, 520 + i) for i, n in enumerate(extra_n)]
    ns += [18]
    ks += [oracle.optimal_iterations(18, 1)]
    marks += [np.array([(1 << 18) - 1], dtype=np.uint64)]
    b = B.Batch(ns, ks, marks)
    b.set_packing(2, 15)
    b.run()
    p = b.success()
    torch.cuda.synchronize()
    for i in range(len(ns)):
        pref = check_instance(b.state(i).cpu().numpy(), ns[i], marks[i], ks[i])
        assert abs(p[i] - pref) <= 1e-4
    s1 = b.amps.cpu().numpy().copy()
    b.run()
    assert np.array_equal(b.success(), p) and np.array_equal(b.amps.cpu().numpy(), s1)
