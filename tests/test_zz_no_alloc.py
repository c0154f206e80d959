"""grover_iterate_noalloc, the entry point for callers that cannot allocate
device memory (a framework's allocator owns the memory, or a loop cannot take
cudaMalloc's device-wide synchronisation): its scratch is a static device
array instead of a cudaMalloc'd one.  Two calls in a row through the C ABI
must give what grover_iterate gives on the same input, and what the FP64
oracle gives from the same stored start, within the tolerances of the other
parity tests.  This file is collected last on purpose; it passes alone in a
fresh process and after the other tests.

Oracle bounds: complex64, the worst-case bound of c64_bounds (FP32 tile sums
of the mean and two roundings per stored amplitude); complex128 (exact sums),
an iteration adds an error vector of norm <= 3u (one rounding per stored
amplitude, norm <= u; the rounding of 2 mu shared by all N amplitudes, norm
<= sqrt(N) u 2|mu| <= 2u, u = 2^-53) and is unitary, so after k iterations
||gpu - oracle||_2 <= 3 k u.
"""
from __future__ import annotations

import numpy as np
import pytest

import c64_bounds
import oracle
from paper_2005_04635_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,m", [(13, 3), (22, 1)])
def test_noalloc_matches_grover_iterate(dtype, n, m):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_04635_gb300 import binding as B
    lib = B.lib()
    marked = inputs.marked_indices(n, m, seed=40 + n)
    psi0 = inputs.gaussian_state(n, seed=41 + n)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    k1, k2 = 7, 12

    # existing entry point (state handle, library-allocated scratch)
    ref = B.State(n, dtype)
    ref.init_state(torch.as_tensor(psi0).to(tdt).cuda())
    mk = B.Marked(n, marked)
    ref.iterate(mk, k1)
    torch.cuda.synchronize()
    want1 = ref.amps.cpu().numpy().astype(np.complex128)
    ref.iterate(mk, k2)
    torch.cuda.synchronize()
    want2 = ref.amps.cpu().numpy().astype(np.complex128)

    # new entry point: caller-owned buffers only, two calls in a row
    amps = torch.as_tensor(psi0).to(tdt).cuda()
    dmarked = torch.as_tensor(marked.astype(np.int64)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    code = 0 if dtype == "c64" else 1
    # the oracle from the same stored start (complex64: the FP32-rounded values)
    start = amps.cpu().numpy().astype(np.complex128)
    u = 2.0 ** -24 if dtype == "c64" else 2.0 ** -53
    ora1 = oracle.grover_operator(start.copy(), n, marked, k1)
    ora2 = oracle.grover_operator(ora1.copy(), n, marked, k2)
    done = 0
    for k, want, ora in ((k1, want1, ora1), (k2, want2, ora2)):
        st = lib.grover_iterate_noalloc(amps.data_ptr(), n, code, dmarked.data_ptr(), m, k, stream)
        assert st == 0, lib.grover_last_error(None)
        torch.cuda.synchronize()
        done += k
        got = amps.cpu().numpy().astype(np.complex128)
        if dtype == "c64":
            # two complex64 paths, each within the worst-case bound of the oracle (c64_bounds)
            E = c64_bounds.norm_bound(done, 1.0, start=0.0)
            assert np.linalg.norm(got - want) <= 2 * E
            assert np.linalg.norm(got - ora) <= E
        else:  # exact sums: 2 mu and the update round once each, 3u per iteration
            assert np.max(np.abs(got - want)) <= 1e-12
            assert np.linalg.norm(got - ora) <= 3 * done * u + 1e-14


def test_noalloc_rejects_bad_sizes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_04635_gb300 import binding as B
    lib = B.lib()
    amps = torch.zeros(1 << 4, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.grover_iterate_noalloc(amps.data_ptr(), 34, 0, None, 0, 1, stream) == 1  # n too large
    assert b"n outside" in lib.grover_last_error(None)
    assert lib.grover_iterate_noalloc(amps.data_ptr(), 33, 1, None, 0, 1, stream) == 1  # c128 n=33
    assert lib.grover_iterate_noalloc(amps.data_ptr(), 4, 0, None, 17, 1, stream) == 7  # m > N
    assert lib.grover_iterate_noalloc(amps.data_ptr() + 8, 4, 0, None, 0, 1, stream) == 1  # misaligned
