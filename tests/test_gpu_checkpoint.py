"""Checkpoint / resume: a search stopped after k1 iterations, saved, loaded
into a new handle and continued for k2 more ends bitwise equal to the search
run k1 + k2 iterations in one go (every reduction has a fixed order, and the
first pass after a load recomputes the mean the stopped run had cached)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2005_04635_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,n,path", [("c64", 14, 0), ("c128", 12, 0), ("c64", 18, 0), ("c64", 12, -1)])
def test_resume_is_bitwise_equal(tmp_path, dtype, n, path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_04635_gb300 import binding, checkpoint
    binding.lib()
    marked = inputs.marked_indices(n, 2, seed=1000 + n)
    k1, k2 = 7, 11
    mk = binding.Marked(n, marked)
    full = binding.State(n, dtype)
    full.set_resident(path)
    full.init_uniform()
    full.iterate(mk, k1)
    part = binding.State(n, dtype)
    part.set_resident(path)
    part.init_uniform()
    part.iterate(mk, k1)
    f = str(tmp_path / "ck.npz")
    checkpoint.save(f, part, marked, k1)
    full.iterate(mk, k2)
    st, mk2, marked2, it = checkpoint.load(f)
    assert it == k1 and np.array_equal(marked2, marked)
    st.set_resident(path)
    st.iterate(mk2, k2)
    torch.cuda.synchronize()
    assert np.array_equal(st.amps.cpu().numpy(), full.amps.cpu().numpy())
