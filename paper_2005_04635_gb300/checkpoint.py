"""Checkpoint / resume of a search: the amplitudes plus a small header.

The state of a running search is its amplitudes, the iteration count done so
far and the marked set; the cached mean is recomputed from the amplitudes on
resume (the first pass after init_state reduces them).  A checkpoint is a numpy
``.npz`` file: ``amps`` (complex64 or complex128, 2^n), ``marked`` (uint64),
and the header fields ``n``, ``dtype``, ``iteration``.  Saving copies device
to host; loading copies host to device through grover_init_state.  Plumbing
only: no arithmetic on the amplitudes happens here.
"""
from __future__ import annotations

import numpy as np

from .binding import Marked, State

FORMAT = "grover-checkpoint-1"


def save(path: str, state: State, marked, iteration: int) -> None:
    import torch
    torch.cuda.synchronize()
    amps = state.amps.detach().cpu().numpy()
    np.savez(path, format=np.array(FORMAT), n=np.int64(state.n), dtype=np.array(state.dtype),
             iteration=np.int64(iteration), marked=np.asarray(marked, dtype=np.uint64), amps=amps)


def load(path: str, stream=None, device=None):
    """Returns (state, Marked, marked indices, iteration)."""
    with np.load(path) as z:
        if str(z["format"]) != FORMAT:
            raise ValueError(f"{path}: not a {FORMAT} file")
        n, dtype, it = int(z["n"]), str(z["dtype"]), int(z["iteration"])
        marked = z["marked"].astype(np.uint64)
        amps = z["amps"]
    want = np.complex64 if dtype == "c64" else np.complex128
    if amps.dtype != want or amps.shape != (1 << n,):
        raise ValueError(f"{path}: amplitudes do not match the header")
    st = State(n, dtype, stream=stream, device=device)
    st.init_state(amps)
    return st, Marked(n, marked), marked, it
