"""Seeded synthetic inputs for the Grover simulator.

This module draws random inputs only; it holds none of the simulator's
arithmetic and imports neither the CUDA binding nor the oracle, so both sides
can be fed the same inputs.  All draws use numpy's PCG64 generator from an
explicit seed.

Workload recipe (the paper fixes only "a search state |i>"; sizes follow the
benchmark configurations):
  * marked indices: M distinct indices drawn uniformly from [0, N), sorted;
  * initial state: uniform (|0> followed by H^{(x)n}), or i.i.d. complex
    Gaussian amplitudes (re, im ~ N(0, 1)) scaled to unit norm in FP64;
  * phases of the phase iterator: i.i.d. uniform on [0, 2 pi).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def marked_indices(n: int, m: int, seed: int) -> np.ndarray:
    """M distinct indices uniform on [0, 2^n), sorted ascending (uint64)."""
    N = 1 << n
    if m < 0 or m > N:
        raise ValueError("m must be in [0, 2^n]")
    g = rng(seed)
    if 2 * m > N:
        # dense case: a random permutation prefix
        sel = g.permutation(N)[:m]
    else:
        chosen: set[int] = set()
        while len(chosen) < m:
            chosen.add(int(g.integers(0, N)))
        sel = np.fromiter(chosen, dtype=np.uint64, count=m)
    return np.sort(np.asarray(sel, dtype=np.uint64))


def bitmask(n: int, marked) -> np.ndarray:
    """ceil(N/32) uint32 words; bit x%32 of word x/32 set for each marked x."""
    N = 1 << n
    words = np.zeros((N + 31) // 32, dtype=np.uint32)
    m = np.asarray(marked, dtype=np.uint64)
    np.bitwise_or.at(words, (m >> np.uint64(5)).astype(np.int64),
                     (np.uint32(1) << (m & np.uint64(31)).astype(np.uint32)))
    return words


def gaussian_state(n: int, seed: int) -> np.ndarray:
    """i.i.d. complex Gaussian amplitudes, unit norm (complex128)."""
    g = rng(seed)
    N = 1 << n
    re = g.standard_normal(N)
    im = g.standard_normal(N)
    psi = re + 1j * im
    psi /= np.sqrt(np.sum(re * re + im * im))
    return psi.astype(np.complex128)


def uniform_phases(K: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Two arrays of K phases i.i.d. uniform on [0, 2 pi) (float64): the
    oracle phases phi and the diffusion phases vphi of the phase iterator."""
    g = rng(seed)
    return g.uniform(0.0, 2.0 * np.pi, K), g.uniform(0.0, 2.0 * np.pi, K)
