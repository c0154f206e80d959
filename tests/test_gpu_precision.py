"""Precision study (complex64 storage, n=26 Gaussian start, M=8, 3000 iterations):
every mean accumulation mode against the FP64 oracle's closed form for an
arbitrary start.

Bounds: P_success within 1e-4 of the FP64 value (the stated tolerance for
FP32 results) in every mode but plain FP32.  The error vector's norm, and so
the largest amplitude error, has a worst-case bound (c64_bounds) for the
default, exact and FP64 modes: per iteration two roundings per stored
amplitude (2u) plus the mean's error, an error e in the computed mean adding
2 e sqrt(N) to the norm (at most 6u for the FP32 pairwise 8-amplitude tile
sums of the streaming pass this study runs, none for the exact mode),
propagated unitarily.  The
compensated mode's running sums and FP32 block tree have no bound of that
size; it is held to the FP64 mode's bound as an observed margin."""
from __future__ import annotations

import pytest

import c64_bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def study():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    return bench.run_precision_study(None)


def _row(study, start, state, mode):
    return next(r for r in study["rows"]
                if r["start"] == start and r["state"] == state and r["accumulation"] == mode)


@pytest.mark.parametrize("start", ["gaussian", "uniform"])
@pytest.mark.parametrize("mode", ["kahan", "fp64", "default", "exact"])
def test_compensated_and_wide_modes(study, start, mode):
    r = _row(study, start, "c64", mode)
    assert r["p_success_err"] <= 1e-4
    n, k = 26, 3000
    rho = {"default": c64_bounds.RHO["tile8"], "exact": c64_bounds.RHO["exact"]}.get(mode, c64_bounds.rho_fp64(n))
    assert r["max_abs_err"] <= c64_bounds.norm_bound(k, 1.0, rho)


@pytest.mark.parametrize("start", ["gaussian", "uniform"])
def test_plain_fp32_is_reported(study, start):
    r = _row(study, start, "c64", "fp32")
    assert r["max_abs_err"] >= 0.0 and r["p_success"] > 0.0  # reported, no bound asserted


@pytest.mark.parametrize("start", ["gaussian", "uniform"])
def test_complex128_reference_run(study, start):
    r = _row(study, start, "c128", "default")
    assert r["max_abs_err"] <= 1e-11 and r["p_success_err"] <= 1e-11
