"""Precision study (complex64 storage, n=26 Gaussian start, M=8, 3000 iterations):
every mean accumulation mode against the FP64 oracle's closed form for an
arbitrary start.

Bounds: the amplitude error of complex64 storage is at most 3k * 2^-24 (one
FP32 rounding per stored amplitude per iteration plus the shared rounding of
2 mu, propagated unitarily; the hi + lo form of 2 mu removes the latter for
these modes but the bound keeps it) plus the effect of the mean's error: an
error e in the computed mean adds 2 e sqrt(N) to the error norm per iteration.
The compensated, FP64 and exact modes keep e far below the storage rounding;
P_success must be within 1e-4 of the FP64 value (the stated tolerance)."""
from __future__ import annotations

import pytest

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
    assert r["max_abs_err"] <= 3 * 3000 * 2.0 ** -24


@pytest.mark.parametrize("start", ["gaussian", "uniform"])
def test_plain_fp32_is_reported(study, start):
    r = _row(study, start, "c64", "fp32")
    assert r["max_abs_err"] >= 0.0 and r["p_success"] > 0.0  # reported, no bound asserted


@pytest.mark.parametrize("start", ["gaussian", "uniform"])
def test_complex128_reference_run(study, start):
    r = _row(study, start, "c128", "default")
    assert r["max_abs_err"] <= 1e-11 and r["p_success_err"] <= 1e-11
