"""The float-float arithmetic of the on-chip phase sweeps (phase_ops.cuh:
ff_add, ff_mul, cff_mul), compiled for the host and checked against exact
rational arithmetic: sums within 2^-44 and products within 2^-43 of the exact
value relative to its magnitude (complex products relative to |a||b|), with
normalised results (|lo| <= ulp(hi) / 2).  These bounds are what the sweeps'
per-step constants rely on (about 48 significant bits, two float32 roundings
of margin), stated against the exact value, not against another float
implementation."""
from __future__ import annotations

import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bits(x: float) -> str:
    return struct.pack(">f", x).hex()


def val(h: str) -> float:
    return struct.unpack(">f", bytes.fromhex(h))[0]


def rand_ff(g: random.Random):
    e = g.randint(-40, 20)
    hi = float(np.float32(g.uniform(1.0, 2.0) * 2.0 ** e * g.choice((-1, 1))))
    ulp = float(np.spacing(np.float32(abs(hi))))
    lo = float(np.float32(g.uniform(-0.5, 0.5) * ulp))
    return hi, lo


def exact(p):
    return Fraction(p[0]) + Fraction(p[1])


def check_norm(hi, lo):
    if hi == 0.0:
        return lo == 0.0
    return abs(lo) <= float(np.spacing(np.float32(abs(hi)))) / 2


def test_float_float_error_bounds(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not available")
    exe = str(tmp_path / "ff_ops")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2005_04635_gb300", "csrc"),
                    "-o", exe, os.path.join(ROOT, "tests", "host", "ff_ops.cu")], check=True)
    g = random.Random(2005)
    cases = []
    for _ in range(1500):
        a, b = rand_ff(g), rand_ff(g)
        if g.random() < 0.2:  # near cancellation
            b = (-a[0], float(np.float32(g.uniform(-1, 1) * abs(a[1]) + 0.0)))
        cases.append((0, a, b))
        cases.append((1, a, b))
    for _ in range(1000):
        cases.append((2, rand_ff(g), rand_ff(g), rand_ff(g), rand_ff(g)))
    lines = []
    for c in cases:
        ws = [bits(x) for p in c[1:] for x in p]
        lines.append(f"{c[0]} " + " ".join(ws))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    for c, line in zip(cases, out):
        r = [val(h) for h in line.split()]
        if c[0] in (0, 1):
            a, b = exact(c[1]), exact(c[2])
            want = a + b if c[0] == 0 else a * b
            got = Fraction(r[0]) + Fraction(r[1])
            # sums: 2^-44 of |a| + |b| (covers cancellation); products: 2^-43 of |a b|
            scale = (abs(a) + abs(b)) if c[0] == 0 else abs(a * b)
            bound = Fraction(1, 2 ** (44 if c[0] == 0 else 43)) * scale
            assert abs(got - want) <= bound, (c, r)
            assert check_norm(r[0], r[1]), (c, r)
        else:
            ar, ai, br, bi = (exact(p) for p in c[1:])
            want_re, want_im = ar * br - ai * bi, ar * bi + ai * br
            got_re = Fraction(r[0]) + Fraction(r[1])
            got_im = Fraction(r[2]) + Fraction(r[3])
            mag = (abs(ar) + abs(ai)) * (abs(br) + abs(bi))
            bound = Fraction(1, 2 ** 42) * mag
            assert abs(got_re - want_re) <= bound and abs(got_im - want_im) <= bound, (c, r)
            assert check_norm(r[0], r[1]) and check_norm(r[2], r[3]), (c, r)
