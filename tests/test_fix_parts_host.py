"""fix_parts (fixed_sum.cuh), the split behind fix_add_cvt (the streaming
pass's exact FP32 accumulation), compiled for the host and checked against the
definition fix_add also implements, with Python integers: every value x with
|x| < 16 contributes round-toward-zero of x 2^100, exactly, the sum taken
modulo 2^128.  Values mix signs, magnitudes from subnormal to just below 16 and
zeros of both signs (values of 16 and more take the FP64 side sum before the
split and are not sent)."""
from __future__ import annotations

import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def f32(x: float) -> float:
    return struct.unpack("<f", struct.pack("<f", x))[0]


def bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def reference(vals):
    total, side = 0, 0.0
    for v in vals:
        if math.isfinite(v) and abs(v) < 16.0:
            q = Fraction(v) * (1 << 100)
            total += int(q)  # int() truncates toward zero
        else:
            side += v
    return total % (1 << 128), side


def sequences(seed=77):
    g = random.Random(seed)
    out = []
    for _ in range(400):
        n = g.choice([1, 2, 7, 64, 512])
        vals = []
        for _ in range(n):
            r = g.random()
            if r < 0.05:
                v = g.choice([0.0, -0.0, 15.999999, -15.999999, 1e-45, -1e-45, 2.0 ** -126, 2.0 ** -50])
            elif r < 0.15:  # subnormals and tiny values
                v = g.uniform(-1, 1) * 2.0 ** g.randint(-149, -100)
            else:
                v = g.uniform(-1, 1) * 2.0 ** g.randint(-60, 3)
            vals.append(f32(v))
        out.append(vals)
    return out


def test_fix_parts_matches_the_fixed_point_definition(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not available")
    exe = str(tmp_path / "fix_parts")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2005_04635_gb300", "csrc"),
                    "-o", exe, os.path.join(ROOT, "tests", "host", "fix_parts.cu")], check=True)
    seqs = sequences()
    inp = "".join(f"{len(s)} " + " ".join(f"{bits(v):x}" for v in s) + "\n" for s in seqs)
    lines = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.splitlines()
    assert len(lines) == len(seqs)
    for s, line in zip(seqs, lines):
        h, l = line.split()
        got = (int(h, 16) << 64) | int(l, 16)
        want, wside = reference(s)
        assert wside == 0.0
        assert got == want, (s[:4], got, want)
