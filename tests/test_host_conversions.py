"""The integer-only conversions used by the FP32-phase kernels, compiled for the host
and checked against exact rational arithmetic (Python fractions) and NumPy casts."""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
EXE = os.path.join(HERE, "host", "_build", "conv_main")


@pytest.fixture(scope="module")
def conv():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    src = os.path.join(HERE, "host", "conv_main.cu")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", EXE, src], check=True)

    def run(lines):
        res = subprocess.run([EXE], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return [int(x) for x in res.stdout.split()]
    return run


def _expected_frac(r, l):
    inv = Fraction(1.0 / l)
    v = Fraction(r) * inv * (1 << 32)
    mag = abs(v)
    n = int(mag)
    if mag - n >= Fraction(1, 2):   # half away from zero on the magnitude
        n += 1
    return (-n if v < 0 else n) % (1 << 32)


def test_fixed_fraction_exact(conv):
    rng = np.random.default_rng(3)
    cases = []
    for l in (10.0, 80.0, 120.0, 342.0, 44.78, 1.0, 3.3):
        rs = np.concatenate([rng.uniform(0, l, 60), rng.uniform(-3 * l, 3 * l, 30), [0.0, -0.0, l, 2 * l, -l, 1e-300,
                             5e-324, l * 1e5, 0.5 * l, 0.25 * l, l * (1 - 2**-40)]])
        cases += [(float(r), l) for r in rs]
    got = conv([f"F {r!r} {l!r}" for r, l in cases])
    for (r, l), g in zip(cases, got):
        exp = 0 if abs(r) < 1e-290 else _expected_frac(r, l)
        assert g == exp, (r, l, g, exp)


def test_double_to_float_matches_numpy(conv):
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.normal(size=200), rng.uniform(-1e30, 1e30, 50), [1.0, -1.0, 0.4238, -0.8476, 3.4e38,
                         1e-30, 0.0, 1.0 + 2**-24, 1.0 + 3 * 2**-24, 1.0 + 2**-24 + 2**-50]])
    got = conv([f"D {float(x)!r}" for x in xs])
    for x, g in zip(xs, got):
        ref = struct.unpack("<I", struct.pack("<f", np.float32(x)))[0]
        assert g == ref, (x, hex(g), hex(ref))


def test_float_to_double_exact(conv):
    rng = np.random.default_rng(5)
    fs = np.concatenate([rng.normal(size=200).astype(np.float32), np.array([0.0, -0.0, 1e-40, -3e-42, 3.4e38,
                         np.inf, -np.inf], dtype=np.float32)])
    bits = [struct.unpack("<I", struct.pack("<f", f))[0] for f in fs]
    got = conv([f"W {b}" for b in bits])
    for f, g in zip(fs, got):
        ref = struct.unpack("<Q", struct.pack("<d", float(f)))[0]
        assert g == ref, (f, hex(g), hex(ref))
