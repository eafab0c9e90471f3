"""The integer helpers of the split-precision path, compiled for the host, against exact
Python integer / fraction arithmetic: fixed point from IEEE bits (round half away from
zero), balanced base-256 digits (reconstruct F exactly, digit ranges of the exactness
bound), and I 2^E back to the correctly rounded double (ties away from zero)."""
import os
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("si") / "split_int_check")
    subprocess.check_call(["nvcc", "-std=c++17", "-o", out, os.path.join(ROOT, "tests", "native", "split_int_check.cu")])
    return out


def run(exe, lines):
    return subprocess.check_output([exe], input="\n".join(lines) + "\n", text=True).splitlines()


def round_half_away(fr):
    n = abs(fr)
    q = int(n + Fraction(1, 2)) if (n - int(n)) == Fraction(1, 2) else round(n)
    if (n - int(n)) == Fraction(1, 2):
        q = int(n) + 1
    return q if fr >= 0 else -q


def test_fixed_point_and_exponent(exe):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.standard_normal(300) * 10.0 ** rng.integers(-12, 12, 300), [1.0, -0.5, 2.0**-1030]])
    lines, cases = [], []
    for x in xs:
        e = int(np.frexp(x)[1]) if x != 0 else 0
        sh = 40 - e + int(rng.integers(-3, 3))
        b = struct.unpack("<Q", struct.pack("<d", float(x)))[0]
        lines.append(f"fp {b:x} {sh}")
        cases.append((float(x), sh))
    out = run(exe, lines)
    for (x, sh), o in zip(cases, out):
        got, ex = map(int, o.split())
        if abs(x) < 2.0**-1022:
            assert got == 0
            continue
        ref = round_half_away(Fraction(x) * Fraction(2) ** sh)
        assert got == ref, (x, sh)
        assert ex == np.frexp(x)[1]


def test_balanced_digits(exe):
    rng = np.random.default_rng(2)
    Fs = [int(v) for v in rng.integers(-(2**40), 2**40, 500)] + [2**40, -(2**40), 0, 127, 128, -128, 2**24 - 1]
    out = run(exe, [f"dg {F}" for F in Fs])
    for F, o in zip(Fs, out):
        d = list(map(int, o.split()))
        d5, d6 = d[:5], d[5:]
        assert sum(v * 256 ** (4 - i) for i, v in enumerate(d5)) == F
        assert sum(v * 256 ** (5 - i) for i, v in enumerate(d6)) == F
        assert abs(d5[0]) <= 256 and all(-128 <= v <= 127 for v in d5[1:])
        assert all(-128 <= v <= 127 for v in d6[1:])


def test_scaled_to_double(exe):
    rng = np.random.default_rng(3)
    cases = [(int(i), int(e)) for i, e in zip(rng.integers(-(2**56), 2**56, 400), rng.integers(-120, 60, 400))]
    cases += [(2**53 + 1, 0), (-(2**53 + 1), 3), (2**54 + 2, -7), (1, -1074 + 60)]
    out = run(exe, [f"sd {i} {e}" for i, e in cases])
    for (i, e), o in zip(cases, out):
        got = struct.unpack("<d", struct.pack("<Q", int(o, 16)))[0]
        exact = Fraction(i) * Fraction(2) ** e
        # correctly rounded to 53 bits with ties away from zero
        if i == 0:
            assert got == 0.0
            continue
        mag = abs(exact)
        k = mag.numerator.bit_length() - mag.denominator.bit_length()
        while Fraction(2) ** k > mag:
            k -= 1
        while Fraction(2) ** (k + 1) <= mag:
            k += 1
        ulp = Fraction(2) ** (k - 52)
        q = mag / ulp
        r = int(q) + (1 if q - int(q) >= Fraction(1, 2) else 0)
        ref = float(r * ulp) * (1 if exact > 0 else -1)
        assert got == ref, (i, e)
