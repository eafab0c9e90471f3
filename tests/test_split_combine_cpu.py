"""Host check of the accumulator recombination of the split-precision epilogue (combine_acc in
paper_1303_4446_gb300/csrc/split.cu): I = sum_g acc_g 2^8(S-1-g) from the S FP32 diagonal
accumulators, with

* diagonals 0 and 1 converted exactly by adding 1.5 2^23 in FP32 (|acc| <= 2^22 when the
  leading digits lie in [-128, 128] and K <= 128),
* the middle diagonals by a float-to-integer conversion,
* the last two merged in FP32 as round((acc_{S-2} + acc_{S-1}/256) / 4),

the constant 0x4B400000 offsets removed by one 64-bit constant.  The device steps are
replayed here with IEEE single-precision rounding (every FP32 add and FMA is computed exactly
in double precision and rounded once to single), so the test pins the bounds the kernel
relies on: exact integer results for the magic additions at the extreme accumulator values,
and an error of at most 2^10 in I from the merge, far below the dropped diagonals g >= S.
"""
import numpy as np
import pytest

KC = np.float32(12582912.0)  # 1.5 2^23
KCB = 0x4B400000


def f32(x):
    return np.float32(x)


def fma32(a, b, c):
    # products of a float32 and a power of two plus a float32 are exact in double precision
    return np.float32(np.float64(np.float32(a)) * np.float64(np.float32(b)) + np.float64(np.float32(c)))


def add32(a, b):
    return np.float32(np.float64(np.float32(a)) + np.float64(np.float32(b)))


def bits(x):
    return int(np.array([x], dtype=np.float32).view(np.uint32)[0])


def combine(acc, S):
    """The device recombination, step for step, in wrapping 64-bit arithmetic."""
    k_last = S - 2
    k_magic = min(k_last, 2)
    off = (KCB << 10) + sum(KCB << (8 * (S - 1 - g)) for g in range(k_magic))
    t = fma32(acc[S - 1], 2.0**-10, fma32(acc[S - 2], 0.25, KC))
    x = bits(t) * 1024 - off
    for g in range(k_magic, k_last):
        x += int(np.rint(np.float32(acc[g]))) << (8 * (S - 1 - g))
    for g in range(k_magic):
        x += bits(add32(acc[g], KC)) << (8 * (S - 1 - g))
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


def bound(g, K):
    # digits within [-128, 128]: diagonal g sums (g + 1) products of at most 2^14 per K term
    return (g + 1) * 2**14 * K


@pytest.mark.parametrize("S", [3, 4, 5, 6])
@pytest.mark.parametrize("K", [60, 96, 128])
def test_combine_error_bound(S, K):
    rng = np.random.default_rng(1000 * S + K)
    worst = 0
    for trial in range(1500):
        acc = []
        for g in range(S):
            b = bound(g, K)
            assert b < 2**24  # exact FP32 accumulation
            if trial % 3 == 0:
                acc.append(int(b) * int(rng.choice([-1, 1])))
            else:
                acc.append(int(rng.integers(-b, b + 1)))
        exact = sum(a << (8 * (S - 1 - g)) for g, a in enumerate(acc))
        got = combine([float(a) for a in acc], S)
        worst = max(worst, abs(got - exact))
    assert worst <= 2**10
    # the dropped diagonal g = S alone can contribute up to bound(S, K) / 256 in I's units:
    # the merge error stays below an eighth of that
    assert 8 * 2**10 < bound(S, K) / 256


@pytest.mark.parametrize("v", [0, 1, -1, 2**22, -(2**22), 2**22 - 1, -(2**22) + 1, 12345, -987654])
def test_magic_conversion_exact(v):
    # acc + 1.5 2^23 keeps the integer in its low mantissa bits for |acc| <= 2^22
    assert bits(add32(float(v), KC)) - KCB == v


def test_leading_diagonals_within_magic_range():
    # |acc_0| <= 2^14 K, |acc_1| <= 2^15 K: at most 2^22 for K <= 128
    assert bound(0, 128) <= 2**22 and bound(1, 128) <= 2**22
    # the merged pair stays in range too: (acc_{S-2} + acc_{S-1}/256) / 4 < 2^22 for S <= 6
    for S in (3, 4, 5, 6):
        assert (bound(S - 2, 128) + bound(S - 1, 128) / 256) / 4 < 2**22
