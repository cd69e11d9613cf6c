"""Host-side check of the exactness argument of the tensor-core A^T u
(paper_1808_03374_gb300/csrc/packed_tc.cu), from the constants and the digit
table written in that file, against the e2m1 format as the OCP Microscaling
specification defines it (no GPU needed):

- the kernel's nibble table maps the balanced base-8 digits -4..3 onto e2m1
  codes of exactly those values, and a 2-bit genotype code c read as an e2m1
  nibble is c/2;
- D digits of kBits = 3 (D - 1) fractional bits write every |z| <= 2^kBits with
  digits in [-4, 3] and a leading digit of -1, 0 or 1;
- every FP32 accumulator value is a multiple of 1/2 below 2^23 over a K-range
  (so exact), and each 16-lane half recombines its digits in 64-bit integers
  without overflow.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "paper_1808_03374_gb300", "csrc", "packed_tc.cu")).read()


def const(name):
    m = re.search(r"\b" + name + r"\s*=\s*(0x[0-9A-Fa-f]+|\d+)u?\b", SRC)
    assert m, name
    return int(m.group(1), 0)


def e2m1(nibble):
    """Value of a 4-bit E2M1 element: sign bit, two exponent bits (bias 1), one
    mantissa bit; exponent 0 is subnormal (mantissa x 2^(1-bias) / 2)."""
    s, e, mnt = (nibble >> 3) & 1, (nibble >> 1) & 3, nibble & 1
    mag = 0.5 * mnt if e == 0 else 2.0 ** (e - 1) * (1 + 0.5 * mnt)
    return -mag if s else mag


def test_e2m1_decoder_reproduces_the_format_table():
    assert [e2m1(x) for x in range(8)] == [0.0, 0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0]
    assert [e2m1(x) for x in range(8, 16)] == [-0.0, -0.5, -1.0, -1.5, -2.0, -3.0, -4.0, -6.0]


def test_digit_table_and_code_values():
    lut = const("lut")
    for k in range(8):  # nibble k holds the code of digit k - 4
        assert e2m1((lut >> (4 * k)) & 0xF) == k - 4
    for c in range(4):  # a genotype code in the low two bits of a nibble
        assert e2m1(c) == c / 2


def balanced_digits(z, D):
    """z = sum_p d_p 8^(D-1-p): D-1 digits in [-4, 3] from the lowest up, then
    the remainder as the leading digit."""
    d, r = [], int(z)
    for _ in range(D - 1):
        dg = ((r + 4) & 7) - 4
        d.append(dg)
        r = (r - dg) >> 3
    return [r] + d[::-1]


@pytest.mark.parametrize("D", [const("kDigitsF32"), const("kDigitsF64")])
def test_balanced_digits_cover_the_fixed_point_range(D):
    assert "kBits = 3 * (D - 1)" in SRC
    bits = 3 * (D - 1)
    assert bits > (24 if D == const("kDigitsF32") else 53)  # finer than the output's significand
    rng = np.random.default_rng(D)
    top = 1 << bits
    zs = [0, 1, -1, 4, -4, 3, -5, top, -top, top - 1, 1 - top, top // 2, -(top // 2)]
    zs += [int(x) for x in rng.integers(-top, top, 2000, endpoint=True)]
    for z in zs:
        d = balanced_digits(z, D)
        assert d[0] in (-1, 0, 1), (z, d[0])
        assert all(-4 <= x <= 3 for x in d[1:])
        assert sum(x * 8 ** (D - 1 - p) for p, x in enumerate(d)) == z


@pytest.mark.parametrize("D", [const("kDigitsF32"), const("kDigitsF64")])
def test_accumulators_exact_and_recombination_fits(D):
    # 2 F_p = sum over a K-range of c d with |c| <= 3, |d| <= 4: an integer
    bound = 3 * 4 * const("kStageSamples") * const("kMaxRangeStages")
    assert bound < 2 ** 24  # so F_p, a multiple of 1/2 below 2^23, is exact in FP32
    assert "kHalf0 = D <= 11 ? D : D / 2" in SRC
    half0 = D if D <= 11 else D // 2
    for lo, hi in ((0, half0), (half0, D)):  # each half weighs its digits relative to its lowest one
        if lo < hi:
            total = sum(8 ** (hi - 1 - p) for p in range(lo, hi)) * bound
            assert total < 2 ** 63
