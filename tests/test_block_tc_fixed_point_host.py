"""Host-side check of the exactness argument of the block tensor-core products
(paper_1808_03374_gb300/csrc/block_tc.cu), from the constants written in that
file, against the e4m3 format as the OCP 8-bit floating point specification
defines it (no GPU needed):

- the code-function tables hold the e4m3 bytes of f1 = g [observed] ->
  {0, 1, 2, 0} and f2 = [observed] -> {1, 1, 1, 0} for codes 0..3 (3 = missing);
- every integer in [-16, 16] is an e4m3 value, and D balanced base-16 digits
  write every |X| <= 2^(4D) with digits 1..D-1 in [-8, 7] and digit 0 in
  [-16, 16];
- the size limits keep every FP32 accumulator an integer below 2^24 (A^T U:
  |f1 d| <= 32 per sample; A V: |f1 d1| + |f2 d2| <= 48 per SNP), and the
  digit recombination in 64-bit integers does not overflow.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "paper_1808_03374_gb300", "csrc", "block_tc.cu")).read()


def const(name):
    m = re.search(r"\b" + name + r"\s*=\s*(0x[0-9A-Fa-f]+|\d+)u?\b", SRC)
    assert m, name
    return int(m.group(1), 0)


def e4m3(byte):
    """Value of an E4M3 byte: sign bit, four exponent bits (bias 7), three
    mantissa bits; exponent 0 is subnormal; S.1111.111 is NaN (no infinities)."""
    s, e, mnt = (byte >> 7) & 1, (byte >> 3) & 15, byte & 7
    if e == 15 and mnt == 7:
        return float("nan")
    mag = mnt / 8 * 2.0 ** -6 if e == 0 else 2.0 ** (e - 7) * (1 + mnt / 8)
    return -mag if s else mag


def test_e4m3_decoder_landmarks():
    assert e4m3(0x38) == 1.0 and e4m3(0x40) == 2.0 and e4m3(0x7E) == 448.0 and e4m3(0x01) == 2.0 ** -9
    assert np.isnan(e4m3(0x7F)) and e4m3(0xB8) == -1.0


def test_code_function_tables():
    f1 = [e4m3((const("kLut1") >> (8 * c)) & 0xFF) for c in range(4)]
    f2 = [e4m3((const("kLut2") >> (8 * c)) & 0xFF) for c in range(4)]
    assert f1 == [0.0, 1.0, 2.0, 0.0]
    assert f2 == [1.0, 1.0, 1.0, 0.0]


def test_small_integers_are_e4m3_values():
    values = {e4m3(b) for b in range(256)}
    assert all(float(v) in values for v in range(-16, 17))
    assert 17.0 not in values  # the digit range is as wide as the format allows


def balanced_digits16(X, D):
    d, r = [], int(X)
    for _ in range(D - 1):
        dg = ((r + 8) & 15) - 8
        d.append(dg)
        r = (r - dg) >> 4
    return [r] + d[::-1]


@pytest.mark.parametrize("D", [4, 8])
def test_balanced_base16_digits(D):
    top = 1 << (4 * D)
    rng = np.random.default_rng(D)
    xs = [0, 1, -1, 8, -8, 7, -9, top, -top, top - 1, 1 - top] + [int(x) for x in
                                                                  rng.integers(-top, top, 2000, endpoint=True)]
    for X in xs:
        d = balanced_digits16(X, D)
        assert -16 <= d[0] <= 16 and all(-8 <= x <= 7 for x in d[1:])
        assert sum(x * 16 ** (D - 1 - p) for p, x in enumerate(d)) == X


def test_size_limits_keep_accumulators_exact():
    assert 2 * 16 * const("kMaxSamplesRmv") < 2 ** 24          # A^T U: |f1| <= 2, |digit| <= 16
    assert (2 * 16 + 1 * 16) * const("kMaxSnpsChunk") < 2 ** 24  # A V: f1 d1 + f2 d2
    for D in (4, 8):  # recombination sum_p 16^(D-1-p) F_p, |F_p| < 2^24
        assert sum(16 ** (D - 1 - p) for p in range(D)) * 2 ** 24 < 2 ** 63
