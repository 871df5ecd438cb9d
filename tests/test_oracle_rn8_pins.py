"""Pins of the balanced 8-bit digit split (the round-to-nearest variant of
the Ozaki split) against exact integer arithmetic: every value is
represented by the rounded integer round(x 2^(8S - e')) (ties to even,
computed here with Python's exact rationals), e' is one more than the
frexp exponent of the row (column) maximum, the lower digits lie in
[-128, 127] and the top one in [-128, 128]; products of small integers are
exact; and the emulated product obeys the a-priori bound of the method."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

U = 2.0 ** -53


@pytest.mark.parametrize("S", [1, 2, 3, 5, 6, 7])
@pytest.mark.parametrize("by_col", [False, True])
def test_digits_are_the_rounded_value_in_balanced_base_256(S, by_col):
    X, _ = inputs.gemm_operands("spread", 24, 40, 8, seed=0, cfg=60 + S)
    e, d = oracle.ozaki_split_rn8(X, by_col, S)
    rows, cols = X.shape
    for i in range(rows):
        for j in range(cols):
            line = X[:, j] if by_col else X[i, :]
            mx = float(np.max(np.abs(line)))
            e1 = math.frexp(mx)[1] + 1 if mx > 0 else 1
            assert e[j if by_col else i] == e1
            x = float(X[i, j])
            V = round(Fraction(x) * Fraction(2) ** (8 * S - e1))  # ties to even
            digits = [int(d[s, i, j]) for s in range(S)]
            assert sum(dg * 256 ** (S - 1 - s) for s, dg in enumerate(digits)) == V
            assert all(-128 <= dg <= 127 for dg in digits[1:])
            assert -128 <= digits[0] <= 128


def test_top_digit_reaches_128_and_ties_go_to_even():
    # x just below the row maximum's binade top: rounds up to 2^(8S-1)
    X = np.array([[1.0 - 2.0 ** -53, 0.5]])
    e, d = oracle.ozaki_split_rn8(X, False, 2)
    assert e[0] == 1 and list(d[:, 0, 0]) == [128, 0]
    # exact ties below the last digit: 2^(8S - e') x = k + 1/2
    X = np.array([[0.75, 2.0 ** -16 * 5, 2.0 ** -16 * 7]])  # e' = 1: V = x 2^15
    e, d = oracle.ozaki_split_rn8(X, False, 2)
    assert e[0] == 1
    got = [int(d[0, 0, j]) * 256 + int(d[1, 0, j]) for j in range(3)]
    assert got == [24576, 2, 4]  # 2.5 -> 2, 3.5 -> 4


@pytest.mark.parametrize("S", [1, 2, 4, 7])
def test_small_integer_products_exact(S):
    A = inputs.int_uniform(0, 70, (33, 65), -8, 8)
    B = inputs.int_uniform(0, 71, (65, 29), -8, 8)
    want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert np.array_equal(oracle.ozaki_gemm_rn8(A, B, S), want)


@pytest.mark.parametrize("S", [3, 5, 6, 7])
def test_a_priori_bound(S):
    """|C - AB| <= k 2^(e'_i + f'_j) 2^(-8S) (S/4 + 1/2) (dropped digit pairs
    and the two roundings of the split) + the FP64 recombination."""
    m, k, n = 40, 500, 36
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=70 + S)
    C = oracle.ozaki_gemm_rn8(A, B, S)
    d2 = oracle.gemm_dot2(A, B)
    ea = np.array([math.frexp(float(np.max(np.abs(A[i]))))[1] + 1 for i in range(m)])
    fb = np.array([math.frexp(float(np.max(np.abs(B[:, j]))))[1] + 1 for j in range(n)])
    scale = np.ldexp(1.0, (ea[:, None] + fb[None, :]).astype(np.int64))
    bound = k * scale * 2.0 ** (-8 * S) * (S / 4 + 0.5) * 1.001 + 4 * U * np.abs(d2)
    assert np.all(np.abs(C - d2) <= bound)


def test_error_decreases_with_slices_and_beats_truncation():
    A, B = inputs.gemm_operands("spread", 32, 800, 32, seed=0, cfg=80)
    d2 = oracle.gemm_dot2(A, B)
    errs = [np.max(np.abs(oracle.ozaki_gemm_rn8(A, B, S) - d2)) for S in range(2, 8)]
    assert all(b <= a for a, b in zip(errs, errs[1:]))
    # rounding to nearest halves the representation error of truncation
    t6 = np.max(np.abs(oracle.ozaki_gemm(A, B, 6, beta=8) - d2))
    assert errs[4] < t6


def test_entries_match_the_full_product_and_limits():
    A, B = inputs.gemm_operands("spread", 50, 70, 45, seed=0, cfg=81)
    C = oracle.ozaki_gemm_rn8(A, B, 6)
    rng = np.random.default_rng(3)
    ii = rng.integers(0, 50, 40)
    jj = rng.integers(0, 45, 40)
    assert np.array_equal(oracle.ozaki_entries_rn8(A, B, ii, jj, 6), C[ii, jj])
    with pytest.raises(FloatingPointError):
        oracle.ozaki_gemm_rn8(A, B, 8)  # V would not fit int64
