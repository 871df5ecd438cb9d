"""Pins of the mod2as oracle (Sec. 3.2: y = A x, A in the 3-array CSR form)
against what the mathematics fixes, independent of the oracle itself:
exact integer products, identity and permutation matrices, the dense
product of the already-pinned GEMM oracle, exact rationals, an
ill-conditioned row for the compensated variant, and the structure checks.
CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

U = 2.0 ** -53


def dense_of(rowp, indx, vals, ncols):
    n = len(rowp) - 1
    D = np.zeros((n, ncols))
    for i in range(n):
        D[i, indx[rowp[i]:rowp[i + 1]]] = vals[rowp[i]:rowp[i + 1]]
    return D


def csr_of(D):
    rowp, indx, vals = [0], [], []
    for row in D:
        nz = np.nonzero(row)[0]
        indx.extend(nz)
        vals.extend(row[nz])
        rowp.append(len(indx))
    return np.array(rowp, np.int32), np.array(indx, np.int32), np.array(vals, np.float64)


def test_integer_entries_exact():
    """Integers in [-8, 8]: every partial sum is an integer below 2^53, so
    y is exact and equals the int64 product."""
    rowp, indx, _ = inputs.csr_random(0, 50, 400, 0.05)
    vals = inputs.int_uniform(0, 51, (len(indx),), -8, 8)
    x = inputs.int_uniform(0, 52, (400,), -8, 8)
    D = dense_of(rowp, indx, vals, 400).astype(np.int64)
    assert np.array_equal(oracle.spmv(rowp, indx, vals, x), (D @ x.astype(np.int64)).astype(float))


def test_identity_and_permutation():
    n = 257
    x = inputs.uniform_pm1(0, 53, (n,))
    rowp = np.arange(n + 1, dtype=np.int32)
    assert np.array_equal(oracle.spmv(rowp, np.arange(n, dtype=np.int32), np.ones(n), x), x)
    p = inputs.permutation(0, 54, n).astype(np.int32)
    assert np.array_equal(oracle.spmv(rowp, p, np.ones(n), x), x[p])


def test_matches_the_dense_oracle():
    """Summing a row's non-zeros in column order is the naive dense loop
    with the zero terms left out (adding +-0 changes no non-zero sum)."""
    rowp, indx, vals = inputs.csr_random(0, 55, 300, 0.06)
    x = inputs.uniform_pm1(0, 56, (300,))
    D = dense_of(rowp, indx, vals, 300)
    ref = oracle.gemm_naive(D, x.reshape(-1, 1)).ravel()
    got = oracle.spmv(rowp, indx, vals, x)
    assert np.all((got == ref) | ((got == 0) & (ref == 0)))


def test_rationals_and_error_bounds():
    """Against exact rational sums: the storage-order loop within
    gamma_len sum|a||x|, Dot2 within u|y| + 2 len^2 u^2 sum|a||x|."""
    rowp, indx, vals = inputs.csr_random(3, 57, 60, 0.3)
    x = inputs.exp_spread(3, 58, (60,), -10, 10)
    y = oracle.spmv(rowp, indx, vals, x)
    y2 = oracle.spmv_dot2(rowp, indx, vals, x)
    ab = oracle.spmv_abs(rowp, indx, vals, x)
    for i in range(60):
        terms = [Fraction(float(vals[j])) * Fraction(float(x[indx[j]]))
                 for j in range(rowp[i], rowp[i + 1])]
        exact = sum(terms, Fraction(0))
        L = rowp[i + 1] - rowp[i]
        absum = float(sum((abs(t) for t in terms), Fraction(0)))
        assert abs(Fraction(float(y[i])) - exact) <= Fraction(L * U / (1 - L * U)) * Fraction(absum)
        assert abs(Fraction(float(y2[i])) - exact) <= Fraction(U) * abs(exact) + \
            Fraction(2 * L * L * U * U) * Fraction(absum)
        assert ab[i] == pytest.approx(absum, rel=L * U * 2)


def test_dot2_ill_conditioned_row():
    """(1e16 + 1 - 1e16) x 1: the storage-order sum loses the 1, Dot2 keeps it."""
    rowp = np.array([0, 3], np.int32)
    indx = np.array([0, 1, 2], np.int32)
    vals = np.array([1e16, 1.0, -1e16])
    x = np.ones(3)
    assert oracle.spmv(rowp, indx, vals, x)[0] != 1.0
    assert oracle.spmv_dot2(rowp, indx, vals, x)[0] == 1.0
    # |-1e16| + |1| + |1e16| in storage order: 1e16 + 1 rounds to 1e16, then 2e16
    assert oracle.spmv_abs(rowp, indx, -vals, x)[0] == 2e16


def test_empty_rows_and_matrix():
    rowp = np.array([0, 0, 2, 2], np.int32)
    y = oracle.spmv(rowp, np.array([1, 2], np.int32), np.array([2.0, -3.0]), np.array([5., 7., 11.]))
    assert list(y) == [0.0, 2 * 7 - 3 * 11.0, 0.0]
    y = oracle.spmv(np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0), np.ones(3))
    assert np.array_equal(y, np.zeros(4))


def test_structure_is_checked():
    x = np.ones(3)
    with pytest.raises(ValueError):  # rowp not monotone
        oracle.spmv(np.array([0, 2, 1, 3], np.int32), np.zeros(3, np.int32), np.ones(3), x)
    with pytest.raises(ValueError):  # column out of range
        oracle.spmv(np.array([0, 1], np.int32), np.array([3], np.int32), np.ones(1), x)
    with pytest.raises(ValueError):  # rowp[n] != nnz
        oracle.spmv(np.array([0, 1], np.int32), np.array([0, 1], np.int32), np.ones(2), x)


def test_generator():
    a = inputs.csr_random(7, 60, 500, 0.045)
    b = inputs.csr_random(7, 60, 500, 0.045)
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    rowp, indx, vals = a
    nnz = rowp[-1]
    assert rowp.dtype == np.int32 and indx.dtype == np.int32 and len(vals) == nnz
    assert abs(nnz / 500 ** 2 - 0.045) < 4 * np.sqrt(0.045 * 0.955 / 500 ** 2)
    for i in range(500):
        c = indx[rowp[i]:rowp[i + 1]]
        assert np.all(np.diff(c) > 0) and (len(c) == 0 or (c[0] >= 0 and c[-1] < 500))
    D = dense_of(rowp, indx, vals, 500)
    r2, i2, v2 = csr_of(D)
    assert np.array_equal(r2, rowp) and np.array_equal(i2, indx) and np.array_equal(v2, vals)


def test_sampled_generator():
    """The per-value generator for large matrices: valid CSR, repeatable,
    mean length and spread those of the binomial fill it stands in for."""
    a = inputs.csr_sampled(7, 61, 20000, 30000, 40.0)
    b = inputs.csr_sampled(7, 61, 20000, 30000, 40.0)
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    rowp, indx, vals = a
    assert rowp.dtype == np.int32 and indx.dtype == np.int32 and len(vals) == rowp[-1]
    lens = np.diff(rowp)
    assert abs(lens.mean() - 40.0) < 0.3 and abs(lens.std() - np.sqrt(40 * (1 - 40 / 30000))) < 0.5
    r = np.repeat(np.arange(20000, dtype=np.int64), lens)
    key = r * 30000 + indx
    assert np.all(np.diff(key) > 0) and indx.min() >= 0 and indx.max() < 30000
