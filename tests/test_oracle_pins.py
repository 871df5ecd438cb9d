"""Pins of the CPU oracle against facts fixed outside the oracle itself.

The oracle (``oracle/``) is what every CUDA result is compared with, so it is
checked first, on the CPU, against: exact rational arithmetic (brute force on
tiny inputs), integer products that FP64 holds exactly, identity/permutation
and rank-1 closed forms, hand-worked examples of the definition (Sec. 3.1)
and of the Ozaki split (tests/golden/), Python's own ``math.frexp``, and the
published error bounds of the methods.  Each pin is chosen so that a plausible
mistake (a dropped term, a wrong sign or index, a transposed operand, a wrong
slice weight) fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

U = 2.0 ** -53  # unit roundoff of FP64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def exact_product(A, B):
    """Exact rational A.B of float matrices (Fractions of the doubles)."""
    m, k = A.shape
    n = B.shape[1]
    Af = [[Fraction(float(A[i, l])) for l in range(k)] for i in range(m)]
    Bf = [[Fraction(float(B[l, j])) for j in range(n)] for l in range(k)]
    return [[sum((Af[i][l] * Bf[l][j] for l in range(k)), Fraction(0)) for j in range(n)]
            for i in range(m)]


def gamma(k):
    return k * U / (1 - k * U)


# ---------------------------------------------------------------- mod2am
def test_worked_examples_from_definition():
    with open(os.path.join(GOLDEN, "mod2am_worked.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            dims, a, b, c = line.split("|")
            m, k, n = map(int, dims.split())
            A = np.array(a.split(), dtype=np.float64).reshape(m, k)
            B = np.array(b.split(), dtype=np.float64).reshape(k, n)
            C = np.array(c.split(), dtype=np.float64).reshape(m, n)
            for f in (oracle.gemm_naive, oracle.gemm_outer, oracle.gemm_dot2):
                assert np.array_equal(f(A, B), C), f.__name__
            assert np.array_equal(oracle.gemm_abs(A, B), np.abs(A) @ np.abs(B))


@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_exact_rational(seed):
    """1x1 .. 8x8: naive within gamma_k |A||B| of the exact product; Dot2
    within u|c| + gamma_k^2 |A||B| (Ogita-Rump-Oishi 2005, Prop. 5.5)."""
    rng = np.random.default_rng(seed)
    m, k, n = (int(v) for v in rng.integers(1, 9, size=3))
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-30, 30, size=(m, k)))
    B = rng.standard_normal((k, n)) * np.exp2(rng.integers(-30, 30, size=(k, n)))
    ex = exact_product(A, B)
    naive = oracle.gemm_naive(A, B)
    dot2 = oracle.gemm_dot2(A, B)
    absp = exact_product(np.abs(A), np.abs(B))
    for i in range(m):
        for j in range(n):
            e = ex[i][j]
            s = absp[i][j]
            assert abs(Fraction(float(naive[i, j])) - e) <= Fraction(gamma(k)) * s
            bound = Fraction(U) * abs(e) + Fraction(gamma(k)) ** 2 * s
            assert abs(Fraction(float(dot2[i, j])) - e) <= bound
    # the abs product is a sum of non-negative terms: within gamma_k too
    ab = oracle.gemm_abs(A, B)
    for i in range(m):
        for j in range(n):
            assert abs(Fraction(float(ab[i, j])) - absp[i][j]) <= Fraction(gamma(k)) * absp[i][j]


def test_bruteforce_catches_transpose():
    """A non-square case where using B^T (or A^T) would give another shape or
    value: the result must equal the exact product entry by entry."""
    A = np.array([[1.0, 2.0, 3.0]])
    B = np.array([[1.0, 0.0], [0.0, 10.0], [100.0, 0.0]])
    assert np.array_equal(oracle.gemm_naive(A, B), np.array([[301.0, 20.0]]))


@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 13, 5), (64, 257, 33), (128, 1024, 96)])
def test_integer_inputs_exact(shape):
    """Integers in [-8, 8]: |c| <= 64k << 2^53, every partial sum is an exact
    integer, so naive, mxm2a order and Dot2 all equal the int64 product."""
    m, k, n = shape
    A, B = inputs.gemm_operands("int8", m, k, n, seed=0, cfg=3)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    for f in (oracle.gemm_naive, oracle.gemm_outer, oracle.gemm_dot2):
        assert np.array_equal(f(A, B), ref), f.__name__
    assert np.array_equal(oracle.gemm_abs(A, B),
                          (np.abs(A).astype(np.int64) @ np.abs(B).astype(np.int64)).astype(np.float64))


def test_identity_and_permutation_exact():
    n = 96
    A, B = inputs.gemm_operands("uniform", n, n, n, seed=0, cfg=0)
    I = np.eye(n)
    assert np.array_equal(oracle.gemm_naive(I, B), B)
    assert np.array_equal(oracle.gemm_naive(A, I), A)
    P = inputs.permutation_matrix(0, 7, n)
    p = inputs.permutation(0, 7, n)
    assert np.array_equal(oracle.gemm_naive(P, B), B[p])
    assert np.array_equal(oracle.gemm_naive(A, P.T), A[:, p])
    assert np.array_equal(oracle.gemm_dot2(P, B), B[p])


def test_rank1_closed_form():
    """A = u v^T, B = w z^T with small dyadic entries: C = (v.w) u z^T
    exactly (every product and partial sum is a short dyadic number)."""
    m, k, n = 20, 31, 17
    rng = np.random.default_rng(5)
    u = rng.integers(-8, 9, m) / 4.0
    v = rng.integers(-8, 9, k) / 8.0
    w = rng.integers(-8, 9, k) / 2.0
    z = rng.integers(-8, 9, n) / 16.0
    A = np.outer(u, v)
    B = np.outer(w, z)
    vw = float(np.dot(v, w))  # exact: short dyadics
    C = vw * np.outer(u, z)
    for f in (oracle.gemm_naive, oracle.gemm_outer, oracle.gemm_dot2):
        assert np.array_equal(f(A, B), C)


def test_ones_closed_form():
    for k in (1, 5, 1000):
        C = oracle.gemm_naive(np.ones((3, k)), np.ones((k, 4)))
        assert np.array_equal(C, np.full((3, 4), float(k)))


def test_empty_k_gives_zeros():
    A = np.zeros((3, 0))
    B = np.zeros((0, 5))
    for f in (oracle.gemm_naive, oracle.gemm_outer, oracle.gemm_dot2, oracle.gemm_abs):
        assert np.array_equal(f(A, B), np.zeros((3, 5)))


@pytest.mark.parametrize("shape", [(5, 9, 7), (33, 100, 65)])
def test_naive_equals_mxm2a_order(shape):
    """The naive loop and the rank-1 update order add the same terms in the
    same order for every entry: equal values."""
    m, k, n = shape
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=1)
    assert np.array_equal(oracle.gemm_naive(A, B), oracle.gemm_outer(A, B))


def test_naive_within_bound_of_dot2_random():
    m, k, n = 40, 700, 30
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=2)
    d = oracle.gemm_dot2(A, B)
    nv = oracle.gemm_naive(A, B)
    ab = oracle.gemm_abs(A, B)
    assert np.all(np.abs(nv - d) <= gamma(k) * ab)
    # and Dot2 is far tighter than that: a few ulps of |C| plus gamma_k^2 |A||B|
    assert np.all(np.abs(d - np.asarray(nv)) >= 0)


def test_entries_match_full():
    m, k, n = 23, 57, 19
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=4)
    ii = np.array([0, 5, 22, 7, 7])
    jj = np.array([0, 18, 3, 7, 8])
    d2, ab = oracle.entries_dot2_abs(A, B, ii, jj)
    assert np.array_equal(d2, oracle.gemm_dot2(A, B)[ii, jj])
    assert np.array_equal(ab, oracle.gemm_abs(A, B)[ii, jj])


# ---------------------------------------------------------------- Ozaki split
def _golden_split_rows():
    with open(os.path.join(GOLDEN, "ozaki_split_digits.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            head, vals, digs = line.split("|")
            beta, S, e = map(int, head.split())
            vals = np.array([float.fromhex(v) for v in vals.split()])
            digs = np.array([[int(x) for x in d.split()] for d in digs.split(";")])
            yield beta, S, e, vals, digs


def test_split_hand_worked_digits():
    rows = list(_golden_split_rows())
    assert len(rows) >= 10
    for beta, S, e, vals, digs in rows:
        ex, d = oracle.ozaki_split(vals[None, :], by_col=False, beta=beta, S=S)
        assert ex[0] == e, (vals, ex)
        assert np.array_equal(d[:, 0, :].T, digs), (vals, d[:, 0, :].T, digs)
        # the same values as a column of a k x 1 matrix (by-column exponent)
        ec, dc = oracle.ozaki_split(vals[:, None], by_col=True, beta=beta, S=S)
        assert ec[0] == e
        assert np.array_equal(dc[:, :, 0].T, digs)


def test_exponent_matches_math_frexp():
    rng = np.random.default_rng(11)
    vals = list(rng.standard_normal(200) * np.exp2(rng.integers(-1070, 1020, 200)))
    vals += [1.0, 0.5, 2.0, -0.75, 5e-324, 2.2250738585072014e-308, 1.7976931348623157e308,
             2.0 ** -1060, 3.0 * 2.0 ** -1070]
    X = np.array(vals)[:, None]
    e, st = oracle.ozaki_exponents(X, by_col=False)
    assert st == oracle.OK
    for x, ei in zip(vals, e):
        assert ei == math.frexp(abs(x))[1]


def test_exponent_is_row_and_column_max():
    A = np.array([[0.1, -3.0, 0.2], [0.0, 0.0, 0.0], [1e-300, 2e-300, -4e-300]])
    e, _ = oracle.ozaki_exponents(A, by_col=False)
    assert list(e) == [math.frexp(3.0)[1], 0, math.frexp(4e-300)[1]]
    f, _ = oracle.ozaki_exponents(A, by_col=True)
    assert list(f) == [math.frexp(0.1)[1], math.frexp(3.0)[1], math.frexp(0.2)[1]]


def test_nonfinite_detected():
    A = np.array([[1.0, np.inf], [0.0, 1.0]])
    _, st = oracle.ozaki_exponents(A, by_col=False)
    assert st == oracle.NONFINITE
    with pytest.raises(FloatingPointError):
        oracle.ozaki_gemm(A, np.eye(2), S=3)
    B = np.array([[np.nan, 0.0], [0.0, 1.0]])
    with pytest.raises(FloatingPointError):
        oracle.ozaki_gemm(np.eye(2), B, S=3)


@pytest.mark.parametrize("beta,S", [(7, 1), (7, 4), (7, 8), (8, 3), (8, 7)])
def test_split_reconstructs_and_digit_range(beta, S):
    """x = 2^e (sum_s d_s 2^{-beta s} + residual), |residual| < 2^{-beta S},
    digits in [-(2^beta - 1), 2^beta - 1], never of opposite sign to x."""
    A = inputs.exp_spread(0, 9, (12, 40))
    e, d = oracle.ozaki_split(A, by_col=False, beta=beta, S=S)
    lim = 2 ** beta - 1
    assert np.abs(d).max() <= lim
    assert np.all(d.astype(np.float64) * np.sign(A)[None] >= 0)
    for i in range(A.shape[0]):
        for l in range(A.shape[1]):
            x = Fraction(float(A[i, l]))
            rec = sum(Fraction(int(d[s, i, l])) * Fraction(2) ** (int(e[i]) - beta * (s + 1))
                      for s in range(S))
            res = x - rec
            assert abs(res) < Fraction(2) ** (int(e[i]) - beta * S)
            assert res * x >= 0  # truncation: the residual keeps the sign of x


def test_split_exact_for_short_values():
    """Values with at most beta*S bits below the row exponent are split
    exactly (zero residual)."""
    beta, S = 7, 3
    rng = np.random.default_rng(3)
    ints = rng.integers(-(2 ** 21 - 1), 2 ** 21, size=(6, 10)).astype(np.float64)
    ints[:, 0] = 2 ** 20 + 1  # pins e = 21 in every row
    A = ints * 2.0 ** -9
    e, d = oracle.ozaki_split(A, by_col=False, beta=beta, S=S)
    rec = sum(d[s].astype(np.float64) * np.exp2(e[:, None] - beta * (s + 1)) for s in range(S))
    assert np.array_equal(rec, A)


# ---------------------------------------------------------------- Ozaki product
def test_ozaki_integer_inputs_exact_at_one_slice():
    """Integers in [-8, 8]: the row max is at most 8 = 0.5 * 2^4, so every
    entry is a multiple of 2^(e - 7) and one 7-bit digit holds it exactly; all
    products are kept and the sums are exact integers."""
    m, k, n = 37, 129, 41
    A, B = inputs.gemm_operands("int8", m, k, n, seed=0, cfg=3)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    for S in (1, 2, 5):
        assert np.array_equal(oracle.ozaki_gemm(A, B, S=S, beta=7), ref)
    assert np.array_equal(oracle.ozaki_gemm(A, B, S=1, beta=8), ref)


def test_ozaki_identity_and_permutation():
    """I.B and P.B: each entry of C is one product a*b with a = 1, whose
    digits are (64, 0, ...); with 7S >= 53 + 1 bits the digits of b hold it
    exactly, so the result is exactly B (or B permuted)."""
    n = 40
    _, B = inputs.gemm_operands("uniform", n, n, n, seed=0, cfg=0)
    P = inputs.permutation_matrix(0, 7, n)
    p = inputs.permutation(0, 7, n)
    # column exponents of B may sit above an entry by up to ~10 bits here;
    # 7*10 = 70 >= 53 + 11 bits covers every entry exactly.
    assert np.array_equal(oracle.ozaki_gemm(np.eye(n), B, S=10, beta=7), B)
    assert np.array_equal(oracle.ozaki_gemm(P, B, S=10, beta=7), B[p])


def test_ozaki_dyadic_inputs_exact():
    """Rows of A use only digits 1..2 and columns of B only digit 1: every
    product pair s + t <= 3 <= S + 1 is kept for S >= 2, so the emulated
    product is the exact product of short dyadic numbers (which fits FP64)."""
    m, k, n = 9, 50, 11
    rng = np.random.default_rng(8)
    A = rng.integers(-(2 ** 13 - 1), 2 ** 13, size=(m, k)).astype(np.float64) * 2.0 ** -14
    B = rng.integers(-127, 128, size=(k, n)).astype(np.float64) * 2.0 ** -7
    A[:, 0] = 0.75  # row exponent 0
    B[0, :] = 0.75  # column exponent 0
    ref = (A * 2 ** 14).astype(np.int64) @ (B * 2 ** 7).astype(np.int64)
    ref = ref.astype(np.float64) * 2.0 ** -21
    assert np.array_equal(oracle.ozaki_gemm(A, B, S=2, beta=7), ref)
    assert np.array_equal(oracle.ozaki_gemm(A, B, S=3, beta=7), ref)


def test_ozaki_dropped_pair_would_show():
    """With S = 1 only the (1,1) product is kept: for this A, B the (1,2) and
    (2,1) pairs carry the low bits, so S = 1 must differ from the exact value
    by exactly those pairs and S = 2 must not."""
    A = np.array([[0.5 + 2.0 ** -10]])  # digits (64, 16)
    B = np.array([[0.5 + 2.0 ** -12]])  # digits (64, 4)
    exact = float(A[0, 0] * B[0, 0])   # exact: short dyadics
    s1 = oracle.ozaki_gemm(A, B, S=1)[0, 0]
    assert s1 == 0.25
    s2 = oracle.ozaki_gemm(A, B, S=2)[0, 0]
    # cross pairs (1,2) + (2,1) carry weight 2^(-7*3)
    assert s2 == 0.25 + (64 * 4 + 16 * 64) * 2.0 ** -21
    s3 = oracle.ozaki_gemm(A, B, S=3)[0, 0]
    assert s3 == exact


@pytest.mark.parametrize("kind", ["uniform", "spread"])
def test_ozaki_error_decreases_with_slices_and_meets_apriori_bound(kind):
    """|C_S - exact| <= (S + 1) k 2^{e_i + f_j} 2^{-beta S} (truncation of both
    operands plus the dropped pairs s + t > S + 1) and the max error does not
    grow with S."""
    m, k, n = 24, 150, 20
    A, B = inputs.gemm_operands(kind, m, k, n, seed=0, cfg=5)
    e, _ = oracle.ozaki_exponents(A, by_col=False)
    f, _ = oracle.ozaki_exponents(B, by_col=True)
    d2 = oracle.gemm_dot2(A, B)
    ab = oracle.gemm_abs(A, B)
    prev = np.inf
    for S in range(1, 9):
        C = oracle.ozaki_gemm(A, B, S=S, beta=7)
        err = np.abs(C - d2)
        scale = np.exp2(e[:, None].astype(np.float64) + f[None, :] - 7 * S)
        # Dot2 itself is within u|c| + gamma_k^2 |A||B| of exact, and the fold
        # rounds at most S times: both far below the a-priori term
        bound = (S + 1) * k * scale + 4 * (S + 2) * U * ab
        assert np.all(err <= bound), S
        assert err.max() <= prev * 1.0000001 + 1e-300
        prev = err.max()


def test_ozaki_high_slice_count_matches_dot2_closely():
    """Uniform inputs, beta*S = 70 bits >> 53: every kept digit pair together
    carries the product to below FP64 resolution, so the emulated product is
    within a few ulps (scaled by |A||B|) of Dot2."""
    m, k, n = 31, 300, 29
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=6)
    d2 = oracle.gemm_dot2(A, B)
    ab = oracle.gemm_abs(A, B)
    for beta, S in ((7, 10), (8, 9)):
        C = oracle.ozaki_gemm(A, B, S=S, beta=beta)
        assert np.all(np.abs(C - d2) <= 8 * U * ab), (beta, S)


def test_ozaki_within_acceptance_bound_at_working_slices():
    """The library's acceptance bound |C - C_dot2| <= 2 k u (|A||B|) holds at
    the slice counts used at scale: 7 slices of 7 bits (6 of 8 bits) for
    uniform entries, 8 of 7 bits (7 of 8 bits) when entries spread over 2^41;
    one slice fewer breaks it on these inputs."""
    m, k, n = 48, 512, 40
    for kind, cases in (("uniform", ((7, 7), (8, 6))), ("spread", ((7, 8), (8, 7)))):
        A, B = inputs.gemm_operands(kind, m, k, n, seed=0, cfg=7)
        d2 = oracle.gemm_dot2(A, B)
        ab = oracle.gemm_abs(A, B)
        for beta, S in cases:
            C = oracle.ozaki_gemm(A, B, S=S, beta=beta)
            assert np.all(np.abs(C - d2) <= 2 * k * U * ab), (kind, beta, S)
            C = oracle.ozaki_gemm(A, B, S=S - 1, beta=beta)
            assert not np.all(np.abs(C - d2) <= 2 * k * U * ab), (kind, beta, S - 1)


def test_ozaki_entries_match_full():
    m, k, n = 17, 70, 13
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=8)
    ii = np.array([0, 16, 5, 5, 3])
    jj = np.array([12, 0, 5, 6, 3])
    for beta, S in ((7, 3), (7, 7), (8, 5)):
        full = oracle.ozaki_gemm(A, B, S=S, beta=beta)
        assert np.array_equal(oracle.ozaki_entries(A, B, ii, jj, S=S, beta=beta), full[ii, jj])


def test_ozaki_sign_symmetry():
    """Negating A negates every digit and hence C exactly."""
    A, B = inputs.gemm_operands("spread", 11, 33, 9, seed=0, cfg=9)
    C = oracle.ozaki_gemm(A, B, S=5)
    assert np.array_equal(oracle.ozaki_gemm(-A, B, S=5), -C)
    assert np.array_equal(oracle.ozaki_gemm(A, -B, S=5), -C)


def test_ozaki_power_of_two_scaling_invariance():
    """Scaling a row of A by 2^p moves e_i by p and nothing else: the row of C
    scales by exactly 2^p (no under/overflow here)."""
    A, B = inputs.gemm_operands("uniform", 6, 45, 7, seed=0, cfg=10)
    C = oracle.ozaki_gemm(A, B, S=6)
    A2 = A.copy()
    A2[2] *= 2.0 ** 37
    C2 = oracle.ozaki_gemm(A2, B, S=6)
    assert np.array_equal(C2[2], C[2] * 2.0 ** 37)
    assert np.array_equal(np.delete(C2, 2, 0), np.delete(C, 2, 0))


# ---------------------------------------------------------------- comparison modes
def test_f32_oracle_small_integers_exact():
    A, B = inputs.gemm_operands("int8", 13, 40, 11, seed=0, cfg=3)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(oracle.gemm_f32(A, B).astype(np.int64), ref)


def test_round_bf16_definition():
    import torch
    # float32-representable values: torch's float32 -> bfloat16 conversion is
    # round-to-nearest-even, and float64 -> float32 is exact for them.
    rng = np.random.default_rng(2)
    x32 = (rng.standard_normal(5000) * np.exp2(rng.integers(-130, 120, 5000))).astype(np.float32)
    x32 = np.concatenate([x32, np.array([1.0, 1.00390625, 1.01171875, -2.0 ** -133,
                                         3.3895313892515355e38], dtype=np.float32)])
    ours = oracle.round_bf16(x32.astype(np.float64))
    ref = torch.from_numpy(x32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1
    assert oracle.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 0x3F80
    assert oracle.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 0x3F82
    # a double just above the tie rounds up (a float32 path would tie)
    assert oracle.round_bf16(np.array([1.0 + 2.0 ** -8 + 2.0 ** -40]))[0] == 0x3F81
