"""Pins of the mod2f oracle (Sec. 3.3): the term-by-term DFT of Eq. 1 and
the radix-2 decimation-in-frequency recursion of Eqs. 2-3, against values
worked by hand from Eq. 1 (tests/golden/mod2f_worked.txt), numpy's FFT
(a library routine), closed forms that are exact in floating point,
Parseval, the shift theorem and Hermitian symmetry.  The error bound of
a radix-2 FFT (Higham, Accuracy and Stability of Numerical Algorithms,
2nd ed., Thm. 24.2): ||F^ - F|| / ||F|| <= log2(N) eta / (1 - log2(N) eta),
eta = mu + gamma_4 (sqrt(2) + mu), mu the twiddle error (here <= 2u)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mod2f_worked.txt")


def fft_bound(N):
    mu = 2 * U
    g4 = 4 * U / (1 - 4 * U)
    eta = mu + g4 * (math.sqrt(2) + mu)
    t = max(math.log2(N), 1) * eta
    return t / (1 - t)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def cplx(seed, stream, n):
    u = inputs.uniform_pm1(seed, stream, (2 * n,))
    return u[0::2] + 1j * u[1::2]


def _value(tok):
    r = math.sqrt(2.0)
    return float(eval(tok, {"__builtins__": {}}, {"r": r}))


def golden_cases():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, f, F = (part.strip() for part in line.split("|"))
        pair = lambda t: complex(*(_value(x) for x in t.split(",")))  # noqa: E731
        cases.append((int(n), np.array([pair(t) for t in f.split()]),
                      np.array([pair(t) for t in F.split()])))
    return cases


@pytest.mark.parametrize("case", range(4))
def test_worked_examples(case):
    N, f, F = golden_cases()[case]
    assert len(f) == N and len(F) == N
    for fn in (oracle.dft, oracle.fft):
        got = fn(f)
        assert np.max(np.abs(got - F)) <= 8 * N * U * max(np.abs(F).max(), 1.0)


@pytest.mark.parametrize("p", list(range(0, 17)) + [20])
def test_fft_against_numpy(p):
    N = 1 << p
    f = cplx(0, 110 + p, N)
    ref = np.fft.fft(f)
    assert rel(oracle.fft(f), ref) <= 2 * fft_bound(N) + 1e-300


@pytest.mark.parametrize("p", [0, 1, 2, 3, 5, 8, 10])
def test_fft_against_definition(p):
    N = 1 << p
    f = cplx(1, 130 + p, N)
    # the term-by-term sum carries up to ~N u of rounding per entry
    assert rel(oracle.fft(f), oracle.dft(f)) <= 2 * fft_bound(N) + 2 * N * U


def test_exact_closed_forms():
    for p in (1, 4, 9, 12):
        N = 1 << p
        delta = np.zeros(N, complex)
        delta[0] = 1.0
        assert np.array_equal(oracle.fft(delta), np.ones(N, complex))  # every twiddle times 0 or W^0
        ones = np.ones(N, complex)
        want = np.zeros(N, complex)
        want[0] = N
        assert np.array_equal(oracle.fft(ones), want)  # f_o = 0 at every level


@pytest.mark.parametrize("m", [0, 1, 7, 300, 1023])
def test_single_tone(m):
    N = 1024
    n = np.arange(N)
    f = np.exp(2j * np.pi * ((m * n) % N) / N)
    want = np.zeros(N, complex)
    want[m] = N
    assert rel(oracle.fft(f), want) <= 2 * fft_bound(N) + 4 * U


def test_parseval_shift_and_symmetry():
    N = 4096
    f = cplx(2, 140, N)
    F = oracle.fft(f)
    assert abs(np.vdot(F, F).real / N - np.vdot(f, f).real) <= 4 * fft_bound(N) * np.vdot(f, f).real
    # shift theorem: f(n - 1) -> W^k F(k)
    k = np.arange(N)
    Fs = oracle.fft(np.roll(f, 1))
    assert rel(Fs, np.exp(-2j * np.pi * k / N) * F) <= 4 * fft_bound(N)
    # real input: F(N - k) = conj F(k)
    R = oracle.fft(f.real.astype(complex))
    assert rel(R[1:][::-1], np.conj(R[1:])) <= 4 * fft_bound(N)


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12, complex))
