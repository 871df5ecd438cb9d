"""mod2f on the GPU (mxm_fft, Sec. 3.3) against the FFT oracle through the C
ABI.  The GPU factors the transform differently (one pass, or two passes
with a twiddle in between) and rounds in another order, so the two are
compared against the radix-2 error bound (Higham, Accuracy and Stability
of Numerical Algorithms, 2nd ed., Thm. 24.2) with one level more for the
twiddle between the passes: each is within
(log2 N + 1) eta / (1 - (log2 N + 1) eta) of the exact transform in the
2-norm, eta = mu + gamma_4 (sqrt 2 + mu), mu = 2u, so they are within twice
that of each other."""
import math

import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def bound(N):
    mu = 2 * U
    eta = mu + 4 * U / (1 - 4 * U) * (math.sqrt(2) + mu)
    t = (math.log2(max(N, 1)) + 1) * eta
    return 2 * t / (1 - t)


def cplx(seed, stream, n, spread=False):
    if spread:
        u = inputs.exp_spread(seed, stream, (2 * n,), -20, 20)
    else:
        u = inputs.uniform_pm1(seed, stream, (2 * n,))
    return u[0::2] + 1j * u[1::2]


def gpu_fft(f, T=None, in_place=False):
    n = len(f)
    plan = mxm.FFT(T or n)
    x = torch.from_numpy(np.ascontiguousarray(f, dtype=np.complex128)).cuda()
    if T is None or T == n:
        out = plan(x, out=x if in_place else None)
    else:
        out = torch.empty_like(x) if not in_place else x
        work = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        mxm._check(mxm.load().mxm_fft(x.data_ptr(), out.data_ptr(), work.data_ptr(),
                                      plan.table.data_ptr(), T, n, None), "mxm_fft")
    torch.cuda.synchronize()
    return out.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("p", list(range(0, 23)))
def test_every_order_against_oracle(p):
    """All orders 2^0 ... 2^22: the paper's 2^8 ... 2^20, the one-pass and
    two-pass forms and their boundary (2^10 / 2^11)."""
    N = 1 << p
    f = cplx(0, 150 + p, N)
    assert rel(gpu_fft(f), oracle.fft(f)) <= bound(N)


@pytest.mark.parametrize("p", [3, 10, 11, 16, 20])
def test_wide_exponent_range(p):
    N = 1 << p
    f = cplx(1, 180 + p, N, spread=True)
    assert rel(gpu_fft(f), oracle.fft(f)) <= bound(N)


def bin_bound(N, mu):
    """Per-bin (componentwise) error of a radix-2 FFT with twiddles accurate
    to mu: every entry of the product of the stages' absolute butterfly
    matrices is 1 (one path from each input to each output, twiddles of
    modulus 1), so the first-order error analysis behind Higham's Thm. 24.2
    gives, for every output bin, |F'(k) - F(k)| <= L eta / (1 - L eta) ||f||_1
    with L = log2 N + 1 levels (one more for the twiddle between the two
    passes) and eta = mu + gamma_4 (sqrt 2 + mu)."""
    eta = mu + 4 * U / (1 - 4 * U) * (math.sqrt(2) + mu)
    t = (math.log2(max(N, 1)) + 1) * eta
    return t / (1 - t)


def dft_bin_bound(N):
    """Per-component error of the oracle's term-by-term DFT (Eq. 1, n in
    order): the twiddle of angle 2 pi m / N has an absolute error of at most
    ~ (4 pi + 1) u <= 14 u per component (the rounded angle, then libm), each
    term a c - b s adds gamma_2 |f(n)|, and the recursive sum of N terms
    gamma_{N-1} sum |term|: in all (gamma_{N+1} + sqrt 2 * 14 u) ||f||_1."""
    g = (N + 1) * U / (1 - (N + 1) * U)
    return g + math.sqrt(2) * 14 * U


def assert_bins(got, want, tol, what):
    err = np.maximum(np.abs(got.real - want.real), np.abs(got.imag - want.imag))
    bad = ~(err <= tol)
    assert not bad.any(), (f"{what}: {int(bad.sum())} bins beyond {tol:.3e}; worst "
                           f"{err.max():.3e} at bin {int(np.argmax(err))}")


@pytest.mark.parametrize("p", list(range(0, 13)))
@pytest.mark.parametrize("spread", [False, True])
def test_every_bin_against_the_definition(p, spread):
    """Bin by bin against the DFT of Eq. 1 summed term by term (the plain
    definition, O(N^2)), N = 2^0 ... 2^12: every bin within the GPU's per-bin
    FFT bound plus the definition's own rounding, both times ||f||_1."""
    N = 1 << p
    f = cplx(3, 230 + p + (40 if spread else 0), N, spread=spread)
    got = gpu_fft(f)
    tol = (bin_bound(N, 2 * U) + dft_bin_bound(N)) * np.sum(np.abs(f))
    assert_bins(got, oracle.dft(f), tol, f"N={N} spread={spread}")


@pytest.mark.parametrize("p", [13, 14, 16, 18, 20, 22])
def test_every_bin_against_oracle_fft(p):
    """The larger orders bin by bin against the oracle's radix-2 recursion:
    each within its per-bin bound of the exact transform (the GPU's table
    from sincospi, mu ~ 2u; the oracle's from libm of a rounded angle,
    mu ~ 8u)."""
    N = 1 << p
    f = cplx(4, 260 + p, N)
    tol = (bin_bound(N, 2 * U) + bin_bound(N, 8 * U)) * np.sum(np.abs(f))
    assert_bins(gpu_fft(f), oracle.fft(f), tol, f"N={N}")


@pytest.mark.parametrize("p", [1, 6, 10, 11, 17, 22])
def test_exact_delta_and_constant(p):
    N = 1 << p
    delta = np.zeros(N, complex)
    delta[0] = 1.0
    assert np.array_equal(gpu_fft(delta), np.ones(N, complex))
    want = np.zeros(N, complex)
    want[0] = N
    assert np.array_equal(gpu_fft(np.ones(N, complex)), want)


@pytest.mark.parametrize("p", [9, 10, 11, 14, 20])
def test_in_place_and_shared_table(p):
    """out == in gives the same values; a table of a larger order gives
    bit-identical results (its entries for this order are the same
    doubles)."""
    N = 1 << p
    f = cplx(2, 200 + p, N)
    ref = gpu_fft(f)
    assert np.array_equal(gpu_fft(f, in_place=True), ref)
    assert np.array_equal(gpu_fft(f, T=1 << 22), ref)


def test_single_tone_and_determinism():
    N = 1 << 18
    m = 12345
    n = np.arange(N)
    f = np.exp(2j * np.pi * ((m * n) % N) / N)
    want = np.zeros(N, complex)
    want[m] = N
    got = gpu_fft(f)
    assert rel(got, want) <= bound(N) + 4 * U
    assert np.array_equal(gpu_fft(f), got)


def test_argument_errors():
    lib = mxm.load()
    x = torch.zeros(2 * 4096, dtype=torch.float64, device="cuda")
    w = torch.zeros(2 * 4096, dtype=torch.float64, device="cuda")
    t = torch.zeros(4096, dtype=torch.float64, device="cuda")
    assert lib.mxm_fft_twiddles(t.data_ptr(), 4096, None) == mxm.MXM_OK
    P = x.data_ptr()
    assert lib.mxm_fft(P, P, w.data_ptr(), t.data_ptr(), 4096, 3000, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft(P, P, w.data_ptr(), t.data_ptr(), 2048, 4096, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft(P, P, None, t.data_ptr(), 4096, 4096, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft(P, P, P + 16, t.data_ptr(), 4096, 4096, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft(P + 8, P + 8, w.data_ptr(), t.data_ptr(), 4096, 2048, None) == \
        mxm.MXM_ERR_ALIGNMENT
    assert lib.mxm_fft(P, P, w.data_ptr(), t.data_ptr(), 4096,
                       lib.mxm_fft_max_n() * 2, None) == mxm.MXM_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
