"""FP64-accurate Ozaki path (mxm_f64_emul / mxm_gemm emulated modes)
against the oracle, through the C ABI.

The digit products are exact integers on both sides and both recombine in
the same fixed order, so the GPU result must be BIT-IDENTICAL to the CPU
emulator (oracle.ozaki_gemm) for every slice count and both digit widths;
through it the result meets |C - C_dot2| <= 2 k u (|A||B|) at the working
slice counts."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs
from helpers import assert_bitwise, assert_within_bound

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu

BETA = {mxm.MODE_EMUL_I8: 7, mxm.MODE_EMUL_BF16: 8}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_emul(A, B, S, mode=mxm.MODE_EMUL_I8, expect=mxm.MXM_OK):
    m, k = A.shape
    n = B.shape[1]
    C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
    mxm.mxm_gemm(mode, dev(A), dev(B), C, slices=S)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == expect
    return C.cpu().numpy()


@pytest.mark.parametrize("mode", [mxm.MODE_EMUL_I8, mxm.MODE_EMUL_BF16])
@pytest.mark.parametrize("S", [1, 2, 3, 5, 7, 8])
def test_emul_bit_identical_n256(mode, S):
    n = 256
    A, B = inputs.gemm_operands("uniform", n, n, n, seed=0, cfg=0)
    C = run_emul(A, B, S, mode)
    assert_bitwise(C, oracle.ozaki_gemm(A, B, S=S, beta=BETA[mode]), f"S={S} mode={mode}")


SHAPES = [(1, 1, 1), (7, 13, 5), (17, 65, 15), (128, 64, 128), (129, 65, 131),
          (300, 200, 257), (64, 1000, 40), (257, 129, 300)]


@pytest.mark.parametrize("shape", SHAPES)
def test_emul_ragged_bit_identical(shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=1)
    for mode, S in ((mxm.MODE_EMUL_I8, 7), (mxm.MODE_EMUL_BF16, 6)):
        C = run_emul(A, B, S, mode)
        assert_bitwise(C, oracle.ozaki_gemm(A, B, S=S, beta=BETA[mode]), f"{shape} mode={mode}")


@pytest.mark.parametrize("kind,S", [("uniform", 7), ("spread", 8)])
def test_emul_within_bound(kind, S):
    m, k, n = 300, 700, 260
    A, B = inputs.gemm_operands(kind, m, k, n, seed=0, cfg=2)
    C = run_emul(A, B, S)
    assert_within_bound(C, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B), k, f"{kind} S={S}")


def test_emul_exact_cases_n256():
    n = 256
    Ai, Bi = inputs.gemm_operands("int8", n, n, n, seed=0, cfg=3)
    ref = (Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float64)
    for S in (1, 7):
        assert_bitwise(run_emul(Ai, Bi, S), ref, f"int [-8,8] S={S}")
    _, B = inputs.gemm_operands("uniform", n, n, n, seed=0, cfg=0)
    P = inputs.permutation_matrix(0, 7, n)
    # 7*10 bits cover the spread of each column of B: exact
    assert_bitwise(run_emul(np.eye(n), B, 10), B, "I.B")
    assert_bitwise(run_emul(P, B, 10), B[inputs.permutation(0, 7, n)], "P.B")


@pytest.mark.parametrize("beta,mode", [(7, mxm.MODE_EMUL_I8), (8, mxm.MODE_EMUL_BF16)])
def test_emul_fp32_accumulation_exact_at_full_window(beta, mode):
    """Every digit at its largest magnitude 2^beta - 1 (entries 1 - 2^-beta*S
    with random signs): each FP32 accumulation window holds the most
    products allowed; any rounding inside the tensor core would break bit
    identity with the int64 oracle."""
    S = 4
    m, k, n = 256, 4096, 256
    v = 1.0 - 2.0 ** (-beta * S)
    sa = np.where(inputs.int_uniform(0, 11, (m, k), 0, 1) > 0, 1.0, -1.0)
    sb = np.where(inputs.int_uniform(0, 12, (k, n), 0, 1) > 0, 1.0, -1.0)
    A = v * sa
    B = v * sb
    B[:, :8] = v  # some columns with every product positive: the largest sums
    A[:8, :] = v
    e, d = oracle.ozaki_split(A, by_col=False, beta=beta, S=S)
    assert np.abs(d).min() == 2 ** beta - 1
    C = run_emul(A, B, S, mode)
    assert_bitwise(C, oracle.ozaki_gemm(A, B, S=S, beta=beta), f"full window beta={beta}")


def test_emul_nonfinite_reported():
    A, B = inputs.gemm_operands("uniform", 64, 64, 64, seed=0, cfg=0)
    A[3, 5] = np.inf
    run_emul(A, B, 3, expect=mxm.MXM_ERR_NONFINITE)
    B[1, 1] = np.nan
    A[3, 5] = 0.0
    run_emul(A, B, 3, expect=mxm.MXM_ERR_NONFINITE)
    # status was read and cleared
    assert mxm.mxm_get_device_status() == mxm.MXM_OK


def test_emul_zero_k_and_zero_rows():
    C = run_emul(np.zeros((5, 0)), np.zeros((0, 7)), 5)
    assert np.array_equal(C, np.zeros((5, 7)))
    A = np.zeros((130, 70))
    A[5] = inputs.uniform_pm1(0, 3, (70,))
    B = inputs.uniform_pm1(0, 4, (70, 9))
    assert_bitwise(run_emul(A, B, 6), oracle.ozaki_gemm(A, B, S=6), "zero rows")


def test_emul_deterministic():
    A, B = inputs.gemm_operands("uniform", 333, 517, 291, seed=0, cfg=4)
    assert_bitwise(run_emul(A, B, 7), run_emul(A, B, 7), "run to run")


def test_emul_int64_running_sums_long_k():
    """k long enough that the per-diagonal integer sums need 64 bits:
    m = n = 128, k = 65536 (the long-k rectangular case)."""
    m, k, n = 128, 65536, 128
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=5)
    C = run_emul(A, B, 7)
    rng = np.random.default_rng(1)
    ii = rng.integers(0, m, 200)
    jj = rng.integers(0, n, 200)
    assert_bitwise(C[ii, jj], oracle.ozaki_entries(A, B, ii, jj, S=7, beta=7), "long k")
    d2, ab = oracle.entries_dot2_abs(A, B, ii, jj)
    assert_within_bound(C[ii, jj], d2, ab, k, "long k bound")


@pytest.mark.parametrize("kind,slices", [("uniform", (7,)), ("spread", (7, 8))])
def test_emul_n8192_sampled(kind, slices):
    """The benchmark configuration (m = k = n = 8192) in the call bench.py
    times; the spread inputs are the benchmark's own (seed 0, streams 4
    and 5) and S = 7 is its slice count: sampled entries bit-identical to the
    CPU emulator and within the bound of Dot2."""
    n = 8192
    A, B = inputs.gemm_operands(kind, n, n, n, seed=0, cfg=2)
    rng = np.random.default_rng(8192)
    ii = rng.integers(0, n, 300)
    jj = rng.integers(0, n, 300)
    ii[:8] = [0, n - 1, 0, n - 1, 127, 128, 255, 256]
    jj[:8] = [0, n - 1, n - 1, 0, 128, 127, 256, 255]
    d2, ab = oracle.entries_dot2_abs(A, B, ii, jj)
    for S in slices:
        C = run_emul(A, B, S)
        assert_bitwise(C[ii, jj], oracle.ozaki_entries(A, B, ii, jj, S=S, beta=7),
                       f"n=8192 {kind} S={S}")
        assert_within_bound(C[ii, jj], d2, ab, n, f"n=8192 {kind} S={S} bound")


# Split-k of the emulated product: the exact per-range D_g are added exactly
# before the fold, so the result stays bit-identical to the CPU emulator
# (1 tile x 8 ranges; 4 tiles x 4 ranges with a ragged last k-block).
@pytest.mark.parametrize("mode,S", [(mxm.MODE_EMUL_I8, 7), (mxm.MODE_EMUL_BF16, 6)])
@pytest.mark.parametrize("shape", [(128, 4096, 128), (130, 2125, 200)])
def test_emul_splitk_bit_identical(mode, S, shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=9)
    C = run_emul(A, B, S, mode)
    assert_bitwise(C, oracle.ozaki_gemm(A, B, S=S, beta=BETA[mode]), f"split-k {shape}")


def test_emul_splitk_64_tiles_sampled():
    """m = k = n = 1024 (64 C tiles, 2 k ranges each), sampled entries."""
    n = 1024
    A, B = inputs.gemm_operands("spread", n, n, n, seed=0, cfg=10)
    C = run_emul(A, B, 7)
    rng = np.random.default_rng(10)
    ii = rng.integers(0, n, 300)
    jj = rng.integers(0, n, 300)
    assert_bitwise(C[ii, jj], oracle.ozaki_entries(A, B, ii, jj, S=7, beta=7), "n=1024")


@pytest.mark.parametrize("S", [4, 7])
@pytest.mark.parametrize("shape", [(2048, 128, 2048), (1024, 64, 1536)])
def test_emul_one_kblock_many_tiles(shape, S):
    """k within one k-block and more C tiles than SMs: every diagonal's
    windows are one to seven steps long (one-step windows included), many
    per CTA; sampled entries bit-identical to the CPU emulator, two runs
    bit-identical to each other."""
    m, k, n = shape
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=11)
    C = run_emul(A, B, S)
    assert_bitwise(run_emul(A, B, S), C, "run to run")
    rng = np.random.default_rng(m + n + S)
    ii = rng.integers(0, m, 400)
    jj = rng.integers(0, n, 400)
    assert_bitwise(C[ii, jj], oracle.ozaki_entries(A, B, ii, jj, S=S, beta=7), f"{shape} S={S}")


# Long k in the paired kernel: a diagonal's int32 digit sum would pass 2^31
# over all of k, so every so many window drains the epilogue moves it into an
# int64 spill area and the fold adds it back.  The integer sums, and so the
# results, stay bit-identical to the CPU emulator.
@pytest.mark.parametrize("mode,S,beta,k", [(mxm.MODE_EMUL_BF16, 6, 8, 8192),
                                           (mxm.MODE_EMUL_BF16, 8, 8, 12000),
                                           (mxm.MODE_EMUL_I8, 7, 7, 20000)])
def test_emul_long_k_spills_bit_identical(mode, S, beta, k):
    m, n = 2048, 2048 + 64  # enough C tiles for no split-k; a ragged column tile
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=40 + S)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    mxm.mxm_gemm(mode, dA, dB, C, slices=S)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    C = C.cpu().numpy()
    rng = np.random.default_rng(k)
    ii = rng.integers(0, m, 160)
    jj = rng.integers(0, n, 160)
    ii[:4] = [0, m - 1, 0, m - 1]
    jj[:4] = [0, n - 1, n - 1, 0]
    assert_bitwise(C[ii, jj], oracle.ozaki_entries(A, B, ii, jj, S=S, beta=beta), "long k spills")


# Products with two or more tile-rows of A run on CTA pairs (256-row C
# tiles); with an odd number of tile-rows the second CTA of the last pair
# has no rows and only feeds its half of B.  More 256-row tiles than pairs
# on the GPU: several tiles per pair.
@pytest.mark.parametrize("shape,S", [((9 * 128 + 5, 640, 700), 7), ((33 * 128, 256, 2048), 5),
                                     ((2 * 128, 1000, 129), 7), ((3 * 128 - 1, 130, 4 * 128), 8)])
def test_emul_cta_pairs_odd_tile_rows(shape, S):
    m, k, n = shape
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=60 + S)
    C = run_emul(A, B, S)
    assert_bitwise(run_emul(A, B, S), C, "run to run")
    rng = np.random.default_rng(m + k + n)
    ii = rng.integers(0, m, 300)
    jj = rng.integers(0, n, 300)
    # the last rows (the odd tile-row), the first rows of each CTA's half of
    # a pair tile, the last columns
    ii[:6] = [m - 1, m - 1, 128, 255, 256 % m, (m - 1) // 128 * 128]
    jj[:6] = [n - 1, 0, 63, 64, n - 1, 127 % n]
    assert_bitwise(C[ii, jj], oracle.ozaki_entries(A, B, ii, jj, S=S, beta=7), f"{shape} S={S}")
