"""The round-to-nearest split with balanced 8-bit digits on the GPU
(MXM_MODE_EMUL_RN8): bit-identical to the CPU emulator of the same split
(oracle.ozaki_*_rn8) for every slice count, ragged shapes, split-k shapes,
long k (spilled digit sums) and the pipelined host path; within the FP64
bound of Dot2 at the benchmark size with 6 slices."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs
from helpers import assert_bitwise, assert_within_bound

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu
RN8 = mxm.MODE_EMUL_RN8


def run(A, B, S, expect=mxm.MXM_OK):
    m, k = A.shape
    n = B.shape[1]
    C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
    mxm.mxm_gemm(RN8, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, slices=S)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == expect
    return C.cpu().numpy()


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5, 6, 7])
def test_bit_identical_n256(S):
    A, B = inputs.gemm_operands("spread", 256, 256, 256, seed=0, cfg=90 + S)
    assert_bitwise(run(A, B, S), oracle.ozaki_gemm_rn8(A, B, S), f"S={S}")


@pytest.mark.parametrize("shape", [(1, 1, 1), (130, 257, 3), (300, 129, 517), (64, 1000, 200)])
def test_ragged_bit_identical(shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=97)
    assert_bitwise(run(A, B, 6), oracle.ozaki_gemm_rn8(A, B, 6), f"{shape}")


def test_integers_exact_and_ties():
    A = inputs.int_uniform(0, 98, (200, 300), -8, 8)
    B = inputs.int_uniform(0, 99, (300, 170), -8, 8)
    want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert np.array_equal(run(A, B, 1), want)
    # values whose rounding is an exact tie at S = 2 (V = x 2^15 = odd / 2)
    A = np.full((128, 128), 0.75)
    A[:, 1::2] = 2.0 ** -16 * np.arange(1, 129, 2)[None, :]
    B = np.eye(128)
    assert_bitwise(run(A, B, 2), oracle.ozaki_gemm_rn8(A, B, 2), "ties")


@pytest.mark.parametrize("shape", [(128, 4096, 128), (130, 2125, 200)])
def test_splitk_bit_identical(shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=100)
    assert_bitwise(run(A, B, 6), oracle.ozaki_gemm_rn8(A, B, 6), f"split-k {shape}")


def test_long_k_spills_sampled():
    m, k, n = 2048, 30000, 2048 + 64
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=101)
    C = run(A, B, 6)
    rng = np.random.default_rng(30000)
    ii = rng.integers(0, m, 120)
    jj = rng.integers(0, n, 120)
    ii[:2] = [0, m - 1]
    jj[:2] = [n - 1, 0]
    assert_bitwise(C[ii, jj], oracle.ozaki_entries_rn8(A, B, ii, jj, 6), "long k")


def test_n8192_six_slices_within_bound():
    n = 8192
    A, B = inputs.gemm_operands("spread", n, n, n, seed=0, cfg=2)
    C = run(A, B, 6)
    rng = np.random.default_rng(8192)
    ii = rng.integers(0, n, 200)
    jj = rng.integers(0, n, 200)
    assert_bitwise(C[ii, jj], oracle.ozaki_entries_rn8(A, B, ii, jj, 6), "n=8192")
    d2, ab = oracle.entries_dot2_abs(A, B, ii, jj)
    assert_within_bound(C[ii, jj], d2, ab, n, "n=8192 bound")


def test_host_path_and_limits():
    m, k, n = 4000, 300, 10000
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=102)
    Ch = np.empty((m, n))
    mxm.mxm_gemm_host(RN8, A, B, Ch, slices=6)
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    assert_bitwise(Ch, run(A, B, 6), "host path vs device")
    lib = mxm.load()
    assert lib.mxm_workspace_size(RN8, 64, 64, 64, 8) == 0  # S <= 7
    with pytest.raises(mxm.MxmError):
        run(np.ascontiguousarray(A[:64, :64]), np.ascontiguousarray(B[:64, :64]), 8)
