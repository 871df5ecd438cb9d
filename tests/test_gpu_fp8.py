"""The 4-bit-digit Ozaki engine on the FP8 tensor path (MXM_MODE_EMUL_FP8):
digits |d| <= 15 carried in E4M3 through tcgen05 kind::f8f6f4.  The digit
products are exact integers and the recombination order is the CPU
emulator's, so every result must be bit-identical to oracle.ozaki_gemm with
beta = 4."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs
from helpers import assert_bitwise, assert_within_bound

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu


def run_fp8(A, B, S, expect=mxm.MXM_OK):
    m, k = A.shape
    n = B.shape[1]
    C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
    mxm.mxm_gemm(mxm.MODE_EMUL_FP8, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C,
                 slices=S)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == expect
    return C.cpu().numpy()


@pytest.mark.parametrize("S", [1, 2, 5, 8, 12, 16])
def test_fp8_bit_identical_n256(S):
    A, B = inputs.gemm_operands("spread", 256, 256, 256, seed=0, cfg=20 + S)
    assert_bitwise(run_fp8(A, B, S), oracle.ozaki_gemm(A, B, S=S, beta=4), f"S={S}")


@pytest.mark.parametrize("shape", [(1, 1, 1), (17, 33, 15), (129, 65, 131), (300, 200, 257),
                                   (64, 1000, 40), (130, 2125, 200)])
def test_fp8_ragged_bit_identical(shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=30)
    assert_bitwise(run_fp8(A, B, 13), oracle.ozaki_gemm(A, B, S=13, beta=4), f"{shape}")


def test_fp8_full_digits_and_bound():
    """Digits at their maximum (|x| 2^-e = 1 - 2^-53: the first 13 4-bit
    digits are 15) over k = 4096, then a uniform product at 16 slices within
    the FP64 bound."""
    k = 4096
    x = 1.0 - 2.0 ** -53
    A = np.full((128, k), x)
    B = np.full((k, 128), -x)
    assert_bitwise(run_fp8(A, B, 16), oracle.ozaki_gemm(A, B, S=16, beta=4), "all-15 digits")
    A, B = inputs.gemm_operands("uniform", 384, 2048, 256, seed=0, cfg=31)
    C = run_fp8(A, B, 16)
    assert_within_bound(C, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B), 2048, "S=16")


def test_fp8_edges():
    A, B = inputs.gemm_operands("uniform", 40, 0, 30, seed=0, cfg=32)
    assert np.all(run_fp8(A, B, 8) == 0.0)  # k = 0: empty sums
    A, B = inputs.gemm_operands("uniform", 40, 50, 30, seed=0, cfg=33)
    A[3, 7] = np.inf
    run_fp8(A, B, 8, expect=mxm.MXM_ERR_NONFINITE)
    Z = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    for S in (0, 17):
        with pytest.raises(mxm.MxmError):
            mxm.mxm_gemm(mxm.MODE_EMUL_FP8, Z, Z, torch.empty_like(Z), slices=S)
    with pytest.raises(mxm.MxmError):  # no grouped form
        table = mxm.problem_table([(Z, Z, torch.empty_like(Z))])
        ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
        mxm.mxm_grouped(table.cuda(), mxm.MODE_EMUL_FP8, 8, ws)
