"""Comparison modes (FP32 and BF16-in/FP32-accumulate): inputs rounded to the
narrow type the way the oracle rounds them, products summed in FP32.  Checked
against Dot2 of the rounded inputs within the FP32 analogue of the bound,
2 k 2^-24 (|A'||B'|).  They are reported beside the FP64 modes, not held to
the FP64 bound."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu


def run(mode, A, B):
    m, k = A.shape
    n = B.shape[1]
    C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
    mxm.mxm_gemm(mode, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, slices=1)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    return C.cpu().numpy()


def check_f32_bound(C, Ar, Br, k):
    ref = oracle.gemm_dot2(Ar, Br)
    ab = oracle.gemm_abs(Ar, Br)
    lim = 2.0 * k * 2.0 ** -24 * ab + 1e-300
    assert np.all(np.abs(C - ref) <= lim)


@pytest.mark.parametrize("shape", [(1, 1, 1), (129, 65, 131), (300, 500, 280)])
def test_f32_mode(shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=0)
    C = run(mxm.MODE_F32, A, B)
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    check_f32_bound(C, A32, B32, k)
    # the result is an FP32 value written as FP64
    assert np.array_equal(C.astype(np.float32).astype(np.float64), C)


@pytest.mark.parametrize("shape", [(1, 1, 1), (129, 65, 131), (300, 500, 280)])
def test_bf16_mode(shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=1)
    C = run(mxm.MODE_BF16_F32ACC, A, B)
    Ab = oracle.bf16_to_f64(oracle.round_bf16(A))
    Bb = oracle.bf16_to_f64(oracle.round_bf16(B))
    check_f32_bound(C, Ab, Bb, k)


def test_bf16_mode_rounding_matches_oracle_exactly():
    """With B = I the product is exactly the rounded A: the device's rounding
    of every input equals the oracle's (a decision taken in the same
    precision on both sides)."""
    n = 256
    A = inputs.exp_spread(0, 5, (n, n), -100, 100)  # bf16 normal range: no flush question
    C = run(mxm.MODE_BF16_F32ACC, A, np.eye(n))
    assert np.array_equal(C, oracle.bf16_to_f64(oracle.round_bf16(A)).astype(np.float32).astype(np.float64))
