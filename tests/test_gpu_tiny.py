"""Operands whose rows or columns hold only tiny values, through the C ABI.

The row and column maxima are taken on the high words of |x| (exponent
field and top mantissa bits), with a second pass over the low words where
every high word of a row or column is zero (all |x| < 2^-1042).  These
operands reach both paths: rows and columns of subnormals with a zero high
word, subnormals with a nonzero high word, zero rows and columns, and a row
with one tiny value among zeros, next to ordinary ones.  Single products
(7-bit, truncated 8-bit, balanced 8-bit and 4-bit digits) and grouped calls
must be bit-identical to the oracle's emulation of the same split."""
import numpy as np
import pytest

import oracle
from helpers import assert_bitwise

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu


def tiny_operands(m, k, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, (m, k))
    B = rng.uniform(-1.0, 1.0, (k, n))
    # subnormals below 2^-1042: integer significands under 2^31, high word zero
    A[0] = rng.integers(-2**31, 2**31, k).astype(np.float64) * 2.0**-1074
    B[:, 0] = rng.integers(-2**31, 2**31, k).astype(np.float64) * 2.0**-1074
    # subnormals with a nonzero high word
    A[1] = rng.uniform(-1.0, 1.0, k) * 2.0**-1030
    B[:, 1] = rng.uniform(-1.0, 1.0, k) * 2.0**-1030
    # zeros, and one tiny value among zeros
    A[2] = 0.0
    B[:, 2] = 0.0
    A[3] = 0.0
    A[3, k // 2] = 3.0 * 2.0**-1074
    B[:, 3] = 0.0
    B[k // 3, 3] = -5.0 * 2.0**-1074
    return A, B


def reference(A, B, mode, S):
    if mode == mxm.MODE_EMUL_RN8:
        return oracle.ozaki_gemm_rn8(A, B, S)
    beta = {mxm.MODE_EMUL_I8: 7, mxm.MODE_EMUL_BF16: 8, mxm.MODE_EMUL_FP8: 4}[mode]
    return oracle.ozaki_gemm(A, B, S=S, beta=beta)


def test_tiny_operands_reach_the_low_word_pass():
    # the premise of the test: high words of rows 0 and 3 are zero
    A, _ = tiny_operands(40, 50, 30, 0)
    hi = (A.view(np.uint64) >> np.uint64(32)) & np.uint64(0x7FFFFFFF)
    assert not hi[0].any() and not hi[3].any() and hi[1].all()
    assert np.count_nonzero(A[0]) > 0 and np.count_nonzero(A[3]) == 1


MODES = [(mxm.MODE_EMUL_I8, 7), (mxm.MODE_EMUL_BF16, 6), (mxm.MODE_EMUL_RN8, 6),
         (mxm.MODE_EMUL_FP8, 14)]


@pytest.mark.parametrize("mode,S", MODES)
@pytest.mark.parametrize("shape", [(40, 50, 30), (150, 300, 140)])
def test_tiny_rows_and_columns_bit_identical(mode, S, shape):
    m, k, n = shape
    A, B = tiny_operands(m, k, n, seed=m + n)
    C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
    mxm.mxm_gemm(mode, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, slices=S)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    assert_bitwise(C.cpu().numpy(), reference(A, B, mode, S), f"{shape} mode={mode} S={S}")


@pytest.mark.parametrize("mode,S", [(mxm.MODE_EMUL_I8, 7), (mxm.MODE_EMUL_RN8, 6)])
def test_tiny_grouped_bit_identical(mode, S):
    dims = [(40, 50, 30), (7, 20, 9), (150, 300, 140), (5, 129, 6)]
    hs, ds = [], []
    for p, (m, k, n) in enumerate(dims):
        A, B = tiny_operands(m, k, n, seed=10 + p)
        hs.append((A, B))
        ds.append((torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                   torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")))
    table_h = mxm.problem_table(ds)
    ws = torch.empty(max(1, mxm.mxm_grouped_workspace_size(table_h, mode, S)),
                     dtype=torch.uint8, device="cuda")
    mxm.mxm_grouped(table_h.cuda(), mode, S, ws)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    for p, ((A, B), (_, _, C)) in enumerate(zip(hs, ds)):
        assert_bitwise(C.cpu().numpy(), reference(A, B, mode, S), f"problem {p} mode={mode}")
