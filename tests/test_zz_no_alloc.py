"""The no-allocation entry point (mxm_f64_emul_noalloc), for callers that
cannot allocate device memory: it must give exactly what mxm_f64_emul gives,
call after call, through the C ABI, from its fixed scratch array.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test first; it also passes alone in a fresh
process."""
import ctypes

import numpy as np
import pytest

from paper_1211_1581_gb300 import inputs
from helpers import assert_bitwise, assert_within_bound

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu


def _call_noalloc(A, B, C, S):
    lib = mxm.load()
    m, k = A.shape
    n = B.shape[1]
    st = lib.mxm_f64_emul_noalloc(A.data_ptr(), B.data_ptr(), C.data_ptr(), m, k, n, S,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


def test_noalloc_matches_mxm_f64_emul_on_two_calls_in_a_row():
    import oracle
    # two different products back to back: the second must not see the
    # first one's leftovers in the shared scratch array
    # (slice counts that meet the bound at these small k; see the oracle pins)
    for idx, ((m, k, n), S, kind) in enumerate((((300, 200, 257), 10, "spread"),
                                                ((129, 500, 131), 8, "uniform"))):
        A_h, B_h = inputs.gemm_operands(kind, m, k, n, seed=0, cfg=40 + idx)
        A = torch.from_numpy(A_h).cuda()
        B = torch.from_numpy(B_h).cuda()
        C_ref = torch.empty((m, n), dtype=torch.float64, device="cuda")
        mxm.mxm_f64_emul(A, B, C_ref, S)
        torch.cuda.synchronize()
        C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        assert _call_noalloc(A, B, C, S) == mxm.MXM_OK
        assert mxm.mxm_get_device_status() == mxm.MXM_OK
        got = C.cpu().numpy()
        assert_bitwise(got, C_ref.cpu().numpy(), f"noalloc vs mxm_f64_emul, call {idx}")
        assert_within_bound(got, oracle.gemm_dot2(A_h, B_h), oracle.gemm_abs(A_h, B_h), k,
                            f"noalloc call {idx}")


def test_noalloc_rejects_products_beyond_its_scratch():
    A = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda")
    B = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda")
    C = torch.full((2048, 2048), 7.0, dtype=torch.float64, device="cuda")
    assert _call_noalloc(A, B, C, 7) == mxm.MXM_ERR_WORKSPACE_TOO_SMALL
    assert torch.all(C == 7.0)  # nothing was launched
