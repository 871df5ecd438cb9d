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


def test_noalloc_split_k_and_fallback_plans_match_mxm_f64_emul():
    """Shapes where mxm_f64_emul splits k (few C tiles): 256 x 2048 x 256 fits
    the scratch with the same split-k plan (4 tiles x 4 k ranges); for
    1024^3 at 7 slices the split plan does not fit and the call runs the
    unsplit product.  Both give mxm_f64_emul's bits, and the oracle's."""
    import oracle
    for idx, ((m, k, n), S) in enumerate((((256, 2048, 256), 7), ((1024, 1024, 1024), 7))):
        A_h, B_h = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=50 + idx)
        A = torch.from_numpy(A_h).cuda()
        B = torch.from_numpy(B_h).cuda()
        C_ref = torch.empty((m, n), dtype=torch.float64, device="cuda")
        mxm.mxm_f64_emul(A, B, C_ref, S)
        torch.cuda.synchronize()
        C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        assert _call_noalloc(A, B, C, S) == mxm.MXM_OK
        assert mxm.mxm_get_device_status() == mxm.MXM_OK
        got = C.cpu().numpy()
        assert_bitwise(got, C_ref.cpu().numpy(), f"noalloc vs mxm_f64_emul {(m, k, n)}")
        rng = np.random.default_rng(m + k)
        ii = rng.integers(0, m, 200)
        jj = rng.integers(0, n, 200)
        assert_bitwise(got[ii, jj], oracle.ozaki_entries(A_h, B_h, ii, jj, S=S, beta=7),
                       f"noalloc vs oracle {(m, k, n)}")


def test_noalloc_empty_sum_writes_zeros():
    """k = 0 needs no scratch: zeros, even when m x n alone is far larger
    than anything the scratch could hold."""
    A = torch.zeros((4096, 0), dtype=torch.float64, device="cuda")
    B = torch.zeros((0, 4096), dtype=torch.float64, device="cuda")
    C = torch.full((4096, 4096), 7.0, dtype=torch.float64, device="cuda")
    assert _call_noalloc(A, B, C, 7) == mxm.MXM_OK
    assert torch.all(C == 0.0)


def test_noalloc_rejects_products_beyond_its_scratch():
    A = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda")
    B = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda")
    C = torch.full((2048, 2048), 7.0, dtype=torch.float64, device="cuda")
    assert _call_noalloc(A, B, C, 7) == mxm.MXM_ERR_WORKSPACE_TOO_SMALL
    assert torch.all(C == 7.0)  # nothing was launched
