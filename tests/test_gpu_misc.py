"""Device status word, the bounded-wait failure path, the host-buffer entry
point and the peak probes."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs
from helpers import assert_bitwise

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    """A wait on a barrier nothing completes gives up after its limit; the
    kernel exits, the status word says MXM_ERR_TIMEOUT, and the next call
    works."""
    mxm.mxm_debug_wait_timeout(50_000_000)  # 50 ms
    assert mxm.mxm_get_device_status() == mxm.MXM_ERR_TIMEOUT
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    A, B = inputs.gemm_operands("int8", 64, 64, 64, seed=0, cfg=3)
    C = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    mxm.mxm_f64(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert_bitwise(C.cpu().numpy(), ref, "after timeout")


@pytest.mark.parametrize("mode,S", [(mxm.MODE_F64, 0), (mxm.MODE_EMUL_I8, 7)])
def test_host_entry_point_matches_device(mode, S):
    m, k, n = 190, 333, 270
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=6)
    Ch = np.empty((m, n))
    mxm.mxm_gemm_host(mode, A, B, Ch, slices=S)
    Cd = torch.empty((m, n), dtype=torch.float64, device="cuda")
    mxm.mxm_gemm(mode, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, slices=S)
    assert_bitwise(Ch, Cd.cpu().numpy(), "host vs device")
    if mode != mxm.MODE_F64:
        assert_bitwise(Ch, oracle.ozaki_gemm(A, B, S=S), "host vs oracle")


def test_caller_workspace():
    m, k, n = 200, 300, 100
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=7)
    need = mxm.mxm_workspace_size(mxm.MODE_EMUL_I8, m, k, n, 7)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    try:
        mxm.mxm_set_workspace(ws)
        C = torch.empty((m, n), dtype=torch.float64, device="cuda")
        mxm.mxm_f64_emul(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, 7)
        assert_bitwise(C.cpu().numpy(), oracle.ozaki_gemm(A, B, S=7), "caller workspace")
        # too small for a bigger problem: rejected, nothing launched
        with pytest.raises(mxm.MxmError) as ei:
            A2 = torch.zeros((2000, 300), dtype=torch.float64, device="cuda")
            C2 = torch.empty((2000, 100), dtype=torch.float64, device="cuda")
            mxm.mxm_f64_emul(A2, torch.from_numpy(B).cuda(), C2, 7)
        assert ei.value.status == mxm.MXM_ERR_WORKSPACE_TOO_SMALL
    finally:
        torch.cuda.synchronize()
        mxm.mxm_set_workspace(None)


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_peak_probes_run(kind):
    v = mxm.mxm_peak_probe(kind)
    assert v > 0.0


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("mode,S,m,n", [(mxm.MODE_EMUL_I8, 7, 3000, 6500),
                                        (mxm.MODE_EMUL_BF16, 6, 3000, 6500),
                                        (mxm.MODE_EMUL_I8, 7, 4000, 10000)])
def test_host_entry_point_panels(mode, S, m, n, pinned):
    """Products large enough for the pipelined host path (A and C moved in
    blocks while earlier blocks compute): 8 panels of 384 rows, the last
    one 312 rows, all columns at once; and 8 panels of 512 rows times two
    column panels of B (5120 and 4880 columns) on a 152-SM GPU.
    Bit-identical to the device call and, on sampled entries, to the CPU
    emulator."""
    k = 300
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=12)
    if pinned:
        Ah = torch.from_numpy(A).pin_memory()
        Bh = torch.from_numpy(B).pin_memory()
        Ch = torch.empty((m, n), dtype=torch.float64).pin_memory()
        mxm.mxm_gemm_host(mode, Ah, Bh, Ch, slices=S)
        Ch = Ch.numpy()
    else:
        Ch = np.empty((m, n))
        mxm.mxm_gemm_host(mode, A, B, Ch, slices=S)
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    Cd = torch.empty((m, n), dtype=torch.float64, device="cuda")
    mxm.mxm_gemm(mode, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, slices=S)
    assert_bitwise(Ch, Cd.cpu().numpy(), "panels vs device")
    rng = np.random.default_rng(13)
    ii = rng.integers(0, m, 300)
    jj = rng.integers(0, n, 300)
    ii[:3] = [0, m - 1, (m - 1) // 8 * 8]  # first row, last row, a row of the last panel
    jj[:3] = [n - 1, 0, n // 2]
    beta = 7 if mode == mxm.MODE_EMUL_I8 else 8
    assert_bitwise(Ch[ii, jj], oracle.ozaki_entries(A, B, ii, jj, S=S, beta=beta), "panels vs oracle")
