"""The engine / slice-count tuner on the GPU: its choice, checked against
the oracle (not against the library it measured), and the cache path."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs
from helpers import assert_within_bound

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm, tune  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["spread", "uniform"])
def test_tuned_choice_is_fp64_accurate(kind, tmp_path):
    m, k, n = 384, 520, 300
    A_h, B_h = inputs.gemm_operands(kind, m, k, n, seed=5, cfg=0)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    cache = tune.TuneCache(str(tmp_path / "t.json"))
    choice = tune.tune(A, B, tag=kind, cache=cache)
    assert choice.err_ratio <= 1.0
    # every emulated scan ended at its first accurate count
    for mode in (mxm.MODE_EMUL_I8, mxm.MODE_EMUL_BF16, mxm.MODE_EMUL_FP8):
        rows = [r for r in choice.measured if r[0] == mode]
        assert rows and rows[-1][2] <= 1.0 and all(r[2] > 1.0 for r in rows[:-1])
        assert [r[1] for r in rows] == list(range(1, len(rows) + 1))
    # the choice, run again, meets the FP64 bound against the oracle's
    # compensated product
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    tune._run(choice.mode, choice.slices, A, B, C, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    ref = oracle.gemm_dot2(A_h, B_h)
    ab = oracle.gemm_abs(A_h, B_h)
    assert_within_bound(C.cpu().numpy(), ref, ab, k, f"tuned {choice.name} S={choice.slices}")
    # the cache holds it under this device, tag and size class
    key = tune.cache_key(torch.cuda.get_device_name(0), kind, m, k, n, 1.0)
    assert tune.TuneCache(cache.path).get(key) == choice


def test_gemm_uses_the_cache(tmp_path, monkeypatch):
    m, k, n = 256, 256, 256
    A_h, B_h = inputs.gemm_operands("spread", m, k, n, seed=6, cfg=0)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    cache = tune.TuneCache(str(tmp_path / "t.json"))
    C1 = torch.empty((m, n), dtype=torch.float64, device="cuda")
    first = tune.gemm(A, B, C1, tag="spread", cache=cache)  # miss: tunes
    torch.cuda.synchronize()

    def no_tuning(*a, **kw):
        raise AssertionError("tuned again on a cache hit")
    monkeypatch.setattr(tune, "tune", no_tuning)
    C2 = torch.empty_like(C1)
    second = tune.gemm(A, B, C2, tag="spread", cache=cache)
    torch.cuda.synchronize()
    assert second == first
    assert torch.equal(C1, C2)
