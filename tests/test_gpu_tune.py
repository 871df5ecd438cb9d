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


def test_tuned_plan_few_tiles(tmp_path):
    """A product with few C tiles and long k: the plan search tries split-k
    counts and CTA forms; the tuned product stays bit-identical to the
    oracle's emulation when an emulated engine is chosen, and within the
    FP64 bound in any case; the cache keeps the plan."""
    m, k, n = 256, 4096, 256
    A_h, B_h = inputs.gemm_operands("spread", m, k, n, seed=7, cfg=0)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    cache = tune.TuneCache(str(tmp_path / "t.json"))
    choice = tune.tune(A, B, tag="spread", cache=cache)
    assert choice.plan_measured and choice.plan_measured[0][0] == {}
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    tune._run(choice.mode, choice.slices, A, B, C, torch.cuda.current_stream(), choice.plan)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    got = C.cpu().numpy()
    assert_within_bound(got, oracle.gemm_dot2(A_h, B_h), oracle.gemm_abs(A_h, B_h), k,
                        f"tuned {choice.name} S={choice.slices} plan={choice.plan}")
    if choice.mode == mxm.MODE_EMUL_I8:
        assert np.array_equal(got, oracle.ozaki_gemm(A_h, B_h, S=choice.slices, beta=7))
    key = tune.cache_key(torch.cuda.get_device_name(0), "spread", m, k, n, 1.0)
    assert tune.TuneCache(cache.path).get(key).plan == choice.plan


def test_tune_grouped_size_classes(tmp_path):
    """The grouped tuner times the size-class boundaries and caches the
    fastest; the call under it gives the oracle's bits."""
    dims = [(100, 40, 90), (300, 700, 200), (64, 1000, 500), (129, 129, 17), (20, 300, 40)]
    hs, ds = [], []
    for p, (m, k, n) in enumerate(dims):
        A_h, B_h = inputs.gemm_operands("spread", m, k, n, seed=8, cfg=p)
        hs.append((A_h, B_h))
        ds.append((torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda(),
                   torch.empty((m, n), dtype=torch.float64, device="cuda")))
    table_h = mxm.problem_table(ds)
    table_d = table_h.cuda()
    cache = tune.TuneCache(str(tmp_path / "g.json"))
    plan = tune.tune_grouped(table_h, table_d, mxm.MODE_EMUL_I8, 8, cache=cache)
    key = tune.grouped_key(torch.cuda.get_device_name(0), "default", len(dims),
                           mxm.MODE_EMUL_I8, 8)
    entry = tune.TuneCache(cache.path).entries[key]
    assert entry["short_kt"] == plan.short_kt and len(entry["measured"]) >= 5
    ws = torch.empty(mxm.mxm_grouped_workspace_size(table_h, mxm.MODE_EMUL_I8, 8, plan),
                     dtype=torch.uint8, device="cuda")
    mxm.mxm_grouped(table_d, mxm.MODE_EMUL_I8, 8, ws, plan=plan)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    for (A_h, B_h), (_, _, C) in zip(hs, ds):
        assert np.array_equal(C.cpu().numpy(), oracle.ozaki_gemm(A_h, B_h, S=8, beta=7))
    # a second call is a cache hit
    assert tune.tune_grouped(table_h, table_d, mxm.MODE_EMUL_I8, 8,
                             cache=cache).short_kt == plan.short_kt
