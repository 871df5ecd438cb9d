"""Host logic of the engine / slice-count tuner (no GPU): the scan, the
choice and the JSON cache."""
import json

import pytest

from paper_1211_1581_gb300 import mxm, tune


def fake_measure(need, cost, calls):
    """err_ratio falls by 2^7 per slice and reaches tol at `need[mode]`
    slices; time = cost[mode] * pairs (native FP64: a fixed cost)."""
    def measure(mode, s):
        calls.append((mode, s))
        if mode == mxm.MODE_F64:
            return 0.5, cost[mode]
        err = 2.0 ** (7 * (need[mode] - s))
        return err, cost[mode] * s * (s + 1) / 2
    return measure


def test_select_fastest_accurate():
    calls = []
    m = fake_measure({mxm.MODE_EMUL_I8: 7, mxm.MODE_EMUL_BF16: 6, mxm.MODE_EMUL_FP8: 13,
                      mxm.MODE_EMUL_RN8: 6},
                     {mxm.MODE_F64: 100.0, mxm.MODE_EMUL_I8: 1.0, mxm.MODE_EMUL_BF16: 1.5,
                      mxm.MODE_EMUL_FP8: 0.6, mxm.MODE_EMUL_RN8: 1.4}, calls)
    c = tune.select(m, tol=1.0)
    # i8: 28 pairs x 1.0 = 28; bf16: 21 x 1.5 = 31.5; fp8: 91 x 0.6 = 54.6; rn8: 21 x 1.4 =
    # 29.4; f64 100
    assert (c.mode, c.slices, c.ms) == (mxm.MODE_EMUL_I8, 7, 28.0)
    # each emulated scan stopped at its first accurate count
    assert [s for (mo, s) in calls if mo == mxm.MODE_EMUL_I8] == list(range(1, 8))
    assert [s for (mo, s) in calls if mo == mxm.MODE_EMUL_BF16] == list(range(1, 7))
    assert len(c.measured) == len(calls)


def test_select_native_wins_when_faster():
    calls = []
    m = fake_measure({mxm.MODE_EMUL_I8: 9, mxm.MODE_EMUL_BF16: 8, mxm.MODE_EMUL_FP8: 16,
                      mxm.MODE_EMUL_RN8: 7},
                     {mxm.MODE_F64: 20.0, mxm.MODE_EMUL_I8: 1.0, mxm.MODE_EMUL_BF16: 1.0,
                      mxm.MODE_EMUL_FP8: 1.0, mxm.MODE_EMUL_RN8: 1.0}, calls)
    c = tune.select(m, tol=1.0)
    assert (c.mode, c.slices) == (mxm.MODE_F64, 0) and c.name == "f64"


def test_select_tolerance_moves_the_count():
    m = fake_measure({mxm.MODE_EMUL_I8: 7, mxm.MODE_EMUL_BF16: 6, mxm.MODE_EMUL_FP8: 14,
                      mxm.MODE_EMUL_RN8: 6},
                     {mxm.MODE_F64: 1e9, mxm.MODE_EMUL_I8: 1.0, mxm.MODE_EMUL_BF16: 9.0,
                      mxm.MODE_EMUL_FP8: 9.0, mxm.MODE_EMUL_RN8: 9.0}, [])
    assert tune.select(m, tol=1.0).slices == 7
    assert tune.select(m, tol=2.0 ** 7).slices == 6  # one slice fewer is 2^7 worse


def test_select_raises_when_nothing_is_accurate():
    def never(mode, s):
        return float("inf"), 1.0
    with pytest.raises(RuntimeError):
        tune.select(never, tol=1.0, max_slices=3)


def test_select_scans_each_engine_to_its_own_limit():
    calls = []

    def never(mode, s):
        calls.append((mode, s))
        return float("inf"), 1.0
    with pytest.raises(RuntimeError):
        tune.select(never, tol=1.0)
    assert max(s for mo, s in calls if mo == mxm.MODE_EMUL_I8) == 12
    assert max(s for mo, s in calls if mo == mxm.MODE_EMUL_FP8) == 16
    assert max(s for mo, s in calls if mo == mxm.MODE_EMUL_RN8) == 7


def test_shape_class_and_key():
    assert tune.shape_class(8192, 8192, 8192) == "m13k13n13"
    assert tune.shape_class(8193, 1, 1000) == "m14k0n10"
    assert tune.shape_class(0, 2, 3) == "m0k1n2"
    assert tune.cache_key("GB300", "spread", 100, 200, 300, 1.0) == "GB300|spread|m7k8n9|tol=1"


def test_cache_round_trip(tmp_path):
    path = tmp_path / "sub" / "tune.json"
    c = tune.TuneCache(str(path))
    assert c.get("x") is None
    choice = tune.Choice(mode=mxm.MODE_EMUL_I8, slices=7, ms=21.5, err_ratio=0.01,
                         measured=[[1, 7, 0.01, 21.5]])
    c.put("x", choice)
    again = tune.TuneCache(str(path))
    assert again.get("x") == choice
    assert json.loads(path.read_text())["x"]["slices"] == 7
    assert [p.name for p in path.parent.iterdir()] == ["tune.json"]  # no temporary left


def test_grouped_slices_takes_the_worst_problem():
    # problem "p" needs need[p] slices; the grouped count is the maximum
    need = {"short": 8, "long": 6, "mid": 7}

    def measure_for(A, B):
        def measure(mode, s):
            return 2.0 ** (7 * (need[A] - s)), float(s)
        return measure
    probs = [("long", None), ("short", None), ("mid", None)]
    assert tune.grouped_slices(probs, measure_for=measure_for) == 8
    assert tune.grouped_slices(probs[:1], measure_for=measure_for) == 6


def test_select_plan_coordinate_search():
    """From the rule (all fields 0), each alternative of one field is tried
    on top of the best plan so far; a change is kept only when accurate and
    more than 1 % faster."""
    cost = {("raster", 2): 0.90, ("raster", 8): 1.05, ("kb_order", 1): 0.95,
            ("cta", 1): 1.20, ("splitk", 1): 0.97}
    tried = []

    def measure(plan):
        tried.append(dict(plan))
        t = 100.0
        for f, v in plan.items():
            t *= cost.get((f, v), 1.0)
        err = 5.0 if plan.get("splitk") == 1 else 0.5  # an inaccurate alternative
        return err, t

    cands = {"raster": [0, 2, 8], "kb_order": [0, 1], "cta": [0, 1], "splitk": [0, 1]}
    plan, err, ms, rows = tune.select_plan(measure, cands, tol=1.0)
    assert plan == {"raster": 2, "kb_order": 1}
    assert abs(ms - 100.0 * 0.90 * 0.95) < 1e-9 and err == 0.5
    assert tried[0] == {} and len(rows) == len(tried) == 1 + 2 + 1 + 1 + 1
    # raster 8 was tried on top of nothing better than raster 2: it came
    # after raster 2 was kept, with raster replaced
    assert {"raster": 8} in tried


def test_plan_candidates_follow_the_shape():
    big = tune.plan_candidates(mxm.MODE_EMUL_I8, 8192, 8192, 8192)
    assert "splitk" not in big and big["cta"] == [0, 1] and big["raster"][0] == 0
    few = tune.plan_candidates(mxm.MODE_EMUL_I8, 128, 65536, 128)
    assert "cta" not in few and few["splitk"][0] == 0 and 1 in few["splitk"]
    native = tune.plan_candidates(mxm.MODE_F64, 128, 65536, 128)
    assert native["splitk"][0] == 0 and "cta" not in native
    assert "splitk" not in tune.plan_candidates(mxm.MODE_EMUL_FP8, 128, 65536, 128)


def test_cache_keeps_the_plan(tmp_path):
    path = str(tmp_path / "c.json")
    c = tune.TuneCache(path)
    ch = tune.Choice(mode=mxm.MODE_EMUL_I8, slices=7, ms=1.5, err_ratio=0.1,
                     plan={"raster": 2, "splitk": 1}, plan_measured=[[{}, 0.1, 1.6]])
    c.put("k", ch)
    back = tune.TuneCache(path).get("k")
    assert back == ch and back.plan == {"raster": 2, "splitk": 1}
    p = tune.make_plan(back.plan)
    assert (p.raster, p.kb_order, p.cta, p.splitk) == (2, 0, 0, 1)
    assert tune.make_plan({}) is None
    # entries written before plans existed still load
    c.entries["old"] = {"mode": 1, "slices": 7, "ms": 1.0, "err_ratio": 0.2, "measured": []}
    assert tune.TuneCache.get(c, "old").plan == {}
