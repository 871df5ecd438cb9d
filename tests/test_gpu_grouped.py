"""Grouped products (mxm_grouped): a device-resident table of uneven problems
computed by one persistent launch sequence, also under CUDA-graph capture.
Every product is checked against the oracle: the emulated modes
bit-identical to the CPU emulator, native FP64 within 2 k u (|A||B|)."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs
from helpers import assert_bitwise, assert_within_bound

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu


def make_group(dims, seed=0, kind="uniform"):
    hs, ds = [], []
    for p, (m, k, n) in enumerate(dims):
        A, B = inputs.gemm_operands(kind, m, k, n, seed=seed, cfg=100 + p)
        hs.append((A, B))
        ds.append((torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                   torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")))
    return hs, ds


def run_group(ds, mode, S, graph=False, plan=None):
    table_h = mxm.problem_table(ds)
    ws_bytes = mxm.mxm_grouped_workspace_size(table_h, mode, S, plan)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device="cuda")
    table_d = table_h.cuda()
    if not graph:
        mxm.mxm_grouped(table_d, mode, S, ws, plan=plan)
    else:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            mxm.mxm_grouped(table_d, mode, S, ws, stream=s, plan=plan)
        for _, _, C in ds:
            C.fill_(float("nan"))
        g.replay()
        g.replay()
    torch.cuda.synchronize()
    return mxm.mxm_get_device_status()


DIMS = [(1, 1, 1), (17, 5, 33), (128, 64, 128), (129, 65, 131), (300, 200, 257), (16, 1024, 16),
        (0, 5, 7), (5, 0, 7), (7, 9, 0), (1000, 33, 20), (64, 300, 500), (256, 256, 256)]


# The emulated problems run on two slice GEMMs split by k (mxm_group_plan):
# the default sends every problem here to the one-diagonal kernel; short_kt
# = 0 sends all of them to the diagonal-pair kernel, 1 splits them.
PLANS = {"default": None, "pair": mxm.GroupPlan(0), "split": mxm.GroupPlan(1)}


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("plan", ["default", "pair", "split"])
@pytest.mark.parametrize("mode,S", [(mxm.MODE_EMUL_I8, 7), (mxm.MODE_EMUL_BF16, 6),
                                    (mxm.MODE_EMUL_RN8, 6), (mxm.MODE_F64, 0)])
def test_grouped_matches_oracle(mode, S, graph, plan):
    if mode == mxm.MODE_F64 and plan != "default":
        pytest.skip("the plan only splits emulated calls")
    hs, ds = make_group(DIMS, kind="spread" if mode != mxm.MODE_F64 else "uniform")
    assert run_group(ds, mode, S, graph=graph, plan=PLANS[plan]) == mxm.MXM_OK
    for (A, B), (_, _, C) in zip(hs, ds):
        got = C.cpu().numpy()
        if mode == mxm.MODE_F64:
            assert_within_bound(got, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B), A.shape[1],
                                f"grouped f64 {A.shape}x{B.shape}")
        elif mode == mxm.MODE_EMUL_RN8:
            assert_bitwise(got, oracle.ozaki_gemm_rn8(A, B, S),
                           f"grouped rn8 {A.shape}x{B.shape}")
        else:
            beta = 8 if mode == mxm.MODE_EMUL_BF16 else 7
            assert_bitwise(got, oracle.ozaki_gemm(A, B, S=S, beta=beta),
                           f"grouped emul {A.shape}x{B.shape}")


# Edge tiles: the grouped kernels cut work at 16 columns and 16 k (the MMA
# steps) and copy only the rows an edge tile reads, and the native kernel
# cuts at 32 x 32 pieces and 4 k; every remainder around those steps.
EDGE_DIMS = [(m, k, n) for m in (1, 9, 40, 130) for k in (1, 15, 16, 17, 64, 65, 129)
             for n in (1, 16, 17, 100)]


@pytest.mark.parametrize("mode,S,plan", [(mxm.MODE_EMUL_I8, 5, "default"),
                                         (mxm.MODE_EMUL_I8, 5, "pair"),
                                         (mxm.MODE_EMUL_RN8, 4, "default"),
                                         (mxm.MODE_EMUL_RN8, 4, "pair"),
                                         (mxm.MODE_F64, 0, "default")])
def test_grouped_edge_tiles(mode, S, plan):
    hs, ds = make_group(EDGE_DIMS, seed=3, kind="spread" if mode != mxm.MODE_F64 else "uniform")
    assert run_group(ds, mode, S, plan=PLANS[plan]) == mxm.MXM_OK
    for (A, B), (_, _, C) in zip(hs, ds):
        got = C.cpu().numpy()
        if mode == mxm.MODE_F64:
            assert_within_bound(got, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B), A.shape[1],
                                f"edge f64 {A.shape}x{B.shape}")
        elif mode == mxm.MODE_EMUL_RN8:
            assert_bitwise(got, oracle.ozaki_gemm_rn8(A, B, S), f"edge rn8 {A.shape}x{B.shape}")
        else:
            assert_bitwise(got, oracle.ozaki_gemm(A, B, S=S, beta=7),
                           f"edge emul {A.shape}x{B.shape}")


def test_grouped_workspace_too_small_reported():
    _, ds = make_group(DIMS[:4])
    table_h = mxm.problem_table(ds)
    need = mxm.mxm_grouped_workspace_size(table_h, mxm.MODE_EMUL_I8, 7)
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    mxm.mxm_grouped(table_h.cuda(), mxm.MODE_EMUL_I8, 7, ws)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_ERR_WORKSPACE_TOO_SMALL
    for _, _, C in ds:  # nothing was computed
        assert torch.isnan(C).all()


def test_grouped_2000_logu_sampled():
    """The grouped workload: 2000 problems, each of m, k, n log-uniform in
    [16, 1024] from seed 0; both modes; 24 problems checked in full plus the
    three with the shortest k.  S = 8: with uniform entries the truncation
    error relative to k u |A||B| grows as 1/k, and at k = 16 seven slices
    leave ~4 k u |A||B|, outside the bound; eight meet it."""
    dims = inputs.grouped_problems(0, 2000)
    hs, ds = make_group([tuple(int(v) for v in d) for d in dims])
    rng = np.random.default_rng(5)
    pick = list(rng.choice(len(dims), 24, replace=False))
    pick += sorted(range(len(dims)), key=lambda p: dims[p][1])[:3]
    for mode, S in ((mxm.MODE_EMUL_I8, 8), (mxm.MODE_F64, 0)):
        assert run_group(ds, mode, S, graph=True) == mxm.MXM_OK
        for p in pick:
            A, B = hs[p]
            got = ds[p][2].cpu().numpy()
            if mode != mxm.MODE_F64:
                assert_bitwise(got, oracle.ozaki_gemm(A, B, S=S), f"p={p}")
            assert_within_bound(got, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B),
                                A.shape[1], f"p={p} mode={mode}")


def test_grouped_many_small_problems():
    """6000 problems with m, k, n uniform in [0, 48], empty ones included:
    thousands of claims on the maxima pass's cursor and on the slice GEMM's
    tile cursor, and every operand tile's and C tile's problem taken from
    the owner map.  300 random problems and every empty one are checked
    against the oracle (bit-identical for the emulated modes)."""
    rng = np.random.default_rng(11)
    dims = [tuple(int(v) for v in rng.integers(0, 49, 3)) for _ in range(6000)]
    hs, ds = make_group(dims, seed=4, kind="spread")
    pick = sorted(set(rng.choice(len(dims), 300, replace=False).tolist())
                  | {p for p, d in enumerate(dims) if 0 in d})
    for mode, S in ((mxm.MODE_EMUL_I8, 7), (mxm.MODE_EMUL_RN8, 6), (mxm.MODE_F64, 0)):
        for _, _, C in ds:
            C.fill_(float("nan"))
        assert run_group(ds, mode, S) == mxm.MXM_OK
        for p in pick:
            A, B = hs[p]
            got = ds[p][2].cpu().numpy()
            if mode == mxm.MODE_F64:
                assert_within_bound(got, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B),
                                    A.shape[1], f"p={p} {dims[p]}")
            elif mode == mxm.MODE_EMUL_RN8:
                assert_bitwise(got, oracle.ozaki_gemm_rn8(A, B, S), f"p={p} {dims[p]}")
            else:
                assert_bitwise(got, oracle.ozaki_gemm(A, B, S=S), f"p={p} {dims[p]}")
