"""Conjugate gradients on the GPU (mxm_cg, Sec. 3.4) against the CG oracle
through the C ABI.  The two differ only in the order their dot products
and row sums are added.  For a well-conditioned matrix (Gershgorin bound
kappa_G <= 1000) r2 after step k and the iterate then differ by rounding
that accumulates over the steps: the tolerance is
4 kappa_G (n + bw) u (k + 1), and the step count must agree unless an r2
of the oracle lies within that tolerance of the stop value.  For a worse
conditioned matrix the recursive residuals of two correct runs drift apart
(late steps can differ by tens of percent), so there only the solution is
compared: each x is within (sqrt(r2) + drift) / lambda_min of the true
one, lambda_min >= the Gershgorin lower bound, drift = k (bw + n) u
|A|_inf |x|_inf sqrt(n) the gap between the recursive and the true
residual."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt).cuda()


def run_cg(rowp, indx, vals, b, stop, max_iters, expect=mxm.MXM_OK, engine=mxm.CG_CLUSTER):
    n = len(rowp) - 1
    x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    hist = torch.full((max(max_iters, 1),), float("nan"), dtype=torch.float64, device="cuda")
    it, r2 = mxm.mxm_cg(dev(vals, torch.float64), dev(indx, torch.int32), dev(rowp, torch.int32),
                        dev(b, torch.float64), x, stop, max_iters, r2_hist=hist, engine=engine)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == expect
    k = int(it.item())
    return {"x": x.cpu().numpy(), "iters": k, "r2": float(r2.item()),
            "hist": hist.cpu().numpy()[:k]}


def gershgorin(rowp, indx, vals):
    """(lower, upper) Gershgorin bounds of the spectrum."""
    n = len(rowp) - 1
    rows = np.repeat(np.arange(n), np.diff(rowp))
    diag = np.zeros(n)
    np.add.at(diag, rows[indx == rows], vals[indx == rows])
    off = np.zeros(n)
    np.add.at(off, rows[indx != rows], np.abs(vals[indx != rows]))
    return float((diag - off).min()), float((diag + off).max())


def csr_times(rowp, indx, vals, x):
    rows = np.repeat(np.arange(len(rowp) - 1), np.diff(rowp))
    y = np.zeros(len(rowp) - 1)
    np.add.at(y, rows, vals * x[indx])
    return y


def compare(rowp, indx, vals, b, stop, max_iters, bw, engine=mxm.CG_CLUSTER):
    n = len(rowp) - 1
    want = oracle.cg(rowp, indx, vals, b, stop, max_iters)
    got = run_cg(rowp, indx, vals, b, stop, max_iters, engine=engine)
    lo, hi = gershgorin(rowp, indx, vals)
    kap = hi / lo
    h = want["hist"]
    if got["iters"]:
        assert got["r2"] == got["hist"][-1]
    if kap <= 1000:
        tol = lambda k: 4 * kap * (n + bw) * U * (k + 1)  # noqa: E731
        near = np.any(np.abs(h / stop - 1.0) <= tol(len(h))) if stop > 0 and len(h) else False
        if near:
            assert abs(got["iters"] - want["iters"]) <= 1
        else:
            assert got["iters"] == want["iters"], (got["iters"], want["iters"])
        m = min(got["iters"], want["iters"])
        for k in range(m):
            assert abs(got["hist"][k] - h[k]) <= tol(k) * h[k], (k, got["hist"][k], h[k])
        if got["iters"] == want["iters"]:
            err = np.max(np.abs(got["x"] - want["x"]))
            assert err <= tol(m) * max(np.max(np.abs(want["x"])), 1e-300), err
    else:
        assert abs(got["iters"] - want["iters"]) <= max(1, want["iters"] // 50)
        k = max(got["iters"], want["iters"])
        amax = max(np.abs(vals).max() * (bw if bw < n else n), 1.0)
        xmax = max(np.abs(want["x"]).max(), 1e-300)
        drift = k * (bw + n) * U * amax * xmax * np.sqrt(n)
        bound = (np.sqrt(got["r2"]) + np.sqrt(want["r2"]) + 2 * drift) / lo
        assert np.linalg.norm(got["x"] - want["x"]) <= bound
        res = np.linalg.norm(b - csr_times(rowp, indx, vals, got["x"]))
        assert res <= np.sqrt(got["r2"]) + drift
    return got, want


ENGINES = [mxm.CG_CLUSTER, mxm.CG_GRAPH]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n,bw", inputs.CG_TABLE2)
def test_table2_against_oracle(n, bw, engine):
    rowp, indx, vals = inputs.banded_spd(6, 91, n, bw)
    b = inputs.uniform_pm1(6, 92, (n,))
    got, want = compare(rowp, indx, vals, b, 1e-24 * float(b @ b), 10 * n, bw, engine)
    assert got["iters"] > 5


@pytest.mark.parametrize("n,bw,shift,steps", [(1024, 31, 1e-3, 60), (512, 255, 1e-2, 20),
                                              (300, 7, 1e-4, 100)])
@pytest.mark.parametrize("engine", ENGINES)
def test_worse_conditioned(n, bw, shift, steps, engine):
    """Off-diagonals made negative (a shifted graph Laplacian: the constant
    vector is nearly in the null space), so the smallest eigenvalue is close
    to the shift and the solve takes many steps."""
    rowp, indx, vals = inputs.banded_spd(8, 93, n, bw, shift=shift)
    rows = np.repeat(np.arange(n), np.diff(rowp))
    vals = np.where(indx != rows, -np.abs(vals), vals)
    b = inputs.uniform_pm1(8, 94, (n,))
    got, _ = compare(rowp, indx, vals, b, 1e-20 * float(b @ b), 10 * n, bw, engine)
    assert got["iters"] > steps


@pytest.mark.parametrize("n,bw", [(12288, 63), (4099, 7), (12288, 3), (1, 3), (33, 65)])
def test_sizes_and_cluster_shapes(n, bw):
    """The largest order, ragged row splits over the cluster, a 1 x 1
    system, and a band wider than the matrix."""
    rowp, indx, vals = inputs.banded_spd(9, 95, n, bw)
    b = inputs.uniform_pm1(9, 96, (n,))
    compare(rowp, indx, vals, b, 1e-22 * float(b @ b), 200, bw)


def test_rows_partly_held_in_shared_memory():
    """At the largest order the shared memory left over holds a diagonal
    block of 768 rows but not a tridiagonal one: the CTA owning the first
    768 rows (tridiagonal there) streams its rows from global memory while
    the 15 others use their copies; the solve is the oracle's all the same.
    The diagonal is random in [2, 8) (distinct eigenvalues: with only a few
    distinct ones the late residuals of any two summation orders drift
    apart beyond the tolerance)."""
    n, head = 12288, 768
    d = 5.0 + 3.0 * inputs.uniform_pm1(15, 107, (n,))
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if j == i:
                rows.append(i), cols.append(j), vals.append(d[i] + (2.0 if i < head else 0.0))
            elif i < head and 0 <= j < head:
                rows.append(i), cols.append(j), vals.append(-1.0)
    rowp = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowp, np.asarray(rows) + 1, 1)
    rowp = np.cumsum(rowp).astype(np.int32)
    indx, vals = np.asarray(cols, dtype=np.int32), np.asarray(vals)
    b = inputs.uniform_pm1(15, 106, (n,))
    got, _ = compare(rowp, indx, vals, b, 1e-24 * float(b @ b), 500, 1)
    assert got["iters"] > 5


@pytest.mark.parametrize("engine", ENGINES)
def test_fixed_step_counts_and_edges(engine):
    n, bw = 700, 31
    rowp, indx, vals = inputs.banded_spd(10, 97, n, bw)
    b = inputs.uniform_pm1(10, 98, (n,))
    for k in (1, 2, 5):
        got, _ = compare(rowp, indx, vals, b, 0.0, k, bw, engine)
        assert got["iters"] == k
    bb = float(b @ b)
    got = run_cg(rowp, indx, vals, b, 0.0, 0, engine=engine)
    assert got["iters"] == 0 and np.array_equal(got["x"], np.zeros(n))
    assert got["r2"] == pytest.approx(bb, rel=n * U)
    assert run_cg(rowp, indx, vals, b, 1.5 * bb, 50, engine=engine)["iters"] == 0
    z = run_cg(rowp, indx, vals, np.zeros(n), 0.0, 50, engine=engine)
    assert z["iters"] == 0 and np.array_equal(z["x"], np.zeros(n))


@pytest.mark.parametrize("engine", ENGINES)
def test_identity_multiple_and_determinism(engine):
    n = 2049
    rowp = np.arange(n + 1, dtype=np.int32)
    indx = np.arange(n, dtype=np.int32)
    b = inputs.uniform_pm1(11, 99, (n,))
    got = run_cg(rowp, indx, np.full(n, 4.0), b, 1e-20 * float(b @ b), 50, engine=engine)
    assert got["iters"] == 1
    assert np.max(np.abs(got["x"] - b / 4.0)) <= 4 * n * U * np.max(np.abs(b))
    rowp, indx, vals = inputs.banded_spd(12, 100, 5000, 63)
    b = inputs.uniform_pm1(12, 101, (5000,))
    a1 = run_cg(rowp, indx, vals, b, 1e-24 * float(b @ b), 500, engine=engine)
    a2 = run_cg(rowp, indx, vals, b, 1e-24 * float(b @ b), 500, engine=engine)
    assert a1["iters"] == a2["iters"] and np.array_equal(a1["x"], a2["x"])
    assert np.array_equal(a1["hist"], a2["hist"])


@pytest.mark.parametrize("engine", ENGINES)
def test_breakdown_and_bad_structure_reported(engine):
    n = 64
    rowp = np.arange(n + 1, dtype=np.int32)
    indx = np.arange(n, dtype=np.int32)
    got = run_cg(rowp, indx, -np.ones(n), np.ones(n), 0.0, 10, expect=mxm.MXM_ERR_BREAKDOWN,
                 engine=engine)
    assert got["iters"] == 0 and np.array_equal(got["x"], np.zeros(n))
    bad = indx.copy()
    bad[7] = 10_000
    run_cg(rowp, bad, np.ones(n), np.ones(n), 0.0, 3, expect=mxm.MXM_ERR_INVALID_ARG,
           engine=engine)
    badp = rowp.copy()
    badp[5] = 1000
    run_cg(badp, indx, np.ones(n), np.ones(n), 0.0, 3, expect=mxm.MXM_ERR_INVALID_ARG,
           engine=engine)
    # the context is intact and the status was cleared
    ok = run_cg(rowp, indx, np.full(n, 2.0), np.ones(n), 1e-30, 10, engine=engine)
    assert ok["iters"] == 1 and np.allclose(ok["x"], 0.5, rtol=1e-15, atol=0)


@pytest.mark.parametrize("n,bw", [(100_000, 7), (1_000_000, 3), (30_000, 63)])
def test_graph_engine_large_orders(n, bw):
    """Orders beyond one cluster's shared memory: the graph engine only."""
    rowp, indx, vals = inputs.banded_spd(13, 102, n, bw)
    b = inputs.uniform_pm1(13, 103, (n,))
    got, want = compare(rowp, indx, vals, b, 1e-22 * float(b @ b), 200, bw, mxm.CG_GRAPH)
    assert got["iters"] > 5


def test_engines_agree_and_auto():
    """Both engines solve the same system to the same tolerance; the
    automatic choice runs without a workspace for a small system."""
    n, bw = 1024, 511
    rowp, indx, vals = inputs.banded_spd(14, 104, n, bw)
    b = inputs.uniform_pm1(14, 105, (n,))
    stop = 1e-24 * float(b @ b)
    c = run_cg(rowp, indx, vals, b, stop, 500, engine=mxm.CG_CLUSTER)
    g = run_cg(rowp, indx, vals, b, stop, 500, engine=mxm.CG_GRAPH)
    a = run_cg(rowp, indx, vals, b, stop, 500, engine=mxm.CG_AUTO)
    assert c["iters"] == g["iters"] == a["iters"]
    scale = np.max(np.abs(c["x"]))
    assert np.max(np.abs(c["x"] - g["x"])) <= 1e-12 * scale
    lib = mxm.load()
    d = lambda arr, dt: torch.from_numpy(np.ascontiguousarray(arr)).to(dtype=dt).cuda()  # noqa: E731
    dv, di, dr, db = d(vals, torch.float64), d(indx, torch.int32), d(rowp, torch.int32), \
        d(b, torch.float64)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    r2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    args = (dv.data_ptr(), di.data_ptr(), dr.data_ptr(), db.data_ptr(), x.data_ptr(), n, len(vals),
            stop, 500)
    tail = (it.data_ptr(), r2.data_ptr(), None, None)
    assert lib.mxm_cg(*args, mxm.CG_AUTO, None, *tail) == mxm.MXM_OK
    assert lib.mxm_cg(*args, mxm.CG_GRAPH, None, *tail) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_cg(*args, 7, None, *tail) == mxm.MXM_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert int(it.item()) == c["iters"] and mxm.mxm_get_device_status() == mxm.MXM_OK
