"""mod2as on the GPU (mxm_spmv, Sec. 3.2) against the CSR oracle, through
the C ABI: every row within 2 len_i u (|A||x|)_i of the Dot2 reference
(len_i the row's length), bit-exact where every partial sum is exact, and
bad structure reported through the device status, never read through."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -53

# Table 1 of the paper: n x n matrices and their fill in percent
TABLE1 = [(100, 3.50), (200, 3.75), (256, 5.0), (400, 4.38), (500, 5.00), (512, 4.00),
          (960, 4.50), (1000, 5.00), (1024, 5.50), (2000, 7.50), (4096, 3.50), (4992, 4.00),
          (5000, 4.00), (9984, 4.50), (10000, 5.00), (10240, 5.72)]


def run_spmv(rowp, indx, vals, x, expect=mxm.MXM_OK):
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt).cuda()  # noqa: E731
    y = torch.full((len(rowp) - 1,), float("nan"), dtype=torch.float64, device="cuda")
    mxm.mxm_spmv(d(vals, torch.float64), d(indx, torch.int32), d(rowp, torch.int32),
                 d(x, torch.float64), y)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == expect
    return y.cpu().numpy()


def check_bound(y, rowp, indx, vals, x, what):
    ref = oracle.spmv_dot2(rowp, indx, vals, x)
    ab = oracle.spmv_abs(rowp, indx, vals, x)
    lens = np.diff(rowp).astype(np.float64)
    lim = 2.0 * np.maximum(lens, 1.0) * U * ab
    bad = ~(np.abs(y - ref) <= lim)
    assert not bad.any(), f"{what}: {int(bad.sum())} rows outside the bound, first {np.argmax(bad)}"


@pytest.mark.parametrize("n,fill", TABLE1)
def test_table1_within_bound(n, fill):
    rowp, indx, vals = inputs.csr_random(0, 70, n, fill / 100.0)
    x = inputs.uniform_pm1(0, 72, (n,))
    check_bound(run_spmv(rowp, indx, vals, x), rowp, indx, vals, x, f"n={n}")


def test_integer_entries_bit_exact():
    rowp, indx, _ = inputs.csr_random(0, 73, 3000, 0.04)
    vals = inputs.int_uniform(0, 74, (len(indx),), -8, 8)
    x = inputs.int_uniform(0, 75, (3000,), -8, 8)
    assert np.array_equal(run_spmv(rowp, indx, vals, x), oracle.spmv(rowp, indx, vals, x))


def test_identity_permutation_and_empty():
    n = 4097
    x = inputs.uniform_pm1(0, 76, (n,))
    rowp = np.arange(n + 1, dtype=np.int32)
    assert np.array_equal(run_spmv(rowp, np.arange(n, dtype=np.int32), np.ones(n), x), x)
    p = inputs.permutation(0, 77, n).astype(np.int32)
    assert np.array_equal(run_spmv(rowp, p, np.ones(n), x), x[p])
    # no values at all, and rows of every length from 0 to 100 000 (every lane-group width)
    assert np.array_equal(run_spmv(np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0),
                                   np.ones(7)), np.zeros(5))
    lens = np.array([0, 1, 3, 0, 7, 15, 31, 64, 0, 100000, 2, 0])
    rowp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ncols = 120000
    indx = np.concatenate([np.sort(inputs.permutation(0, 78 + i, ncols)[:L]) for i, L in
                           enumerate(lens)]).astype(np.int32)
    vals = inputs.uniform_pm1(0, 90, (len(indx),))
    x = inputs.uniform_pm1(0, 91, (ncols,))
    check_bound(run_spmv(rowp, indx, vals, x), rowp, indx, vals, x, "mixed lengths")


@pytest.mark.parametrize("avg,n", [(3, 160_000), (12, 160_000), (48, 160_000), (200, 40_000),
                                   (600, 20_000), (48, 2_000)])
def test_every_lane_group_width(avg, n):
    """Average row lengths and row counts that select 2, 4, 8, 16 and 32
    lanes per row (and a short matrix widened for occupancy), with rounds
    of 2 or 4 values per lane and ragged last rounds."""
    rowp, indx, vals = inputs.csr_sampled(1, 92, n, n, avg)
    x = inputs.exp_spread(1, 94, (n,), -10, 10)
    check_bound(run_spmv(rowp, indx, vals, x), rowp, indx, vals, x, f"avg={avg}")


def test_bad_structure_is_reported_not_read():
    x = np.ones(8)
    vals = np.ones(4)
    # a column out of range in row 1: row 1 skipped, the others written
    y = run_spmv(np.array([0, 2, 4], np.int32), np.array([0, 1, 2, 99], np.int32), vals, x,
                 expect=mxm.MXM_ERR_INVALID_ARG)
    assert y[0] == 2.0 and np.isnan(y[1])
    # rowp decreasing and past nnz
    y = run_spmv(np.array([0, 3, 1, 9], np.int32), np.array([0, 1, 2, 3], np.int32), vals, x,
                 expect=mxm.MXM_ERR_INVALID_ARG)
    assert y[0] == 3.0 and np.isnan(y[1]) and np.isnan(y[2])
    # the context is intact and the status was cleared
    assert np.array_equal(run_spmv(np.array([0, 1], np.int32), np.array([0], np.int32),
                                   np.array([2.0]), np.array([3.0])), np.array([6.0]))


def test_large_beyond_l2():
    """A matrix of 50 million values (600 MB of values and columns: larger
    than L2), as the benchmark's large case: all rows within the bound."""
    n = 200_000
    rowp, indx, vals = inputs.csr_sampled(2, 95, n, n, 250)
    x = inputs.uniform_pm1(2, 97, (n,))
    check_bound(run_spmv(rowp, indx, vals, x), rowp, indx, vals, x, "n=200000")
