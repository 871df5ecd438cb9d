"""Native FP64 path (mxm_f64) against the oracle, through the C ABI.

Acceptance (per entry): |C - C_dot2| <= 2 k u (|A||B|), u = 2^-53; bit-exact
on inputs whose products and partial sums are all exact (identity,
permutation, small integers)."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs
from helpers import assert_bitwise, assert_within_bound

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_f64(A, B):
    m, k = A.shape
    n = B.shape[1]
    C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
    mxm.mxm_f64(dev(A), dev(B), C)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    return C.cpu().numpy()


SHAPES = [(1, 1, 1), (7, 13, 5), (17, 33, 15), (128, 16, 128), (129, 65, 131),
          (255, 17, 129), (300, 200, 257), (256, 256, 256), (64, 1000, 40)]


@pytest.mark.parametrize("shape", SHAPES)
def test_f64_uniform_within_bound(shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=0)
    C = run_f64(A, B)
    assert_within_bound(C, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B), k, f"f64 {shape}")


def test_f64_spread_within_bound():
    m, k, n = 200, 300, 190
    A, B = inputs.gemm_operands("spread", m, k, n, seed=0, cfg=2)
    C = run_f64(A, B)
    assert_within_bound(C, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B), k, "f64 spread")


def test_f64_exact_cases_n256():
    """The small exact-check cases at m = k = n = 256: identity, random
    permutation, integer entries in [-8, 8] -- bit-exact."""
    n = 256
    A, B = inputs.gemm_operands("uniform", n, n, n, seed=0, cfg=0)
    I = np.eye(n)
    assert_bitwise(run_f64(I, B), B, "I.B")
    assert_bitwise(run_f64(A, I), A, "A.I")
    P = inputs.permutation_matrix(0, 7, n)
    assert_bitwise(run_f64(P, B), B[inputs.permutation(0, 7, n)], "P.B")
    Ai, Bi = inputs.gemm_operands("int8", n, n, n, seed=0, cfg=3)
    ref = (Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float64)
    assert_bitwise(run_f64(Ai, Bi), ref, "int [-8,8]")


def test_f64_empty_and_zero_k():
    A = np.zeros((5, 0))
    B = np.zeros((0, 6))
    C = run_f64(A, B)
    assert np.array_equal(C, np.zeros((5, 6)))
    # m == 0: nothing written, nothing launched
    C = torch.zeros((0, 4), dtype=torch.float64, device="cuda")
    mxm.mxm_f64(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                torch.zeros((3, 4), dtype=torch.float64, device="cuda"), C)


def test_f64_deterministic():
    A, B = inputs.gemm_operands("uniform", 333, 517, 291, seed=0, cfg=4)
    assert_bitwise(run_f64(A, B), run_f64(A, B), "run to run")


def _sample(n_rows, n_cols, count, seed):
    """Seeded entries of an n_rows x n_cols result: `count` at random plus
    the corners of the matrix and of the 128 x 128 tiles around its middle
    and its last tile row and column (the edges a tiling gets wrong)."""
    rng = np.random.default_rng(seed)
    ii = list(rng.integers(0, n_rows, count))
    jj = list(rng.integers(0, n_cols, count))
    for r in (0, 127, 128, 129, n_rows // 2, n_rows - 129, n_rows - 128, n_rows - 1):
        for c in (0, 127, 128, n_cols // 2, n_cols - 128, n_cols - 1):
            if 0 <= r < n_rows and 0 <= c < n_cols:
                ii.append(r)
                jj.append(c)
    return np.array(ii, dtype=np.int64), np.array(jj, dtype=np.int64)


@pytest.mark.parametrize("n", [1024, 2048, 4096, 8192])
def test_f64_sweep_sampled(n):
    """The square sweep sizes: seeded entries (random, and the tile corners)
    checked one by one against Dot2 with the bound 2 k u (|A||B|)."""
    A, B = inputs.gemm_operands("uniform", n, n, n, seed=0, cfg=1)
    C = run_f64(A, B)
    ii, jj = _sample(n, n, 600, n)
    d2, ab = oracle.entries_dot2_abs(A, B, ii, jj)
    assert_within_bound(C[ii, jj], d2, ab, n, f"f64 n={n}")


def test_f64_sweep_n16384_sampled():
    """The largest sweep size, 16384^3 (2 GiB per operand): 300 seeded
    entries and the tile corners against Dot2."""
    n = 16384
    A, B = inputs.gemm_operands("uniform", n, n, n, seed=0, cfg=1)
    dA, dB = dev(A), dev(B)
    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
    mxm.mxm_f64(dA, dB, C)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    del dA, dB
    ii, jj = _sample(n, n, 300, n)
    got = C[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
    del C
    torch.cuda.empty_cache()
    d2, ab = oracle.entries_dot2_abs(A, B, ii, jj)
    assert_within_bound(got, d2, ab, n, "f64 n=16384")


def test_f64_rectangular_sampled():
    for (m, k, n) in [(4096, 256, 1024), (128, 16384, 128), (8192, 1024, 64)]:
        A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=3)
        C = run_f64(A, B)
        rng = np.random.default_rng(m + k + n)
        ii = rng.integers(0, m, 300)
        jj = rng.integers(0, n, 300)
        d2, ab = oracle.entries_dot2_abs(A, B, ii, jj)
        assert_within_bound(C[ii, jj], d2, ab, k, f"f64 {(m, k, n)}")


# Split-k: products with fewer C tiles than SMs cut k into ranges computed by
# separate CTAs and added in range order (1 tile x 32 ranges; 3 tiles x 23
# ranges with a ragged last k-block; 64 tiles x 4 ranges).
@pytest.mark.parametrize("shape", [(128, 4096, 128), (257, 3001, 65), (1024, 1024, 1024)])
def test_f64_splitk_within_bound(shape):
    m, k, n = shape
    A, B = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=7)
    C = run_f64(A, B)
    if m * n <= 300 * 300:
        assert_within_bound(C, oracle.gemm_dot2(A, B), oracle.gemm_abs(A, B), k, f"{shape}")
    else:
        rng = np.random.default_rng(k)
        ii = rng.integers(0, m, 400)
        jj = rng.integers(0, n, 400)
        d2, ab = oracle.entries_dot2_abs(A, B, ii, jj)
        assert_within_bound(C[ii, jj], d2, ab, k, f"{shape}")


def test_f64_splitk_exact_integers_and_deterministic():
    """Integers in [-8, 8] with k = 4096: every partial sum is an integer
    below 2^18, so any summation order (split or not) is exact."""
    A, B = inputs.gemm_operands("int8", 100, 4096, 90, seed=0, cfg=8)
    C = run_f64(A, B)
    assert_bitwise(C, oracle.gemm_naive(A, B), "split-k integers")
    assert_bitwise(run_f64(A, B), C, "split-k run to run")
