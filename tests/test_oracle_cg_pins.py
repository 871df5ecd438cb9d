"""Pins of the conjugate-gradient oracle (Sec. 3.4, Fig. 6) to facts that
do not come from the oracle itself: the k-th iterate minimises the A-norm
of the error over the Krylov space K_k(A, b) (solved here by a projected
dense system), exact termination after n steps, the recursive residual
equal to the true one, mutually orthogonal residuals, closed forms for
multiples of the identity, and the paper's stopping rule."""
import numpy as np
import pytest

import oracle
from paper_1211_1581_gb300 import inputs

U = 2.0 ** -53


def dense_of(rowp, indx, vals, n):
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(rowp[i], rowp[i + 1]):
            D[i, indx[j]] += vals[j]
    return D


def csr_of(D):
    rowp, indx, vals = [0], [], []
    for i in range(D.shape[0]):
        nz = np.nonzero(D[i])[0]
        indx += list(nz)
        vals += list(D[i, nz])
        rowp.append(len(indx))
    return np.array(rowp, np.int32), np.array(indx, np.int32), np.array(vals, np.float64)


def krylov_minimiser(A, b, k):
    """argmin over x in span{b, Ab, ..., A^{k-1} b} of (x* - x)^T A (x* - x),
    i.e. V y with (V^T A V) y = V^T b for an orthonormal basis V."""
    K = np.empty((len(b), k))
    v = b.copy()
    for t in range(k):
        K[:, t] = v
        v = A @ v
    V, _ = np.linalg.qr(K)
    y = np.linalg.solve(V.T @ A @ V, V.T @ b)
    return V @ y


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_iterates_minimise_a_norm_over_krylov_space(k):
    n = 14
    rowp, indx, vals = inputs.banded_spd(0, 80, n, 5)
    b = inputs.uniform_pm1(0, 81, (n,))
    A = dense_of(rowp, indx, vals, n)
    got = oracle.cg(rowp, indx, vals, b, 0.0, k)
    assert got["iters"] == k and not got["breakdown"]
    ref = krylov_minimiser(A, b, k)
    assert np.max(np.abs(got["x"] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_first_step_closed_form():
    """x1 = (b.b / b.Ab) b and r2 after it = |b - x1-step residual|^2."""
    n = 40
    rowp, indx, vals = inputs.banded_spd(1, 82, n, 7)
    b = inputs.uniform_pm1(1, 83, (n,))
    A = dense_of(rowp, indx, vals, n)
    got = oracle.cg(rowp, indx, vals, b, 0.0, 1)
    alpha = (b @ b) / (b @ (A @ b))
    assert np.allclose(got["x"], alpha * b, rtol=1e-14, atol=0)
    r1 = b - alpha * (A @ b)
    assert got["hist"][0] == pytest.approx(r1 @ r1, rel=1e-12)


def test_exact_termination_after_n_steps():
    n = 10
    rowp, indx, vals = inputs.banded_spd(2, 84, n, 9)
    b = inputs.uniform_pm1(2, 85, (n,))
    A = dense_of(rowp, indx, vals, n)
    got = oracle.cg(rowp, indx, vals, b, 0.0, n)
    xs = np.linalg.solve(A, b)
    assert np.max(np.abs(got["x"] - xs)) <= 1e-11 * np.max(np.abs(xs))


def test_recursive_residual_is_true_residual_and_residuals_orthogonal():
    n = 30
    rowp, indx, vals = inputs.banded_spd(3, 86, n, 5)
    b = inputs.uniform_pm1(3, 87, (n,))
    A = dense_of(rowp, indx, vals, n)
    res = []
    for k in range(1, 7):
        got = oracle.cg(rowp, indx, vals, b, 0.0, k)
        r = b - A @ got["x"]
        assert got["hist"][k - 1] == pytest.approx(r @ r, rel=1e-9)
        res.append(r)
    res.insert(0, b)
    for i in range(len(res)):
        for j in range(i):
            c = abs(res[i] @ res[j]) / (np.linalg.norm(res[i]) * np.linalg.norm(res[j]))
            assert c < 1e-8, (i, j, c)


def test_multiple_of_identity_one_step_exact():
    n = 33
    rowp = np.arange(n + 1, dtype=np.int32)
    indx = np.arange(n, dtype=np.int32)
    b = inputs.uniform_pm1(4, 88, (n,))
    got = oracle.cg(rowp, indx, np.full(n, 4.0), b, 0.0, 50)
    assert got["iters"] == 1 and got["r2"] == 0.0
    assert np.array_equal(got["x"], b / 4.0)


def test_stopping_rule_and_edges():
    n = 64
    rowp, indx, vals = inputs.banded_spd(5, 89, n, 3)
    b = inputs.uniform_pm1(5, 90, (n,))
    bb = float(b @ b)
    # r2 > stop is the loop test: stop >= (b, b) takes no step
    got = oracle.cg(rowp, indx, vals, b, 1.5 * bb, 100)
    assert got["iters"] == 0 and np.array_equal(got["x"], np.zeros(n))
    assert got["r2"] == pytest.approx(bb, rel=n * U)
    assert oracle.cg(rowp, indx, vals, b, 0.5 * bb, 100)["iters"] >= 1
    # max_iters = 0 takes no step either; b = 0 stops at once
    assert oracle.cg(rowp, indx, vals, b, 0.0, 0)["iters"] == 0
    z = oracle.cg(rowp, indx, vals, np.zeros(n), 0.0, 100)
    assert z["iters"] == 0 and np.array_equal(z["x"], np.zeros(n))
    # converged run: the step count is the first k with r2_k <= stop
    stop = 1e-20 * bb
    got = oracle.cg(rowp, indx, vals, b, stop, 1000)
    h = got["hist"]
    assert h[-1] <= stop and np.all(h[:-1] > stop) and not got["breakdown"]
    A = dense_of(rowp, indx, vals, n)
    r = b - A @ got["x"]
    assert r @ r <= 4 * stop + (n * U * np.abs(A).sum(axis=1).max() * np.abs(got["x"]).max()) ** 2 * n


def test_one_by_one_and_breakdown():
    got = oracle.cg(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([8.0]),
                    np.array([3.0]), 0.0, 5)
    assert got["iters"] == 1 and got["x"][0] == 3.0 / 8.0
    # negative definite: (p, A p) < 0 at the first step, nothing taken
    n = 5
    got = oracle.cg(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                    -np.ones(n), np.ones(n), 0.0, 5)
    assert got["breakdown"] and got["iters"] == 0 and np.array_equal(got["x"], np.zeros(n))
    with pytest.raises(ValueError):
        oracle.cg(np.array([0, 1], np.int32), np.array([2], np.int32), np.ones(1), np.ones(1), 0.0, 3)


@pytest.mark.parametrize("n,bw", inputs.CG_TABLE2)
def test_table2_converges_to_the_solution(n, bw):
    rowp, indx, vals = inputs.banded_spd(6, 91, n, bw)
    b = inputs.uniform_pm1(6, 92, (n,))
    A = dense_of(rowp, indx, vals, n)
    xs = np.linalg.solve(A, b)
    got = oracle.cg(rowp, indx, vals, b, 1e-24 * float(b @ b), 10 * n)
    assert not got["breakdown"] and got["iters"] < 10 * n
    # eigenvalues in [1, lam_max] (Gershgorin): |x - x*| <= |r| / lam_min + drift
    assert np.linalg.norm(got["x"] - xs) <= 1e-11 * np.linalg.norm(xs) + 1e-12


def test_generator():
    for n, bw in ((1, 3), (5, 3), (20, 9), (8, 31)):
        rowp, indx, vals = inputs.banded_spd(7, 93, n, bw)
        D = dense_of(rowp, indx, vals, n)
        assert np.array_equal(D, D.T)
        h = (bw - 1) // 2
        i, j = np.nonzero(D)
        assert np.all(np.abs(i - j) <= h)
        if n > h:
            assert np.count_nonzero(D) == n * (2 * h + 1) - h * (h + 1)
        off = np.abs(D).sum(axis=1) - np.diag(D)
        assert np.all(np.diag(D) == 1.0 + off) or np.allclose(np.diag(D), 1.0 + off, rtol=1e-15)
        r2, i2, v2 = csr_of(D)
        assert np.array_equal(r2, rowp) and np.array_equal(i2, indx) and np.array_equal(v2, vals)
    with pytest.raises(ValueError):
        inputs.banded_spd(0, 0, 4, 4)
