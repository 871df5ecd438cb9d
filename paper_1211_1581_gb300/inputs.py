"""Seeded synthetic inputs for the mod2am product (Sec. 3.1) and its variants,
the mod2as sparse product (Sec. 3.2) and the conjugate-gradient solver
(Sec. 3.4).

This module only draws numbers; it holds none of the product's arithmetic.
Both the CUDA path and the CPU oracle are fed from it.  The paper measured
on the EuroBen reference input sets, which are not available; these
generators stand in for them with the shapes and value distributions of
the workloads the library is benchmarked on.

Generator: counter-based SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Word ``i`` of stream
``(seed, stream)`` is ``mix(key + (i + 1) * GAMMA)`` with
``key = mix(seed * GAMMA ^ (stream + 1) * STREAM_MUL)`` and ``mix`` the
SplitMix64 finaliser; all arithmetic modulo 2^64.  A uniform double in
[0, 1) is the top 53 bits times 2^-53.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
STREAM_MUL = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


_CHUNK = 1 << 21


def _key(seed: int, stream: int):
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        st = np.array([(stream + 1) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix(s * GAMMA ^ st * STREAM_MUL)[0]


def _words_chunk(key, start: int, lo: int, hi: int) -> np.ndarray:
    """Words lo .. hi - 1 (after ``start``) of the stream with this key."""
    with np.errstate(over="ignore"):
        z = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
        z *= GAMMA
        z += key
        t = np.empty_like(z)
        np.right_shift(z, np.uint64(30), out=t)
        z ^= t
        z *= _M1
        np.right_shift(z, np.uint64(27), out=t)
        z ^= t
        z *= _M2
        np.right_shift(z, np.uint64(31), out=t)
        z ^= t
    return z


def _chunked(count: int, fill) -> None:
    """fill(lo, hi) over chunks of [0, count), by a pool of host threads
    (numpy releases the interpreter lock inside its array operations, and
    the output pages are first touched by the thread that fills them).
    Every value depends only on its own counter: the chunking changes
    nothing."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    starts = range(0, count, _CHUNK)
    if count <= _CHUNK:
        for lo in starts:
            fill(lo, min(count, lo + _CHUNK))
        return
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(lambda lo: fill(lo, min(count, lo + _CHUNK)), starts))


def words(seed: int, stream: int, count: int, *, start: int = 0) -> np.ndarray:
    """``count`` 64-bit words of stream (seed, stream), from word ``start``."""
    key = _key(seed, stream)
    out = np.empty(count, dtype=np.uint64)

    def fill(lo, hi):
        out[lo:hi] = _words_chunk(key, start, lo, hi)

    _chunked(count, fill)
    return out


def _unit_of(w: np.ndarray) -> np.ndarray:
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def unit(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of each word times 2^-53."""
    key = _key(seed, stream)
    out = np.empty(count, dtype=np.float64)

    def fill(lo, hi):
        out[lo:hi] = _unit_of(_words_chunk(key, 0, lo, hi))

    _chunked(count, fill)
    return out


def uniform_pm1(seed: int, stream: int, shape) -> np.ndarray:
    """Entries uniform in [-1, 1): 2u - 1 (exact in FP64)."""
    shape = tuple(shape)
    count = int(np.prod(shape))
    key = _key(seed, stream)
    out = np.empty(count, dtype=np.float64)

    def fill(lo, hi):
        out[lo:hi] = 2.0 * _unit_of(_words_chunk(key, 0, lo, hi)) - 1.0

    _chunked(count, fill)
    return out.reshape(shape)


def int_uniform(seed: int, stream: int, shape, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (as float64), word mod (hi - lo + 1)."""
    shape = tuple(shape)
    w = words(seed, stream, int(np.prod(shape)))
    span = np.uint64(hi - lo + 1)
    return ((w % span).astype(np.int64) + lo).astype(np.float64).reshape(shape)


def exp_spread(seed: int, stream: int, shape, emin: int = -20, emax: int = 20) -> np.ndarray:
    """Entries s * u * 2^e: u uniform in [1, 2), s a random sign, e a
    uniform integer in [emin, emax].  u comes from one word, s and e from
    a second word of the same counter (stream + 1000003)."""
    shape = tuple(shape)
    cnt = int(np.prod(shape))
    k1 = _key(seed, stream)
    k2 = _key(seed, stream + 1000003)
    span = np.uint64(emax - emin + 1)
    out = np.empty(cnt, dtype=np.float64)

    def fill(lo, hi):
        u = 1.0 + _unit_of(_words_chunk(k1, 0, lo, hi))
        w2 = _words_chunk(k2, 0, lo, hi)
        sign = np.where((w2 & np.uint64(1)) == 1, -1.0, 1.0)
        e = ((w2 >> np.uint64(1)) % span).astype(np.int64) + emin
        out[lo:hi] = sign * np.ldexp(u, e)

    _chunked(cnt, fill)
    return out.reshape(shape)


def permutation(seed: int, stream: int, n: int) -> np.ndarray:
    """A permutation of range(n): argsort of n random words (stable)."""
    return np.argsort(words(seed, stream, n), kind="stable")


def permutation_matrix(seed: int, stream: int, n: int) -> np.ndarray:
    p = permutation(seed, stream, n)
    P = np.zeros((n, n), dtype=np.float64)
    P[np.arange(n), p] = 1.0
    return P


def logu_dims(seed: int, stream: int, count: int, lo: int = 16, hi: int = 1024) -> np.ndarray:
    """``count`` sizes round(exp(U[ln lo, ln hi]))."""
    u = unit(seed, stream, count)
    v = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return np.clip(np.rint(v), lo, hi).astype(np.int64)


def grouped_problems(seed: int, count: int, lo: int = 16, hi: int = 1024):
    """Sizes (m, k, n) of ``count`` problems, each dimension log-uniform
    in [lo, hi]: m from stream 0, k from stream 1, n from stream 2."""
    m = logu_dims(seed, 0, count, lo, hi)
    k = logu_dims(seed, 1, count, lo, hi)
    n = logu_dims(seed, 2, count, lo, hi)
    return np.stack([m, k, n], axis=1)


def gemm_operands(kind: str, m: int, k: int, n: int, seed: int = 0, cfg: int = 0):
    """A (m x k) and B (k x n) for one workload.

    kind: ``"uniform"`` (U[-1,1)), ``"int8"`` (integers in [-8, 8]),
    ``"spread"`` (s u 2^e, e in [-20, 20]).  A uses stream 2*cfg, B stream
    2*cfg + 1.
    """
    if kind == "uniform":
        return uniform_pm1(seed, 2 * cfg, (m, k)), uniform_pm1(seed, 2 * cfg + 1, (k, n))
    if kind == "int8":
        return (int_uniform(seed, 2 * cfg, (m, k), -8, 8),
                int_uniform(seed, 2 * cfg + 1, (k, n), -8, 8))
    if kind == "spread":
        return exp_spread(seed, 2 * cfg, (m, k)), exp_spread(seed, 2 * cfg + 1, (k, n))
    raise ValueError(f"unknown input kind {kind!r}")


def csr_random(seed: int, stream: int, n: int, fill: float, *, rows_per_block: int = 256):
    """A random n x n sparse matrix in the 3-array CSR form of mod2as
    (Sec. 3.2): entry (i, j) is present when word i*n + j of stream
    (seed, stream) is below ``fill`` as a uniform in [0, 1) (so the fill
    fraction of Table 1 holds in expectation, rows of binomial length);
    values uniform in [-1, 1) from stream + 1, one per present entry in
    row-major order.  Returns (rowp int32[n + 1], indx int32[nnz],
    matvals float64[nnz]), columns increasing within a row."""
    rowp = np.zeros(n + 1, dtype=np.int64)
    cols = []
    for r0 in range(0, n, rows_per_block):
        r1 = min(n, r0 + rows_per_block)
        w = words(seed, stream, (r1 - r0) * n, start=r0 * n)
        u = (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        present = (u < fill).reshape(r1 - r0, n)
        rowp[r0 + 1:r1 + 1] = present.sum(axis=1)
        cols.append(np.nonzero(present)[1])
    rowp = np.cumsum(rowp)
    indx = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    nnz = int(rowp[-1])
    vals = uniform_pm1(seed, stream + 1, (nnz,))
    return rowp.astype(np.int32), indx.astype(np.int32), vals


def csr_sampled(seed: int, stream: int, nrows: int, ncols: int, mean_len: float):
    """A large random sparse matrix in the same CSR form, drawn per value
    rather than per (i, j) cell: row i asks for round(mean_len + sd * z_i)
    columns (z_i standard normal by Box-Muller from stream + 2, sd the
    binomial spread sqrt(mean_len (1 - mean_len / ncols)), clipped to
    [0, ncols]), each column word mod ncols from stream; repeated columns
    in a row are merged, so rows hold distinct increasing columns and
    lengths close to binomial, as in ``csr_random``.  Values uniform in
    [-1, 1) from stream + 1.  Returns (rowp, indx, matvals) like
    ``csr_random``."""
    p = min(1.0, mean_len / max(ncols, 1))
    sd = float(np.sqrt(mean_len * (1.0 - p)))
    u = unit(seed, stream + 2, 2 * nrows).reshape(2, nrows)
    z = np.sqrt(-2.0 * np.log1p(-u[0])) * np.cos(2.0 * np.pi * u[1])
    want = np.clip(np.rint(mean_len + sd * z), 0, ncols).astype(np.int64)
    total = int(want.sum())
    rows = np.repeat(np.arange(nrows, dtype=np.int64), want)
    cols = (words(seed, stream, total) % np.uint64(max(ncols, 1))).astype(np.int64)
    key = np.sort(rows * ncols + cols)
    if len(key):
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    r = key // max(ncols, 1)
    rowp = np.zeros(nrows + 1, dtype=np.int64)
    rowp[1:] = np.cumsum(np.bincount(r, minlength=nrows))
    vals = uniform_pm1(seed, stream + 1, (len(key),))
    return rowp.astype(np.int32), (key % max(ncols, 1)).astype(np.int32), vals


def banded_spd(seed: int, stream: int, n: int, bw: int, shift: float = 1.0):
    """A random symmetric positive definite band matrix in CSR, as the
    conjugate-gradient inputs of Sec. 3.4 (Table 2): ``bw`` diagonals
    (bw odd; h = (bw - 1) / 2 on each side of the main one).  Entry
    (i, i + d), 1 <= d <= h, equals entry (i + d, i) and is word
    i * h + d - 1 of stream (seed, stream) as a uniform in [-1, 1); the
    diagonal entry is ``shift`` + the sum of the row's off-diagonal
    magnitudes, so the matrix is strictly diagonally dominant with a
    positive diagonal (hence SPD, eigenvalues in [shift, shift + 2 * max
    off-diagonal row sum] by Gershgorin; a small shift gives a worse
    conditioned system and more steps).
    Returns (rowp int32[n + 1], indx int32[nnz], matvals float64[nnz])."""
    if bw < 1 or bw % 2 == 0:
        raise ValueError("bw must be odd and positive")
    h = min((bw - 1) // 2, max(n - 1, 0))
    up = uniform_pm1(seed, stream, (max(n * h, 1),))[:n * h].reshape(n, h) if h else \
        np.zeros((n, 0))
    # band[i, h + d] = a(i, i + d) for -h <= d <= h
    band = np.zeros((n, 2 * h + 1))
    for d in range(1, h + 1):
        band[:n - d, h + d] = up[:n - d, d - 1]
        band[d:, h - d] = up[:n - d, d - 1]
    band[:, h] = shift + np.abs(band).sum(axis=1)
    cols = np.arange(n)[:, None] + np.arange(-h, h + 1)[None, :]
    keep = (cols >= 0) & (cols < n)
    rowp = np.zeros(n + 1, dtype=np.int64)
    rowp[1:] = np.cumsum(keep.sum(axis=1))
    return rowp.astype(np.int32), cols[keep].astype(np.int32), band[keep]


# Table 2 of the paper: (n, bw) of the conjugate-gradient runs
CG_TABLE2 = [(128, 3), (128, 31), (128, 63), (256, 3), (256, 31), (256, 63), (256, 127),
             (512, 3), (512, 31), (512, 63), (512, 127), (512, 255), (1024, 3), (1024, 31),
             (1024, 63), (1024, 127), (1024, 255), (1024, 511)]
