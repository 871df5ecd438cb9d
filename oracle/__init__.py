"""CPU oracle for the mod2am product C = A.B (Sec. 3.1) and its Ozaki-split
FP64-accurate emulation.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU
baseline leg of ``bench.py`` use this module; the CUDA library never does.
It shares no code with the CUDA path.  Everything here is a thin numpy /
ctypes wrapper around ``mxm_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``).

Functions (all take and return numpy arrays, row-major float64):

* ``gemm_naive``   - the definition c_ij = sum_l a_il b_lj, l in order.
* ``gemm_outer``   - the same sum in arbb_mxm2a's rank-1 update order.
* ``gemm_dot2``    - each entry by Dot2 (Ogita-Rump-Oishi 2005): the
  accuracy reference.
* ``gemm_abs``     - |A|.|B|, the scale of the elementwise error bound.
* ``entries_dot2_abs`` - Dot2 and |A|.|B| at selected (i, j) only.
* ``ozaki_split``  - steps 1-2 of the Ozaki split (exponents + digits).
* ``ozaki_gemm`` / ``ozaki_entries`` - the full emulated product.
* ``ozaki_split_rn8`` / ``ozaki_gemm_rn8`` / ``ozaki_entries_rn8`` - the same
  with balanced 8-bit digits (the value rounded once to nearest).
* ``gemm_f32``, ``round_bf16`` - comparison-mode references.
* ``spmv`` / ``spmv_dot2`` / ``spmv_abs`` - mod2as (Sec. 3.2), CSR y = A x
  in storage order, by Dot2, and |A||x|.
* ``cg``           - conjugate gradients (Sec. 3.4, Fig. 6) on a CSR SPD
  matrix, the paper's step order.
* ``dft`` / ``fft`` - mod2f (Sec. 3.3): the DFT of Eq. 1 term by term, and
  the radix-2 decimation-in-frequency recursion of Eqs. 2-3.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mxm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmxm_oracle.so")

OK = 0
INVALID = 1
NONFINITE = 4

_lib = None


def build(force: bool = False) -> str:
    """Compile ``mxm_oracle.c`` into ``oracle/_build/libmxm_oracle.so``."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    if shutil.which(cc) is None:
        raise RuntimeError(f"oracle build needs a C compiler ({cc} not found)")
    base = [cc, "-std=c11", "-O2", "-fno-fast-math", "-ffp-contract=off",
            "-shared", "-fPIC", _SRC, "-lm"]
    tmp = _LIB + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:] + ["-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB)
            return _LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # MXM_ORACLE_LIB points the pins at a deliberately broken copy of the
    # oracle (tests/test_oracle_mutations.py); unset, the real one is built.
    override = os.environ.get("MXM_ORACLE_LIB")
    if override:
        lib = ctypes.CDLL(override)
    else:
        build()
        lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    for name in ("oracle_gemm_naive", "oracle_gemm_outer", "oracle_gemm_dot2",
                 "oracle_gemm_abs", "oracle_gemm_f32"):
        f = getattr(lib, name)
        f.argtypes = [P, P, P, I64, I64, I64]
        f.restype = None
    lib.oracle_entries_dot2_abs.argtypes = [P, P, I64, I64, I64, I64, P, P, P, P]
    lib.oracle_entries_dot2_abs.restype = None
    lib.oracle_ozaki_exponents.argtypes = [P, I64, I64, I, P]
    lib.oracle_ozaki_exponents.restype = I
    lib.oracle_ozaki_split.argtypes = [P, I64, I64, I, I, I, P, P]
    lib.oracle_ozaki_split.restype = I
    lib.oracle_ozaki_gemm.argtypes = [P, P, P, I64, I64, I64, I, I]
    lib.oracle_ozaki_gemm.restype = I
    lib.oracle_ozaki_entries.argtypes = [P, P, I64, I64, I64, I, I, I64, P, P, P]
    lib.oracle_ozaki_entries.restype = I
    lib.oracle_ozaki_split_rn8.argtypes = [P, I64, I64, I, I, P, P]
    lib.oracle_ozaki_split_rn8.restype = I
    lib.oracle_ozaki_gemm_rn8.argtypes = [P, P, P, I64, I64, I64, I]
    lib.oracle_ozaki_gemm_rn8.restype = I
    lib.oracle_ozaki_entries_rn8.argtypes = [P, P, I64, I64, I64, I, I64, P, P, P]
    lib.oracle_ozaki_entries_rn8.restype = I
    lib.oracle_round_bf16.argtypes = [P, P, I64]
    lib.oracle_round_bf16.restype = None
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = I
    lib.oracle_set_threads.argtypes = [I]
    lib.oracle_set_threads.restype = I
    for name in ("oracle_spmv", "oracle_spmv_dot2", "oracle_spmv_abs"):
        f = getattr(lib, name)
        f.argtypes = [P, P, P, P, P, I64, I64, I64]
        f.restype = I
    lib.oracle_cg.argtypes = [P, P, P, P, P, I64, I64, ctypes.c_double, I64, P, P, P]
    lib.oracle_cg.restype = I
    lib.oracle_dft.argtypes = [P, P, I64]
    lib.oracle_dft.restype = None
    lib.oracle_fft_dif.argtypes = [P, P, I64]
    lib.oracle_fft_dif.restype = I
    _lib = lib
    return lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(A, B):
    A = _f64(A)
    B = _f64(B)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError(f"shape mismatch {A.shape} x {B.shape}")
    return A, B, A.shape[0], A.shape[1], B.shape[1]


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's loops from now on; returns the count."""
    return int(_load().oracle_set_threads(int(n)))


def _gemm(name, A, B):
    A, B, m, k, n = _dims(A, B)
    C = np.empty((m, n), dtype=np.float64)
    getattr(_load(), name)(_ptr(A), _ptr(B), _ptr(C), m, k, n)
    return C


def gemm_naive(A, B):
    return _gemm("oracle_gemm_naive", A, B)


def gemm_outer(A, B):
    return _gemm("oracle_gemm_outer", A, B)


def gemm_dot2(A, B):
    return _gemm("oracle_gemm_dot2", A, B)


def gemm_abs(A, B):
    return _gemm("oracle_gemm_abs", A, B)


def entries_dot2_abs(A, B, ii, jj):
    A, B, m, k, n = _dims(A, B)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    if ii.shape != jj.shape:
        raise ValueError("ii and jj differ in shape")
    if ii.size and (ii.min() < 0 or ii.max() >= m or jj.min() < 0 or jj.max() >= n):
        raise ValueError("entry index out of range")
    d2 = np.empty(ii.shape, dtype=np.float64)
    ab = np.empty(ii.shape, dtype=np.float64)
    _load().oracle_entries_dot2_abs(_ptr(A), _ptr(B), m, k, n, ii.size,
                                    _ptr(ii), _ptr(jj), _ptr(d2), _ptr(ab))
    return d2, ab


def ozaki_exponents(X, by_col: bool):
    X = _f64(X)
    r, c = X.shape
    e = np.empty(c if by_col else r, dtype=np.int32)
    st = _load().oracle_ozaki_exponents(_ptr(X), r, c, int(by_col), _ptr(e))
    return e, st


def ozaki_split(X, by_col: bool, beta: int, S: int):
    """Exponents (int32, per row or per column) and digits [S][rows][cols]
    (int16) of X.  Raises on non-finite input."""
    X = _f64(X)
    r, c = X.shape
    e = np.empty(c if by_col else r, dtype=np.int32)
    d = np.empty((S, r, c), dtype=np.int16)
    st = _load().oracle_ozaki_split(_ptr(X), r, c, int(by_col), beta, S, _ptr(e), _ptr(d))
    if st != OK:
        raise FloatingPointError(f"oracle_ozaki_split status {st}")
    return e, d


def ozaki_gemm(A, B, S: int, beta: int = 7):
    A, B, m, k, n = _dims(A, B)
    C = np.empty((m, n), dtype=np.float64)
    st = _load().oracle_ozaki_gemm(_ptr(A), _ptr(B), _ptr(C), m, k, n, S, beta)
    if st != OK:
        raise FloatingPointError(f"oracle_ozaki_gemm status {st}")
    return C


def ozaki_entries(A, B, ii, jj, S: int, beta: int = 7):
    A, B, m, k, n = _dims(A, B)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    if ii.size and (ii.min() < 0 or ii.max() >= m or jj.min() < 0 or jj.max() >= n):
        raise ValueError("entry index out of range")
    out = np.empty(ii.shape, dtype=np.float64)
    st = _load().oracle_ozaki_entries(_ptr(A), _ptr(B), m, k, n, S, beta, ii.size,
                                      _ptr(ii), _ptr(jj), _ptr(out))
    if st != OK:
        raise FloatingPointError(f"oracle_ozaki_entries status {st}")
    return out


def ozaki_split_rn8(X, by_col: bool, S: int):
    """The balanced 8-bit digit split: exponents e + 1 (int32) and digits
    [S][rows][cols] (int16), sum_s d_s 2^(8(S-s)) = round(x 2^(8S - e - 1))."""
    X = _f64(X)
    r, c = X.shape
    e = np.empty(c if by_col else r, dtype=np.int32)
    d = np.empty((S, r, c), dtype=np.int16)
    st = _load().oracle_ozaki_split_rn8(_ptr(X), r, c, int(by_col), S, _ptr(e), _ptr(d))
    if st != OK:
        raise FloatingPointError(f"oracle_ozaki_split_rn8 status {st}")
    return e, d


def ozaki_gemm_rn8(A, B, S: int):
    A, B, m, k, n = _dims(A, B)
    C = np.empty((m, n), dtype=np.float64)
    st = _load().oracle_ozaki_gemm_rn8(_ptr(A), _ptr(B), _ptr(C), m, k, n, S)
    if st != OK:
        raise FloatingPointError(f"oracle_ozaki_gemm_rn8 status {st}")
    return C


def ozaki_entries_rn8(A, B, ii, jj, S: int):
    A, B, m, k, n = _dims(A, B)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    if ii.size and (ii.min() < 0 or ii.max() >= m or jj.min() < 0 or jj.max() >= n):
        raise ValueError("entry index out of range")
    out = np.empty(ii.shape, dtype=np.float64)
    st = _load().oracle_ozaki_entries_rn8(_ptr(A), _ptr(B), m, k, n, S, ii.size, _ptr(ii),
                                          _ptr(jj), _ptr(out))
    if st != OK:
        raise FloatingPointError(f"oracle_ozaki_entries_rn8 status {st}")
    return out


def gemm_f32(A, B):
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("shape mismatch")
    C = np.empty((m, n), dtype=np.float32)
    _load().oracle_gemm_f32(_ptr(A), _ptr(B), _ptr(C), m, k, n)
    return C


def round_bf16(x):
    """bfloat16 bit patterns (uint16) of x rounded to nearest even."""
    x = _f64(x)
    out = np.empty(x.shape, dtype=np.uint16)
    _load().oracle_round_bf16(_ptr(x), _ptr(out), x.size)
    return out


def bf16_to_f64(bits):
    """Values of bfloat16 bit patterns (exact)."""
    b = np.ascontiguousarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)



def _spmv(name, rowp, indx, vals, x, ncols=None):
    rowp = np.ascontiguousarray(rowp, dtype=np.int32)
    indx = np.ascontiguousarray(indx, dtype=np.int32)
    vals = _f64(vals)
    x = _f64(x)
    nrows = rowp.shape[0] - 1
    ncols = x.shape[0] if ncols is None else ncols
    if vals.shape[0] != indx.shape[0] or x.shape[0] != ncols:
        raise ValueError("CSR array lengths do not match")
    y = np.empty(nrows, dtype=np.float64)
    st = getattr(_load(), name)(_ptr(vals), _ptr(indx), _ptr(rowp), _ptr(x), _ptr(y), nrows,
                                ncols, vals.shape[0])
    if st != 0:
        raise ValueError(f"{name}: invalid CSR structure")
    return y


def spmv(rowp, indx, vals, x):
    """y = A x, A in CSR (rowp, indx, matvals), rows in storage order (Sec. 3.2)."""
    return _spmv("oracle_spmv", rowp, indx, vals, x)


def spmv_dot2(rowp, indx, vals, x):
    """y = A x with every row by Dot2 (the accuracy reference)."""
    return _spmv("oracle_spmv_dot2", rowp, indx, vals, x)


def spmv_abs(rowp, indx, vals, x):
    """|A| |x| (the scale of the elementwise error bound)."""
    return _spmv("oracle_spmv_abs", rowp, indx, vals, x)


CG_BREAKDOWN = 9


def cg(rowp, indx, vals, b, stop, max_iters):
    """Conjugate gradients for A x = b (Sec. 3.4, Fig. 6), A SPD in CSR,
    x0 = 0.  Returns a dict: x, iters, r2 (the last (r, r)), hist (r2
    after every step), breakdown (True when (p, A p) <= 0 ended the loop)."""
    rowp = np.ascontiguousarray(rowp, dtype=np.int32)
    indx = np.ascontiguousarray(indx, dtype=np.int32)
    vals = _f64(vals)
    b = _f64(b)
    n = rowp.shape[0] - 1
    if b.shape[0] != n or vals.shape[0] != indx.shape[0]:
        raise ValueError("CSR array lengths do not match")
    x = np.empty(n, dtype=np.float64)
    hist = np.full(int(max_iters) + 1, np.nan)
    it = ctypes.c_int64(0)
    r2 = ctypes.c_double(0.0)
    st = _load().oracle_cg(_ptr(vals), _ptr(indx), _ptr(rowp), _ptr(b), _ptr(x), n,
                           vals.shape[0], float(stop), int(max_iters), ctypes.byref(it),
                           ctypes.byref(r2), _ptr(hist))
    if st not in (0, CG_BREAKDOWN):
        raise ValueError("oracle_cg: invalid CSR structure")
    return {"x": x, "iters": it.value, "r2": r2.value, "hist": hist[:it.value].copy(),
            "breakdown": st == CG_BREAKDOWN}


def _complex_io(f):
    f = np.ascontiguousarray(f, dtype=np.complex128)
    if f.ndim != 1:
        raise ValueError("1-D data expected")
    return f, np.empty_like(f)


def dft(f):
    """F(k) = sum_n f(n) exp(-2 pi i k n / N), term by term (Eq. 1)."""
    f, F = _complex_io(f)
    _load().oracle_dft(_ptr(f), _ptr(F), f.shape[0])
    return F


def fft(f):
    """The same transform by the radix-2 DIF recursion (Eqs. 2-3); N a
    power of two."""
    f, F = _complex_io(f)
    if _load().oracle_fft_dif(_ptr(f), _ptr(F), f.shape[0]) != 0:
        raise ValueError("fft: N must be a power of two")
    return F


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
