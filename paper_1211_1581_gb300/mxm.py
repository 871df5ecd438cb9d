"""Python binding of libmxm.so (include/mxm.h), argument marshalling only.

Every function has the name of the C entry point it calls and takes torch
tensors where the C call takes device pointers; streams are
``torch.cuda.Stream`` objects (default: the current stream).  All arithmetic
runs in the library's CUDA kernels.  If the library is missing or cannot be
loaded the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MXM_OK = 0
MXM_ERR_INVALID_ARG = 1
MXM_ERR_ALIGNMENT = 2
MXM_ERR_UNSUPPORTED = 3
MXM_ERR_NONFINITE = 4
MXM_ERR_TIMEOUT = 5
MXM_ERR_CUDA = 6
MXM_ERR_NO_WORKSPACE = 7
MXM_ERR_WORKSPACE_TOO_SMALL = 8
MXM_ERR_BREAKDOWN = 9
CG_AUTO, CG_CLUSTER, CG_GRAPH = 0, 1, 2

MODE_F64 = 0
MODE_EMUL_I8 = 1
MODE_EMUL_BF16 = 2
MODE_F32 = 3
MODE_BF16_F32ACC = 4
MODE_EMUL_FP8 = 5
MODE_EMUL_RN8 = 6



class Plan(ctypes.Structure):
    """mxm_plan: how one product is laid out (see include/mxm.h); all zero
    is the library's own rule."""
    _fields_ = [("raster", ctypes.c_int32), ("kb_order", ctypes.c_int32),
                ("cta", ctypes.c_int32), ("splitk", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class GroupPlan(ctypes.Structure):
    """mxm_group_plan: problems of a grouped emulated call with at most
    ``short_kt`` k-blocks of 128 run on the one-diagonal slice GEMM, the
    others on the diagonal-pair GEMM (-1: the library's default)."""
    _fields_ = [("short_kt", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


# Every symbol include/mxm.h declares, with (restype, argtypes).
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_SZ = ctypes.c_size_t
SIGNATURES = {
    "mxm_version": (_I, []),
    "mxm_status_string": (ctypes.c_char_p, [_I]),
    "mxm_f64": (_I, [_P, _P, _P, _I64, _I64, _I64, _P]),
    "mxm_f64_emul": (_I, [_P, _P, _P, _I64, _I64, _I64, _I, _P]),
    "mxm_gemm": (_I, [_I, _P, _P, _P, _I64, _I64, _I64, _I, _P]),
    "mxm_gemm_plan": (_I, [_I, _P, _P, _P, _I64, _I64, _I64, _I, ctypes.POINTER(Plan), _P]),
    "mxm_workspace_size_plan": (_SZ, [_I, _I64, _I64, _I64, _I, ctypes.POINTER(Plan)]),
    "mxm_gemm_host": (_I, [_I, _P, _P, _P, _I64, _I64, _I64, _I, _P]),
    "mxm_workspace_size": (_SZ, [_I, _I64, _I64, _I64, _I]),
    "mxm_set_workspace": (_I, [_P, _SZ, _P]),
    "mxm_grouped_workspace_size": (_I, [_I64, _P, _I, _I, ctypes.POINTER(_SZ)]),
    "mxm_grouped": (_I, [_I64, _P, _I, _I, _P, _SZ, _P]),
    "mxm_grouped_plan": (_I, [_I64, _P, _I, _I, ctypes.POINTER(GroupPlan), _P, _SZ, _P]),
    "mxm_grouped_workspace_size_plan": (_I, [_I64, _P, _I, _I, ctypes.POINTER(GroupPlan),
                                             ctypes.POINTER(_SZ)]),
    "mxm_get_device_status": (_I, [_P]),
    "mxm_peak_probe": (_I, [_I, ctypes.POINTER(ctypes.c_double)]),
    "mxm_debug_wait_timeout": (_I, [ctypes.c_uint64, _P]),
    "mxm_profile_enable": (_I, [_I]),
    "mxm_profile_read": (_I, [ctypes.POINTER(ctypes.c_double), _I, ctypes.POINTER(_I64)]),
    "mxm_f64_emul_noalloc": (_I, [_P, _P, _P, _I64, _I64, _I64, _I, _P]),
    "mxm_spmv": (_I, [_P, _P, _P, _P, _P, _I64, _I64, _I64, _P]),
    "mxm_cg": (_I, [_P, _P, _P, _P, _P, _I64, _I64, ctypes.c_double, ctypes.c_int32,
                    ctypes.c_int32, _P, _P, _P, _P, _P]),
    "mxm_cg_max_n": (_I64, []),
    "mxm_cg_workspace_size": (_SZ, [_I64]),
    "mxm_fft": (_I, [_P, _P, _P, _P, _I64, _I64, _P]),
    "mxm_fft_twiddles": (_I, [_P, _I64, _P]),
    "mxm_fft_max_n": (_I64, []),
}

_lib = None


class MxmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def library_path() -> str:
    """libmxm.so, or the bounds-checked build when MXM_DEBUG_BOUNDS=1 is set
    in the environment (the process loads one or the other)."""
    return _build.LIB_DEBUG if os.environ.get("MXM_DEBUG_BOUNDS") == "1" else _build.LIB


def load(build_if_missing: bool = True):
    """Load libmxm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing:
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not found at {path}; run build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().mxm_status_string(int(status)).decode()


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _check(st: int, what: str):
    if st != MXM_OK:
        raise MxmError(st, what)


def _operands(A, B, C):
    import torch
    for name, t in (("A", A), ("B", B), ("C", C)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA float64 tensor")
        if t.dim() != 2 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 2-D (row-major) tensor")
    m, k = A.shape
    k2, n = B.shape
    if k != k2 or tuple(C.shape) != (m, n):
        raise ValueError(f"shapes {tuple(A.shape)} x {tuple(B.shape)} -> {tuple(C.shape)}")
    return m, k, n


def mxm_gemm(mode: int, A, B, C, slices: int = 7, stream=None):
    """C = A.B in ``mode`` (see include/mxm.h), asynchronously on ``stream``."""
    m, k, n = _operands(A, B, C)
    st = load().mxm_gemm(int(mode), A.data_ptr(), B.data_ptr(), C.data_ptr(), m, k, n,
                         int(slices), _stream_ptr(stream))
    _check(st, "mxm_gemm")
    return C


def mxm_gemm_plan(mode: int, A, B, C, slices: int = 7, plan: Plan | None = None, stream=None):
    """mxm_gemm under an explicit plan (None: the library's rule)."""
    m, k, n = _operands(A, B, C)
    st = load().mxm_gemm_plan(int(mode), A.data_ptr(), B.data_ptr(), C.data_ptr(), m, k, n,
                              int(slices), ctypes.byref(plan) if plan is not None else None,
                              _stream_ptr(stream))
    _check(st, "mxm_gemm_plan")
    return C


def mxm_workspace_size_plan(mode: int, m: int, k: int, n: int, slices: int = 7,
                            plan: Plan | None = None) -> int:
    return int(load().mxm_workspace_size_plan(int(mode), m, k, n, int(slices),
                                              ctypes.byref(plan) if plan is not None else None))


def mxm_f64(A, B, C, stream=None):
    m, k, n = _operands(A, B, C)
    _check(load().mxm_f64(A.data_ptr(), B.data_ptr(), C.data_ptr(), m, k, n, _stream_ptr(stream)),
           "mxm_f64")
    return C


def mxm_f64_emul(A, B, C, slices: int = 7, stream=None):
    m, k, n = _operands(A, B, C)
    _check(load().mxm_f64_emul(A.data_ptr(), B.data_ptr(), C.data_ptr(), m, k, n, int(slices),
                               _stream_ptr(stream)), "mxm_f64_emul")
    return C


def mxm_f64_emul_noalloc(A, B, C, slices: int = 7, stream=None):
    """mxm_f64_emul with scratch from the library's fixed device array: no
    allocation anywhere (for callers that cannot allocate); products whose
    scratch exceeds the array raise MxmError(MXM_ERR_WORKSPACE_TOO_SMALL)."""
    m, k, n = _operands(A, B, C)
    _check(load().mxm_f64_emul_noalloc(A.data_ptr(), B.data_ptr(), C.data_ptr(), m, k, n,
                                       int(slices), _stream_ptr(stream)), "mxm_f64_emul_noalloc")
    return C


def mxm_gemm_host(mode: int, A, B, C, slices: int = 7, stream=None):
    """Host-buffer form: A, B, C are C-contiguous float64 numpy arrays (or
    CPU tensors, ideally pinned); returns after C holds the result."""
    import numpy as np
    import torch

    def ptr_shape(x):
        if isinstance(x, torch.Tensor):
            if x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
                raise TypeError("host tensors must be contiguous CPU float64")
            return x.data_ptr(), tuple(x.shape)
        if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
            raise TypeError("host arrays must be C-contiguous float64")
        return x.ctypes.data, x.shape

    pa, sa = ptr_shape(A)
    pb, sb = ptr_shape(B)
    pc, sc = ptr_shape(C)
    m, k = sa
    if sb[0] != k or tuple(sc) != (m, sb[1]):
        raise ValueError("shape mismatch")
    _check(load().mxm_gemm_host(int(mode), pa, pb, pc, m, k, sb[1], int(slices),
                                _stream_ptr(stream)), "mxm_gemm_host")
    return C


def mxm_workspace_size(mode: int, m: int, k: int, n: int, slices: int = 7) -> int:
    return int(load().mxm_workspace_size(int(mode), m, k, n, int(slices)))


def mxm_set_workspace(ws=None, stream=None):
    """Use a caller-owned uint8 CUDA tensor as workspace (None: library-owned);
    the switch waits for the work queued on ``stream``."""
    if ws is None:
        _check(load().mxm_set_workspace(None, 0, _stream_ptr(stream)), "mxm_set_workspace")
    else:
        _check(load().mxm_set_workspace(ws.data_ptr(), ws.numel() * ws.element_size(),
                                        _stream_ptr(stream)), "mxm_set_workspace")


def problem_table(problems):
    """Pack [(A, B, C), ...] (CUDA float64 tensors) into the int64 layout of
    ``mxm_problem``: 6 int64 words per problem (A, B, C, m, k, n)."""
    import torch
    rows = []
    for A, B, C in problems:
        m, k, n = _operands(A, B, C)
        rows.append([A.data_ptr(), B.data_ptr(), C.data_ptr(), m, k, n])
    return torch.tensor(rows, dtype=torch.int64).reshape(-1, 6)


def mxm_grouped_workspace_size(table_host, mode: int, slices: int = 7,
                               plan: GroupPlan | None = None) -> int:
    size = ctypes.c_size_t(0)
    t = table_host.contiguous()
    _check(load().mxm_grouped_workspace_size_plan(
        t.shape[0], t.data_ptr(), int(mode), int(slices),
        ctypes.byref(plan) if plan is not None else None, ctypes.byref(size)),
        "mxm_grouped_workspace_size")
    return int(size.value)


def mxm_grouped(table_device, mode: int, slices: int, ws, stream=None,
                plan: GroupPlan | None = None):
    _check(load().mxm_grouped_plan(table_device.shape[0], table_device.data_ptr(), int(mode),
                                   int(slices), ctypes.byref(plan) if plan is not None else None,
                                   ws.data_ptr(), ws.numel() * ws.element_size(),
                                   _stream_ptr(stream)), "mxm_grouped")


def mxm_get_device_status(stream=None) -> int:
    return int(load().mxm_get_device_status(_stream_ptr(stream)))


def mxm_peak_probe(kind: int) -> float:
    out = ctypes.c_double(0.0)
    _check(load().mxm_peak_probe(int(kind), ctypes.byref(out)), "mxm_peak_probe")
    return float(out.value)


def mxm_debug_wait_timeout(limit_ns: int, stream=None):
    _check(load().mxm_debug_wait_timeout(int(limit_ns), _stream_ptr(stream)),
           "mxm_debug_wait_timeout")


def mxm_profile_enable(on: bool = True):
    _check(load().mxm_profile_enable(1 if on else 0), "mxm_profile_enable")


def mxm_profile_read():
    """(ms per phase [scale, split/pack, product], number of calls) since
    the last read."""
    ms = (ctypes.c_double * 3)()
    calls = ctypes.c_int64(0)
    _check(load().mxm_profile_read(ms, 3, ctypes.byref(calls)), "mxm_profile_read")
    return [float(x) for x in ms], int(calls.value)


def mxm_version() -> int:
    return int(load().mxm_version())


def mxm_spmv(matvals, indx, rowp, x, y, stream=None):
    """y = A x for A in CSR (matvals float64, indx and rowp int32; CUDA
    tensors), asynchronously on ``stream`` (mod2as, Sec. 3.2)."""
    import torch
    for name, t, dt in (("matvals", matvals, torch.float64), ("indx", indx, torch.int32),
                        ("rowp", rowp, torch.int32), ("x", x, torch.float64),
                        ("y", y, torch.float64)):
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA {dt} tensor")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 1-D tensor")
    nrows = rowp.shape[0] - 1
    if nrows < 0 or y.shape[0] != nrows or indx.shape[0] != matvals.shape[0]:
        raise ValueError("CSR array lengths do not match")
    _check(load().mxm_spmv(matvals.data_ptr(), indx.data_ptr(), rowp.data_ptr(), x.data_ptr(),
                           y.data_ptr(), nrows, x.shape[0], matvals.shape[0],
                           _stream_ptr(stream)), "mxm_spmv")
    return y


def mxm_cg(matvals, indx, rowp, b, x, stop, max_iters, iters=None, r2=None, r2_hist=None,
           stream=None, engine=CG_AUTO, work=None):
    """Conjugate gradients for A x = b (Sec. 3.4), A SPD in CSR (CUDA
    tensors: matvals float64, indx and rowp int32, b and x float64), the
    loop on the device (``engine``: CG_AUTO, CG_CLUSTER or CG_GRAPH).
    ``iters`` (int32[1]), ``r2`` (float64[1]) and, for the graph engine,
    ``work`` (mxm_cg_workspace_size(n) bytes) are allocated when not given;
    ``r2_hist`` (float64[max_iters]) is optional.  Returns (iters, r2) as
    device tensors; read them after the stream (and check
    mxm_get_device_status for MXM_ERR_BREAKDOWN)."""
    import torch
    for name, t, dt in (("matvals", matvals, torch.float64), ("indx", indx, torch.int32),
                        ("rowp", rowp, torch.int32), ("b", b, torch.float64),
                        ("x", x, torch.float64)):
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA {dt} tensor")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 1-D tensor")
    n = rowp.shape[0] - 1
    if n < 1 or b.shape[0] != n or x.shape[0] != n or indx.shape[0] != matvals.shape[0]:
        raise ValueError("CSR array lengths do not match")
    dev = b.device
    iters = torch.zeros(1, dtype=torch.int32, device=dev) if iters is None else iters
    r2 = torch.zeros(1, dtype=torch.float64, device=dev) if r2 is None else r2
    if work is None and engine != CG_CLUSTER:
        nbytes = load().mxm_cg_workspace_size(n)
        work = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=dev)
    if r2_hist is not None and (r2_hist.dtype != torch.float64 or r2_hist.numel() < max_iters):
        raise ValueError("r2_hist must be a float64 tensor of max_iters entries")
    _check(load().mxm_cg(matvals.data_ptr(), indx.data_ptr(), rowp.data_ptr(), b.data_ptr(),
                         x.data_ptr(), n, matvals.shape[0], float(stop), int(max_iters),
                         int(engine), work.data_ptr() if work is not None else None,
                         iters.data_ptr(), r2.data_ptr(),
                         r2_hist.data_ptr() if r2_hist is not None else None,
                         _stream_ptr(stream)), "mxm_cg")
    return iters, r2


class FFT:
    """The mod2f transform (Sec. 3.3) of order n on the current CUDA device:
    owns the twiddle table (mxm_fft_twiddles, written once) and the work
    array; ``fft(x, out=None)`` runs mxm_fft on a complex128 CUDA tensor of
    n values (``out`` may be ``x``)."""

    def __init__(self, n, stream=None):
        import torch
        if n < 1 or n & (n - 1):
            raise ValueError("n must be a power of two")
        self.n = n
        self.table = torch.empty(max(n // 2, 1) * 2, dtype=torch.float64, device="cuda")
        self.work = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        _check(load().mxm_fft_twiddles(self.table.data_ptr(), n, _stream_ptr(stream)),
               "mxm_fft_twiddles")

    def __call__(self, x, out=None, stream=None):
        import torch
        if not isinstance(x, torch.Tensor) or x.dtype != torch.complex128 or not x.is_cuda:
            raise TypeError("x must be a CUDA complex128 tensor")
        if x.dim() != 1 or x.shape[0] != self.n or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous tensor of {self.n} values")
        out = torch.empty_like(x) if out is None else out
        if out.dtype != torch.complex128 or out.shape != x.shape or not out.is_contiguous():
            raise ValueError("out must match x")
        _check(load().mxm_fft(x.data_ptr(), out.data_ptr(), self.work.data_ptr(),
                              self.table.data_ptr(), self.n, self.n, _stream_ptr(stream)),
               "mxm_fft")
        return out
