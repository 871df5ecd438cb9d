"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/mxm.h declares; argument errors are
rejected before any device work.  Runs without a GPU."""
import ctypes
import os
import re
import shutil

import pytest

from paper_1211_1581_gb300 import build as mxm_build
from paper_1211_1581_gb300 import mxm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mxm.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and
                                not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="needs nvcc to build libmxm.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(mxm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mxm_f64", "mxm_f64_emul", "mxm_grouped", "mxm_gemm",
                     "mxm_get_device_status", "mxm_workspace_size", "mxm_set_workspace"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(mxm_build.build())
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in mxm.h but not exported"
    # and the binding knows every one of them
    assert set(declared_functions()) == set(mxm.SIGNATURES)


def test_status_strings_and_version():
    assert mxm.mxm_version() >= 100
    assert mxm.status_string(mxm.MXM_OK) == "MXM_OK"
    assert mxm.status_string(mxm.MXM_ERR_TIMEOUT) == "MXM_ERR_TIMEOUT"
    assert mxm.status_string(99) == "MXM_ERR_UNKNOWN"


def test_argument_errors_need_no_device():
    lib = mxm.load()
    P = ctypes.c_void_p
    fake = P(0x10000)  # never dereferenced: the checks fail first
    assert lib.mxm_gemm(0, fake, fake, fake, -1, 4, 4, 0, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_gemm(0, fake, fake, None, 4, 4, 4, 0, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_gemm(1, fake, fake, fake, 4, 4, 4, 0, None) == mxm.MXM_ERR_UNSUPPORTED
    assert lib.mxm_gemm(1, fake, fake, fake, 4, 4, 4, 13, None) == mxm.MXM_ERR_UNSUPPORTED
    assert lib.mxm_gemm(9, fake, fake, fake, 4, 4, 4, 7, None) == mxm.MXM_ERR_UNSUPPORTED
    assert lib.mxm_gemm(0, P(0x10004), fake, P(0x20000), 4, 4, 4, 0, None) == mxm.MXM_ERR_ALIGNMENT
    # C overlapping A
    assert lib.mxm_gemm(0, P(0x10000), P(0x90000), P(0x10008), 4, 4, 4, 0, None) == \
        mxm.MXM_ERR_INVALID_ARG
    # empty products are no-ops
    assert lib.mxm_gemm(0, None, None, None, 0, 5, 5, 0, None) == mxm.MXM_OK
    assert lib.mxm_f64(None, None, None, 5, 5, 0, None) == mxm.MXM_OK
    assert lib.mxm_f64_emul(fake, fake, fake, 4, 4, 4, 0, None) == mxm.MXM_ERR_UNSUPPORTED


def test_noalloc_size_limits_need_no_device():
    """Sizes beyond 2^31 are refused before any byte count is formed (their
    products would wrap around in 64 bits), as by mxm_f64_emul; nothing is
    launched."""
    lib = mxm.load()
    P = ctypes.c_void_p
    a, b, c = P(0x100000), P(0x200000), P(0x300000)
    for m, k, n in ((1 << 61, 1, 1), (1, 1 << 40, 1), (1, 1, (1 << 31) + 1)):
        assert lib.mxm_f64_emul_noalloc(a, b, c, m, k, n, 7, None) == mxm.MXM_ERR_UNSUPPORTED
        assert lib.mxm_f64_emul(a, b, c, m, k, n, 7, None) == mxm.MXM_ERR_UNSUPPORTED
    assert lib.mxm_f64_emul_noalloc(a, b, c, -1, 4, 4, 7, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_f64_emul_noalloc(a, b, c, 4, 4, 4, 13, None) == mxm.MXM_ERR_UNSUPPORTED
    assert lib.mxm_f64_emul_noalloc(P(0x100004), b, c, 4, 4, 4, 7, None) == mxm.MXM_ERR_ALIGNMENT
    assert lib.mxm_f64_emul_noalloc(a, b, P(0x100008), 4, 4, 4, 7, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_f64_emul_noalloc(None, None, None, 0, 4, 4, 7, None) == mxm.MXM_OK


def test_workspace_size_is_host_arithmetic():
    # FP64: zero-padded 128x16 tiles of A and B
    assert mxm.mxm_workspace_size(0, 128, 16, 128) == 2 * 128 * 16 * 8
    assert mxm.mxm_workspace_size(0, 0, 16, 128) == 0
    # emulated: exponents + S slices of 128x128 bf16 tiles of A and of B^T
    # (Mt = 2, Nt = 1, Kt = 1) + a 128x128 FP64 running-sum tile per C tile
    ws = mxm.mxm_workspace_size(1, 256, 128, 128, 7)
    tiles = 7 * (2 * 1 + 1 * 1)
    sums = 2 * 128 * 128 * 8
    assert ws >= tiles * 128 * 128 * 2 + sums
    assert ws < tiles * 128 * 128 * 2 + sums + 8 * 1024
    assert mxm.mxm_workspace_size(1, 256, 128, 128, 0) == 0


def test_fp8_workspace_size_and_slices():
    # E4M3 digit tiles are 16 KiB: S slices x (2 A tiles + 1 B tile) + sums
    ws = mxm.mxm_workspace_size(5, 256, 128, 128, 16)
    planes = 16 * (2 + 1) * 128 * 128
    sums = 2 * 128 * 128 * 8
    assert planes + sums <= ws < planes + sums + 8 * 1024
    assert mxm.mxm_workspace_size(5, 256, 128, 128, 17) == 0
    assert mxm.mxm_workspace_size(5, 256, 128, 128, 0) == 0


def test_splitk_workspace_size():
    """Products with fewer C tiles than half the 304 split-k units cut k
    into ranges (FP64: at least 8 k-blocks of 16 each; emulated: at least 4
    k-blocks of 128) and add room for the partial tiles."""
    # FP64, m = n = 128, k = 65536: 1 tile, Kt = 4096 -> 304 ranges
    packs = 2 * 4096 * 128 * 16 * 8
    assert mxm.mxm_workspace_size(0, 128, 65536, 128) == packs + 304 * 128 * 128 * 8
    # FP64 with 152 or more tiles is not split
    assert mxm.mxm_workspace_size(0, 152 * 128, 1024, 128) == (152 + 1) * 64 * 128 * 16 * 8
    # emulated, S = 6, m = n = 128, k = 65536: Kt = 512 -> 128 ranges, each
    # holding S diagonals' int64 128 x 128 partials
    ws = mxm.mxm_workspace_size(1, 128, 65536, 128, 6)
    planes = 6 * 2 * 512 * 128 * 128 * 2
    partials = 128 * 6 * 128 * 128 * 8
    assert planes + partials <= ws < planes + partials + 8 * 1024


def test_grouped_workspace_size_on_host():
    import numpy as np
    rows = np.array([[0, 0, 0, 128, 64, 128], [0, 0, 0, 129, 65, 1], [0, 0, 0, 0, 5, 5]],
                    dtype=np.int64)
    lib = mxm.load()
    size = ctypes.c_size_t(0)
    st = lib.mxm_grouped_workspace_size(3, rows.ctypes.data, 1, 7, ctypes.byref(size))
    assert st == mxm.MXM_OK
    # A tiles: 1*1 + 2*1 ; B tiles: 1*1 + 1*1 ; 7 planes of 32 KiB tiles; the
    # spill areas of up to 256 CTAs of the diagonal-pair GEMM (2 x 128 x 128 x
    # 8 bytes each); no running sums: both problems are short-k (one k-block)
    fixed = 7 * (3 + 2) * 32768 + 256 * 2 * 128 * 128 * 8
    assert fixed <= size.value < fixed + 16 * 1024
    # with every problem on the diagonal-pair GEMM (short_kt = 0): the
    # running sums of the 3 C tiles (128 x 128 x 8 bytes each) as well
    plan = mxm.GroupPlan(0)
    st = lib.mxm_grouped_workspace_size_plan(3, rows.ctypes.data, 1, 7, ctypes.byref(plan),
                                             ctypes.byref(size))
    assert st == mxm.MXM_OK
    assert fixed + 3 * 128 * 128 * 8 <= size.value < fixed + 3 * 128 * 128 * 8 + 16 * 1024
    bad_plan = mxm.GroupPlan(-2)
    assert lib.mxm_grouped_workspace_size_plan(3, rows.ctypes.data, 1, 7, ctypes.byref(bad_plan),
                                               ctypes.byref(size)) == mxm.MXM_ERR_INVALID_ARG
    # native: the plan only (the operands are read in place): a 256-byte
    # header and one record per problem, rounded to 1 KiB
    st = lib.mxm_grouped_workspace_size(3, rows.ctypes.data, 0, 0, ctypes.byref(size))
    assert st == mxm.MXM_OK and size.value == 1024
    bad = rows.copy()
    bad[0, 3] = -1
    assert lib.mxm_grouped_workspace_size(3, bad.ctypes.data, 1, 7, ctypes.byref(size)) == \
        mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_grouped_workspace_size(3, rows.ctypes.data, 3, 7, ctypes.byref(size)) == \
        mxm.MXM_ERR_UNSUPPORTED
    assert lib.mxm_grouped(0, None, 1, 7, None, 0, None) == mxm.MXM_OK
    assert lib.mxm_grouped(4, ctypes.c_void_p(0x1000), 1, 7, ctypes.c_void_p(0x10000), 16, None) == \
        mxm.MXM_ERR_WORKSPACE_TOO_SMALL


def test_spmv_argument_errors_on_host():
    lib = mxm.load()
    P = ctypes.c_void_p
    fake = P(0x10000)
    assert lib.mxm_spmv(fake, fake, fake, fake, fake, -1, 4, 4, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_spmv(fake, fake, fake, fake, fake, 0, 4, 4, None) == mxm.MXM_OK
    assert lib.mxm_spmv(fake, fake, None, fake, fake, 4, 4, 4, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_spmv(P(0x10004), fake, fake, fake, fake, 4, 4, 4, None) == mxm.MXM_ERR_ALIGNMENT
    assert lib.mxm_spmv(fake, P(0x10002), fake, fake, fake, 4, 4, 4, None) == mxm.MXM_ERR_ALIGNMENT
    assert lib.mxm_spmv(fake, fake, fake, fake, fake, 1 << 32, 4, 4, None) == \
        mxm.MXM_ERR_UNSUPPORTED


def test_cg_argument_errors_on_host():
    lib = mxm.load()
    P = ctypes.c_void_p
    f = P(0x10000)
    x = P(0x30000)
    b = P(0x40000)
    it = P(0x50000)
    r2 = P(0x60000)
    w = P(0x1000000)

    def call(n=8, nnz=8, vals=f, indx=P(0x70000), rowp=P(0x80000), bb=b, xx=x, iters=it, rr=r2,
             hist=None, max_iters=5, engine=mxm.CG_CLUSTER, work=None):
        return lib.mxm_cg(vals, indx, rowp, bb, xx, n, nnz, 0.0, max_iters, engine, work, iters,
                          rr, hist, None)

    assert lib.mxm_cg_max_n() >= 1024
    assert lib.mxm_cg_workspace_size(1000) >= 3 * 1000 * 8 and lib.mxm_cg_workspace_size(0) == 0
    assert call(n=0) == mxm.MXM_ERR_INVALID_ARG
    assert call(n=-1) == mxm.MXM_ERR_INVALID_ARG
    assert call(max_iters=-1) == mxm.MXM_ERR_INVALID_ARG
    assert call(engine=3) == mxm.MXM_ERR_INVALID_ARG
    assert call(n=lib.mxm_cg_max_n() + 1) == mxm.MXM_ERR_UNSUPPORTED
    assert call(engine=mxm.CG_GRAPH) == mxm.MXM_ERR_INVALID_ARG               # no work
    assert call(iters=None) == mxm.MXM_ERR_INVALID_ARG
    assert call(rr=None) == mxm.MXM_ERR_INVALID_ARG
    assert call(xx=P(0x30004)) == mxm.MXM_ERR_ALIGNMENT
    assert call(iters=P(0x50002)) == mxm.MXM_ERR_ALIGNMENT
    assert call(engine=mxm.CG_GRAPH, work=P(0x1000004)) == mxm.MXM_ERR_ALIGNMENT
    assert call(xx=P(0x40000 + 8)) == mxm.MXM_ERR_INVALID_ARG    # x overlaps b
    assert call(xx=f) == mxm.MXM_ERR_INVALID_ARG                 # x aliases the values
    assert call(engine=mxm.CG_GRAPH, work=P(0x30000)) == mxm.MXM_ERR_INVALID_ARG  # work on x
    assert call(engine=mxm.CG_GRAPH, work=P(0x40000)) == mxm.MXM_ERR_INVALID_ARG  # work on b
    assert mxm.load().mxm_status_string(mxm.MXM_ERR_BREAKDOWN) == b"MXM_ERR_BREAKDOWN"


def test_fft_argument_errors_on_host():
    lib = mxm.load()
    P = ctypes.c_void_p
    a, w, t = P(0x100000), P(0x200000), P(0x300000)
    assert lib.mxm_fft_max_n() == 1 << 22
    assert lib.mxm_fft(a, a, w, t, 64, 48, None) == mxm.MXM_ERR_INVALID_ARG      # not 2^p
    assert lib.mxm_fft(a, a, w, t, 64, 0, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft(a, a, w, t, 32, 64, None) == mxm.MXM_ERR_INVALID_ARG      # table too small
    assert lib.mxm_fft(a, a, w, t, 96, 64, None) == mxm.MXM_ERR_INVALID_ARG      # table not 2^p
    assert lib.mxm_fft(a, a, w, None, 64, 64, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft(None, a, w, t, 64, 64, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft(a, a, None, t, 4096, 4096, None) == mxm.MXM_ERR_INVALID_ARG  # two passes
    assert lib.mxm_fft(a, a, P(0x100000 + 4096 * 8), t, 4096, 4096, None) == \
        mxm.MXM_ERR_INVALID_ARG                                                     # work overlaps
    assert lib.mxm_fft(P(0x100008), P(0x100008), w, t, 64, 64, None) == mxm.MXM_ERR_ALIGNMENT
    assert lib.mxm_fft(a, P(0x100000 + 16), w, t, 64, 64, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft_twiddles(t, 48, None) == mxm.MXM_ERR_INVALID_ARG
    assert lib.mxm_fft_twiddles(t, 1, None) == mxm.MXM_OK
    assert lib.mxm_fft_twiddles(P(0x300008), 64, None) == mxm.MXM_ERR_ALIGNMENT
