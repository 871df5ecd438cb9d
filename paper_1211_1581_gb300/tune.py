"""Choice of engine and slice count for the FP64-accurate product, measured.

Several engines compute C = A.B (Sec. 3.1) to FP64 accuracy: the native
FP64 tensor path (DMMA) and the Ozaki split (Ozaki, Ogita, Oishi, Rump 2012;
integer-slice form of Ootomo, Ozaki, Yokota 2024) with S slices of 7-bit
digits (MODE_EMUL_I8), 8-bit digits (MODE_EMUL_BF16) or balanced 8-bit
digits of the value rounded to nearest (MODE_EMUL_RN8) on the bf16 tensor
pipe, or of 4-bit digits on the FP8 tensor pipe (MODE_EMUL_FP8).  The cost of the split grows as S(S+1)/2 digit products;
the slice count needed for FP64 accuracy depends on the data: a term
a_il b_lj far below the row / column maxima 2^{e_i}, 2^{f_j} loses its low
digits first, so wide exponent spreads need more slices.  Which engine is
fastest depends on the shape and on that slice count.

``tune`` runs every candidate on the caller's operands and keeps the fastest
one whose error stays within ``tol`` times the classical FP64 bound
k u (|A||B|)_ij (u = 2^-53), entry by entry.  The error is taken against the
Ozaki split at 12 slices of 8-bit digits (truncation 2^-96 below the row and
column maxima), computed by the same library; |A||B| by the native FP64
product of |A| and |B|.  Per emulated mode the slice count is scanned
upwards and the scan stops at the first accurate count (more slices only
cost more).  Results are kept in a JSON cache keyed by device, a tag the
caller gives for the kind of data, the power-of-two size class of (m, k, n)
and ``tol``; ``gemm`` looks the choice up and tunes on a miss.

The tile shapes are not tuned: they are fixed by the tensor instructions
(128 x 128 output tiles, the MMA shape of tcgen05 and the TMEM column
budget), and the persistent kernels size their grids to the SM count.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
from dataclasses import asdict, dataclass, field

from . import mxm

U = 2.0 ** -53
REFERENCE = (mxm.MODE_EMUL_BF16, 12)
MODE_NAMES = {mxm.MODE_F64: "f64", mxm.MODE_EMUL_I8: "emul_i8", mxm.MODE_EMUL_BF16: "emul_bf16",
              mxm.MODE_EMUL_FP8: "emul_fp8", mxm.MODE_EMUL_RN8: "emul_rn8"}
MAX_SLICES = {mxm.MODE_EMUL_I8: 12, mxm.MODE_EMUL_BF16: 12, mxm.MODE_EMUL_FP8: 16,
              mxm.MODE_EMUL_RN8: 7}
ENGINES = (mxm.MODE_F64, mxm.MODE_EMUL_I8, mxm.MODE_EMUL_BF16, mxm.MODE_EMUL_FP8,
           mxm.MODE_EMUL_RN8)


@dataclass
class Choice:
    mode: int
    slices: int
    ms: float
    err_ratio: float
    measured: list = field(default_factory=list)  # [mode, slices, err_ratio, ms] per candidate

    @property
    def name(self) -> str:
        return MODE_NAMES.get(self.mode, str(self.mode))


def shape_class(m: int, k: int, n: int) -> str:
    """Power-of-two size class: ceil(log2) of each dimension."""
    return "m{}k{}n{}".format(*(max(0, int(x) - 1).bit_length() for x in (m, k, n)))


def cache_key(device: str, tag: str, m: int, k: int, n: int, tol: float) -> str:
    return f"{device}|{tag}|{shape_class(m, k, n)}|tol={tol:g}"


class TuneCache:
    """A JSON file of choices; written whole through a temporary file and a
    rename, so a reader never sees half a file."""

    def __init__(self, path: str | None = None):
        self.path = path or os.environ.get(
            "MXM_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "mxm_tune.json"))
        self.entries: dict[str, dict] = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                self.entries = json.load(f)

    def get(self, key: str) -> Choice | None:
        e = self.entries.get(key)
        return Choice(**e) if e is not None else None

    def put(self, key: str, choice: Choice):
        self.entries[key] = asdict(choice)
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".mxm_tune.")
        with os.fdopen(fd, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def select(measure, tol: float, modes=ENGINES, max_slices=None) -> Choice:
    """Pick the fastest accurate candidate.

    ``measure(mode, slices) -> (err_ratio, ms)``.  Native FP64 is one
    candidate; each emulated mode is scanned from 1 slice upwards and its
    scan stops at the first count with ``err_ratio <= tol``.  Raises if no
    candidate is accurate."""
    measured = []
    best = None
    for mode in modes:
        top = max_slices if isinstance(max_slices, int) else MAX_SLICES.get(mode, 12)
        counts = [0] if mode == mxm.MODE_F64 else range(1, top + 1)
        for s in counts:
            err, ms = measure(mode, s)
            measured.append([mode, s, float(err), float(ms)])
            if err <= tol:
                if best is None or ms < best[3]:
                    best = measured[-1]
                break
    if best is None:
        raise RuntimeError(f"no candidate within {tol} x k u |A||B|: {measured}")
    return Choice(mode=best[0], slices=best[1], ms=best[3], err_ratio=best[2], measured=measured)


def _run(mode, slices, A, B, C, stream):
    if mode == mxm.MODE_F64:
        mxm.mxm_f64(A, B, C, stream=stream)
    else:
        mxm.mxm_gemm(mode, A, B, C, slices=slices, stream=stream)


def accuracy_reference(A, B, stream=None):
    """(ref, bound): the 12-slice 8-bit-digit split of A.B and the
    classical FP64 bound k u (|A||B|)_ij (|A||B| by the native FP64
    product of |A| and |B|), both on the device."""
    import torch
    stream = stream or torch.cuda.current_stream()
    m, k = A.shape
    n = B.shape[1]
    ref = torch.empty((m, n), dtype=torch.float64, device=A.device)
    _run(REFERENCE[0], REFERENCE[1], A, B, ref, stream)
    absprod = torch.empty_like(ref)
    mxm.mxm_f64(A.abs(), B.abs(), absprod, stream=stream)
    return ref, (max(k, 1) * U) * absprod


def error_ratio(C, ref, bound) -> float:
    """max_ij |C - ref|_ij / bound_ij; where the bound is 0 (an exactly
    zero |A||B| entry) anything but equality is an infinite ratio."""
    diff = (C - ref).abs()
    zero = bound == 0
    if bool((diff[zero] != 0).any()):
        return math.inf
    return (diff[~zero] / bound[~zero]).max().item() if bool((~zero).any()) else 0.0


def device_measure(A, B, reps: int = 3, stream=None):
    """The measuring function ``select`` calls, on the GPU: error ratio
    against the 12-slice 8-bit-digit split, time by CUDA events on
    ``stream`` (median of ``reps`` after one warm-up run)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    ref, bound = accuracy_reference(A, B, stream)
    C = torch.empty_like(ref)

    def measure(mode, slices):
        _run(mode, slices, A, B, C, stream)  # warm-up (and workspace growth)
        times = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _run(mode, slices, A, B, C, stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        st = mxm.mxm_get_device_status(stream)
        if st != mxm.MXM_OK:
            raise mxm.MxmError(st, "tune")
        return error_ratio(C, ref, bound), sorted(times)[len(times) // 2]

    return measure


def grouped_slices(problems, mode: int = mxm.MODE_EMUL_I8, tol: float = 1.0,
                   measure_for=None) -> int:
    """Slice count for one grouped call (a single count serves every
    problem): the largest of the smallest accurate counts of ``problems``
    [(A, B), ...], a sample the caller picks.  Short-k problems need the
    most slices: the truncation error scales with the row / column maxima
    while k u |A||B| shrinks with k.  ``measure_for(A, B)`` builds the
    measuring function (default: ``device_measure`` with one timed run)."""
    measure_for = measure_for or (lambda A, B: device_measure(A, B, reps=1))
    need = 1
    for A, B in problems:
        c = select(measure_for(A, B), tol, modes=(mode,))
        need = max(need, c.slices)
    return need


def tune(A, B, tag: str = "default", tol: float = 1.0, cache: TuneCache | None = None,
         reps: int = 3, stream=None) -> Choice:
    """Measure every candidate on A, B and store the choice under
    (device, tag, size class, tol)."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    choice = select(device_measure(A, B, reps=reps, stream=stream), tol)
    cache = cache if cache is not None else TuneCache()
    cache.put(cache_key(torch.cuda.get_device_name(A.device), tag, m, k, n, tol), choice)
    return choice


def gemm(A, B, C, tag: str = "default", tol: float = 1.0, cache: TuneCache | None = None,
         stream=None) -> Choice:
    """C = A.B with the cached choice for this device, tag and size class;
    on a miss, tune on these operands first."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    cache = cache if cache is not None else TuneCache()
    choice = cache.get(cache_key(torch.cuda.get_device_name(A.device), tag, m, k, n, tol))
    if choice is None:
        choice = tune(A, B, tag=tag, tol=tol, cache=cache, stream=stream)
    _run(choice.mode, choice.slices, A, B, C, stream)
    return choice
