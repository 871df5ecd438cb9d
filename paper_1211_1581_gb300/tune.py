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

After the engine and slice count, ``tune`` chooses the product's layout on
the GPU (``mxm_plan``) by measuring it: the C-tile shape of the slice GEMM
(256 x 128 tiles on CTA pairs, cta_group::2, or 128 x 128 on single CTAs),
the raster group of the persistent tile walk (how many tile-rows the CTAs
working at the same time share), the k-block order, and split-k (none, the
library's rule, or other range counts) for products with few C tiles.  The
search changes one field at a time from the library's rule and keeps a
change only when it is more than 1 % faster and still accurate (for the
emulated engines every plan gives the same bits; the native FP64 product's
rounding depends on split-k, so its error is checked again).  The choice,
plan included, is kept in the cache.  For grouped calls ``tune_grouped``
chooses the size classes: the k (in blocks of 128) up to which problems run
on the one-diagonal slice GEMM rather than the diagonal-pair one.
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


PLAN_FIELDS = ("raster", "kb_order", "cta", "splitk")


@dataclass
class Choice:
    mode: int
    slices: int
    ms: float
    err_ratio: float
    measured: list = field(default_factory=list)  # [mode, slices, err_ratio, ms] per candidate
    plan: dict = field(default_factory=dict)      # mxm_plan fields ({}: the library's rule)
    plan_measured: list = field(default_factory=list)  # [plan, err_ratio, ms] per plan tried

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
        self.save()

    def save(self):
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


def make_plan(plan: dict | None):
    """An mxm.Plan from a dict of its fields (missing fields: 0, the rule)."""
    if not plan:
        return None
    return mxm.Plan(*(int(plan.get(f, 0)) for f in PLAN_FIELDS))


def _run(mode, slices, A, B, C, stream, plan: dict | None = None):
    if plan:
        mxm.mxm_gemm_plan(mode, A, B, C, slices=slices, plan=make_plan(plan), stream=stream)
    elif mode == mxm.MODE_F64:
        mxm.mxm_f64(A, B, C, stream=stream)
    else:
        mxm.mxm_gemm(mode, A, B, C, slices=slices, stream=stream)


def plan_candidates(mode: int, m: int, k: int, n: int) -> dict:
    """Per plan field, the values worth trying for this product (the rule,
    0, first).  CTA pairs need two or more tile-rows of A and bf16 digits;
    split-k is only considered for products with fewer C tiles than SMs."""
    tiles = -(-m // 128) * -(-n // 128)
    emul_bf16 = mode in (mxm.MODE_EMUL_I8, mxm.MODE_EMUL_BF16, mxm.MODE_EMUL_RN8)
    c = {}
    if mode == mxm.MODE_F64:
        c["raster"] = [0, 4, 16]
        kt = -(-k // 16)
        if tiles < 152 and kt >= 16:
            rule = max(1, min(304 // tiles, kt // 8))
            c["splitk"] = [0] + sorted({1, max(2, rule // 2), min(kt, 2 * rule)} - {rule})
        return c
    if emul_bf16 or mode == mxm.MODE_EMUL_FP8:
        c["raster"] = [0, 2, 8]
        c["kb_order"] = [0, 1]
    if emul_bf16:
        if -(-m // 128) >= 2:
            c["cta"] = [0, 1]
        kt = -(-k // 128)
        if tiles < 152 and kt >= 2:
            rule = max(1, min(304 // tiles, kt // 4))
            c["splitk"] = [0] + sorted({1, max(2, rule // 2), min(kt, 2 * rule)} - {rule})
    return c


def select_plan(measure, candidates: dict, tol: float, gain: float = 0.01):
    """Coordinate search over the plan fields: from the rule (every field
    0), try each alternative of one field at a time on top of the best plan
    so far; keep it when it is accurate and more than ``gain`` faster.
    ``measure(plan) -> (err_ratio, ms)``.  Returns (plan, err, ms, tried)."""
    best = {}
    err, ms = measure(best)
    tried = [[dict(best), float(err), float(ms)]]
    for f, values in candidates.items():
        for v in values:
            if v == best.get(f, 0):
                continue
            p = dict(best)
            p[f] = v
            e, t = measure(p)
            tried.append([dict(p), float(e), float(t)])
            if e <= tol and t < ms * (1.0 - gain):
                best, err, ms = p, e, t
    best = {f: v for f, v in best.items() if v != 0}
    return best, float(err), float(ms), tried


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

    def measure(mode, slices, plan=None):
        _run(mode, slices, A, B, C, stream, plan)  # warm-up (and workspace growth)
        times = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _run(mode, slices, A, B, C, stream, plan)
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
         reps: int = 3, stream=None, plans: bool = True) -> Choice:
    """Measure every candidate on A, B (engine and slice count, then the
    plan of the chosen one) and store the choice under (device, tag, size
    class, tol)."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    measure = device_measure(A, B, reps=reps, stream=stream)
    choice = select(measure, tol)
    if plans:
        cands = plan_candidates(choice.mode, m, k, n)
        if cands:
            plan, err, ms, tried = select_plan(
                lambda p: measure(choice.mode, choice.slices, p), cands, tol)
            choice.plan, choice.err_ratio, choice.ms, choice.plan_measured = plan, err, ms, tried
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
    _run(choice.mode, choice.slices, A, B, C, stream, choice.plan)
    return choice


def grouped_key(device: str, tag: str, count: int, mode: int, slices: int) -> str:
    return f"{device}|grouped|{tag}|count={count}|{MODE_NAMES.get(mode, mode)}|S={slices}"


def tune_grouped(table_h, table_d, mode: int, slices: int, tag: str = "default",
                 cache: TuneCache | None = None, candidates=(0, 1, 2, 4, 8), reps: int = 2,
                 stream=None):
    """The size classes of a grouped emulated call: the largest k (in
    blocks of 128) that still runs on the one-diagonal slice GEMM, chosen by
    timing the whole call (every boundary gives the same bits) and cached
    under (device, tag, count, mode, slices).  Returns an mxm.GroupPlan."""
    import torch
    cache = cache if cache is not None else TuneCache()
    key = grouped_key(torch.cuda.get_device_name(table_d.device), tag, table_h.shape[0], mode,
                      slices)
    hit = cache.entries.get(key)
    if hit is not None:
        return mxm.GroupPlan(int(hit["short_kt"]))
    stream = stream or torch.cuda.current_stream()
    kmax = int(table_h[:, 4].max().item()) if table_h.shape[0] else 0
    cands = sorted(set(int(c) for c in candidates) | {-(-kmax // 128)})
    measured = []
    for skt in cands:
        plan = mxm.GroupPlan(skt)
        ws = torch.empty(max(1, mxm.mxm_grouped_workspace_size(table_h, mode, slices, plan)),
                         dtype=torch.uint8, device=table_d.device)
        mxm.mxm_grouped(table_d, mode, slices, ws, stream=stream, plan=plan)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            mxm.mxm_grouped(table_d, mode, slices, ws, stream=stream, plan=plan)
        e1.record(stream)
        e1.synchronize()
        st = mxm.mxm_get_device_status(stream)
        if st != mxm.MXM_OK:
            raise mxm.MxmError(st, "tune_grouped")
        measured.append([skt, e0.elapsed_time(e1) / reps])
        del ws
    best = min(measured, key=lambda r: r[1])
    cache.entries[key] = {"short_kt": best[0], "ms": best[1], "measured": measured}
    cache.save()
    return mxm.GroupPlan(best[0])
