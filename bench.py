#!/usr/bin/env python3
"""Benchmark of the FP64-accurate mod2am product C = A.B (Sec. 3.1) on GB300.

One step = one FP64-accurate product (Ozaki split, int8-range digits on
tcgen05, exact windows, FP64 recombination) of m = k = n = 8192 synthetic
matrices with entries s*u*2^e (u in [1,2), e in [-20,20]), through the C ABI
(mxm_f64_emul) with inputs resident in HBM.  value = 2 m n k / t in TFLOP/s
(FP64-equivalent work).  The same line reports the native FP64 product
(mxm_f64) and the 8-bit-digit variant at the same size, the roofline of the
product kernel, the end-to-end figure through mxm_gemm_host (host buffers,
copies inside the timed region), the CPU oracle timed on a bounded sample,
and SM clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica (the products
do not exchange data): weak scaling, value = all ranks' work / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64-accurate GEMM TFLOP/s at n=8192 (Ozaki-INT8 vs native FP64), % roofline"
U = 2.0 ** -53


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--kind", default="spread", choices=["spread", "uniform"])
    p.add_argument("--slices", type=int, default=0, help="0: the tuned choice for the input kind")
    p.add_argument("--native-steps", type=int, default=2)
    p.add_argument("--no-native", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-check", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--suite", nargs="?", const="all",
                   choices=("all", "gemm", "grouped", "spmv", "cg", "fft", "probes"),
                   help="instead of the benchmark line: one JSON line per case of the "
                        "workload suite (FP64 sweep, slice counts and modes, rectangular "
                        "shapes, grouped batch under a CUDA graph; mod2as sparse products; "
                        "conjugate-gradient solves; mod2f transforms)")
    p.add_argument("--only", default="",
                   help="with --suite spmv / cg / fft: run only the rows whose key (case:n, "
                        "cg:n:bw, fft:n) is this string or extends it by ':...', e.g. "
                        "spmv_large:200000, cg:1024, cg:1024:511 or fft:1048576")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def profiled_traffic():
    """DRAM bytes per launch of the product kernel from the committed ncu
    summary, if the kernel sources still hash as they did at capture."""
    import hashlib
    import re
    summary = os.path.join(ROOT, "profiles", "oz_gemm2_n8192_dram.md")
    if not os.path.exists(summary):
        return None
    text = open(summary).read()
    mt = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    mh = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", text)
    if not mt or not mh:
        return None
    h = hashlib.sha256()
    for rel in ("csrc/ozaki.cu", "csrc/ptx.cuh", "csrc/mxm_internal.h"):
        with open(os.path.join(ROOT, "paper_1211_1581_gb300", rel), "rb") as fh:
            h.update(fh.read())
    return int(mt.group(1)) if h.hexdigest() == mh.group(1) else None


def choose_bf16_peak(peaks, clk):
    """The bf16 roofline denominator for the product kernel: the burst
    figure (cuBLAS timed alone, at full clock) when the SM clock sampled in
    the timed region stays within 3 % of its maximum, else the sustained
    figure (cuBLAS in a seconds-long loop, measured at the power cap's
    lower clock).  Returns (peak, key, reason)."""
    burst = peaks["bf16_tflops"]
    sustained = peaks.get("bf16_tflops_sustained", burst)
    mhz, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if mhz and mx and mhz >= 0.97 * mx:
        return burst, "bf16_tflops", (f"burst: SM clock median {mhz:.0f} MHz of max {mx:.0f} "
                                      f"in the timed region (reasons seen: "
                                      f"{', '.join(clk.get('reasons', [])) or 'none'})")
    return sustained, "bf16_tflops_sustained", (
        f"sustained: SM clock median {mhz} MHz below 97 % of max {mx} in the timed region")


def sample_entries(n_rows, n_cols, count, seed):
    """Seeded entries of a result: `count` at random plus the corners of the
    matrix and of the tiles at its middle and its last tile row / column."""
    import numpy as np
    rng = np.random.default_rng(seed)
    ii = list(rng.integers(0, n_rows, count))
    jj = list(rng.integers(0, n_cols, count))
    for r in (0, 127, 128, 255, 256, n_rows // 2, n_rows - 129, n_rows - 128, n_rows - 1):
        for c in (0, 127, 128, n_cols // 2, n_cols - 128, n_cols - 1):
            if 0 <= r < n_rows and 0 <= c < n_cols:
                ii.append(r)
                jj.append(c)
    return np.array(ii, dtype=np.int64), np.array(jj, dtype=np.int64)


def default_slices(kind: str, beta: int) -> int:
    """Smallest slice count meeting 2ku|A||B| at n = 8192 on sampled entries
    of each input kind, found with the oracle on sampled entries."""
    table = {("spread", 7): 7, ("spread", 8): 6, ("uniform", 7): 6, ("uniform", 8): 5}
    return table[(kind, beta)]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names[1:], parts[5:9]):
                    if v.lower() in ("active", "0x1", "1"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [v for v in sm if v >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ distributed
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def _reduce_device():
    """Device of the tensors the collectives reduce: CUDA under NCCL, the
    host under gloo (the CPU multi-process path)."""
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def barrier(world):
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.zeros(1, device=_reduce_device())
        dist.all_reduce(t)


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_operands(kind, n, rank):
    """The problem rank `rank` multiplies: its own seeded n x n pair (stream
    configuration 2 + rank), so replicas share no data and need no exchange;
    rank 0's pair is the single-GPU workload."""
    from paper_1211_1581_gb300 import inputs
    return inputs.gemm_operands(kind, n, n, n, seed=0, cfg=2 + rank)


def aggregate_rate(world, flops_per_step, steps, ms_max):
    """Whole-job throughput in TFLOP/s: every rank runs `steps` independent
    products of `flops_per_step` flops (replicas, weak scaling), and the
    job takes the slowest rank's time `ms_max`."""
    return world * flops_per_step * steps / (ms_max * 1e-3) / 1e12


# ------------------------------------------------------------------ CPU oracle leg
def cpu_oracle_rate(A, B, seconds: float):
    """The oracle's naive FP64 loop (OpenMP over rows, as the paper's OpenMP
    baseline) on a band of rows of the same product, sized to ~`seconds`."""
    import numpy as np

    import oracle
    m, k = A.shape
    n = B.shape[1]
    threads = oracle.num_threads()
    rows = max(1, threads)
    t0 = time.perf_counter()
    oracle.gemm_naive(A[:rows], B)
    t1 = time.perf_counter() - t0
    total_rows = rows
    elapsed = t1
    if t1 < seconds:
        more = int(max(0, (seconds - t1) / max(t1, 1e-6) * rows))
        more = min(more, m - rows)
        more = (more // max(1, threads)) * max(1, threads)
        if more > 0:
            t0 = time.perf_counter()
            oracle.gemm_naive(np.ascontiguousarray(A[rows:rows + more]), B)
            t2 = time.perf_counter() - t0
            total_rows += more
            elapsed += t2
    flops = 2.0 * total_rows * n * k
    return flops / elapsed / 1e12, threads, total_rows, elapsed


# ------------------------------------------------------------------ main legs
def run_ours(args):
    import numpy as np
    import torch

    from paper_1211_1581_gb300 import inputs, mxm

    world, rank, local = dist_setup(args)
    n = args.n
    beta = 7
    S = args.slices or default_slices(args.kind, beta)
    peaks, peak_src = load_peaks()
    mxm.load()

    A_h, B_h = rank_operands(args.kind, n, rank)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        mxm.mxm_gemm(mxm.MODE_EMUL_I8, A, B, C, slices=S, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    st = mxm.mxm_get_device_status()
    if st != mxm.MXM_OK:
        raise RuntimeError(f"device status after warm-up: {mxm.status_string(st)}")

    # ---- timed region (device time, CUDA events on the launching stream)
    mxm.mxm_profile_enable(True)
    mxm.mxm_profile_read()  # reset
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    phase_ms, calls = mxm.mxm_profile_read()
    mxm.mxm_profile_enable(False)
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    flops = 2.0 * n * n * n
    value = aggregate_rate(world, flops, args.steps, ms_total)

    # entries of the last timed result kept for the oracle comparison of the
    # CPU-baseline leg (the oracle runs only there)
    ii, jj = sample_entries(n, n, 1024, seed=8192)
    C_sampled = C[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()

    pairs = S * (S + 1) // 2
    gemm_ms = phase_ms[2] / max(calls, 1)
    achieved = pairs * flops / (gemm_ms * 1e-3) / 1e12
    peak, peak_key, peak_why = choose_bf16_peak(peaks, clk)
    roofline = {"bound": "tensor", "kernel": "oz_gemm2_kernel", "achieved": round(achieved, 1),
                "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "peak_source": f"{peak_key} of {peak_src} (MEASURED_PEAKS.json)",
                "peak_choice": peak_why,
                "frac_of_burst_peak": round(achieved / peaks["bf16_tflops"], 4),
                "frac_of_sustained_peak": round(achieved / peaks["bf16_tflops_sustained"], 4),
                "traffic": profiled_traffic() if (n == 8192 and S == 7) else None,
                "traffic_unit": "bytes per launch (dram read + write, ncu)",
                "algorithmic": f"{pairs} digit-pair products x 2mnk bf16 flops per launch",
                "phase_ms_per_step": {"scale": round(phase_ms[0] / max(calls, 1), 4),
                                      "split": round(phase_ms[1] / max(calls, 1), 4),
                                      "product": round(gemm_ms, 4)}}

    # ---- accuracy of the last timed result, every entry, on the device:
    # against the 12-slice 8-bit-digit split, in units of k u (|A||B|)_ij
    check_all = None
    if not args.no_check and rank == 0:
        from paper_1211_1581_gb300 import tune
        ref, bnd = tune.accuracy_reference(A, B, stream)
        check_all = {"entries": n * n, "max_err_over_ku_AB": tune.error_ratio(C, ref, bnd),
                     "reference": "12-slice 8-bit-digit split of the library (truncation "
                                  "2^-96 below the row and column maxima); |A||B| by the "
                                  "native FP64 product"}
        del ref, bnd
        torch.cuda.empty_cache()

    # ---- other modes at the same size
    modes = {}
    if rank == 0:
        S8 = default_slices(args.kind, 8)
        for name, mode, s_, steps in (("emul_bf16digits", mxm.MODE_EMUL_BF16, S8, args.steps),
                                      ("emul_rn8digits", mxm.MODE_EMUL_RN8, S8, args.steps)):
            for _ in range(2):
                mxm.mxm_gemm(mode, A, B, C, slices=s_)
            torch.cuda.synchronize()
            mxm.mxm_profile_enable(True)
            mxm.mxm_profile_read()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            for _ in range(steps):
                mxm.mxm_gemm(mode, A, B, C, slices=s_)
            a1.record()
            torch.cuda.synchronize()
            ph, c_ = mxm.mxm_profile_read()
            mxm.mxm_profile_enable(False)
            t = a0.elapsed_time(a1) / steps
            p_ = s_ * (s_ + 1) // 2
            gms = ph[2] / max(c_, 1)
            modes[name] = {"slices": s_, "digit_bits": 8,
                           "digits": "balanced, rounded to nearest" if mode == mxm.MODE_EMUL_RN8
                           else "truncated", "ms": round(t, 3),
                           "tflops": round(flops / (t * 1e-3) / 1e12, 2),
                           "product_kernel_frac_of_bf16": round(
                               p_ * flops / (gms * 1e-3) / 1e12 / peak, 4)}
        if not args.no_native:
            probe = None
            try:
                probe = mxm.mxm_peak_probe(1)
            except Exception:
                pass
            mxm.mxm_gemm(mxm.MODE_F64, A, B, C)
            torch.cuda.synchronize()
            mxm.mxm_profile_enable(True)
            mxm.mxm_profile_read()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            for _ in range(args.native_steps):
                mxm.mxm_gemm(mxm.MODE_F64, A, B, C)
            a1.record()
            torch.cuda.synchronize()
            ph, c_ = mxm.mxm_profile_read()
            mxm.mxm_profile_enable(False)
            t = a0.elapsed_time(a1) / args.native_steps
            ach = flops / (t * 1e-3) / 1e12
            gach = flops / (ph[2] / max(c_, 1) * 1e-3) / 1e12
            modes["native_f64"] = {"ms": round(t, 2), "tflops": round(ach, 4),
                                   "dmma_peak_probe_tflops": probe,
                                   "product_kernel_frac_of_probe": (round(gach / probe, 4)
                                                                    if probe else None),
                                   "emul_speedup": round(value / world / ach, 2)}

    # ---- end to end through the public host-buffer call, over the same
    # number of steps as the device-timed line
    e2e = None
    if not args.no_e2e:
        Ap = torch.from_numpy(A_h).pin_memory()
        Bp = torch.from_numpy(B_h).pin_memory()
        Cp = torch.empty((n, n), dtype=torch.float64).pin_memory()
        mxm.mxm_gemm_host(mxm.MODE_EMUL_I8, Ap, Bp, Cp, slices=S)
        e2e_steps = args.steps
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            mxm.mxm_gemm_host(mxm.MODE_EMUL_I8, Ap, Bp, Cp, slices=S)
        t_e2e = time.perf_counter() - t0
        barrier(world)
        t_e2e = max_over_ranks(t_e2e, world)
        e2e = {"value": round(world * flops * e2e_steps / t_e2e / 1e12, 3), "unit": "TFLOP/s",
               "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": n * n * 8,
               "call": "mxm_gemm_host(MXM_MODE_EMUL_I8), pinned host buffers", "steps": e2e_steps,
               "ms_per_step": round(t_e2e / e2e_steps * 1e3, 3)}
        del Ap, Bp, Cp

    # ---- CPU-baseline leg: the oracle on a bounded sample, timed on the
    # host cores; then the oracle's values of the sampled entries of the
    # timed result (Dot2, and the emulation of the same split)
    cpu = None
    check = None
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle
        rate, threads, rows, secs = cpu_oracle_rate(A_h, B_h, args.cpu_seconds)
        cpu = {"value": rate, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
               "sample": f"naive FP64 triple loop (OpenMP over rows) on {rows} of {n} rows "
                         f"of the same product, {secs:.1f} s"}
        # the same loop on one core, as the paper's single-core panels
        oracle.set_threads(1)
        try:
            rate1, _, rows1, secs1 = cpu_oracle_rate(A_h, B_h, args.cpu_seconds / 3)
        finally:
            oracle.set_threads(threads)
        cpu["one_core"] = {"value": rate1, "unit": "TFLOP/s", "cores": 1,
                           "sample": f"{rows1} of {n} rows, {secs1:.1f} s"}
        if not args.no_check:
            d2, ab = oracle.entries_dot2_abs(A_h, B_h, ii, jj)
            emu = oracle.ozaki_entries(A_h, B_h, ii, jj, S=S, beta=beta)
            ratio = np.abs(C_sampled - d2) / (n * U * ab)
            check = {"entries": int(len(ii)), "reference": "oracle: Dot2 (compensated FP64 "
                     "dot product) per entry; |A||B| by the oracle",
                     "max_err_over_ku_AB": float(np.max(ratio)),
                     "bound_over_ku_AB": 2.0,
                     "within_bound": bool(np.all(ratio <= 2.0)),
                     "bit_identical_to_oracle_emulation": int(np.sum(C_sampled == emu)),
                     "sample": "1024 seeded entries of the last timed result, tile corners "
                               "included"}

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms_step, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "precision": f"FP64-accurate (Ozaki split, {S} slices of 7-bit digits, exact "
                             "FP32 windows, FP64 recombination)",
                "data": "synthetic",
                "config": {"workload": f"emulated FP64 GEMM m=k=n={n}, entries s*u*2^e "
                                       "(u in [1,2), e in [-20,20]), Ozaki-INT8",
                           "m": n, "k": n, "n": n, "slices": S, "digit_bits": beta,
                           "inputs": args.kind, "seed": 0,
                           "l2": "inputs larger than L2 (A, B 512 MiB each)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                # per step: column maxima of B, the fused scale + split of A, the
                # split of B, the product (and one memset of the column maxima)
                "gpu_launches": 4 * args.steps, "modes": modes, "check": check,
                "check_all_entries": check_all}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ workload suite
def _timed_ms(fn, reps, stream):
    """Mean device time of ``fn`` over ``reps`` runs after one warm-up run,
    CUDA events on ``stream``."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def run_suite(args):
    """The workload suite: every case prints one JSON line with its time,
    FP64-equivalent TFLOP/s (2mnk/t) and error in units of k u (|A||B|)_ij
    against the 12-slice 8-bit-digit split (all entries)."""
    import numpy as np
    import torch

    from paper_1211_1581_gb300 import inputs, mxm, tune
    torch.cuda.set_device(0)
    mxm.load()
    stream = torch.cuda.current_stream()
    peaks, _ = load_peaks()
    names = {mxm.MODE_F64: "f64", mxm.MODE_EMUL_I8: "emul_i8", mxm.MODE_EMUL_BF16: "emul_bf16",
             mxm.MODE_F32: "f32", mxm.MODE_BF16_F32ACC: "bf16_f32acc", mxm.MODE_EMUL_FP8: "emul_fp8",
             mxm.MODE_EMUL_RN8: "emul_rn8"}

    def emit(**d):
        print(json.dumps(dict(suite=True, **d)), flush=True)

    if args.suite in ("all", "probes"):
        run_probe_suite(emit)
    if args.suite == "probes":
        return
    if args.suite in ("all", "spmv"):
        run_spmv_suite(emit, stream, peaks, args.only)
    if args.suite in ("all", "cg"):
        run_cg_suite(emit, stream, args.only)
    if args.suite in ("all", "fft"):
        run_fft_suite(emit, stream, args.only)
    if args.suite in ("spmv", "cg", "fft"):
        return
    if args.suite == "grouped":
        run_grouped_suite(emit, stream, names)
        return
    dmma = mxm.mxm_peak_probe(1)

    def one(case, kind, m, k, n, runs, reps=3, seed=0, cfg=2, tuned=False):
        A_h, B_h = inputs.gemm_operands(kind, m, k, n, seed=seed, cfg=cfg)
        A = torch.from_numpy(A_h).cuda()
        B = torch.from_numpy(B_h).cuda()
        C = torch.empty((m, n), dtype=torch.float64, device="cuda")
        ref, bnd = tune.accuracy_reference(A, B, stream)
        flops = 2.0 * m * n * k
        for mode, S in runs:
            ms = _timed_ms(lambda: tune._run(mode, S, A, B, C, stream), reps, stream)
            st = mxm.mxm_get_device_status()
            d = {"case": case, "inputs": kind, "m": m, "k": k, "n": n, "mode": names[mode],
                 "slices": S or None, "ms": round(ms, 4),
                 "tflops": round(flops / (ms * 1e-3) / 1e12, 3),
                 "err_over_ku_AB": tune.error_ratio(C, ref, bnd), "status": st}
            if mode == mxm.MODE_F64:
                d["frac_of_dmma_probe"] = round(flops / (ms * 1e-3) / 1e12 / dmma, 4)
            emit(**d)
        if tuned:
            with tempfile.TemporaryDirectory() as td:
                c = tune.tune(A, B, tag=kind, cache=tune.TuneCache(os.path.join(td, "t.json")))
            emit(case=case, inputs=kind, m=m, k=k, n=n, tuner_choice=c.name,
                 slices=c.slices or None, plan=c.plan, ms=round(c.ms, 4),
                 err_over_ku_AB=c.err_ratio)
        del A, B, C, ref, bnd
        torch.cuda.empty_cache()

    # native FP64 sweep (uniform entries), against the measured DMMA rate
    for n in (1024, 2048, 4096, 8192, 16384):
        one("f64_sweep", "uniform", n, n, n, [(mxm.MODE_F64, 0)], reps=3 if n <= 4096 else 1)
    # emulated FP64 per slice count, with the comparison modes beside it
    for n in (4096, 8192):
        runs = ([(mxm.MODE_EMUL_I8, S) for S in range(5, 10)] +
                [(mxm.MODE_EMUL_BF16, S) for S in range(4, 9)] +
                [(mxm.MODE_EMUL_RN8, S) for S in range(4, 8)] +
                [(mxm.MODE_EMUL_FP8, S) for S in range(11, 17)] +
                [(mxm.MODE_F32, 0), (mxm.MODE_BF16_F32ACC, 0), (mxm.MODE_F64, 0)])
        one("emul_slices", "spread", n, n, n, runs, reps=3 if n == 4096 else 2)
    # rectangular shapes, both engines and the tuner's choice
    for (m, k, n) in ((16384, 256, 16384), (128, 65536, 128), (32768, 1024, 64)):
        one("rectangular", "uniform", m, k, n,
            [(mxm.MODE_F64, 0), (mxm.MODE_EMUL_I8, 6), (mxm.MODE_EMUL_BF16, 5)], tuned=True)
    run_grouped_suite(emit, stream, names)


def run_grouped_suite(emit, stream, names):
    """The grouped batch: 2000 problems, m, k, n log-uniform in [16, 1024],
    one launch sequence per mode captured in a CUDA graph and replayed."""
    import numpy as np
    import torch

    from paper_1211_1581_gb300 import inputs, mxm, tune
    dims = [tuple(int(v) for v in d) for d in inputs.grouped_problems(0, 2000)]
    ds = []
    for p, (m, k, n) in enumerate(dims):
        A_h, B_h = inputs.gemm_operands("uniform", m, k, n, seed=0, cfg=100 + p)
        ds.append((torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda(),
                   torch.empty((m, n), dtype=torch.float64, device="cuda")))
    flops = sum(2.0 * m * k * n for m, k, n in dims)
    # one slice count serves the whole call: the tuner's largest need over
    # a sample (the three shortest k, the two longest, eight at random)
    by_k = sorted(range(len(dims)), key=lambda p: dims[p][1])
    rng = np.random.default_rng(6)
    sample = sorted(set(by_k[:3] + by_k[-2:] + list(rng.choice(len(dims), 8, replace=False))))
    s_i8 = tune.grouped_slices([(ds[p][0], ds[p][1]) for p in sample], mxm.MODE_EMUL_I8)
    s_rn8 = tune.grouped_slices([(ds[p][0], ds[p][1]) for p in sample], mxm.MODE_EMUL_RN8)
    table_h = mxm.problem_table(ds)
    table_d = table_h.cuda()
    check = np.random.default_rng(5).choice(len(dims), 24, replace=False)
    refs = [tune.accuracy_reference(ds[p][0], ds[p][1], stream) for p in check]
    for mode, S in ((mxm.MODE_F64, 0), (mxm.MODE_EMUL_I8, s_i8), (mxm.MODE_EMUL_RN8, s_rn8)):
        # the size classes of the emulated call from the grouped tuner
        plan = None
        if mode != mxm.MODE_F64:
            with tempfile.TemporaryDirectory() as td:
                plan = tune.tune_grouped(table_h, table_d, mode, S,
                                         cache=tune.TuneCache(os.path.join(td, "g.json")))
        ws = torch.empty(max(1, mxm.mxm_grouped_workspace_size(table_h, mode, S, plan)),
                         dtype=torch.uint8, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            mxm.mxm_grouped(table_d, mode, S, ws, stream=side, plan=plan)
        ms = _timed_ms(g.replay, 3, stream)
        st = mxm.mxm_get_device_status()
        err = max(tune.error_ratio(ds[p][2], r, b) for p, (r, b) in zip(check, refs))
        emit(case="grouped", inputs="uniform", problems=len(dims), mode=names[mode],
             slices=S or None, slices_from=f"tuner: largest need over {len(sample)} sampled problems" if S else None,
             short_kt=plan.short_kt if plan is not None else None,
             ms=round(ms, 4), tflops=round(flops / (ms * 1e-3) / 1e12, 3),
             err_over_ku_AB_24_checked=err, status=st, graph=True)
        del ws, g


def run_probe_suite(emit, repeats=12, rounds=2):
    """The unit probes behind the roofline denominators the driver does not
    measure (FP64 DFMA and DMMA, legacy IMMA) and tcgen05 BF16 beside them:
    each repeated back to back with SM clocks sampled around the repeats;
    median TFLOP/s and TFLOP/s per GHz."""
    from paper_1211_1581_gb300 import mxm
    names = {0: "fp64_dfma", 1: "fp64_dmma", 4: "imma_s8", 2: "tcgen05_bf16_128x128"}
    for rnd in range(rounds):
        for kind, name in names.items():
            clk = ClockSampler(0)
            clk.start()
            vals = [mxm.mxm_peak_probe(kind) for _ in range(repeats)]
            c = clk.stop()
            v = statistics.median(vals)
            mhz = c.get("sm_mhz")
            emit(case="probe", probe=name, kind=kind, round=rnd, tflops=round(v, 4),
                 spread=[round(min(vals), 4), round(max(vals), 4)], sm_mhz=mhz,
                 reasons=c.get("reasons"),
                 tflops_per_ghz=round(v / (mhz / 1000.0), 4) if mhz else None)


def _selected(key, only):
    """--only: the key itself, or a key that extends it by ':...'."""
    return not only or key == only or key.startswith(only + ":")


# Table 1 of the paper: mod2as orders and fill in percent
SPMV_TABLE1 = [(100, 3.50), (200, 3.75), (256, 5.0), (400, 4.38), (500, 5.00), (512, 4.00),
               (960, 4.50), (1000, 5.00), (1024, 5.50), (2000, 7.50), (4096, 3.50),
               (4992, 4.00), (5000, 4.00), (9984, 4.50), (10000, 5.00), (10240, 5.72)]


def spmv_bytes(nrows, ncols, nnz):
    """Algorithmic bytes of one y = A x in CSR: 8 + 4 per value (matvals,
    indx), 4 per row pointer, 8 per y entry written, x read once."""
    return 12 * nnz + 4 * (nrows + 1) + 8 * nrows + 8 * ncols


def run_spmv_suite(emit, stream, peaks, only=""):
    """mod2as (Sec. 3.2) rows: the Table 1 orders and fills (operands well
    inside L2: repeated calls, L2-warm, as the paper's repeated kernel
    loop), then two matrices of 400-600 MB (larger than L2, cold between
    calls) against the measured HBM copy rate.  The CPU line beside each
    Table 1 case is the storage-order oracle loop, timed on the host."""
    import numpy as np
    import torch

    import oracle
    from paper_1211_1581_gb300 import inputs, mxm

    def dev(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt).cuda()

    hbm = peaks.get("hbm_gbs") if peaks else None
    for n, fill in SPMV_TABLE1 + [(2_000_000, None), (200_000, None)]:
        if not _selected(f"{'spmv_table1' if fill is not None else 'spmv_large'}:{n}", only):
            continue
        if fill is not None:
            rowp, indx, vals = inputs.csr_random(0, 70, n, fill / 100.0)
            case, reps = "spmv_table1", 50
        else:
            mean = 16 if n > 1_000_000 else 250
            rowp, indx, vals = inputs.csr_sampled(2, 95, n, n, mean)
            case, reps = "spmv_large", 10
        x = inputs.uniform_pm1(0, 72, (n,))
        nnz = len(vals)
        dv, di, dr, dx = dev(vals, torch.float64), dev(indx, torch.int32), dev(rowp, torch.int32), \
            dev(x, torch.float64)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        ms = _timed_ms(lambda: mxm.mxm_spmv(dv, di, dr, dx, y, stream=stream), reps, stream)
        st = mxm.mxm_get_device_status()
        gbs = spmv_bytes(n, n, nnz) / (ms * 1e-3) / 1e9
        d = {"case": case, "n": n, "nnz": nnz, "fill_pct": fill, "mode": "spmv_f64",
             "ms": round(ms, 5), "gflops": round(2.0 * nnz / (ms * 1e-3) / 1e9, 2),
             "algorithmic_gbs": round(gbs, 1), "status": st,
             "l2": "warm (operands inside L2)" if fill is not None else "operands larger than L2"}
        if fill is None and hbm:
            d["frac_of_measured_hbm"] = round(gbs / hbm, 3)
        if fill is not None:
            t0 = time.perf_counter()
            k = 0
            while time.perf_counter() - t0 < 0.2 or k < 3:
                oracle.spmv(rowp, indx, vals, x)
                k += 1
            cms = (time.perf_counter() - t0) / k * 1e3
            d["cpu_oracle"] = {"ms": round(cms, 4), "gflops": round(2.0 * nnz / (cms * 1e-3) / 1e9, 3),
                               "cores": oracle.num_threads()}
        emit(**d)
        del dv, di, dr, dx, y
        torch.cuda.empty_cache()


def run_cg_suite(emit, stream, only=""):
    """Conjugate gradients (Sec. 3.4): the Table 2 orders and bandwidths,
    the largest order of the cluster engine and a 10^6 order, each solved
    to r2 <= 1e-24 (b, b) by each engine that takes it (the cluster engine:
    one launch; the graph engine: one graph launch).  Rate in the paper's
    terms: FP64 operations of the steps taken (2 nnz + 10 n per step) over
    the solve time (CUDA events).  The CPU line is the oracle's solve,
    timed on the host."""
    import numpy as np
    import torch

    import oracle
    from paper_1211_1581_gb300 import inputs, mxm

    def dev(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt).cuda()

    for n, bw in inputs.CG_TABLE2 + [(12288, 63), (12288, 511), (1_000_000, 7)]:
        if not _selected(f"cg:{n}:{bw}", only):
            continue
        rowp, indx, vals = inputs.banded_spd(6, 91, n, bw)
        b = inputs.uniform_pm1(6, 92, (n,))
        stop = 1e-24 * float(b @ b)
        dv, di, dr, db = dev(vals, torch.float64), dev(indx, torch.int32), dev(rowp, torch.int32), \
            dev(b, torch.float64)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        it = torch.zeros(1, dtype=torch.int32, device="cuda")
        r2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        work = torch.empty((mxm.load().mxm_cg_workspace_size(n) + 7) // 8, dtype=torch.float64,
                           device="cuda")
        nnz = len(vals)
        d = {"case": "cg", "n": n, "bw": bw, "nnz": nnz}
        engines = [("cluster", mxm.CG_CLUSTER)] if n <= mxm.load().mxm_cg_max_n() else []
        engines.append(("graph", mxm.CG_GRAPH))
        for name, eng in engines:
            ms = _timed_ms(lambda: mxm.mxm_cg(dv, di, dr, db, x, stop, 10 * n, it, r2,
                                              stream=stream, engine=eng, work=work), 20, stream)
            k = int(it.item())
            flops = k * (2.0 * nnz + 10.0 * n)
            d[name] = {"iters": k, "ms": round(ms, 4), "us_per_step": round(ms * 1e3 / max(k, 1), 2),
                       "gflops": round(flops / (ms * 1e-3) / 1e9, 3),
                       "status": mxm.mxm_get_device_status()}
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 0.2 or reps < 2:
            o = oracle.cg(rowp, indx, vals, b, stop, 10 * n)
            reps += 1
        cms = (time.perf_counter() - t0) / reps * 1e3
        d["cpu_oracle"] = {"ms": round(cms, 4), "iters": o["iters"],
                           "gflops": round(o["iters"] * (2.0 * nnz + 10.0 * n) / (cms * 1e-3) / 1e9, 3),
                           "cores": oracle.num_threads()}
        emit(**d)
        del dv, di, dr, db, x, work
        torch.cuda.empty_cache()


def run_fft_suite(emit, stream, only=""):
    """mod2f (Sec. 3.3): the paper's orders 2^8 ... 2^20 and 2^22, complex
    FP64.  Rate in the usual FFT convention, 5 N log2 N flops per transform;
    FP64 instructions issued are about 4 N log2 N (8 per butterfly).  Data
    of 2^20 points and more exceeds the 16 MB that stays in L2 only at
    2^22 (64 MB); smaller orders run from L2 between repeated calls.  The
    CPU line is the oracle's radix-2 recursion, timed on the host."""
    import torch

    import oracle
    from paper_1211_1581_gb300 import inputs, mxm

    for p in list(range(8, 21)) + [22]:
        N = 1 << p
        if not _selected(f"fft:{N}", only):
            continue
        u = inputs.uniform_pm1(0, 150 + p, (2 * N,))
        f = u[0::2] + 1j * u[1::2]
        plan = mxm.FFT(N, stream=stream)
        x = torch.from_numpy(f).cuda()
        out = torch.empty_like(x)
        reps = 50 if N <= (1 << 16) else 10
        ms = _timed_ms(lambda: plan(x, out=out, stream=stream), reps, stream)
        st = mxm.mxm_get_device_status()
        flops = 5.0 * N * p
        d = {"case": "fft", "n": N, "ms": round(ms, 5), "gflops": round(flops / (ms * 1e-3) / 1e9, 2),
             "launches": 1 if N <= 8192 else 2, "status": st}
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 0.2 or k < 2:
            oracle.fft(f)
            k += 1
        cms = (time.perf_counter() - t0) / k * 1e3
        d["cpu_oracle"] = {"ms": round(cms, 4), "gflops": round(flops / (cms * 1e-3) / 1e9, 3),
                           "cores": 1}
        emit(**d)
        del plan, x, out
        torch.cuda.empty_cache()


def run_reference(args):
    """The reference arm: the CPU oracle (the plain definition, naive FP64
    loop with OpenMP over rows) on the host cores; rank 0 only.  A step is
    one bounded band of rows of the same product (the whole 8192^3 product
    would take minutes per step on the host), so ms_per_step is the measured
    time of a band and value the band's 2 rows n k flops over that time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    A_h, B_h = rank_operands(args.kind, n, 0)
    per = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    vals, secs_steps, rows_steps = [], [], []
    threads = 0
    for i in range(args.warmup + args.steps):
        rate, threads, rows, secs = cpu_oracle_rate(A_h, B_h, per)
        if i >= args.warmup:
            vals.append(rate)
            secs_steps.append(secs)
            rows_steps.append(rows)
    total_flops = sum(2.0 * r * n * n for r in rows_steps)
    total_s = sum(secs_steps)
    value = total_flops / total_s / 1e12
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_s / len(secs_steps) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"emulated FP64 GEMM m=k=n={n}, entries s*u*2^e "
                                   "(u in [1,2), e in [-20,20]), Ozaki-INT8",
                       "m": n, "k": n, "n": n, "inputs": args.kind, "seed": 0},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step: the naive FP64 loop on a band of "
                                       f"{min(rows_steps)}-{max(rows_steps)} of {n} rows of the "
                                       f"same product (measured band time; the rate is the "
                                       f"band's work over it, not extrapolated in time)"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.suite:
        run_suite(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
