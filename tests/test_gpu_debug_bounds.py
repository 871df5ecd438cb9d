"""The bounds-checked build (libmxm_debug.so, -DMXM_DEBUG_BOUNDS): in its
kernels every bulk-copy source is checked against the digit planes or packed
tiles it must come from, every accumulator against the tensor-memory
columns, every running-sum tile against its region and every piece of a
grouped native call against its problem; a failed check is recorded in the
device status word (MXM_ERR_INVALID_ARG), never trapped.  A run of each
kernel family through that build must leave the status clear and give the
same results as the oracle (the checks change nothing else).  The build is
loaded in a child process, since a process loads one of the two libraries."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle
from paper_1211_1581_gb300 import inputs, mxm
assert mxm.library_path().endswith("libmxm_debug.so")
U = 2.0 ** -53

def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()

def product(mode, m, k, n, S, kind="spread", plan=None):
    A, B = inputs.gemm_operands(kind, m, k, n, seed=0, cfg=77)
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    if plan is None:
        mxm.mxm_gemm(mode, dev(A), dev(B), C, slices=S)
    else:
        mxm.mxm_gemm_plan(mode, dev(A), dev(B), C, slices=S, plan=plan)
    torch.cuda.synchronize()
    st = mxm.mxm_get_device_status()
    assert st == mxm.MXM_OK, (mode, m, k, n, mxm.status_string(st))
    got = C.cpu().numpy()
    if mode == mxm.MODE_F64:
        err = np.abs(got - oracle.gemm_dot2(A, B))
        assert np.all(err <= 2 * k * U * oracle.gemm_abs(A, B)), (m, k, n)
    elif mode == mxm.MODE_EMUL_RN8:
        assert np.array_equal(got, oracle.ozaki_gemm_rn8(A, B, S)), (m, k, n)
    else:
        beta = 7 if mode == mxm.MODE_EMUL_I8 else 8
        assert np.array_equal(got, oracle.ozaki_gemm(A, B, S=S, beta=beta)), (m, k, n)

# CTA pairs with an odd tile-row count; single CTAs; split-k; long k with spills
product(mxm.MODE_EMUL_I8, 3 * 128 - 1, 300, 257, 7)
product(mxm.MODE_EMUL_I8, 300, 300, 257, 7, plan=mxm.Plan(2, 2, 1, 0))
product(mxm.MODE_EMUL_I8, 130, 2125, 200, 7)
product(mxm.MODE_EMUL_BF16, 256, 8192, 300, 6)
product(mxm.MODE_EMUL_RN8, 200, 300, 100, 5)
product(mxm.MODE_F64, 300, 200, 257, 0, kind="uniform")
product(mxm.MODE_F64, 128, 4096, 128, 0, kind="uniform")
# grouped: both slice GEMMs (short and long k), and the native pieces
dims = [(1, 1, 1), (17, 5, 33), (129, 65, 131), (300, 200, 257), (16, 1024, 16), (5, 0, 7)]
for mode, S, plan in ((mxm.MODE_EMUL_I8, 6, None), (mxm.MODE_EMUL_I8, 6, mxm.GroupPlan(0)),
                      (mxm.MODE_F64, 0, None)):
    hs, ds = [], []
    for p, (m, k, n) in enumerate(dims):
        A, B = inputs.gemm_operands("spread" if S else "uniform", m, k, n, seed=1, cfg=p)
        hs.append((A, B))
        ds.append((dev(A), dev(B), torch.empty((m, n), dtype=torch.float64, device="cuda")))
    th = mxm.problem_table(ds)
    ws = torch.empty(max(1, mxm.mxm_grouped_workspace_size(th, mode, S, plan)),
                     dtype=torch.uint8, device="cuda")
    mxm.mxm_grouped(th.cuda(), mode, S, ws, plan=plan)
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK, ("grouped", mode, plan)
    for (A, B), (_, _, C) in zip(hs, ds):
        got = C.cpu().numpy()
        if S:
            assert np.array_equal(got, oracle.ozaki_gemm(A, B, S=S, beta=7))
        else:
            k = A.shape[1]
            assert np.all(np.abs(got - oracle.gemm_dot2(A, B)) <= 2 * max(k, 1) * U * oracle.gemm_abs(A, B))
print("debug-bounds ok")
"""


def test_debug_bounds_build_runs_clean():
    env = dict(os.environ, MXM_DEBUG_BOUNDS="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "debug-bounds ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
