"""The sparse, CG and FFT entry points inside a CUDA graph: mxm_spmv,
mxm_fft and the cluster engine of mxm_cg are captured into one graph and
replayed (bit-identical to the eager calls); the graph engine of mxm_cg
refuses a capturing stream with MXM_ERR_UNSUPPORTED and leaves the capture
usable."""
import numpy as np
import pytest

from paper_1211_1581_gb300 import inputs

torch = pytest.importorskip("torch")
from paper_1211_1581_gb300 import mxm  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt).cuda()


def test_capture_and_replay():
    # mod2as operands
    rowp, indx, vals = inputs.csr_random(0, 70, 4096, 0.035)
    x = inputs.uniform_pm1(0, 72, (4096,))
    sv, si, sr, sx = dev(vals, torch.float64), dev(indx, torch.int32), dev(rowp, torch.int32), \
        dev(x, torch.float64)
    y = torch.empty(4096, dtype=torch.float64, device="cuda")
    # CG operands (cluster engine)
    crowp, cindx, cvals = inputs.banded_spd(6, 91, 1024, 63)
    b = inputs.uniform_pm1(6, 92, (1024,))
    cv, ci, cr, cb = dev(cvals, torch.float64), dev(cindx, torch.int32), dev(crowp, torch.int32), \
        dev(b, torch.float64)
    xs = torch.empty(1024, dtype=torch.float64, device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    r2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    stop = 1e-24 * float(b @ b)
    # FFT operands, one-launch and two-pass orders
    plans = {N: mxm.FFT(N) for N in (4096, 1 << 16)}
    fin = {N: dev(inputs.uniform_pm1(0, 300 + N % 97, (2 * N,)).view(np.complex128),
                  torch.complex128) for N in plans}
    fout = {N: torch.empty_like(fin[N]) for N in plans}

    def work(stream):
        mxm.mxm_spmv(sv, si, sr, sx, y, stream=stream)
        mxm.mxm_cg(cv, ci, cr, cb, xs, stop, 10240, it, r2, stream=stream,
                   engine=mxm.CG_CLUSTER)
        for N, plan in plans.items():
            plan(fin[N], out=fout[N], stream=stream)

    torch.cuda.synchronize()
    work(torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    eager = [t.clone() for t in (y, xs, it, r2, *fout.values())]
    for t in (y, xs, r2, *fout.values()):
        t.zero_()
    it.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        work(s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert mxm.mxm_get_device_status() == mxm.MXM_OK
    for a, e in zip((y, xs, it, r2, *fout.values()), eager):
        assert torch.equal(a, e)


def test_graph_engine_refuses_capture():
    rowp, indx, vals = inputs.banded_spd(6, 91, 2048, 7)
    b = inputs.uniform_pm1(6, 92, (2048,))
    cv, ci, cr, cb = dev(vals, torch.float64), dev(indx, torch.int32), dev(rowp, torch.int32), \
        dev(b, torch.float64)
    xs = torch.empty(2048, dtype=torch.float64, device="cuda")
    work = torch.empty((mxm.load().mxm_cg_workspace_size(2048) + 7) // 8, dtype=torch.float64,
                       device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    r2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert mxm.mxm_get_device_status() == mxm.MXM_OK  # the device state exists before capture
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        with pytest.raises(mxm.MxmError) as err:
            mxm.mxm_cg(cv, ci, cr, cb, xs, 0.0, 50, it, r2, stream=s, engine=mxm.CG_GRAPH,
                       work=work)
        xs.fill_(1.0)  # the capture goes on
    assert err.value.status == mxm.MXM_ERR_UNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(xs == 1.0)


def test_set_workspace_refuses_a_capturing_stream():
    """Switching the workspace synchronises its stream, so it is refused while
    that stream is being captured (MXM_ERR_UNSUPPORTED) and the capture goes
    on; the switch itself works outside the capture."""
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    mxm.mxm_set_workspace(ws)
    mxm.mxm_set_workspace(None)
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        with pytest.raises(mxm.MxmError) as err:
            mxm.mxm_set_workspace(ws, stream=s)
        y.fill_(2.0)
    assert err.value.status == mxm.MXM_ERR_UNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(y == 2.0)
