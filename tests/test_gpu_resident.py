"""The resident evaluation kernel (fp_resident_*): persistent blocks with a
device work queue in mapped host memory.  Jobs published while the kernel
runs give fp_eval's result bit for bit and meet their value type's bar
against the oracle; the device-side idle wait runs out by design (no fault,
no trap) and the kernel is launched again by the next submission; host-side
waits give up with FP_E_TIMEOUT; oversized and invalid jobs are refused."""
import time

import numpy as np
import pytest

import workloads as W
import paper_1307_5655_gb300 as fpl
from checks import check_any
from test_gpu_batch import _mixed_jobs

pytestmark = pytest.mark.gpu


def _np(out, dtype):
    a = out.cpu().numpy()
    return a.view(np.uint64) if dtype == "modp" else a


@pytest.mark.parametrize("dtype", ["f64", "f32c", "iv64", "modp"])
def test_jobs_published_while_running(dtype):
    import torch
    host = []
    jobs = _mixed_jobs(dtype, 40, {"f64": 11, "f32c": 12, "iv64": 13, "modp": 14}[dtype], host)
    for _, _, out in jobs:
        out.fill_(0)
    torch.cuda.synchronize()  # the resident kernel follows no stream: inputs complete before submitting
    res = fpl.Resident(dtype, max_jobs=256, idle_exit_s=2.0)
    r = W.rng(5)
    tickets = []
    for t, d, out in jobs:
        if d.shape[-1] == 0:
            continue
        tickets.append((res.submit(t, d, out), t, d, out))
        if r.random() < 0.3:
            time.sleep(float(r.uniform(0, 0.002)))  # arrivals while the kernel works
    for tk, _, _, _ in tickets:
        res.wait(tk, 60.0)
    st = res.state()
    assert st["jobs"] == len(tickets)
    res.close()
    for (t, d, out), (e, c, scheme, pts) in zip(jobs, host):
        if d.shape[-1] == 0:
            continue
        alone = fpl.fp_eval(t, dtype, d)
        assert torch.equal(alone.view(torch.uint8), out.view(torch.uint8))
        check_any(dtype, e, c, pts, scheme, _np(out, dtype))


def test_idle_exit_and_relaunch():
    """A short idle time: every block leaves on the device-side timeout (the
    state records it and the kernel is no longer running); the next
    submission launches the kernel again and the job completes."""
    import torch
    e, c, x = W.univariate_case(300, 5000, 71)
    t = fpl.fp_compile(e, c, "B")
    res = fpl.Resident("f64", max_jobs=8, idle_exit_s=0.002)
    time.sleep(0.2)
    st = res.state()
    assert st["idle_exits"] and not st["running"]
    d = torch.from_numpy(x).cuda()
    out = torch.zeros(5000, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    tk = res.submit(t, d, out)
    res.wait(tk, 60.0)
    assert torch.equal(out, fpl.fp_eval(t, "f64", d))
    res.close()


def test_host_wait_times_out_then_completes():
    """A long interval job: a wait of zero seconds gives up with FP_E_TIMEOUT
    and loses nothing; a second wait completes."""
    import torch
    k = 1 << 14
    e = W.dense_univariate_exps(k)
    t = fpl.fp_compile(e, W.uniform_f64(k, 81), "E")
    lo, hi = W.boxes(1, 1 << 19, 82)
    d = torch.from_numpy(np.ascontiguousarray(np.stack([lo, hi], axis=1))).cuda()
    out = torch.zeros((2, 1 << 19), dtype=torch.float64, device="cuda")
    res = fpl.Resident("iv64", max_jobs=4, idle_exit_s=1.0)
    torch.cuda.synchronize()
    tk = res.submit(t, d, out)
    with pytest.raises(fpl.FastPolyError) as ex:
        res.wait(tk, 0.0)
    assert ex.value.code == -8
    res.wait(tk, 120.0)
    assert torch.equal(out, fpl.fp_eval(t, "iv64", d))
    res.close()


def test_refusals():
    import torch
    res = fpl.Resident("f64", max_jobs=2, smem_bytes=4096, idle_exit_s=0.5)
    x = torch.from_numpy(W.points_f64(1, 100, 1)).cuda()
    out = torch.empty(100, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    big = fpl.fp_compile(W.dense_univariate_exps(10007), W.uniform_f64(10007, 2), "B")
    with pytest.raises(fpl.FastPolyError) as ex:  # its table does not fit in 4 KB per block
        res.submit(big, x, out)
    assert ex.value.code == -6
    zero = fpl.fp_compile(W.dense_univariate_exps(3), np.zeros(3), "E")
    with pytest.raises(fpl.FastPolyError):
        res.submit(zero, x, out)
    small = fpl.fp_compile(W.dense_univariate_exps(3), W.uniform_f64(3, 3), "E")
    res.wait(res.submit(small, x, out))
    res.wait(res.submit(small, x, out))
    with pytest.raises(fpl.FastPolyError) as ex:  # the job table (2) is full
        res.submit(small, x, out)
    assert ex.value.code == -6
    res.stop()
    res.close()
    res = fpl.Resident("f64", max_jobs=4, idle_exit_s=0.5)
    res.stop()
    with pytest.raises(fpl.FastPolyError):  # no submissions after a stop
        res.submit(small, x, out)
    res.close()
