"""Batched evaluation: every job's result in a batch meets its value type's
parity bar against the CPU oracle (tests/checks.py) and equals fp_eval's
result for that job alone (bit for bit: the batch kernel runs the same
per-tile code), for mixed tree sizes, schemes, variable counts and point
counts; and a planned batch replays correctly from a captured CUDA graph."""
import numpy as np
import pytest

import workloads as W
import paper_1307_5655_gb300 as fpl
from checks import check_any
from gpu_util import device_points

pytestmark = pytest.mark.gpu


def _mixed_jobs(dtype, n, seed, host=None):
    """n jobs of mixed shape; when host is a list, (exps, coeffs, scheme,
    host points) of every job are appended to it for the oracle."""
    import torch
    r = W.rng(seed)
    jobs = []
    modp = dtype == "modp"
    for j in range(n):
        nv = 1 if r.random() < 0.6 else int(r.integers(2, 4))
        if nv == 1:
            k = int(np.exp(r.uniform(0, np.log(3000))))
            e = W.dense_univariate_exps(max(1, k))
        else:
            e = W.graded_prefix_exps(int(r.integers(1, 200)), nv)
        scheme = ["D", "H", "E", "B"][int(r.integers(0, 4))] if len(e) < 300 else ["H", "E", "B"][int(r.integers(0, 3))]
        c = W.residues(len(e), seed * 100 + j) if modp else W.uniform_f64(len(e), seed * 100 + j)
        t = fpl.fp_compile(e, c, scheme, modp=modp)
        npts = int(np.exp(r.uniform(0, np.log(5000)))) if r.random() > 0.05 else 0
        if dtype == "iv64":
            pts = W.boxes(nv, npts, seed * 100 + j)
        elif modp:
            pts = W.points_modp(nv, npts, seed * 100 + j)
        else:
            pts = W.points_f64(nv, npts, seed * 100 + j)
        d = device_points(dtype, pts)
        out = torch.empty(fpl.out_shape(dtype, npts), dtype=fpl._torch_dtype(dtype), device="cuda")
        jobs.append((t, d, out))
        if host is not None:
            host.append((e, c, scheme, pts))
    return jobs


@pytest.mark.parametrize("dtype", ["f64", "f32c", "iv64", "modp"])
def test_batch_equals_individual_launches(dtype):
    import torch
    host = []
    jobs = _mixed_jobs(dtype, 40, {"f64": 1, "f32c": 2, "iv64": 3, "modp": 4}[dtype], host)
    for _, _, out in jobs:
        out.fill_(0)
    fpl.fp_eval_batch(dtype, jobs)
    torch.cuda.synchronize()
    for (t, d, out), (e, c, scheme, pts) in zip(jobs, host):
        alone = fpl.fp_eval(t, dtype, d)
        assert torch.equal(alone.view(torch.uint8) if alone.numel() else alone,
                           out.view(torch.uint8) if out.numel() else out)
        if out.numel():
            got = out.cpu().numpy()
            check_any(dtype, e, c, pts, scheme, got.view(np.uint64) if dtype == "modp" else got)


def test_planned_batch_replays_from_cuda_graph():
    import torch
    jobs = _mixed_jobs("f64", 24, 9)
    b = fpl.Batch("f64", jobs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.launch()  # warm (sets kernel attributes before capture)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.launch()
    for _, d, out in jobs:
        out.zero_()
        d.mul_(0.5)  # new inputs in the same buffers
    g.replay()
    torch.cuda.synchronize()
    for t, d, out in jobs:
        assert torch.equal(fpl.fp_eval(t, "f64", d), out)
    b.free()
