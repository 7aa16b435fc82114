"""Argument checks of the Python binding (host logic, no GPU).  A buffer that
would send a kernel or a copy outside its memory -- a CPU tensor where the
library reads device memory, another element type, fewer elements than the
layout needs, a non-contiguous view, another device -- is refused with
ValueError before any CUDA call; the layouts the tests and the benchmark pass
are accepted."""
import numpy as np
import pytest
import torch

import paper_1307_5655_gb300 as fpl
import workloads as W


def _host_tree(nvars, k=10):
    e = W.dense_univariate_exps(k) if nvars == 1 else W.graded_prefix_exps(k, nvars)
    return fpl.fp_compile_host(e, W.uniform_f64(len(e), 1), "E")


def _points(dtype, nvars, npts):
    """Points in the layouts of fp_eval, as the GPU tests build them."""
    if dtype == "iv64":
        lo, hi = W.boxes(nvars, npts, 2)
        return torch.from_numpy(np.ascontiguousarray(np.stack([lo, hi], axis=1)))
    if dtype == "modp":
        return torch.from_numpy(W.points_modp(nvars, npts, 3).view(np.int64))
    x = W.points_f64(nvars, npts, 4)
    return torch.from_numpy(W.to_f32(x) if dtype == "f32c" else x)


def _out(dtype, npts):
    return torch.empty(fpl.out_shape(dtype, npts), dtype=fpl._torch_dtype(dtype))


@pytest.fixture
def as_cuda(monkeypatch):
    """CPU tensors report is_cuda, so the checks' layout logic runs on this
    machine (the checks alone: no library call is made under it)."""
    monkeypatch.setattr(torch.Tensor, "is_cuda", property(lambda self: True), raising=False)


def test_cpu_tensors_are_refused_before_any_cuda_call():
    t = _host_tree(1)
    x = _points("f64", 1, 100)
    o = _out("f64", 100)
    calls = [
        lambda: fpl.fp_eval(t, "f64", x),
        lambda: fpl.fp_eval_ex(t, "f64", x, kernel="ops", ppt=1),
        lambda: fpl.fp_tune(t, "f64", x),
        lambda: fpl.fp_eval_plain_f64(torch.zeros(10, dtype=torch.float64), x),
        lambda: fpl.fp_eval_batch("f64", [(t, x, o)]),
        lambda: fpl.Batch("f64", [(t, x, o)]),
        lambda: fpl.fp_crt(torch.zeros((2, 5), dtype=torch.int64)),
        lambda: fpl.fp_eval_rns(t, _points("modp", 1, 100)),
    ]
    for i, call in enumerate(calls):
        with pytest.raises(ValueError):
            call()
    t.free()


@pytest.mark.parametrize("dtype", ["f64", "f32c", "iv64", "modp"])
def test_layouts_of_fp_eval_are_accepted(dtype, as_cuda):
    for nvars in (1, 2, 3):
        t = _host_tree(nvars)
        for npts in (0, 1, 1000):
            x = _points(dtype, nvars, npts)
            fpl._check_eval_io("fp_eval", t, dtype, x, npts, _out(dtype, npts))
            fpl._check_job("fp_eval_batch", t, dtype, x, _out(dtype, npts))
        t.free()
    # the benchmark's forms: a [1, m] result for one value, a row of a [1, m] tensor
    t = _host_tree(1)
    if dtype == "f64":
        o = torch.empty((1, 50), dtype=torch.float64)
        fpl._check_job("Resident.submit", t, "f64", _points("f64", 1, 50), o)
        fpl._check_eval_io("fp_eval", t, "f64", _points("f64", 1, 50), 50, o[0])
    if dtype == "modp" and hasattr(torch, "uint64"):
        fpl._check_eval_io("fp_eval", t, "modp", _points("modp", 1, 7).view(torch.uint64), 7, _out("modp", 7))
    t.free()


@pytest.mark.parametrize("dtype", ["f64", "f32c", "iv64", "modp"])
def test_layouts_that_would_leave_the_buffers_are_refused(dtype, as_cuda):
    t = _host_tree(2)
    x = _points(dtype, 2, 64)
    o = _out(dtype, 64)
    other = torch.float32 if dtype != "f32c" else torch.float64
    bad = [
        (x.to(other), o),                         # another element type
        (x[:1].contiguous(), o),                  # one variable's row for a bivariate tree
        (x, o.flatten()[:-1].contiguous()),       # one result short
        (x, o.to(other)),                         # result of another element type
    ]
    if x.dim() == 2 and x.shape[1] > 1:
        bad.append((x.t(), o))                    # a non-contiguous view
    for pts, out in bad:
        with pytest.raises(ValueError):
            fpl._check_eval_io("fp_eval", t, dtype, pts, 64, out)
    with pytest.raises(ValueError):               # more points than the buffers hold
        fpl._check_eval_io("fp_eval", t, dtype, x, 65, _out(dtype, 65))
    t.free()


def test_plain_rns_and_crt_extents(as_cuda):
    f64 = fpl._elem_types("f64")
    fpl._check_device("fp_eval_plain_f64", "out", torch.empty(100, dtype=torch.float64), f64, 100)
    with pytest.raises(ValueError):
        fpl._check_device("fp_eval_plain_f64", "out", torch.empty(99, dtype=torch.float64), f64, 100)
    with pytest.raises(ValueError):  # residues are one matrix [k][npts]
        fpl.fp_crt(torch.zeros(10, dtype=torch.int64))
    with pytest.raises(ValueError):  # limbs [npts][k] one short
        fpl.fp_crt(torch.zeros((3, 5), dtype=torch.int64), out=torch.zeros((5, 2), dtype=torch.int64))
    t = fpl.Tree(None, 2, "rns")
    t.rns_k = 3
    with pytest.raises(ValueError):  # [k][nvars][npts] with one variable for a bivariate tree
        fpl.fp_eval_rns(t, torch.zeros((3, 1, 8), dtype=torch.int64))
    with pytest.raises(ValueError):  # [k][npts] results for two of the three primes
        fpl.fp_eval_rns(t, torch.zeros((3, 2, 8), dtype=torch.int64), out=torch.zeros((2, 8), dtype=torch.int64))


def test_host_buffers_of_the_server_and_fp_eval_host():
    """The host forms: numpy arrays (pinned pools sliced and reshaped, uint64
    views of int64 buffers) and CPU tensors are accepted; device tensors,
    short or strided arrays and other element types are refused."""
    t = _host_tree(2)
    pool = np.zeros(4 * 2 * 100, dtype=np.float64)
    fpl._check_host_io("Server.submit", t, "iv64", pool[: 2 * 2 * 100].reshape(2, 2, 100), 100, np.zeros((2, 100)))
    m = np.zeros(2 * 100, dtype=np.int64).view(np.uint64).reshape(2, 100)
    fpl._check_host_io("Server.submit", t, "modp", m, 100, np.zeros(100, dtype=np.uint64))
    fpl._check_host_io("Server.submit", t, "f32c", np.zeros((2, 100), dtype=np.float32),
                       100, torch.zeros((2, 100), dtype=torch.float32))
    bad = [
        ("f64", np.zeros((1, 100)), np.zeros(100)),                  # one variable's row
        ("f64", np.zeros((2, 100)), np.zeros(99)),                    # one result short
        ("f32c", np.zeros((2, 100)), np.zeros((2, 100), np.float32)),  # FP64 points for FP32C
        ("f64", np.zeros((100, 2)).T, np.zeros(100)),                 # not C-contiguous
    ]
    for dt, pts, out in bad:
        with pytest.raises(ValueError):
            fpl._check_host_io("Server.submit", t, dt, pts, 100, out)
    with pytest.raises(ValueError):
        fpl.fp_eval_host(t, "f64", np.zeros((1, 100)))  # refused before the copies
    t.free()
