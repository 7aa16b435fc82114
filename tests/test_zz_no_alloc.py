"""The allocation-free composition entry point (fp_compose_noalloc) against
fp_compose, through the C ABI.

fp_compose_noalloc exists for callers that may not allocate device memory
(a serving engine owning all of HBM, or code where allocation calls are not
allowed): its work space is a fixed region in the library, shared by every
call.  This file is collected last so that a failure here comes after every
other test has run; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
import paper_1307_5655_gb300 as fpl

pytestmark = pytest.mark.gpu


def _dev(a, modp):
    import torch
    a = np.ascontiguousarray(a, dtype=np.uint64 if modp else np.float64)
    return torch.from_numpy(a.view(np.int64) if modp else a).cuda()


def _call(fn, tree, dtype, q, pc, out):
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(tree.handle, fpl.DTYPES[dtype], ctypes.c_void_p(pc.data_ptr()), ctypes.c_void_p(q.data_ptr()),
            q.shape[1] - 1, q.shape[0], ctypes.c_void_p(out.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("dtype,scheme", [("modp", "E"), ("modp", "B"), ("f64", "E"), ("f64", "B")])
def test_noalloc_matches_compose_twice(dtype, scheme):
    import torch
    modp = dtype == "modp"
    degp, degq, npairs = 96, 24, 12
    e = W.dense_univariate_exps(degp + 1)
    t = fpl.fp_compile(e, np.ones(degp + 1, dtype=np.uint64 if modp else np.float64), scheme, modp=modp)
    for call in range(2):  # two calls in a row, with different inputs
        pc, qc = W.composition_case(npairs, degp, degq, 900 + call, dtype)
        q = _dev(qc, modp)
        p = _dev(pc[:, ::-1], modp)
        shape = (npairs, degp * degq + 1)
        ref = torch.empty(shape, dtype=torch.int64 if modp else torch.float64, device="cuda")
        got = torch.full(shape, -1, dtype=ref.dtype, device="cuda")
        assert _call(fpl._lib.fp_compose, t, dtype, q, p, ref) == 0
        assert _call(fpl._lib.fp_compose_noalloc, t, dtype, q, p, got) == 0
        # the same kernels in the same order on the same inputs: bit for bit
        assert np.array_equal(ref.cpu().numpy().view(np.uint8), got.cpu().numpy().view(np.uint8)), call


@pytest.mark.parametrize("dtype", ["modp", "f64"])
def test_noalloc_at_the_limit_of_the_region(dtype):
    """Products longer than 4096 (two-pass transforms and their twiddle
    tables): the largest pair count whose work space (fp_compose_workspace)
    fits the fixed region runs and equals fp_compose bit for bit; one pair
    more is refused with FP_E_TOO_LARGE before anything is written."""
    import torch
    modp = dtype == "modp"
    degp, degq = 128, 64
    e = W.dense_univariate_exps(degp + 1)
    t = fpl.fp_compile(e, np.ones(degp + 1, dtype=np.uint64 if modp else np.float64), "E", modp=modp)
    lo, hi = 1, 4096
    while lo < hi:  # largest npairs that fits
        mid = (lo + hi + 1) // 2
        if fpl.fp_compose_workspace(t, dtype, degq, mid) <= fpl.NOALLOC_SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid - 1
    npairs = lo
    assert fpl.fp_compose_workspace(t, dtype, degq, npairs + 1) > fpl.NOALLOC_SCRATCH_BYTES
    pc, qc = W.composition_case(npairs + 1, degp, degq, 950, dtype)
    q = _dev(qc, modp)
    p = _dev(pc[:, ::-1], modp)
    shape = (npairs + 1, degp * degq + 1)
    tdt = torch.int64 if modp else torch.float64
    untouched = torch.zeros(shape, dtype=tdt, device="cuda")
    assert _call(fpl._lib.fp_compose_noalloc, t, dtype, q, p, untouched) == -6
    assert int((untouched != 0).sum().item()) == 0
    q1, p1 = q[:npairs].contiguous(), p[:npairs].contiguous()
    ref = torch.empty((npairs, shape[1]), dtype=tdt, device="cuda")
    got = torch.full((npairs, shape[1]), -1, dtype=tdt, device="cuda")
    assert _call(fpl._lib.fp_compose, t, dtype, q1, p1, ref) == 0
    assert _call(fpl._lib.fp_compose_noalloc, t, dtype, q1, p1, got) == 0
    assert np.array_equal(ref.cpu().numpy().view(np.uint8), got.cpu().numpy().view(np.uint8))


def test_noalloc_binding_checks_tensors():
    """Tensors of the wrong shape or type never reach the C ABI."""
    import torch
    e = W.dense_univariate_exps(9)
    t = fpl.fp_compile(e, np.ones(9), "E")
    q = torch.ones((3, 5), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        fpl.fp_compose_noalloc(t, "f64", q, out=torch.empty((3, 32), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        fpl.fp_compose_noalloc(t, "f64", q, pcoeffs=torch.ones((3, 8), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        fpl.fp_compose_noalloc(t, "f64", q.to(torch.float32))
    with pytest.raises(ValueError):
        fpl.fp_compose_noalloc(t, "f64", q.t())


def test_noalloc_rejects_oversized_problems():
    import torch
    degp, degq, npairs = 512, 64, 64  # work space far above the fixed region
    e = W.dense_univariate_exps(degp + 1)
    t = fpl.fp_compile(e, np.ones(degp + 1, dtype=np.uint64), "E", modp=True)
    pc, qc = W.composition_case(npairs, degp, degq, 5, "modp")
    out = torch.zeros((npairs, degp * degq + 1), dtype=torch.int64, device="cuda")
    rc = _call(fpl._lib.fp_compose_noalloc, t, "modp", _dev(qc, True), _dev(pc[:, ::-1], True), out)
    assert rc == -6  # FP_E_TOO_LARGE, nothing enqueued
    assert int(out.abs().sum().item()) == 0
