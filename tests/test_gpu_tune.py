"""The autotuner and the points-per-thread launch shapes: every count gives
the same result bit for bit within a kernel variant; fp_tune's choice is what
fp_eval then uses, for the tuned tree and for untuned trees of the same shape."""
import numpy as np
import pytest

import workloads as W
import paper_1307_5655_gb300 as fpl
from gpu_util import device_points
from checks import check_f32c, check_f64, check_modp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f64", "f32c", "iv64", "modp"])
@pytest.mark.parametrize("scheme", ["H", "E", "B"])
def test_points_per_thread_do_not_change_results(dtype, scheme):
    import torch
    modp = dtype == "modp"
    k = 1500
    e = W.dense_univariate_exps(k)
    c = W.residues(k, 1) if modp else W.uniform_f64(k, 1)
    t = fpl.fp_compile(e, c, scheme, modp=modp)
    npts = 3000 + 7
    pts = (W.boxes(1, npts, 2) if dtype == "iv64" else
           (W.points_modp(1, npts, 2) if modp else W.points_f64(1, npts, 2)))
    d = device_points(dtype, pts)
    kernels = ["node"] if dtype == "iv64" else ["ops", "node"]
    ppts = [1, 2] if dtype in ("f64", "iv64") else [1, 2, 4]
    for kern in kernels:
        outs = []
        for p in ppts:
            try:
                outs.append(fpl.fp_eval_ex(t, dtype, d, kernel=kern, ppt=p).cpu())
            except fpl.FastPolyError as err:
                assert err.code == -6  # a shape whose tables do not fit
        assert len(outs) >= 1
        for o in outs[1:]:
            assert torch.equal(o.view(torch.uint8), outs[0].view(torch.uint8))


@pytest.mark.parametrize("dtype", ["f64", "f32c", "modp"])
def test_tune_choice_is_used(dtype):
    import torch
    modp = dtype == "modp"
    k = 3000
    e = W.dense_univariate_exps(k)
    c = W.residues(k, 3) if modp else W.uniform_f64(k, 3)
    t = fpl.fp_compile(e, c, "B", modp=modp)
    npts = 1 << 16
    pts = W.points_modp(1, npts, 4) if modp else W.points_f64(1, npts, 4)
    d = device_points(dtype, pts)
    kern, ppt = fpl.fp_tune(t, dtype, d)
    assert kern in ("ops", "node") and ppt in (1, 2, 4)
    a = fpl.fp_eval(t, dtype, d)
    b = fpl.fp_eval_ex(t, dtype, d, kernel=kern, ppt=ppt)
    assert torch.equal(a.view(torch.uint8), b.view(torch.uint8))
    # an untuned tree of the same shape (same bucket) uses the cached choice
    c2 = W.residues(k, 5) if modp else W.uniform_f64(k, 5)
    t2 = fpl.fp_compile(e, c2, "B", modp=modp)
    a2 = fpl.fp_eval(t2, dtype, d)
    b2 = fpl.fp_eval_ex(t2, dtype, d, kernel=kern, ppt=ppt)
    assert torch.equal(a2.view(torch.uint8), b2.view(torch.uint8))


@pytest.mark.parametrize("dtype", ["f64", "f32c", "modp"])
def test_tune_scheme_picks_a_valid_tree(dtype):
    """fp_tune_scheme returns a tuned tree of one of its candidates (k0 a power
    of two up to the first one >= k, or 0 for Balanced) whose result, left in
    `out` and from fp_eval, equals the oracle's (MODP) or meets the bound."""
    import torch
    k = 300
    modp = dtype == "modp"
    e, c, x = W.univariate_case(k, 4096 + 7, 77, "modp" if modp else "f64")
    d = device_points(dtype, x)
    out = torch.empty((4096 + 7,) if dtype != "f32c" else (2, 4096 + 7),
                      dtype=torch.int64 if modp else (torch.float32 if dtype == "f32c" else torch.float64),
                      device="cuda")
    tree, k0 = fpl.fp_tune_scheme(e, c, dtype, d, out=out, modp=modp)
    assert k0 == 0 or ((k0 & (k0 - 1)) == 0 and 1 <= k0 <= 512)
    again = fpl.fp_eval(tree, dtype, d)
    torch.cuda.synchronize()
    assert torch.equal(out, again)
    got = out.cpu().numpy()
    if modp:
        check_modp(e, c, x, got.view(np.uint64))
    elif dtype == "f64":
        check_f64(e, c, x, got)
    else:
        check_f32c(e, c, x, got)
    tree.free()
