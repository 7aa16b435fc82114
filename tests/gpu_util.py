"""Helpers for the GPU parity tests: move seeded inputs to the device in the
layouts of fp_eval and bring results back as numpy arrays."""
import numpy as np

import paper_1307_5655_gb300 as fpl


def device_points(dtype, pts):
    """pts: f64/f32c/modp -> array [nvars, npts]; iv64 -> (lo, hi) each [nvars, npts]."""
    import torch
    if dtype == "iv64":
        lo, hi = pts
        a = np.ascontiguousarray(np.stack([lo, hi], axis=1))
    elif dtype == "f32c":
        a = np.ascontiguousarray(np.asarray(pts, dtype=np.float32))
    elif dtype == "modp":
        a = np.ascontiguousarray(np.asarray(pts, dtype=np.uint64)).view(np.int64)
    else:
        a = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    return torch.from_numpy(a).cuda()


def run(tree, dtype, pts, stream=None, kernel=None):
    d = device_points(dtype, pts)
    if kernel is None:
        out = fpl.fp_eval(tree, dtype, d, stream=stream).cpu().numpy()
    else:
        out = fpl.fp_eval_ex(tree, dtype, d, kernel=kernel, stream=stream).cpu().numpy()
    if dtype == "modp":
        out = out.view(np.uint64)
    return out
