"""Parity bars shared by the GPU tests: the CUDA path's results against the
CPU oracle on the same seeded inputs.

  MODP   bit-exact against the plain sum mod p.
  IV64   bit-exact (both bounds) against the oracle's directed-rounding walk
         on the oracle's own tree.
  FP64   |gpu - oracle| <= (4k + g) u S, S = sum |c_e x^e|, u = 2^-53,
         4k u S the stated bound of the GPU path, g u S the oracle's own
         bound (g = max total degree + nvars + k).
  FP32C  inputs rounded to float; |hi + lo - oracle| <= 2 gamma_{2k+64}(2^-24)^2 S
         + g u S, and the median error below k 2^-48 S.
"""
import numpy as np

import oracle as O
import workloads as W

U = 2.0 ** -53
U32 = 2.0 ** -24


def g32(k):
    return k * U32 / (1 - k * U32)


def check_f64(e, c, x, got):
    want, S = O.eval_f64(e, c, x)
    k = len(e)
    g = int(np.asarray(e).sum(axis=1).max()) + np.asarray(e).shape[1] + k
    tol = (4 * k + g) * U * S
    bad = np.abs(got - want) > tol
    assert not bad.any(), (np.nonzero(bad)[0][:5], got[bad][:5], want[bad][:5])


def check_f32c(e, c, x, got):
    c32 = W.to_f32(c).astype(np.float64)
    x32 = W.to_f32(x).astype(np.float64)
    want, S = O.eval_f64(e, c32, x32)
    k = len(e)
    g = int(np.asarray(e).sum(axis=1).max()) + np.asarray(e).shape[1] + k
    val = got[0].astype(np.float64) + got[1].astype(np.float64)
    err = np.abs(val - want)
    tol = 2 * g32(2 * k + 64) ** 2 * S + g * U * S + 1e-300
    assert np.all(err <= tol), (err / S).max()
    assert np.median(err / S) <= k * 2.0 ** -48
    return err / S


def check_modp(e, c, x, got):
    assert np.array_equal(got, O.eval_modp(e, c, x))


def check_iv64(e, c, lo, hi, scheme, got, ftab=None):
    t = O.build_tree(e, scheme, ftab)
    rlo, rhi = O.walk_iv64(t, t.node_coeffs(c, np.float64), lo, hi)
    assert np.array_equal(got[0], rlo), np.nonzero(got[0] != rlo)[0][:5]
    assert np.array_equal(got[1], rhi), np.nonzero(got[1] != rhi)[0][:5]


def check_any(dtype, e, c, pts, scheme, got):
    """The bar of dtype for one evaluation: pts in the layout the oracle takes
    (iv64: (lo, hi))."""
    if dtype == "f64":
        check_f64(e, c, pts, got)
    elif dtype == "f32c":
        check_f32c(e, c, pts, got)
    elif dtype == "modp":
        check_modp(e, c, pts, got)
    else:
        check_iv64(e, c, pts[0], pts[1], scheme, got)


def local_scale(absw, radius=128):
    """max of absw over [j - radius, j + radius]: the scale of the largest
    block products that meet at coefficient j in the tensor-core FP64
    composition (64-coefficient blocks: a block product lands in its own
    output block or one of the two beside it)."""
    from scipy.ndimage import maximum_filter1d
    return maximum_filter1d(np.asarray(absw, dtype=np.float64), size=2 * radius + 1, mode="constant", cval=0.0)


def check_compose_f64(got, want, absw, K, local):
    """FP64 composition bar: |got - want| <= K u s_j with s_j = (|p| o |q|)_j
    (componentwise: the direct convolution) or its local maximum
    (local_scale: the tensor-core products, blockwise accurate)."""
    scale = local_scale(absw) if local else absw
    err = np.abs(got - want)
    ok = err <= K * U * scale + 1e-300
    assert ok.all(), (int(np.argmin(ok)), float((err / np.maximum(scale, 1e-300)).max()))
    return err
