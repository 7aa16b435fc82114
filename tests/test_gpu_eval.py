"""GPU parity: the CUDA evaluation path against the CPU oracle, element by
element on seeded inputs, for every value type, scheme and edge case.

Bars (tests/checks.py): MODP and IV64 bit-exact, FP64 within (4k + g) u S,
FP32C within the compensated bound; at full size, FP64 and FP32C also against
exact rationals.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1307_5655_gb300 as fpl
from gpu_util import run
from checks import check_f32c, check_f64, check_iv64, check_modp, g32

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
U32 = 2.0 ** -24


# ----------------------------------------------------------------- univariate
KS = [1, 2, 3, 17, 100, 1000, 1024]
SCHEMES = ["D", "H", "E", "B"]


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("scheme", SCHEMES)
def test_f64_univariate(k, scheme):
    e, c, x = W.univariate_case(k, 3000 + 17, 10 + k)
    t = fpl.fp_compile(e, c, scheme)
    check_f64(e, c, x, run(t, "f64", x))


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("scheme", SCHEMES)
def test_f32c_univariate(k, scheme):
    e, c, x = W.univariate_case(k, 3000 + 17, 20 + k)
    t = fpl.fp_compile(e, c, scheme)
    check_f32c(e, c, x, run(t, "f32c", x))


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("scheme", SCHEMES)
def test_modp_univariate(k, scheme):
    e, c, x = W.univariate_case(k, 3000 + 17, 30 + k, "modp")
    t = fpl.fp_compile(e, c, scheme, modp=True)
    check_modp(e, c, x, run(t, "modp", x))


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("scheme", SCHEMES)
def test_iv64_univariate(k, scheme):
    e, c, (lo, hi) = W.univariate_case(k, 1000 + 17, 40 + k, "iv64")
    t = fpl.fp_compile(e, c, scheme)
    check_iv64(e, c, lo, hi, scheme, run(t, "iv64", (lo, hi)))


# ----------------------------------------------------------------- multivariate
MULTI = [(2, "graded", 60), (3, "total", 10), (3, "sparse", 80), (4, "graded", 50)]


def _multi(nvars, kind, size, seed):
    if kind == "graded":
        e = W.graded_prefix_exps(size, nvars)
    elif kind == "total":
        e = W.total_degree_exps(nvars, size)
    else:
        r = W.rng(seed)
        e = np.array(sorted({tuple(int(v) for v in r.integers(0, 7, size=nvars)) for _ in range(size)}),
                     dtype=np.int32)
    return e


@pytest.mark.parametrize("nvars,kind,size", MULTI)
@pytest.mark.parametrize("scheme", SCHEMES)
def test_multivariate_all_types(nvars, kind, size, scheme):
    e = _multi(nvars, kind, size, 5)
    c = W.uniform_f64(len(e), 6)
    e, c = W.shuffled(e, c, 7)
    npts = 2000 + 3
    x = W.points_f64(nvars, npts, 8)
    t = fpl.fp_compile(e, c, scheme)
    check_f64(e, c, x, run(t, "f64", x))
    check_f32c(e, c, x, run(t, "f32c", x))
    lo, hi = W.boxes(nvars, 500 + 3, 9)
    check_iv64(e, c, lo, hi, scheme, run(t, "iv64", (lo, hi)))
    cm = W.residues(len(e), 10)
    xm = W.points_modp(nvars, npts, 11)
    tm = fpl.fp_compile(e, cm, scheme, modp=True)
    check_modp(e, cm, xm, run(tm, "modp", xm))


# ----------------------------------------------------------------- edge cases
def test_zero_points_is_noop():
    t = fpl.fp_compile(W.dense_univariate_exps(5), W.uniform_f64(5, 1), "E")
    import torch
    x = torch.zeros((1, 0), dtype=torch.float64, device="cuda")
    out = fpl.fp_eval(t, "f64", x)
    assert out.numel() == 0


def test_single_point_and_single_term():
    e = np.array([[7]], dtype=np.int32)
    c = np.array([0.75])
    x = np.array([[0.5]])
    t = fpl.fp_compile(e, c, "E")
    assert run(t, "f64", x)[0] == 0.75 * 0.5 ** 7
    lo, hi = W.boxes(1, 1, 3)
    check_iv64(e, c, lo, hi, "E", run(t, "iv64", (lo, hi)))


def test_zero_polynomial_all_types():
    e = np.array([[3], [1]], dtype=np.int32)
    t = fpl.fp_compile(e, np.zeros(2), "E")
    x = W.points_f64(1, 257, 1)
    assert np.all(run(t, "f64", x) == 0)
    assert np.all(run(t, "f32c", x) == 0)
    assert np.all(run(t, "iv64", (x, x)) == 0)
    tm = fpl.fp_compile(e, np.zeros(2, dtype=np.uint64), "E", modp=True)
    assert np.all(run(tm, "modp", W.points_modp(1, 257, 2)) == 0)


def test_sparse_root_degree_and_gaps():
    e = np.array([[900], [512], [77], [40], [13]], dtype=np.int32)
    c = W.uniform_f64(5, 4)
    x = W.points_f64(1, 999, 5)
    for s in SCHEMES:
        t = fpl.fp_compile(e, c, s)
        check_f64(e, c, x, run(t, "f64", x))
        lo, hi = W.boxes(1, 999, 6)
        check_iv64(e, c, lo, hi, s, run(t, "iv64", (lo, hi)))


def _wide_boxes(nvars, npts, seed):
    """Boxes of every sign class (non-negative, non-positive, straddling 0):
    centres U[-1, 1], widths from {0.3, 1, 1.5}, and a few with a bound that
    is exactly zero or a degenerate [0, 0]."""
    c = W.points_f64(nvars, npts, seed)
    w = np.array([0.3, 1.0, 1.5])[W.rng(seed + 1).integers(0, 3, size=c.shape)]
    lo, hi = c - w / 2, c + w / 2
    lo[:, 0], hi[:, 0] = 0.0, 0.5
    lo[:, 1], hi[:, 1] = -0.5, 0.0
    lo[:, 2], hi[:, 2] = 0.0, 0.0
    lo[:, 3], hi[:, 3] = -0.7, 0.7
    return lo, hi


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("k", [5, 64, 300])
def test_iv64_wide_boxes_every_sign_case(k, scheme):
    """Interval products in all nine sign cases (Moore's table): boxes wide
    enough that points and partial sums straddle zero, bit-exact against the
    oracle's walk, whose product takes the min and max of all four products."""
    e = W.dense_univariate_exps(k)
    c = W.uniform_f64(k, 70 + k)
    lo, hi = _wide_boxes(1, 1000 + 9, 71 + k)
    cls = np.where(lo >= 0, 0, np.where(hi <= 0, 1, 2))
    assert set(np.unique(cls)) == {0, 1, 2}
    t = fpl.fp_compile(e, c, scheme)
    check_iv64(e, c, lo, hi, scheme, run(t, "iv64", (lo, hi)))


def test_iv64_wide_boxes_bivariate():
    e = _multi(2, "total", 12, 72)
    c = W.uniform_f64(len(e), 73)
    lo, hi = _wide_boxes(2, 700 + 5, 74)
    for s in SCHEMES:
        t = fpl.fp_compile(e, c, s)
        check_iv64(e, c, lo, hi, s, run(t, "iv64", (lo, hi)))


def test_deep_lazy_height_custom_scheme():
    """Random function schemes give lazy heights well above E/B's."""
    k = 3000
    r = W.rng(3)
    ft = np.zeros(k + 1, dtype=np.int32)
    for n in range(1, k + 1):
        ft[n] = max(1, min(n, int(r.integers(1, 4)) if n % 3 else n // 2 + 1))
    e, c, x = W.univariate_case(k, 1000 + 1, 12)
    t = fpl.fp_compile(e, c, "CUSTOM", ft)
    assert t.info()["max_lazy_height"] >= 2
    check_f64(e, c, x, run(t, "f64", x))
    cm = W.residues(k, 4)
    tm = fpl.fp_compile(e, cm, "CUSTOM", ft, modp=True)
    xm = W.points_modp(1, 1001, 5)
    check_modp(e, cm, xm, run(tm, "modp", xm))


def test_modp_noncanonical_points_are_reduced():
    e, c, x = W.univariate_case(50, 300, 7, "modp")
    t = fpl.fp_compile(e, c, "E", modp=True)
    xr = x.copy()
    big = np.array([O.P_MODP + 5, 2 ** 64 - 1], dtype=np.uint64)
    xr[0, :2] = big
    want = O.eval_modp(e, c, np.array([[5, (2 ** 64 - 1) - O.P_MODP]], dtype=np.uint64))
    got = run(t, "modp", xr)
    assert np.array_equal(got[:2], want)


def test_dtype_mismatch_rejected():
    t = fpl.fp_compile(W.dense_univariate_exps(3), W.residues(3, 1), "E", modp=True)
    with pytest.raises(fpl.FastPolyError):
        run(t, "f64", W.points_f64(1, 10, 1))


def test_host_entry_point_matches_device():
    e, c, x = W.univariate_case(300, 4097, 13)
    t = fpl.fp_compile(e, c, "B")
    assert np.array_equal(fpl.fp_eval_host(t, "f64", x), run(t, "f64", x))


@pytest.mark.parametrize("dtype", ["f64", "f32c", "iv64", "modp"])
def test_host_entry_point_pipelined(dtype):
    """Above 2^22 points fp_eval_host runs chunks as a copy/compute pipeline
    (strided 2D copies of the structure-of-arrays rows, a ragged last chunk):
    bit-identical to fp_eval on the same points, two variables."""
    npts = 3 * (1 << 21) + 7
    e = W.graded_prefix_exps(40, 2)
    modp = dtype == "modp"
    c = W.residues(len(e), 15) if modp else W.uniform_f64(len(e), 15)
    t = fpl.fp_compile(e, c, "E", modp=modp)
    if dtype == "iv64":
        lo, hi = W.boxes(2, npts, 16)
        pts = np.ascontiguousarray(np.stack([lo, hi], axis=1))
        dev = (lo, hi)
    elif modp:
        pts = dev = W.points_modp(2, npts, 16)
    else:
        x = W.points_f64(2, npts, 16)
        pts = W.to_f32(x) if dtype == "f32c" else x
        dev = x
    got = fpl.fp_eval_host(t, dtype, pts)
    want = run(t, dtype, dev)
    assert np.array_equal(np.asarray(got).view(np.uint8), np.asarray(want).view(np.uint8))


def test_plain_baseline_kernel():
    import torch
    e, c, x = W.univariate_case(1024, 5000, 14)
    by_degree = torch.from_numpy(c[::-1].copy()).cuda()
    got = fpl.fp_eval_plain_f64(by_degree, torch.from_numpy(x).cuda()).cpu().numpy()
    check_f64(e, c, x, got)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("k", [5, 17, 300, 1024])
def test_grouped_and_node_kernels(scheme, k):
    """Both kernels on every fused type: MODP identical bit for bit; FP64 and
    FP32C identical where no block template reorders sums (H, D), and within
    the bound everywhere."""
    e, c, x = W.univariate_case(k, 2000 + 11, 50 + k)
    t = fpl.fp_compile(e, c, scheme)
    em, cm, xm = W.univariate_case(k, 2000 + 11, 52 + k, "modp")
    tm = fpl.fp_compile(em, cm, scheme, modp=True)
    for dt, tree, pts in (("f64", t, x), ("f32c", t, x), ("modp", tm, xm)):
        try:
            a = run(tree, dt, pts, kernel="ops")
        except fpl.FastPolyError as err:
            # the Direct scheme's power table (one power per node) does not fit
            assert scheme == "D" and k > 17 and err.code == -6
            continue
        b = run(tree, dt, pts, kernel="node")
        if dt == "modp" or scheme in ("H", "D"):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), dt
        if dt == "f64":
            check_f64(e, c, x, a)
            check_f64(e, c, x, b)
        elif dt == "f32c":
            check_f32c(e, c, x, a)
            check_f32c(e, c, x, b)
        else:
            check_modp(em, cm, xm, a)
    lo, hi = W.boxes(1, 500, 53 + k)
    with pytest.raises(fpl.FastPolyError):
        run(t, "iv64", (lo, hi), kernel="ops")  # intervals keep the paper's node order


@pytest.mark.parametrize("scheme", ["E", "B"])
@pytest.mark.parametrize("nvars,kind,size", [(3, "total", 14), (2, "graded", 300), (3, "sparse", 150)])
def test_grouped_and_node_kernels_multivariate(scheme, nvars, kind, size):
    """Blocks and partial blocks over the innermost variable of a multivariate
    tree: MODP identical to the node-by-node kernel bit for bit, FP64 and
    FP32C within the bound."""
    e = _multi(nvars, kind, size, 21)
    c = W.uniform_f64(len(e), 22)
    x = W.points_f64(nvars, 3000 + 5, 23)
    t = fpl.fp_compile(e, c, scheme)
    cm = W.residues(len(e), 24)
    xm = W.points_modp(nvars, 3000 + 5, 25)
    tm = fpl.fp_compile(e, cm, scheme, modp=True)
    sched = tm.schedule()
    assert (sched["op_words"][:, 0] & 3 >= 2).any()  # the grouped kernel has blocks here
    for dt, tree, pts in (("f64", t, x), ("f32c", t, x), ("modp", tm, xm)):
        a = run(tree, dt, pts, kernel="ops")
        b = run(tree, dt, pts, kernel="node")
        if dt == "modp":
            assert np.array_equal(a, b)
            check_modp(e, cm, xm, a)
        elif dt == "f64":
            check_f64(e, c, x, a)
        else:
            check_f32c(e, c, x, a)


def deep_ftab(kmax):
    """A function scheme maximising the lazy height (dynamic programming over
    the split f at every size): lh grows linearly, about (k - 1) / 2."""
    neg = -10 ** 9
    best = {1: (0, neg, None)}
    for m in range(2, kmax + 1):
        cand = None
        for f in range(1, m):
            la, ma, _ = best[m - f]
            lb, mb, _ = best[f]
            key = (max(la, 1 + mb) if mb > neg else la, max(la, mb))
            if cand is None or key > cand[0]:
                cand = (key, f)
        best[m] = (cand[0][0], cand[0][1], cand[1])
    ft = np.ones(kmax + 1, dtype=np.int32)
    for m in range(2, kmax + 1):
        ft[m - 1] = best[m][2]
    return ft


def test_deep_trees():
    """Lazy heights 16..63 run on both kernels; above 63 fp_compile refuses
    the tree."""
    k = 61
    ft = deep_ftab(k)
    e, c, x = W.univariate_case(k, 1300, 61)
    t = fpl.fp_compile(e, c, "CUSTOM", ft)
    assert t.info()["max_lazy_height"] == O.build_tree(e, "CUSTOM", ft).lh.max() >= 16
    check_f64(e, c, x, run(t, "f64", x, kernel="ops"))
    check_f64(e, c, x, run(t, "f64", x, kernel="node"))
    lo, hi = W.boxes(1, 500, 62)
    check_iv64(e, c, lo, hi, "CUSTOM", run(t, "iv64", (lo, hi)), ftab=ft)
    cm = W.residues(k, 63)
    tm = fpl.fp_compile(e, cm, "CUSTOM", ft, modp=True)
    xm = W.points_modp(1, 1300, 64)
    check_modp(e, cm, xm, run(tm, "modp", xm))
    check_f32c(e, c, x, run(t, "f32c", x))
    kb = 200
    fb = deep_ftab(kb)
    with pytest.raises(fpl.FastPolyError):
        fpl.fp_compile(W.dense_univariate_exps(kb), W.uniform_f64(kb, 1), "CUSTOM", fb)


# ----------------------------------------------------------------- full sizes, sampled
def _sample(npts, m, seed):
    return np.sort(W.rng(seed).choice(npts, size=m, replace=False))


def test_config1_full():
    """1024 terms, Estrin, 65536 points: every point checked."""
    e, c, x = W.univariate_case(1024, 65536, 101)
    t = fpl.fp_compile(e, c, "E")
    check_f64(e, c, x, run(t, "f64", x))


@pytest.mark.parametrize("k", [1000, 3000, 10007])
def test_config2_full_size_sampled(k):
    """2^24 points per (k, scheme); 512 sampled outputs checked per launch."""
    npts = 1 << 24
    e, c, x = W.univariate_case(k, npts, 200 + k)
    idx = _sample(npts, 512, k)
    for s in ("H", "E", "B"):
        t = fpl.fp_compile(e, c, s)
        got = run(t, "f64", x)
        check_f64(e, c, x[:, idx], got[idx])
        got32 = run(t, "f32c", x)
        check_f32c(e, c, x[:, idx], got32[:, idx])


@pytest.mark.parametrize("k", [1000, 3000, 10007])
def test_config2_exact_rational_bound(k):
    """Spec bounds against the exact value at 256 sampled points of the
    2^24-point launch, under each of H, E and B:
      FP64   |r - p(x)| <= 4 n u sum |c_i||x|^i  (n = k - 1, u = 2^-53);
      FP32C  on the float-rounded inputs, |hi + lo - p(x)| <= 2 gamma_{2k+64}(2^-24)^2
             sum |c_i||x|^i, and the median of |hi + lo - p| / sum below k 2^-48.
    The exact value and condition sum come from oracle.exact.horner_enclosure
    (fixed point with 1200 fractional bits, error at most k units of 2^-1200,
    pinned against the exact rational Horner): the test takes the enclosure's
    error against itself, so the bounds hold for the exact values."""
    from fractions import Fraction
    from oracle import exact as X
    npts = 1 << 24
    F = 1200
    e, c, x = W.univariate_case(k, npts, 777 + k)
    idx = _sample(npts, 256, 900 + k)
    xs = x[0, idx]
    c32 = W.to_f32(c).astype(np.float64)
    xs32 = W.to_f32(xs).astype(np.float64)
    ex64 = [X.horner_enclosure(c[::-1], xv, F) for xv in xs]
    ex32 = [X.horner_enclosure(c32[::-1], xv, F) for xv in xs32]

    def fixed(v):  # a double (or a sum of two) as an integer number of units 2^-F
        f = Fraction(v) * 2 ** F
        assert f.denominator == 1
        return f.numerator

    bound32 = 2 * Fraction(g32(2 * k + 64)) ** 2
    for s in ("H", "E", "B"):
        t = fpl.fp_compile(e, c, s)
        got = run(t, "f64", x)[idx]
        for j, (V, A, E) in enumerate(ex64):
            # |r - p| <= |R - V| + E units and S >= A - E units
            assert 2 ** 53 * (abs(fixed(got[j]) - V) + E) <= 4 * (k - 1) * (A - E), (s, j)
        got32 = run(t, "f32c", x)[:, idx]
        rel = []
        for j, (V, A, E) in enumerate(ex32):
            R = fixed(Fraction(float(got32[0, j])) + Fraction(float(got32[1, j])))
            assert abs(R - V) + E <= bound32 * (A - E), (s, j)
            rel.append((abs(R - V) + E) / (A - E))
        assert np.median(rel) <= k * 2.0 ** -48, (s, np.median(rel))
        t.free()


@pytest.mark.parametrize("scheme", ["E", "H"])
def test_maximum_term_count(scheme):
    """FP_MAX_TERMS = 2^24 terms (dense univariate, degree 2^24 - 1): the
    grouped kernel at the size limit, checked at sampled points (MODP exact,
    FP64 within the bound)."""
    k = fpl.MAX_TERMS
    npts = 1000 + 3
    idx = _sample(npts, 6, 5)
    e = W.dense_univariate_exps(k)
    cm = W.residues(k, 91)
    xm = W.points_modp(1, npts, 92)
    tm = fpl.fp_compile(e, cm, scheme, modp=True)
    assert tm.info()["nnodes"] == k
    gm = run(tm, "modp", xm)
    check_modp(e, cm, xm[:, idx], gm[idx])
    tm.free()
    c = W.uniform_f64(k, 93)
    x = W.points_f64(1, npts, 94)
    t = fpl.fp_compile(e, c, scheme)
    g = run(t, "f64", x)
    check_f64(e, c, x[:, idx], g[idx])
    t.free()


def test_config3_full_size_sampled():
    """Trivariate total degree 40 (12341 terms), 2^22 boxes and residues,
    under E and B: sampled boxes bit-exact, sampled residues exact."""
    npts = 1 << 22
    e, c, (lo, hi) = W.trivariate_case(40, npts, 300, "iv64")
    idx = _sample(npts, 48, 3)
    for s in ("E", "B"):
        t = fpl.fp_compile(e, c, s)
        got = run(t, "iv64", (lo, hi))
        check_iv64(e, c, lo[:, idx], hi[:, idx], s, got[:, idx])
        t.free()
    em, cm, xm = W.trivariate_case(40, npts, 301, "modp")
    idx = _sample(npts, 256, 4)
    for s in ("E", "B"):
        tm = fpl.fp_compile(em, cm, s, modp=True)
        gm = run(tm, "modp", xm)
        check_modp(em, cm, xm[:, idx], gm[idx])
        tm.free()
