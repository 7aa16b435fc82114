"""Pins of the oracle's values against closed forms, exact rationals, brute
force over the integers, and interval containment / tightness."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle import exact as X
import workloads as W

U = 2.0 ** -53
P = O.P_MODP


def gamma(k):
    return k * U / (1 - k * U)


# ---------------------------------------------------------------- FP64 plain sum
@pytest.mark.parametrize("nvars,k", [(1, 1), (1, 7), (1, 64), (2, 30), (3, 40)])
def test_f64_plain_vs_exact_rationals(nvars, k):
    if nvars == 1:
        e = W.dense_univariate_exps(k)
    else:
        e = W.graded_prefix_exps(k, nvars)
    c = W.uniform_f64(len(e), 5)
    x = W.points_f64(nvars, 16, 6)
    got, absum = O.eval_f64(e, c, x)
    bound_k = int(e.sum(axis=1).max()) + nvars + len(e)
    for j in range(x.shape[1]):
        v, s = X.exact_value(e.tolist(), c, x[:, j])
        assert abs(Fraction(got[j]) - v) <= Fraction(gamma(bound_k)) * s
        assert abs(Fraction(absum[j]) - s) <= Fraction(gamma(bound_k)) * s


@pytest.mark.parametrize("n", [0, 1, 5, 50, 400])
def test_f64_geometric_closed_form(n):
    """sum_{i<=n} x^i = (x^{n+1} - 1)/(x - 1)."""
    e = W.dense_univariate_exps(n + 1)
    x = W.points_f64(1, 12, 9)
    got, absum = O.eval_f64(e, np.ones(n + 1), x)
    for j in range(12):
        xf = Fraction(x[0, j])
        want = (xf ** (n + 1) - 1) / (xf - 1)
        assert abs(Fraction(got[j]) - want) <= Fraction(gamma(2 * n + 2)) * Fraction(absum[j]) * 2


def _chebyshev_coeffs(n):
    """Integer coefficients of T_n by T_{k+1} = 2x T_k - T_{k-1}."""
    t0, t1 = [1], [0, 1]
    if n == 0:
        return t0
    for _ in range(n - 1):
        t2 = [0] + [2 * v for v in t1]
        for i, v in enumerate(t0):
            t2[i] -= v
        t0, t1 = t1, t2
    return t1


@pytest.mark.parametrize("n", [3, 10, 20])
def test_f64_chebyshev(n):
    """T_n(x) via the three-term recurrence in exact arithmetic."""
    cb = _chebyshev_coeffs(n)
    e = np.array([[i] for i in range(n, -1, -1) if cb[i]], dtype=np.int32)
    c = np.array([float(cb[i]) for i in range(n, -1, -1) if cb[i]])
    x = W.points_f64(1, 10, 12)
    got, absum = O.eval_f64(e, c, x)
    for j in range(10):
        xf = Fraction(x[0, j])
        a, b = Fraction(1), xf
        for _ in range(n - 1):
            a, b = b, 2 * xf * b - a
        assert abs(Fraction(got[j]) - b) <= Fraction(gamma(2 * n + 2)) * Fraction(absum[j])


def test_f64_walk_within_bound_all_schemes():
    """The FP64 walk (Sec. 2.1) of every scheme stays within the plain bound."""
    k = 200
    e, c, x = W.univariate_case(k, 32, 21)
    for s in "DHEB":
        got = O.eval_walk_f64(e, c, x, s)
        for j in range(8):
            v, sabs = X.exact_value(e.tolist(), c, x[:, j])
            assert abs(Fraction(got[j]) - v) <= Fraction(gamma(4 * k)) * sabs


# ---------------------------------------------------------------- MODP
def test_modp_brute_force():
    for seed in range(10):
        nv = 1 + seed % 3
        e = W.graded_prefix_exps(20, nv) if nv > 1 else W.dense_univariate_exps(20)
        c = W.residues(len(e), seed)
        x = W.points_modp(nv, 5, seed + 1)
        got = O.eval_modp(e, c, x)
        for j in range(5):
            assert int(got[j]) == X.modp_value(e.tolist(), c.tolist(), x[:, j].tolist())


@pytest.mark.parametrize("n", [1, 10, 255, 1000])
def test_modp_binomial_closed_form(n):
    """(1 + x)^n expanded with binomial coefficients mod p."""
    e = W.dense_univariate_exps(n + 1)
    c = np.array([math.comb(n, n - i) % P for i in range(n + 1)], dtype=np.uint64)
    x = W.points_modp(1, 6, n)
    want = [pow(1 + int(v), n, P) for v in x[0]]
    assert [int(v) for v in O.eval_modp(e, c, x)] == want
    for s in "DHEB":
        assert [int(v) for v in O.eval_walk_modp(e, c, x, s)] == want


def test_modp_geometric_closed_form():
    n = 777
    e = W.dense_univariate_exps(n + 1)
    x = W.points_modp(1, 6, 3)
    got = O.eval_modp(e, np.ones(n + 1, dtype=np.uint64), x)
    for j in range(6):
        xv = int(x[0, j])
        want = (pow(xv, n + 1, P) - 1) * pow(xv - 1, P - 2, P) % P
        assert int(got[j]) == want


def test_modp_rejects_noncanonical():
    with pytest.raises(O.OracleError):
        O.eval_modp(W.dense_univariate_exps(2), np.array([P, 1], dtype=np.uint64),
                    np.zeros((1, 1), dtype=np.uint64))


# ---------------------------------------------------------------- intervals
def _rand_intervals(seed, n):
    r = W.rng(seed)
    a = r.uniform(-2, 2, size=n)
    b = r.uniform(-2, 2, size=n)
    kinds = r.integers(0, 4, size=n)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    lo = np.where(kinds == 0, np.abs(lo), lo)          # some non-negative
    hi = np.where(kinds == 0, np.maximum(np.abs(lo), np.abs(hi)), hi)
    hi = np.where(kinds == 1, -np.abs(hi), hi)         # some non-positive
    lo = np.where(kinds == 1, -np.maximum(np.abs(lo), np.abs(hi)), lo)
    lo = np.where(kinds == 2, 0.0, lo)                 # touching zero
    lo, hi = np.minimum(lo, hi), np.maximum(lo, hi)
    return lo, hi


def test_interval_product_is_tight_rounding_of_exact_extremes():
    alo, ahi = _rand_intervals(1, 400)
    blo, bhi = _rand_intervals(2, 400)
    rlo, rhi = O.iv_mul(alo, ahi, blo, bhi)
    for i in range(400):
        prods = [Fraction(a) * Fraction(b) for a in (alo[i], ahi[i]) for b in (blo[i], bhi[i])]
        assert rlo[i] == X.round_down(min(prods)), i
        assert rhi[i] == X.round_up(max(prods)), i


@pytest.mark.parametrize("d", [1, 2, 3, 7, 8, 40])
def test_interval_power_contains_and_is_narrow(d):
    lo, hi = _rand_intervals(3, 100)
    lo, hi = lo / 2, hi / 2
    rlo, rhi = O.iv_pow(lo, hi, d)
    for i in range(100):
        for t in (Fraction(lo[i]), Fraction(hi[i]), (Fraction(lo[i]) + Fraction(hi[i])) / 2):
            assert Fraction(rlo[i]) <= t ** d <= Fraction(rhi[i])
        m = max(abs(Fraction(lo[i])), abs(Fraction(hi[i]))) ** d
        slack = Fraction(gamma(4 * d)) * m
        if lo[i] < 0 < hi[i]:
            # straddling zero: interval powers overestimate (dependency), but
            # stay within [-max|x|^d, max|x|^d]
            assert Fraction(rlo[i]) >= -m - slack and Fraction(rhi[i]) <= m + slack
        else:
            # single sign: x^d is monotone on the box, the result is its range
            ends = [Fraction(lo[i]) ** d, Fraction(hi[i]) ** d]
            assert Fraction(rlo[i]) >= min(ends) - slack and Fraction(rhi[i]) <= max(ends) + slack


@pytest.mark.parametrize("scheme", ["D", "H", "E", "B"])
def test_interval_walk_contains_exact_values(scheme):
    e, c, (lo, hi) = W.trivariate_case(6, 24, 4, "iv64")
    rlo, rhi = O.eval_iv64(e, c, lo, hi, scheme)
    assert np.all(rlo <= rhi)
    el = e.tolist()
    for j in range(24):
        corners = [[lo[v, j] if (m >> v) & 1 else hi[v, j] for v in range(3)] for m in range(8)]
        centre = [(Fraction(lo[v, j]) + Fraction(hi[v, j])) / 2 for v in range(3)]
        for pt in corners:
            val, _ = X.exact_value(el, c, pt)
            assert Fraction(rlo[j]) <= val <= Fraction(rhi[j])
        # centre is not a double in general: evaluate exactly with Fractions
        val = sum(Fraction(cc) * math.prod(centre[v] ** ev[v] for v in range(3)) for ev, cc in zip(el, c))
        assert Fraction(rlo[j]) <= val <= Fraction(rhi[j])


def test_interval_walk_degenerate_points_are_narrow():
    k = 300
    e, c, x = W.univariate_case(k, 16, 8)
    rlo, rhi = O.eval_iv64(e, c, x, x, "E")
    for j in range(16):
        v, s = X.exact_value(e.tolist(), c, x[:, j])
        assert Fraction(rlo[j]) <= v <= Fraction(rhi[j])
        assert Fraction(rhi[j]) - Fraction(rlo[j]) <= Fraction(gamma(8 * k)) * s


# ---------------------------------------------------------------- composition
def _poly_eval_mod(c, y):
    r = 0
    for v in reversed([int(t) for t in c]):
        r = (r * y + v) % P
    return r


def test_compose_modp_schwartz_zippel():
    pc, qc = W.composition_case(3, 20, 6, 5, "modp")
    for i in range(3):
        r = O.compose_modp(pc[i], qc[i])
        assert len(r) == 20 * 6 + 1
        for y in [3, 12345, int(W.residues(1, i)[0])]:
            assert _poly_eval_mod(r, y) == _poly_eval_mod(pc[i], _poly_eval_mod(qc[i], y))


def test_compose_modp_identities():
    qc = W.residues(9, 1)
    # x^n o q = q^n
    n = 5
    pc = np.zeros(n + 1, dtype=np.uint64)
    pc[n] = 1
    r = O.compose_modp(pc, qc)
    qn = [1]
    for _ in range(n):
        nx = [0] * (len(qn) + len(qc) - 1)
        for i, a in enumerate(qn):
            for j, b in enumerate(qc):
                nx[i + j] = (nx[i + j] + a * int(b)) % P
        qn = nx
    assert [int(v) for v in r] == qn
    # p o x = p
    pc = W.residues(12, 2)
    assert np.array_equal(O.compose_modp(pc, np.array([0, 1], dtype=np.uint64)), pc)


def test_compose_f64_vs_exact():
    pc, qc = W.composition_case(2, 12, 4, 7, "f64")
    for i in range(2):
        r, ra = O.compose_f64(pc[i], qc[i])
        pf = [Fraction(v) for v in pc[i]]
        qf = [Fraction(v) for v in qc[i]]
        acc = [Fraction(0)] * len(r)
        pw = [Fraction(1)]
        for e in range(len(pf)):
            for j, v in enumerate(pw):
                acc[j] += pf[e] * v
            nx = [Fraction(0)] * (len(pw) + len(qf) - 1)
            for a_i, a in enumerate(pw):
                for b_i, b in enumerate(qf):
                    nx[a_i + b_i] += a * b
            pw = nx
        for j in range(len(r)):
            assert abs(Fraction(r[j]) - acc[j]) <= Fraction(gamma(12 * 5 * 3)) * Fraction(ra[j])


# ------------------------------------------------------------ exact Horner (reference of the FP64 bound)
@pytest.mark.parametrize("k", [1, 2, 5, 17, 64])
def test_exact_horner_equals_exact_plain_sum(k):
    """exact_horner_univariate (coefficients indexed by degree) equals the
    exact plain sum exact_value (terms with exponents), value and condition
    sum sum |c_i||x|^i, at dyadic points of both signs."""
    e, c, x = W.univariate_case(k, 7, 500 + k)  # exps k-1..0, c[j] is the coefficient of x^(k-1-j)
    for xv in list(x[0]) + [-0.5, 0.0, 1.0]:
        want_v, want_s = X.exact_value(e, c, (xv,))
        got_v, got_s = X.exact_horner_univariate(c[::-1], xv)
        assert got_v == want_v and got_s == want_s, xv


def test_exact_horner_coefficient_order_and_signs():
    """Hand-worked values: the coefficient of x^i sits at index i, and the
    condition sum takes |c_i| |x|^i (not |sum|)."""
    assert X.exact_horner_univariate([1.0, 2.0, 3.0], 2.0) == (Fraction(17), Fraction(17))
    assert X.exact_horner_univariate([0.0, 1.0], 0.5) == (Fraction(1, 2), Fraction(1, 2))
    assert X.exact_horner_univariate([1.0, 3.0], -0.5) == (Fraction(-1, 2), Fraction(5, 2))
    assert X.exact_horner_univariate([-1.0, 3.0, -2.0], -0.25) == (Fraction(-15, 8), Fraction(15, 8))
    assert X.exact_horner_univariate([0.25], -3.0) == (Fraction(1, 4), Fraction(1, 4))


@pytest.mark.parametrize("xv", [0.75, -0.99609375, 1.0 + 2.0 ** -20])
def test_exact_horner_geometric_closed_form_10007(xv):
    """k = 10007 ones: sum x^i = (x^k - 1) / (x - 1) and the condition sum is
    (|x|^k - 1) / (|x| - 1), exactly."""
    k = 10007
    v, s = X.exact_horner_univariate(np.ones(k), xv)
    x = Fraction(xv)
    ax = abs(x)
    assert v == (x ** k - 1) / (x - 1)
    assert s == (ax ** k - 1) / (ax - 1)


# ------------------------------------------------------------ fixed-point enclosure (fast reference)
@pytest.mark.parametrize("k", [1, 2, 17, 64, 300])
def test_horner_enclosure_contains_exact_value(k):
    """The enclosure V 2^-F +- k 2^-F contains the exact value (exact rational
    Horner) and the condition sum, at points of both signs in [-1, 1]; with
    F large the interval is far below 2^-1000."""
    e, c, x = W.univariate_case(k, 6, 700 + k)
    F = 1200
    for xv in list(x[0]) + [-1.0, 1.0, 0.0, -0.5]:
        v, s = X.exact_horner_univariate(c[::-1], xv)
        V, A, E = X.horner_enclosure(c[::-1], xv, F)
        assert E == k
        scale = Fraction(2) ** -F
        assert abs(v - V * scale) <= E * scale, xv
        assert abs(s - A * scale) <= E * scale, xv


def test_horner_enclosure_geometric_10007():
    """k = 10007 ones at x = -0.99609375: the enclosure contains (x^k - 1)/(x - 1)
    and (|x|^k - 1)/(|x| - 1)."""
    k, xv, F = 10007, -0.99609375, 1200
    V, A, E = X.horner_enclosure(np.ones(k), xv, F)
    x = Fraction(xv)
    scale = Fraction(2) ** -F
    assert abs((x ** k - 1) / (x - 1) - V * scale) <= E * scale
    assert abs((abs(x) ** k - 1) / (abs(x) - 1) - A * scale) <= E * scale


def test_horner_enclosure_rounds_down_only():
    """A planted error is caught: dropping the coefficient of x^1 moves the
    enclosure away from the exact value by that coefficient."""
    c = np.array([0.5, 0.25, -0.75])
    V, A, E = X.horner_enclosure(c, 0.5, 64)
    v, _ = X.exact_horner_univariate(c, 0.5)
    assert abs(v - Fraction(V, 2 ** 64)) <= Fraction(E, 2 ** 64)
    c2 = c.copy()
    c2[1] = 0.0
    V2, _, _ = X.horner_enclosure(c2, 0.5, 64)
    assert abs(v - Fraction(V2, 2 ** 64)) > Fraction(1, 10)
