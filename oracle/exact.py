"""Exact rational evaluation of the plain definition p(x) = sum c_e x^e.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Doubles are dyadic
rationals, so every value here is exact: a double m * 2^k is carried as the
integer pair (m, k) and sums align exponents with shifts.  Pure Python, meant
for a few points at a time.
"""
from fractions import Fraction
import math

P_MODP = 0xFFFFFFFF00000001


def _split(x):
    """x = m * 2^k exactly, m an int."""
    x = float(x)
    if x == 0.0:
        return 0, 0
    m, e = math.frexp(x)          # x = m * 2^e, 0.5 <= |m| < 1
    mi = int(m * (1 << 53))       # exact: m has at most 53 significant bits
    return mi, e - 53


def _mul(a, b):
    return a[0] * b[0], a[1] + b[1]


def _pow(a, d):
    return a[0] ** d, a[1] * d


def _sum(items):
    items = [t for t in items if t[0] != 0]
    if not items:
        return 0, 0
    k = min(t[1] for t in items)
    return sum(m << (e - k) for m, e in items), k


def to_fraction(v):
    m, k = v
    return Fraction(m) * (Fraction(2) ** k)


def exact_value(exps, coeffs, point):
    """Exact p(point) and exact sum |c_e||point^e| as Fractions.  exps: list of
    exponent tuples, coeffs: doubles, point: one double per variable."""
    nv = len(point)
    xs = [_split(v) for v in point]
    cache = [dict() for _ in range(nv)]

    def pw(v, d):
        if d not in cache[v]:
            cache[v][d] = _pow(xs[v], d)
        return cache[v][d]

    terms, aterms = [], []
    for e, c in zip(exps, coeffs):
        t = _split(c)
        for v in range(nv):
            if e[v]:
                t = _mul(t, pw(v, int(e[v])))
        terms.append(t)
        aterms.append((abs(t[0]), t[1]))
    return to_fraction(_sum(terms)), to_fraction(_sum(aterms))


def exact_horner_univariate(coeffs_by_degree, x):
    """Exact value of sum_i c_i x^i for a dense univariate polynomial given as
    coefficients indexed by degree; Horner over (int, exponent) pairs, which
    keeps large degrees affordable.  Returns (value, sum |c_i||x|^i)."""
    xm, xk = _split(x)
    axm = abs(xm)
    r = (0, 0)
    ar = (0, 0)
    for c in reversed(list(coeffs_by_degree)):
        cm, ck = _split(c)
        r = _sum([_mul(r, (xm, xk)), (cm, ck)])
        ar = _sum([_mul(ar, (axm, xk)), (abs(cm), ck)])
    return to_fraction(r), to_fraction(ar)


def horner_enclosure(coeffs_by_degree, x, frac_bits=1200):
    """Fixed-point Horner with a rigorous error bound, for |x| <= 1: returns
    integers (V, A, E) with |p(x) - V 2^-F| <= E 2^-F and |sum |c_i||x|^i -
    A 2^-F| <= E 2^-F, F = frac_bits.  Every coefficient must be a multiple
    of 2^-F (doubles of exponent >= -F + 52).  Each step multiplies by x and
    rounds down to the unit 2^-F (an error in [0, 1) unit) and adds the
    coefficient exactly; |x| <= 1 keeps the earlier errors from growing, so
    after k steps E = k.  Linear in k per step (numbers of about F bits),
    where the exact rational Horner's numbers grow by 53 bits per step."""
    xm, xk = _split(x)
    assert abs(float(x)) <= 1.0
    F = frac_bits
    axm = abs(xm)

    def times_x(v, m):
        t = v * m
        return t << xk if xk >= 0 else t >> -xk  # floor

    V, A, k = 0, 0, 0
    for c in reversed(list(coeffs_by_degree)):
        cm, ck = _split(c)
        assert cm == 0 or F + ck >= 0, "coefficient finer than the fixed-point unit"
        C = cm << (F + ck) if cm else 0
        V = times_x(V, xm) + C
        A = times_x(A, axm) + abs(C)
        k += 1
    return V, A, k


def modp_value(exps, coeffs, point):
    """p(point) mod 2^64 - 2^32 + 1 with Python integers."""
    s = 0
    for e, c in zip(exps, coeffs):
        t = int(c)
        for v, xv in enumerate(point):
            t = t * pow(int(xv), int(e[v]), P_MODP) % P_MODP
        s = (s + t) % P_MODP
    return s


def int_value(exps, coeffs, point):
    """Exact p(point) over the integers (Python integers of any size):
    sum_e c_e prod_v x_v^(e_v), the plain definition.  exps: exponent tuples,
    coeffs and point: integers."""
    s = 0
    for e, c in zip(exps, coeffs):
        t = int(c)
        for v, xv in enumerate(point):
            if e[v]:
                t *= int(xv) ** int(e[v])
        s += t
    return s


def round_down(q):
    """Largest double <= the Fraction q (q within the finite double range)."""
    f = float(q)  # round to nearest
    while Fraction(f) > q:
        f = math.nextafter(f, -math.inf)
    while Fraction(math.nextafter(f, math.inf)) <= q:
        f = math.nextafter(f, math.inf)
    return f


def round_up(q):
    """Smallest double >= the Fraction q."""
    return -round_down(-q)
