"""Host-side checks of the residue path (no GPU): the oracle's exact integer
value against closed forms, the library's primes, input validation and the
limb conversion."""
import math

import numpy as np
import pytest

import workloads as W
import paper_1307_5655_gb300 as fpl
from oracle import exact as X


def test_int_value_closed_forms():
    # binomial theorem: sum_i C(n, i) x^i = (x + 1)^n
    n = 60
    exps = [(i,) for i in range(n + 1)]
    coeffs = [math.comb(n, i) for i in range(n + 1)]
    for x in (-(3 ** 40), -1, 0, 2, 12345678901234567890):
        assert X.int_value(exps, coeffs, (x,)) == (x + 1) ** n
    # geometric series: sum_{i<k} x^i = (x^k - 1) / (x - 1)
    k = 37
    for x in (-7, 3, 2 ** 70 + 1):
        assert X.int_value([(i,) for i in range(k)], [1] * k, (x,)) == (x ** k - 1) // (x - 1)
    # two variables: (x + y)^n
    n = 12
    exps = [(i, n - i) for i in range(n + 1)]
    coeffs = [math.comb(n, i) for i in range(n + 1)]
    for x, y in ((5, -3), (2 ** 65, 7)):
        assert X.int_value(exps, coeffs, (x, y)) == (x + y) ** n


def test_primes():
    sympy = pytest.importorskip("sympy")
    q = fpl.fp_rns_primes(fpl.RNS_MAX_PRIMES).astype(object)
    assert all(q[i] > q[i + 1] for i in range(len(q) - 1))
    # the largest primes of the form 2^64 - c, c < 2^32, none skipped
    want = []
    c = 1
    while len(want) < len(q):
        if sympy.isprime(2 ** 64 - c):
            want.append(2 ** 64 - c)
        c += 2
    assert list(q) == want
    assert all(2 ** 64 - int(v) < 2 ** 32 for v in q)


def test_compile_rns_rejects_noncanonical_residues():
    q = fpl.fp_rns_primes(3)
    e = W.dense_univariate_exps(5)
    r = np.zeros((3, 5), dtype=np.uint64)
    r[1, 2] = q[1]  # not < q_1
    with pytest.raises(fpl.FastPolyError) as ex:
        fpl.fp_compile_rns(e, r, "E")
    assert ex.value.code == -1
    with pytest.raises(fpl.FastPolyError):
        fpl.fp_compile_rns(e, np.zeros((fpl.RNS_MAX_PRIMES + 1, 5), dtype=np.uint64), "E")


def test_limbs_to_int():
    for v in (0, 1, -1, 2 ** 127 - 5, -(2 ** 191) + 17):
        k = 4
        limbs = [(v >> (64 * i)) & (2 ** 64 - 1) for i in range(k)]
        assert fpl.limbs_to_int(np.array(limbs, dtype=np.uint64)) == v
