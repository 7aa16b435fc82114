"""Exact integer evaluation through residues on the GPU: every residue equals
p(x) mod q_i, and the Chinese remainder reconstruction equals the exact
integer p(x) of the oracle (Python integers), for random coefficients and
points of several hundred bits, both signs, several schemes and shapes."""
import numpy as np
import pytest

import workloads as W
import paper_1307_5655_gb300 as fpl
from oracle import exact as X

pytestmark = pytest.mark.gpu


def _ints(n, bits, seed):
    """n signed integers below 2^bits in magnitude (seeded)."""
    r = W.rng(seed)
    words = (bits + 63) // 64
    out = []
    for _ in range(n):
        v = 0
        for w in r.integers(0, 2 ** 63, size=words, dtype=np.int64).tolist():
            v = (v << 63) | int(w)
        v &= (1 << bits) - 1
        out.append(-v if r.random() < 0.5 else v)
    return out


def _primes_for(bound_bits):
    k = (bound_bits + 2 + 63) // 64 + 1  # Q > 2 |p(x)|
    assert k <= fpl.RNS_MAX_PRIMES
    return [int(v) for v in fpl.fp_rns_primes(k)]


def _check(exps, coeffs, points, scheme, cbits, xbits):
    import torch
    e = np.asarray(exps, dtype=np.int32)
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    nv = e.shape[1]
    deg = int(e.sum(axis=1).max()) if len(e) else 0
    qs = _primes_for(cbits + deg * xbits + max(1, len(e)).bit_length())
    k = len(qs)
    res = np.array([[c % q for c in coeffs] for q in qs], dtype=np.uint64).reshape(k, len(coeffs))
    t = fpl.fp_compile_rns(e, res, scheme)
    npts = len(points)
    pts = np.array([[[p[v] % q for p in points] for v in range(nv)] for q in qs], dtype=np.uint64)
    d = torch.from_numpy(pts.view(np.int64)).cuda()
    out = fpl.fp_eval_rns(t, d)
    limbs = fpl.fp_crt(out)
    torch.cuda.synchronize()
    got_res = out.cpu().numpy().view(np.uint64)
    got_limbs = limbs.cpu().numpy().view(np.uint64)
    for j, p in enumerate(points):
        want = X.int_value(e.tolist(), coeffs, p)
        for i, q in enumerate(qs):
            assert int(got_res[i, j]) == want % q, (j, i)
        assert fpl.limbs_to_int(got_limbs[j]) == want, j
    t.free()


@pytest.mark.parametrize("scheme", ["H", "E", "B"])
@pytest.mark.parametrize("k,cbits,xbits", [(1, 64, 64), (2, 130, 17), (17, 200, 40), (300, 256, 8)])
def test_univariate_exact_integers(scheme, k, cbits, xbits):
    e = W.dense_univariate_exps(k)
    c = _ints(k, cbits, 10 + k)
    pts = [(x,) for x in _ints(1000 + 3, xbits, 20 + k)]
    _check(e, c, pts, scheme, cbits, xbits)


@pytest.mark.parametrize("scheme", ["E", "B"])
def test_trivariate_exact_integers(scheme):
    e = W.total_degree_exps(3, 6)
    c = _ints(len(e), 200, 31)
    pts = list(zip(_ints(500 + 1, 48, 32), _ints(500 + 1, 48, 33), _ints(500 + 1, 48, 34)))
    _check(e, c, pts, scheme, 200, 48)


def test_sparse_and_partly_zero_residues():
    # a coefficient divisible by one of the primes (zero residue there, not
    # elsewhere), a sparse exponent set and extreme points
    qs = [int(v) for v in fpl.fp_rns_primes(8)]
    e = np.array([[90], [64], [63], [7], [0]], dtype=np.int32)
    c = [qs[2] * 3, -1, 2 ** 200 + 1, -(2 ** 120), 5]
    pts = [(x,) for x in (0, 1, -1, 2 ** 5 - 1, -(2 ** 5), 3)]
    _check(e, c, pts, "E", 201, 5)


def test_boundaries_of_the_crt_range():
    # values near +-Q/2 for two primes: constants placed at the ends of the range
    import torch
    qs = [int(v) for v in fpl.fp_rns_primes(2)]
    Q = qs[0] * qs[1]
    vals = [Q // 2, -(Q // 2), Q // 2 - 1, -(Q // 2) + 1, 0, -1]
    res = np.array([[v % q for v in vals] for q in qs], dtype=np.uint64)
    d = torch.from_numpy(res.view(np.int64)).cuda()
    limbs = fpl.fp_crt(d)
    got = [fpl.limbs_to_int(row) for row in limbs.cpu().numpy().view(np.uint64)]
    assert got == vals


def test_noncanonical_points_and_zero_polynomial():
    import torch
    qs = [int(v) for v in fpl.fp_rns_primes(3)]
    e = W.dense_univariate_exps(4)
    c = [3, -2, 0, 7]
    res = np.array([[v % q for v in c] for q in qs], dtype=np.uint64)
    t = fpl.fp_compile_rns(e, res, "E")
    xs = [5, -9]
    raw = np.array([[[(x % q) + (q if (x % q) + q < 2 ** 64 else 0) for x in xs]] for q in qs], dtype=np.uint64)
    out = fpl.fp_eval_rns(t, torch.from_numpy(raw.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
    for j, x in enumerate(xs):
        want = X.int_value(e.tolist(), c, (x,))
        assert [int(out[i, j]) for i in range(3)] == [want % q for q in qs]
    z = fpl.fp_compile_rns(e, np.zeros((3, 4), dtype=np.uint64), "E")
    outz = fpl.fp_eval_rns(z, torch.from_numpy(raw.view(np.int64)).cuda())
    assert int(outz.abs().sum()) == 0
