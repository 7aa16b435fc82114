"""FP64 composition products on the tensor cores (bf16 slices of
64-coefficient blocks, exact integer recombination), through the C ABI.

Exact cases: p and q with small integer coefficients keep every coefficient
of every product below 2^53, so the FP64 composition is exact and must equal
the integer composition (Python integers) bit for bit -- any slicing,
Toeplitz, window or recombination index error shows.  Operand lengths from
256 up (the tensor path), ragged against the 64-coefficient blocks and the
128-block tiles, both operand orders, every scheme and slice count.
Random FP64 cases, against the oracle with K = 8 (deg p (deg q + 1) + deg p
+ 2) and s = |p| o |q| (the plain FP64 walk on absolute values):
  tensor cores  |r - oracle|_i <= K u max(s over i +- 128): accurate relative
                to the largest products meeting in the neighbourhood of i
                (64-coefficient blocks with one exponent each), not to each
                coefficient: a coefficient far below its block's scale (the
                steep tails of q^e) keeps only the block's absolute accuracy;
  direct        |r - oracle|_i <= K u s_i (componentwise).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1307_5655_gb300 as fpl
from checks import check_compose_f64

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(autouse=True)
def _default_settings():
    fpl.fp_set_compose_f64(0, 0)
    yield
    fpl.fp_set_compose_f64(0, 0)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _compose(pc, qc, scheme):
    """pc [npairs, degp + 1] (index = degree), qc [npairs, degq + 1]."""
    degp = pc.shape[1] - 1
    t = fpl.fp_compile(W.dense_univariate_exps(degp + 1), np.ones(degp + 1), scheme)
    out = fpl.fp_compose(t, "f64", _dev(qc), pcoeffs=_dev(pc[:, ::-1]))
    return out.cpu().numpy()


def _int_compose(pc, qc):
    """sum_e c_e q^e over the integers, exact: int64 convolutions under a
    bound that keeps every partial sum below 2^62."""
    q = np.asarray(qc, dtype=np.int64)
    c = np.asarray(pc, dtype=np.int64)
    assert float(np.abs(c).sum()) * float(np.abs(q).sum()) ** (len(c) - 1) < 2.0 ** 62
    r = np.zeros((len(c) - 1) * (len(q) - 1) + 1, dtype=np.int64)
    pw = np.ones(1, dtype=np.int64)
    for e, ce in enumerate(c):
        r[: len(pw)] += ce * pw
        if e + 1 < len(c):
            pw = np.convolve(pw, q)
    return r


def _int_case(npairs, degp, degq, seed, cmax=7):
    """Small integer coefficients; |q| small enough that every value of the
    walk (powers, slots, result) stays below 2^53 (sum|c| (sum|q|)^deg p)."""
    r = W.rng(seed)
    qmax = 15 if degp <= 3 else 2
    pc = r.integers(-cmax, cmax + 1, size=(npairs, degp + 1)).astype(np.float64)
    pc[:, -1] = np.where(pc[:, -1] == 0, 1, pc[:, -1])
    qc = r.integers(-qmax, qmax + 1, size=(npairs, degq + 1)).astype(np.float64)
    assert (cmax * (degp + 1)) * (qmax * (degq + 1)) ** degp < 2.0 ** 53
    return pc, qc


@pytest.mark.parametrize("slices", [6, 7, 8])
@pytest.mark.parametrize("scheme", ["H", "E", "B", "D"])
@pytest.mark.parametrize("degp,degq", [(2, 255), (3, 300), (2, 1000), (5, 257)])
def test_integer_compositions_are_exact(slices, scheme, degp, degq):
    fpl.fp_set_compose_f64(slices, 256)
    npairs = 3
    pc, qc = _int_case(npairs, degp, degq, 100 * degp + degq)
    got = _compose(pc, qc, scheme)
    for j in range(npairs):
        want = _int_compose(pc[j], qc[j])
        assert max(abs(v) for v in want) < 2 ** 53
        assert np.array_equal(got[j], np.array(want, dtype=np.float64)), (j, slices, scheme)


def test_integer_compositions_many_pairs_and_scales():
    """129 pairs (more tiles than one wave for the largest product), every
    pair's q scaled by its own power of two (block exponents from 2^-30 to
    2^30 across pairs) and a run of q's coefficients scaled by 2^-12 (blocks
    of very different exponents inside one operand): still exact, and equal
    to the exact rational composition."""
    from fractions import Fraction
    npairs, degp, degq = 129, 2, 700
    pc, qc = _int_case(npairs, degp, degq, 77)
    qc[:, 300:400] *= 2.0 ** -12
    ks = W.rng(78).integers(-30, 30, size=npairs)
    got = _compose(pc, qc * np.exp2(ks)[:, None], "B")
    for j in (0, 1, 64, 128):
        qi = np.round(qc[j] * 4096).astype(np.int64)  # q = 2^k qi / 4096 exactly
        powers = [np.ones(1, dtype=np.int64), qi, np.convolve(qi, qi)]
        want = [Fraction(0)] * (degp * degq + 1)
        for e in range(degp + 1):
            scale = Fraction(2) ** (int(ks[j]) * e - 12 * e)
            for i, v in enumerate(powers[e]):
                want[i] += int(pc[j, e]) * int(v) * scale
        assert all(Fraction(float(g)) == w for g, w in zip(got[j], want)), j


@pytest.mark.parametrize("scheme", ["E", "B"])
@pytest.mark.parametrize("degp,degq", [(12, 64), (40, 32), (9, 300)])
def test_f64_random_against_oracle(scheme, degp, degq):
    n = 4
    pc, qc = W.composition_case(n, degp, degq, 31 * degp + degq, "f64")
    K = 8 * (degp * (degq + 1) + degp + 2)
    got = _compose(pc, qc, scheme)
    fpl.fp_set_compose_f64(0, -1)
    direct = _compose(pc, qc, scheme)
    for j in range(n):
        want, absw = O.compose_f64(pc[j], qc[j])
        check_compose_f64(got[j], want, absw, K, local=True)
        check_compose_f64(direct[j], want, absw, K, local=False)


@pytest.mark.parametrize("slices", [7, 8])
def test_tensor_path_close_to_direct_convolution(slices):
    """The same composition with every product by direct FP64 convolution
    (min_len < 0) and on the tensor cores: the two differ by less than
    2^-40 of the largest coefficient of the result, per pair (both are
    FP64-accurate evaluations of the same walk)."""
    npairs, degp, degq = 8, 16, 64
    pc, qc = W.composition_case(npairs, degp, degq, 555, "f64")
    fpl.fp_set_compose_f64(slices, -1)
    direct = _compose(pc, qc, "B")
    fpl.fp_set_compose_f64(slices, 256)
    tensor = _compose(pc, qc, "B")
    assert not np.array_equal(direct, tensor)  # the tensor path did run
    for j in range(npairs):
        scale = np.abs(direct[j]).max()
        assert np.abs(direct[j] - tensor[j]).max() <= 2.0 ** -40 * scale, j


def test_settings_are_checked():
    with pytest.raises(fpl.FastPolyError):
        fpl.fp_set_compose_f64(5, 0)
    with pytest.raises(fpl.FastPolyError):
        fpl.fp_set_compose_f64(9, 0)
