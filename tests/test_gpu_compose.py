"""GPU parity for batched composition p_j(q_j(y)) against the oracle.

MODP: bit-exact against the schoolbook plain definition sum c_e q^e (small
and transform-crossing sizes), and at the full size (4096 pairs, deg p 512,
deg q 64) by the identity r_j(y) = p_j(q_j(y)) at a random y for every pair
plus a full schoolbook check of sampled pairs.
FP64: componentwise, |gpu - oracle|_i <= K u (|p| o |q|)_i with
K = 8 (deg p (deg q + 1) + deg p + 2): both the GPU walk and the oracle's
plain sum accumulate at most deg p (deg q + 1) + deg p roundings per
coefficient, each relative to the absolute-value computation (products
shorter than 256: direct convolution); at the full size, where the products
run on the tensor cores, blockwise (tests/checks.py: check_compose_f64).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1307_5655_gb300 as fpl
from checks import check_compose_f64

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
P = O.P_MODP


def _to_dev_u64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _to_dev_f64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def compose_modp(pc, qc, scheme, per_pair=True):
    """pc [npairs, degp+1] (index = degree), qc [npairs, degq+1]."""
    degp = pc.shape[1] - 1
    e = W.dense_univariate_exps(degp + 1)          # terms highest degree first
    cols = pc[:, ::-1]                             # coefficients in that term order
    ones = np.ones(degp + 1, dtype=np.uint64)      # non-zero placeholders: the tree keeps every term
    t = fpl.fp_compile(e, ones if per_pair else cols[0], scheme, modp=True)
    out = fpl.fp_compose(t, "modp", _to_dev_u64(qc), pcoeffs=_to_dev_u64(cols) if per_pair else None)
    return out.cpu().numpy().view(np.uint64)


def compose_f64(pc, qc, scheme):
    degp = pc.shape[1] - 1
    e = W.dense_univariate_exps(degp + 1)
    t = fpl.fp_compile(e, np.ones(degp + 1), scheme)
    out = fpl.fp_compose(t, "f64", _to_dev_f64(qc), pcoeffs=_to_dev_f64(pc[:, ::-1]))
    return out.cpu().numpy()


@pytest.mark.parametrize("scheme", ["D", "H", "E", "B"])
@pytest.mark.parametrize("degp,degq", [(1, 1), (2, 3), (7, 5), (16, 8), (33, 4), (64, 1)])
def test_modp_small_exact(scheme, degp, degq):
    n = 7
    pc, qc = W.composition_case(n, degp, degq, 10 * degp + degq, "modp")
    got = compose_modp(pc, qc, scheme)
    for j in range(n):
        assert np.array_equal(got[j], O.compose_modp(pc[j], qc[j])), j


@pytest.mark.parametrize("scheme", ["E", "B"])
def test_modp_four_step_sizes_exact(scheme):
    """deg p 128, deg q 64: products up to length 16384 (two-pass transform)."""
    n = 3
    pc, qc = W.composition_case(n, 128, 64, 5, "modp")
    got = compose_modp(pc, qc, scheme)
    for j in range(n):
        assert np.array_equal(got[j], O.compose_modp(pc[j], qc[j])), j


def test_modp_shared_coefficients():
    pc, qc = W.composition_case(5, 20, 6, 8, "modp")
    pc[:] = pc[0]
    got = compose_modp(pc, qc, "E", per_pair=False)
    for j in range(5):
        assert np.array_equal(got[j], O.compose_modp(pc[0], qc[j]))


def test_modp_edge_cases():
    # q constant: p(q) is the constant p(q0)
    pc, qc = W.composition_case(4, 9, 0, 3, "modp")
    got = compose_modp(pc, qc, "B")
    for j in range(4):
        assert np.array_equal(got[j], O.compose_modp(pc[j], qc[j]))
    # q = y: p o q = p
    pc, _ = W.composition_case(4, 17, 1, 4, "modp")
    qc = np.tile(np.array([0, 1], dtype=np.uint64), (4, 1))
    assert np.array_equal(compose_modp(pc, qc, "E"), pc)
    # single term c y^5 o q
    e = np.array([[5]], dtype=np.int32)
    t = fpl.fp_compile(e, np.array([3], dtype=np.uint64), "E", modp=True)
    _, qc = W.composition_case(2, 1, 3, 6, "modp")
    got = fpl.fp_compose(t, "modp", _to_dev_u64(qc)).cpu().numpy().view(np.uint64)
    for j in range(2):
        pcj = np.zeros(6, dtype=np.uint64)
        pcj[5] = 3
        assert np.array_equal(got[j], O.compose_modp(pcj, qc[j]))


def _poly_at(c, y):
    r = 0
    for v in reversed([int(t) for t in c]):
        r = (r * y + v) % P
    return r


@pytest.mark.parametrize("scheme", ["E", "B"])
def test_modp_full_size(scheme):
    """4096 pairs, deg p 512, deg q 64: r_j(y) = p_j(q_j(y)) at a random y for
    every pair (a wrong coefficient passes with probability <= 32768/p), and
    the full schoolbook result for one sampled pair."""
    npairs = 4096
    pc, qc = W.composition_case(npairs, 512, 64, 4000, "modp")
    got = compose_modp(pc, qc, scheme)
    assert got.shape == (npairs, 512 * 64 + 1)
    y = int(W.residues(1, 77)[0])
    ye = np.array([[y]], dtype=np.uint64)
    er = W.dense_univariate_exps(512 * 64 + 1)
    ep = W.dense_univariate_exps(513)
    eq = W.dense_univariate_exps(65)
    for j in range(npairs):
        rj = int(O.eval_modp(er, got[j, ::-1].copy(), ye)[0])
        qy = int(O.eval_modp(eq, qc[j, ::-1].copy(), ye)[0])
        pq = int(O.eval_modp(ep, pc[j, ::-1].copy(), np.array([[qy]], dtype=np.uint64))[0])
        assert rj == pq, j
    j = int(W.rng(5).integers(npairs))
    assert np.array_equal(got[j], O.compose_modp(pc[j], qc[j]))


@pytest.mark.parametrize("scheme", ["D", "H", "E", "B"])
@pytest.mark.parametrize("degp,degq", [(1, 1), (5, 3), (16, 8), (40, 6)])
def test_f64_componentwise(scheme, degp, degq):
    n = 5
    pc, qc = W.composition_case(n, degp, degq, 20 * degp + degq, "f64")
    got = compose_f64(pc, qc, scheme)
    K = 8 * (degp * (degq + 1) + degp + 2)
    for j in range(n):
        want, absw = O.compose_f64(pc[j], qc[j])
        err = np.abs(got[j] - want)
        assert np.all(err <= K * U * absw + 1e-300), (j, (err / absw).max())


def _oracle_f64_pairs(pc, qc, js):
    """The oracle's schoolbook composition for the pairs js, on all host
    cores (the C oracle runs outside the interpreter lock)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda j: O.compose_f64(pc[j], qc[j]), js))


@pytest.mark.parametrize("scheme", ["E", "B"])
def test_f64_full_size_sampled(scheme):
    """The benchmark's FP64 composition, 4096 pairs of deg p 512 and deg q 64,
    in one call (products on the tensor cores): 16 sampled pairs against the
    oracle within K u max((|p| o |q|) over i +- 128), K = 8 (deg p (deg q + 1)
    + deg p + 2) -- the blockwise bar of the tensor-core products."""
    import torch
    npairs, degp, degq = 4096, 512, 64
    pc, qc = W.composition_case(npairs, degp, degq, 4000, "f64")
    e = W.dense_univariate_exps(degp + 1)
    t = fpl.fp_compile(e, np.ones(degp + 1), scheme)
    out = fpl.fp_compose(t, "f64", _to_dev_f64(qc), pcoeffs=_to_dev_f64(pc[:, ::-1]))
    js = np.sort(W.rng(17).choice(npairs, 16, replace=False))
    got = out[torch.from_numpy(js).cuda()].cpu().numpy()
    del out
    K = 8 * (degp * (degq + 1) + degp + 2)
    for row, (want, absw), j in zip(got, _oracle_f64_pairs(pc, qc, js), js):
        check_compose_f64(row, want, absw, K, local=True)


def test_compose_rejects_bad_input():
    t = fpl.fp_compile(W.graded_prefix_exps(6, 2), np.ones(6), "E")
    with pytest.raises(fpl.FastPolyError):
        fpl.fp_compose(t, "f64", _to_dev_f64(np.ones((2, 3))), degp=2)
    tm = fpl.fp_compile(W.dense_univariate_exps(3), np.ones(3, dtype=np.uint64), "E", modp=True)
    with pytest.raises(fpl.FastPolyError):
        fpl.fp_compose(tm, "f64", _to_dev_f64(np.ones((2, 3))))
