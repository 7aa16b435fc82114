"""Balanced trees whose grouped schedules use the extended kernels: runs of 17
to 24 nodes evaluated as two parts joined with x^f, and edge powers that few
ops read recomputed from a kept binary prefix instead of read from the
per-point table.  Every value type that runs the grouped schedule -- FP64,
FP32C, MODP and residues -- through fp_eval, the batch launch and the
residue path, against the oracle (FP64 / FP32C within the bars of
tests/checks.py, MODP and residues bit-exact), with plain Balanced trees in
the same batch."""
import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1307_5655_gb300 as fpl
from gpu_util import device_points, run
from checks import check_f32c, check_f64, check_modp
from oracle import exact as X

pytestmark = pytest.mark.gpu


def _uses_ext(t):
    """The schedule has two-part blocks or recomputed edge powers."""
    ow = t.schedule()["op_words"]
    two_part = ((ow[:, 1].astype(np.int64) >> 8) & 255) > 0
    recompute = (ow[:, 0] >> 17) == 0x7FFF
    return bool(two_part.any() or recompute.any()), bool(recompute.any())


@pytest.mark.parametrize("k", [40, 10007])
def test_floating_point_balanced_with_two_part_blocks(k):
    e, c, x = W.univariate_case(k, 4096 + 33, 500 + k)
    t = fpl.fp_compile(e, c, "B")
    ext, rec = _uses_ext(t)
    assert ext and (rec or k < 10007)  # 10007 terms: the table also drops rare powers
    check_f64(e, c, x, run(t, "f64", x))
    check_f32c(e, c, x, run(t, "f32c", x))
    for ppt in (1, 2, 4):  # every launch width of the grouped kernel
        d = device_points("f32c", x)
        got = fpl.fp_eval_ex(t, "f32c", d, kernel="ops", ppt=ppt).cpu().numpy()
        check_f32c(e, c, x, got)
    t.free()


@pytest.mark.parametrize("k", [10007, 30000])
def test_modp_balanced_with_recomputed_powers(k):
    e, c, x = W.univariate_case(k, 256 + 5, 600 + k, "modp")
    t = fpl.fp_compile(e, c, "B", modp=True)
    assert _uses_ext(t)[1]
    check_modp(e, c, x, run(t, "modp", x))
    t.free()


def test_batch_mixes_extended_and_plain_balanced_trees():
    """One batch launch with trees that need the extended kernel and trees
    that do not (small Balanced, Estrin): each job equals its own fp_eval and
    the oracle."""
    import torch
    cases = [(10007, "B"), (1000, "B"), (3000, "B"), (1000, "E"), (40, "B"), (30000, "B")]
    jobs, keep = [], []
    for i, (k, s) in enumerate(cases):
        e, c, x = W.univariate_case(k, 2048 + 7 * i, 700 + k)
        t = fpl.fp_compile(e, c, s)
        d = device_points("f64", x)
        out = torch.empty(x.shape[1], dtype=torch.float64, device="cuda")
        jobs.append((t, d, out))
        keep.append((e, c, x, t))
    assert _uses_ext(keep[0][3])[0] and not _uses_ext(keep[1][3])[0] and not _uses_ext(keep[3][3])[0]
    fpl.fp_eval_batch("f64", jobs)
    torch.cuda.synchronize()
    for (t, d, out), (e, c, x, _) in zip(jobs, keep):
        got = out.cpu().numpy()
        assert np.array_equal(got, run(t, "f64", x))
        check_f64(e, c, x, got)
    for *_, t in keep:
        t.free()


def test_residues_balanced_with_recomputed_powers():
    """Residues of a 10007-term Balanced integer polynomial (its schedule
    recomputes edge powers): at points of 60 bits every residue equals p(x)
    mod q_i (Horner's rule mod q_i in Python integers); at points in {-1, 0,
    1}, where p(x) fits the primes' product, the reconstruction equals the
    exact integer."""
    import torch
    k = 10007
    e = W.dense_univariate_exps(k)
    r = W.rng(61)
    coeffs = [int(v) for v in r.integers(-(1 << 40), 1 << 40, size=k)]
    big = [int(v) for v in r.integers(1, 1 << 60, size=4)]
    small = [-1, 0, 1, -1]
    pts = big + small
    qs = [int(v) for v in fpl.fp_rns_primes(3)]  # |p(x)| < 2^54 at the small points
    res = np.array([[cc % q for cc in coeffs] for q in qs], dtype=np.uint64)
    t = fpl.fp_compile_rns(e, res, "B")
    assert _uses_ext(t)[1]
    d = torch.from_numpy(np.array([[[p % q for p in pts]] for q in qs], dtype=np.uint64).view(np.int64)).cuda()
    out = fpl.fp_eval_rns(t, d)
    limbs = fpl.fp_crt(out)
    torch.cuda.synchronize()
    got_res = out.cpu().numpy().view(np.uint64)
    got_limbs = limbs.cpu().numpy().view(np.uint64)
    by_degree = [0] * k
    for ex, cc in zip(e[:, 0].tolist(), coeffs):
        by_degree[ex] = cc
    for j, p in enumerate(pts):
        for i, q in enumerate(qs):
            h = 0
            for cc in reversed(by_degree):
                h = (h * p + cc) % q
            assert int(got_res[i, j]) == h, (j, i)
    for j, p in enumerate(small, start=len(big)):
        assert fpl.limbs_to_int(got_limbs[j]) == X.int_value(e.tolist(), coeffs, (p,)), j
    t.free()
