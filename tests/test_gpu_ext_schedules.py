"""Balanced trees whose grouped schedules use the extended kernels: runs of 17
to 22 nodes evaluated as two parts joined with x^f, and edge powers that few
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


@pytest.mark.parametrize("seed", range(12))
def test_small_grid_split_is_bit_identical(seed):
    """The small-grid split (one point per thread, the root's two parts in two
    warps, the second's root edges applied after the first's) against the
    same tree at two points per thread (never split): FP64, FP32C and MODP
    results equal bit for bit, over random univariate and multivariate trees
    under E, B and random split tables (7 of the 12 trees have a split, and
    the grids of 2000-40000 points take it); plus each against the oracle's
    bar."""
    r = W.rng(7100 + seed)
    nvars = int(r.integers(1, 4))
    if nvars == 1:
        k = int(r.integers(60, 3000))
        e = W.dense_univariate_exps(k)
    else:
        e = W.total_degree_exps(nvars, int(r.integers(6, 16 if nvars == 2 else 10)))
    k = len(e)
    scheme = ["E", "B", "CUSTOM"][int(r.integers(0, 3))]
    ftab = None
    if scheme == "CUSTOM":
        nmax = int(e.max()) + 1
        ftab = np.zeros(nmax + 1, dtype=np.int32)
        for n in range(1, nmax + 1):
            ftab[n] = max(1, n // 2 if r.random() < 0.5 else 2 ** int(np.log2(n)))
    npts = int(r.integers(2000, 40000))
    c = W.uniform_f64(k, 7200 + seed)
    x = W.uniform_f64(nvars * npts, 7300 + seed).reshape(nvars, npts)
    t = fpl.fp_compile(e, c, scheme, ftab)
    res = W.residues(k, 7400 + seed)
    tm = fpl.fp_compile(e, res, scheme, ftab, modp=True)
    xm = W.points_modp(nvars, npts, 7500 + seed)
    for dt, tree, pts in (("f64", t, x), ("f32c", t, x), ("modp", tm, xm)):
        d = device_points(dt, pts)
        one = fpl.fp_eval_ex(tree, dt, d, kernel="ops", ppt=1).cpu().numpy()
        two = fpl.fp_eval_ex(tree, dt, d, kernel="ops", ppt=2).cpu().numpy()
        assert np.array_equal(one.view(np.uint8), two.view(np.uint8)), (dt, scheme, nvars, k, npts)
        if dt == "f64":
            check_f64(e, c, pts, one)
        elif dt == "f32c":
            check_f32c(e, c, pts, one)
        else:
            check_modp(e, res, pts, one.view(np.uint64))
    t.free()
    tm.free()
