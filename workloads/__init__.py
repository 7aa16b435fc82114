"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds input generation only -- no step of the method (no tree,
no walk, no arithmetic on polynomial values).  Both the CUDA path and the CPU
oracle receive these arrays.  The workloads mirror the shapes of the paper's
setting (dense univariate polynomials of growing term count, multivariate
polynomials, polynomial composition) at GPU scale.

Every generator takes an explicit integer seed and uses numpy's PCG64.
"""
import numpy as np

P_MODP = 0xFFFFFFFF00000001  # 2^64 - 2^32 + 1


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# terms
# --------------------------------------------------------------------------
def dense_univariate_exps(k):
    """Exponents k-1, ..., 0 (one variable), shape [k, 1]."""
    return np.arange(k - 1, -1, -1, dtype=np.int32).reshape(-1, 1)


def total_degree_exps(nvars, deg):
    """Every monomial of total degree <= deg in nvars variables, shape [K, nvars]
    (K = C(deg + nvars, nvars); 12341 for three variables and degree 40)."""
    out = []

    def rec(prefix, left, v):
        if v == nvars - 1:
            for e in range(left + 1):
                out.append(prefix + [e])
            return
        for e in range(left + 1):
            rec(prefix + [e], left - e, v + 1)

    rec([], deg, 0)
    return np.array(out, dtype=np.int32)


def graded_prefix_exps(k, nvars=2):
    """The first k monomials in graded order (total degree, then lex): a
    downward-closed term set."""
    out = []
    d = 0
    while len(out) < k:
        level = []

        def rec(prefix, left, v):
            if v == nvars - 1:
                level.append(prefix + [left])
                return
            for e in range(left, -1, -1):
                rec(prefix + [e], left - e, v + 1)

        rec([], d, 0)
        out.extend(level)
        d += 1
    return np.array(out[:k], dtype=np.int32)


def shuffled(exps, coeffs, seed):
    """The same polynomial with its terms in a random order."""
    perm = rng(seed).permutation(len(exps))
    return np.ascontiguousarray(exps[perm]), np.ascontiguousarray(coeffs[perm])


# --------------------------------------------------------------------------
# values
# --------------------------------------------------------------------------
def uniform_f64(n, seed, lo=-1.0, hi=1.0):
    """i.i.d. uniform[lo, hi) doubles."""
    return rng(seed).uniform(lo, hi, size=n)


def residues(n, seed):
    """i.i.d. uniform residues in [0, p-1], p = 2^64 - 2^32 + 1."""
    return rng(seed).integers(0, P_MODP, size=n, dtype=np.uint64, endpoint=False)


def points_f64(nvars, npts, seed):
    """SoA points, shape [nvars, npts], uniform in [-1, 1)."""
    return uniform_f64(nvars * npts, seed).reshape(nvars, npts)


def points_modp(nvars, npts, seed):
    return residues(nvars * npts, seed).reshape(nvars, npts)


def boxes(nvars, npts, seed, width=1e-6):
    """Interval points: centres uniform in [-1, 1), half-width width/2;
    returns (lo, hi), each SoA [nvars, npts], lo <= hi."""
    c = points_f64(nvars, npts, seed)
    return c - width / 2, c + width / 2


def to_f32(x):
    """Inputs of the FP32 path: round-to-nearest FP32 of the FP64 draw."""
    return np.asarray(x, dtype=np.float64).astype(np.float32)


# --------------------------------------------------------------------------
# named workloads (sizes of the benchmark configurations)
# --------------------------------------------------------------------------
def univariate_case(k, npts, seed, dtype="f64"):
    """Dense univariate polynomial with k terms and npts points."""
    exps = dense_univariate_exps(k)
    if dtype == "modp":
        return exps, residues(k, seed), points_modp(1, npts, seed + 1)
    if dtype == "iv64":
        lo, hi = boxes(1, npts, seed + 1)
        return exps, uniform_f64(k, seed), (lo, hi)
    return exps, uniform_f64(k, seed), points_f64(1, npts, seed + 1)


def trivariate_case(deg, npts, seed, dtype="iv64"):
    """All monomials of total degree <= deg in three variables."""
    exps = total_degree_exps(3, deg)
    if dtype == "modp":
        return exps, residues(len(exps), seed), points_modp(3, npts, seed + 1)
    if dtype == "iv64":
        return exps, uniform_f64(len(exps), seed), boxes(3, npts, seed + 1)
    return exps, uniform_f64(len(exps), seed), points_f64(3, npts, seed + 1)


def composition_case(npairs, degp, degq, seed, dtype="modp"):
    """npairs pairs (p, q): p dense of degree degp (coefficients [npairs, degp+1],
    index = degree), q dense of degree degq (coefficients [npairs, degq+1]).
    FP64 draws q from uniform[-1, 1] scaled by 1/(degq+1), so that q^e stays
    inside the FP64 range (unscaled, the coefficients of q^512 overflow)."""
    if dtype == "modp":
        pc = residues(npairs * (degp + 1), seed).reshape(npairs, degp + 1)
        qc = residues(npairs * (degq + 1), seed + 1).reshape(npairs, degq + 1)
        return pc, qc
    pc = uniform_f64(npairs * (degp + 1), seed).reshape(npairs, degp + 1)
    qc = uniform_f64(npairs * (degq + 1), seed + 1).reshape(npairs, degq + 1) / (degq + 1)
    return pc, qc
