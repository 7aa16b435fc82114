"""Exact rational values of dense univariate polynomials at many points, on
all host cores (spawned worker processes: safe after CUDA is initialised in
the parent).  Test infrastructure over oracle.exact."""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

from oracle import exact as X


def _one(args):
    coeffs_by_degree, x = args
    return X.exact_horner_univariate(coeffs_by_degree, x)


def exact_horner_many(coeffs_by_degree, xs):
    """[(p(x), sum |c_i||x|^i) as Fractions for x in xs], exactly."""
    cb = [float(v) for v in coeffs_by_degree]
    work = [(cb, float(x)) for x in xs]
    with ProcessPoolExecutor(max_workers=max(1, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_one, work, chunksize=1))
