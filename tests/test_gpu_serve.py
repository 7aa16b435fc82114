"""Serving with continuous batching: each served result meets its value
type's parity bar against the CPU oracle (tests/checks.py) and equals the
same request evaluated alone (bit for bit), requests arriving while batches
run are admitted, the HBM budget bounds what is admitted at once, and several
threads may submit concurrently."""
import threading
import time

import numpy as np
import pytest

import workloads as W
import paper_1307_5655_gb300 as fpl
from checks import check_any

pytestmark = pytest.mark.gpu
DTYPES = ["f64", "f32c", "iv64", "modp"]


def _host_points(dtype, nv, npts, seed):
    if dtype == "iv64":
        lo, hi = W.boxes(nv, npts, seed)
        return np.ascontiguousarray(np.stack([lo, hi], axis=1))
    if dtype == "modp":
        return W.points_modp(nv, npts, seed)
    if dtype == "f32c":
        return W.to_f32(W.points_f64(nv, npts, seed))
    return W.points_f64(nv, npts, seed)


def _out(dtype, npts):
    npdt = {"f64": np.float64, "f32c": np.float32, "iv64": np.float64, "modp": np.uint64}[dtype]
    return np.full(fpl.out_shape(dtype, npts), 7, dtype=npdt)


def _requests(n, seed, terms=None):
    """n requests of mixed value type, variable count, term count and point
    count; terms (a dict) receives (exps, coeffs, scheme) per tree key."""
    r = W.rng(seed)
    trees = {}
    reqs = []
    for j in range(n):
        dt = DTYPES[int(r.integers(0, 4))]
        nv = 1 if r.random() < 0.5 else 2
        k = int(np.exp(r.uniform(np.log(8), np.log(4000))))
        key = (dt == "modp", nv, k)
        if key not in trees:
            e = W.dense_univariate_exps(k) if nv == 1 else W.graded_prefix_exps(k, 2)
            c = W.residues(len(e), k) if dt == "modp" else W.uniform_f64(len(e), k)
            scheme = "E" if (k & (k - 1)) == 0 else "B"
            trees[key] = fpl.fp_compile(e, c, scheme, modp=dt == "modp")
            if terms is not None:
                terms[trees[key].handle] = (e, c, scheme)
        npts = int(np.exp(r.uniform(0, np.log(20000))))
        reqs.append((trees[key], dt, _host_points(dt, nv, npts, seed * 1000 + j), _out(dt, npts)))
    return trees, reqs


def _alone(tree, dt, pts):
    return fpl.fp_eval_host(tree, dt, pts)


def _oracle_points(dt, pts):
    """Host request points in the oracle's layout (iv64: (lo, hi))."""
    if dt == "iv64":
        return pts[:, 0, :], pts[:, 1, :]
    return pts


def test_served_results_equal_alone():
    terms = {}
    trees, reqs = _requests(80, 1, terms)
    srv = fpl.Server(hbm_budget_bytes=64 << 20, max_batch_jobs=16, streams=3)
    r = W.rng(2)
    for tree, dt, pts, out in reqs:
        srv.submit(tree, dt, pts, out)
        if r.random() < 0.3:
            time.sleep(float(r.uniform(0, 0.002)))  # arrivals while batches run
    srv.drain(120)
    done = srv.poll()
    assert len(done) == len(reqs) and all(st == 0 for _, st, _ in done)
    for tree, dt, pts, out in reqs:
        assert np.array_equal(out.view(np.uint8), _alone(tree, dt, pts).view(np.uint8))
        e, c, scheme = terms[tree.handle]
        check_any(dt, e, c, _oracle_points(dt, pts), scheme, out)
    assert srv.stats()["batches"] > 1
    srv.close()


def test_admission_respects_the_budget():
    trees, reqs = _requests(40, 3)
    budget = 2 << 20
    srv = fpl.Server(hbm_budget_bytes=budget, max_batch_jobs=64, streams=4)
    for tree, dt, pts, out in reqs:
        srv.submit(tree, dt, pts, out)
    srv.drain(120)
    assert len(srv.poll()) == len(reqs)
    biggest = max(pts.nbytes + out.nbytes for _, _, pts, out in reqs)
    assert srv.stats()["peak_bytes"] <= max(budget, biggest)
    for tree, dt, pts, out in reqs:
        assert np.array_equal(out.view(np.uint8), _alone(tree, dt, pts).view(np.uint8))
    srv.close()


def test_request_larger_than_budget_runs_alone():
    e = W.dense_univariate_exps(100)
    t = fpl.fp_compile(e, W.uniform_f64(100, 1), "E")
    pts = W.points_f64(1, 200000, 2)
    out = _out("f64", 200000)
    srv = fpl.Server(hbm_budget_bytes=1 << 20)
    srv.submit(t, "f64", pts, out)
    srv.drain(60)
    assert srv.poll()[0][1] == 0
    assert np.array_equal(out, _alone(t, "f64", pts))
    srv.close()


def test_concurrent_submitters():
    trees, reqs = _requests(48, 5)
    srv = fpl.Server(hbm_budget_bytes=32 << 20, max_batch_jobs=8, streams=4)

    def worker(part):
        for tree, dt, pts, out in part:
            srv.submit(tree, dt, pts, out)

    th = [threading.Thread(target=worker, args=(reqs[i::4],)) for i in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    srv.drain(120)
    assert len(srv.poll()) == len(reqs)
    for tree, dt, pts, out in reqs:
        assert np.array_equal(out.view(np.uint8), _alone(tree, dt, pts).view(np.uint8))
    srv.close()


def test_drain_deadline_then_completion():
    """The bounded wait: a drain whose deadline passes while a long request
    runs returns FP_E_TIMEOUT (the server keeps working, nothing is lost);
    a second drain then completes and the result equals the request alone."""
    k = 1 << 15
    e = W.dense_univariate_exps(k)
    c = W.uniform_f64(k, 41)
    tree = fpl.fp_compile(e, c, "E")
    pts = _host_points("iv64", 1, 1 << 20, 42)  # about 0.4 s of interval work
    out = _out("iv64", 1 << 20)
    srv = fpl.Server(hbm_budget_bytes=1 << 30, max_batch_jobs=4, streams=1)
    srv.submit(tree, "iv64", pts, out)
    with pytest.raises(fpl.FastPolyError) as ex:
        srv.drain(1e-3)
    assert ex.value.code == -8
    srv.drain(120)
    done = srv.poll()
    assert len(done) == 1 and done[0][1] == 0
    srv.close()
    assert np.array_equal(out, _alone(tree, "iv64", pts))
