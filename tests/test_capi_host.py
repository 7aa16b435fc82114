"""Host-side checks of the C ABI (no GPU): the library loads and exports every
symbol the header declares, and the host compiler builds exactly the tree
the oracle builds (index work is compared bit for bit)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1307_5655_gb300 as fpl

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fastpoly.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fp_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert "fp_compile" in names and "fp_eval" in names
    lib = ctypes.CDLL(fpl.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def _enum(name_prefix):
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(%s[A-Z0-9_]+)\s*=\s*(-?\d+)" % name_prefix, src)}


def test_binding_constants_match_header():
    """The binding's names and codes are the header's: rates in enum order,
    value types, schemes and status codes."""
    rates = _enum("FP_RATE_")
    count = rates.pop("FP_RATE_COUNT")
    assert count == len(fpl.RATE_NAMES) == len(rates)
    assert sorted(rates.values()) == list(range(count))
    by_index = [k[len("FP_RATE_"):].lower() for k, _ in sorted(rates.items(), key=lambda kv: kv[1])]
    assert by_index == list(fpl.RATE_NAMES)
    dtypes = _enum("FP_")
    for name, code in fpl.DTYPES.items():
        assert dtypes["FP_" + name.upper()] == code, name
    assert dtypes["FP_OK"] == 0 and dtypes["FP_E_TIMEOUT"] == -8 and dtypes["FP_E_INTERNAL"] == -9


def _compare(exps, coeffs, scheme, ftab=None):
    t = fpl.fp_compile_host(exps, coeffs, scheme, ftab)
    got = t.export()
    ref = O.build_tree(exps, scheme, ftab)
    assert np.array_equal(got["node_e"], ref.node_e)
    assert np.array_equal(got["term_of_node"], ref.term_of_node)
    assert np.array_equal(got["parent"], ref.parent)
    assert np.array_equal(got["pd_var"], ref.pd_var)
    assert np.array_equal(got["pd"], ref.pd)
    assert np.array_equal(got["lh"], ref.lh)
    info = t.info()
    assert info["nnodes"] == ref.n and info["max_lazy_height"] == int(ref.lh.max())
    t.free()


def _ftab(kind, nmax, seed=0):
    ft = np.zeros(nmax + 1, dtype=np.int32)
    r = W.rng(seed)
    for n in range(1, nmax + 1):
        if kind == "random":
            ft[n] = r.integers(1, n + 1)
        else:  # Estrin above 10 terms, Horner below (Remark of Sec. 1.1)
            ft[n] = 2 ** int(math.floor(math.log2(n))) if n > 10 else 1
    return ft


@pytest.mark.parametrize("k", [1, 2, 3, 9, 100, 1000, 1024, 3000, 10007])
@pytest.mark.parametrize("scheme", ["D", "H", "E", "B", "random", "hybrid"])
def test_univariate_tree_matches_oracle(k, scheme):
    if scheme == "D" and k > 3000:
        pytest.skip("direct scheme oracle recursion is linear in depth")
    e = W.dense_univariate_exps(k)
    c = W.uniform_f64(k, k)
    ft = None
    if scheme in ("random", "hybrid"):
        ft, scheme = _ftab(scheme, k, k), "CUSTOM"
    e, c = W.shuffled(e, c, 3)
    _compare(e, c, scheme, ft)


@pytest.mark.parametrize("nvars", [2, 3, 4])
@pytest.mark.parametrize("scheme", ["D", "H", "E", "B"])
def test_multivariate_tree_matches_oracle(nvars, scheme):
    for seed in range(6):
        r = W.rng(seed)
        if seed % 2 == 0:
            e = W.graded_prefix_exps(int(r.integers(1, 60)), nvars)
        else:
            pts = {tuple(int(v) for v in r.integers(0, 6, size=nvars)) for _ in range(40)}
            e = np.array(sorted(pts), dtype=np.int32)
        c = W.uniform_f64(len(e), seed) + 2.0  # non-zero
        e, c = W.shuffled(e, c, seed)
        _compare(e, c, scheme)


def test_trivariate_degree40_tree_matches_oracle():
    e = W.total_degree_exps(3, 40)
    c = W.uniform_f64(len(e), 1)
    for s in "EB":
        _compare(e, c, s)


def test_sparse_univariate_root_degree():
    e = np.array([[40], [17], [5]], dtype=np.int32)
    _compare(e, np.array([1.0, -2.0, 3.0]), "E")


def test_zero_coefficients_dropped_and_zero_polynomial():
    t = fpl.fp_compile_host(np.array([[3], [2], [1]]), np.array([1.0, 0.0, 2.0]), "H")
    assert t.info()["nnodes"] == 2
    z = fpl.fp_compile_host(np.array([[3], [1]]), np.array([0.0, 0.0]), "E")
    assert z.info()["nnodes"] == 0
    z0 = fpl.fp_compile_host(np.zeros((0, 1), dtype=np.int32), np.zeros(0), "E")
    assert z0.info()["nnodes"] == 0


@pytest.mark.parametrize("bad,code", [
    ((np.array([[1], [1]]), np.array([1.0, 2.0]), "E", None, False), -2),      # duplicate
    ((np.array([[1], [-1]]), np.array([1.0, 2.0]), "E", None, False), -1),     # negative exponent
    ((np.array([[2], [1], [0]]), np.array([1.0, 2.0, 3.0]), "CUSTOM", np.array([0, 0, 1]), False), -3),
    ((np.array([[1], [0]]), np.array([O.P_MODP, 1], dtype=np.uint64), "E", None, True), -1),
    ((np.zeros((1, 9), dtype=np.int32), np.array([1.0]), "E", None, False), -6),  # too many variables
])
def test_compile_errors(bad, code):
    with pytest.raises(fpl.FastPolyError) as ei:
        fpl.fp_compile_host(*bad)
    assert ei.value.code == code


def test_more_compile_errors():
    """The documented error codes for bad schemes, split tables, value types
    and pointers (host-only compile: no GPU)."""
    e3, c3 = np.array([[2], [1], [0]]), np.array([1.0, 2.0, 3.0])
    cases = [
        ((e3, c3, 9), -3),                                    # unknown scheme
        ((e3, c3, "CUSTOM", np.array([0, 2, 3])), -3),        # f(1) = 2 > 1
        ((e3, c3, "CUSTOM", np.array([0, 1])), -3),           # table shorter than n
        ((e3, c3, "CUSTOM", None), -3),                       # no table
        ((np.zeros((1, 0), dtype=np.int32), np.array([1.0]), "E"), -1),  # no variable
        ((e3, np.array([np.nan, 1.0, 2.0]), "E"), -1),        # NaN coefficient
    ]
    for args, code in cases:
        with pytest.raises(fpl.FastPolyError) as ei:
            fpl.fp_compile_host(*args)
        assert ei.value.code == code, args
    h = ctypes.c_void_p()
    lib = fpl._lib
    assert lib.fp_compile_host(1, 2, None, None, 0, 2, None, 0, ctypes.byref(h)) == -1   # NULL arrays
    assert lib.fp_compile_host(1, 0, None, None, 0, 2, None, 0, None) == -1              # NULL out
    assert lib.fp_compile_host(1, -1, None, None, 0, 2, None, 0, ctypes.byref(h)) == -1  # negative count
    assert lib.fp_compile_host(1, 0, None, None, 2, 2, None, 0, ctypes.byref(h)) == -4   # IV64 coefficients
    assert lib.fp_compile_host(1, 0, None, None, 7, 2, None, 0, ctypes.byref(h)) == -4   # no such type


def test_term_count_limit():
    """One term above FP_MAX_TERMS is refused before any work."""
    n = fpl.MAX_TERMS + 1
    e = np.arange(n, dtype=np.int32).reshape(-1, 1)
    with pytest.raises(fpl.FastPolyError) as ex:
        fpl.fp_compile_host(e, np.ones(n), "E")
    assert ex.value.code == -6


def test_eval_on_host_only_tree_is_rejected():
    t = fpl.fp_compile_host(np.array([[1], [0]]), np.array([1.0, 2.0]), "E")
    rc = fpl._lib.fp_eval(t.handle, 0, None, 0, None, None)
    assert rc == -4


@pytest.mark.parametrize("seed", range(48))
def test_random_sparse_trees_match_oracle(seed):
    """Fuzz: random sparse term sets in 1-4 variables, given in random order,
    under random schemes (including random split tables): the host compiler's
    tree equals the oracle's index for index."""
    r = W.rng(29000 + seed)
    nvars = int(r.integers(1, 5))
    deg = int(r.integers(1, 60 if nvars == 1 else 10))
    full = W.total_degree_exps(nvars, deg) if nvars > 1 else np.arange(deg + 1)[::-1].reshape(-1, 1)
    keep = r.random(len(full)) < r.uniform(0.1, 1.0)
    e = np.ascontiguousarray(full[keep].astype(np.int32))
    if len(e) == 0:
        e = np.ascontiguousarray(full[:1].astype(np.int32))
    e, c = W.shuffled(e, W.uniform_f64(len(e), seed), seed + 1)
    scheme = ["H", "E", "B", "D", "CUSTOM"][int(r.integers(0, 5))]
    ftab = None
    if scheme == "CUSTOM":
        nmax = max(len(e), int(e.max()) + 1)
        ftab = np.zeros(nmax + 1, dtype=np.int32)
        for n in range(1, nmax + 1):
            ftab[n] = r.integers(1, n + 1)
    _compare(e, c, scheme, ftab)


def test_argument_checks_before_any_cuda_call():
    """Entry points refuse bad arguments with FP_E_BAD_VALUE before touching
    the device, and every status has its own message."""
    lib = fpl._lib
    h = ctypes.c_void_p()
    assert lib.fp_server_create(None, ctypes.byref(h)) == -1
    cfg = fpl._ServerCfg(0, 0, 0)  # no HBM budget
    assert lib.fp_server_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    rates = np.zeros(2)
    assert lib.fp_measure_rates(None, 2, None) == -1
    assert lib.fp_measure_rates(rates.ctypes.data_as(ctypes.c_void_p), -1, None) == -1
    msgs = [lib.fp_strerror(c) for c in range(0, -10, -1)]
    assert msgs[0] == b"ok" and len(set(msgs)) == len(msgs) and all(msgs)
    assert lib.fp_strerror(-99) == b"unknown status"


def test_compose_binding_rejects_host_tensors():
    """The composition bindings check their tensors before the C ABI sees a
    host pointer: CPU tensors and unsupported value types raise ValueError."""
    import torch
    t = fpl.fp_compile_host(W.dense_univariate_exps(4), np.ones(4), "E")
    q = torch.ones((2, 3), dtype=torch.float64)
    for fn in (fpl.fp_compose, fpl.fp_compose_noalloc):
        with pytest.raises(ValueError):
            fn(t, "f64", q)
        with pytest.raises(ValueError):
            fn(t, "iv64", q)
        with pytest.raises(ValueError):
            fn(t, "f64", [[1.0, 2.0]])


@pytest.mark.parametrize("dtype,scheme", [("modp", "E"), ("modp", "B"), ("f64", "E"), ("f64", "B")])
def test_compose_workspace_is_affine_in_pairs(dtype, scheme):
    """The work-space count (a dry run of the composition driver, no CUDA
    call): per-pair buffers grow exactly linearly in the number of pairs (a
    multiple of 32 keeps every 8-byte row set a whole number of 256-byte
    granules), shared tables do not; the tree's own coefficients add one
    shared row of nterms; transforms longer than 4096 add their tables."""
    modp = dtype == "modp"
    degp, degq = 128, 64  # products up to length 16385: four-step transforms
    e = W.dense_univariate_exps(degp + 1)
    t = fpl.fp_compile_host(e, np.ones(degp + 1, dtype=np.uint64 if modp else np.float64), scheme, modp=modp)
    ws = [fpl.fp_compose_workspace(t, dtype, degq, n) for n in (64, 128, 192)]
    assert ws[0] < ws[1] < ws[2]
    assert ws[1] - ws[0] == ws[2] - ws[1]
    shared = fpl.fp_compose_workspace(t, dtype, degq, 128, per_pair_coeffs=False)
    assert shared - ws[1] == ((degp + 1) * 8 + 255) // 256 * 256
    # at least the slots, the powers and the two product buffers per pair
    assert ws[1] - ws[0] >= 64 * 8 * (degp * degq + 1)
    assert fpl.fp_compose_workspace(t, dtype, degq, 0) == 0
    with pytest.raises(fpl.FastPolyError):
        fpl.fp_compose_workspace(t, "f64" if modp else "modp", degq, 32)
