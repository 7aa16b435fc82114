"""Plain CPU oracle for fast polynomial evaluation and composition.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product path never does.
It shares no code with the CUDA library.  Each function names the passage of
Moroz, "Fast polynomial evaluation and composition" (arXiv:1307.5655) that it
follows; the C source ``oracle.c`` lists the readings taken where the paper
is silent.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(worked example of Sec. 1, Table 1, closed forms, exact rationals, brute
force, interval containment).
"""
import ctypes
import os

import numpy as np

from . import build as _build

P_MODP = 0xFFFFFFFF00000001  # 2^64 - 2^32 + 1
SCHEMES = {"D": 0, "H": 1, "E": 2, "B": 3, "CUSTOM": 4}

_lib = None


def _L():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, i32, P = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.or_scheme_f.restype = i64
        lib.or_scheme_f.argtypes = [i32, P, i64, i64]
        lib.or_build_tree.restype = i64
        lib.or_build_tree.argtypes = [i32, i64, P, i32, P, i64, i32, i64, P, P, P, P, P, P]
        for name in ("or_eval_f64_plain", "or_eval_modp_plain"):
            getattr(lib, name).restype = i32
        lib.or_eval_f64_plain.argtypes = [i32, i64, P, P, i64, P, P, P]
        lib.or_eval_modp_plain.argtypes = [i32, i64, P, P, i64, P, P]
        lib.or_walk_f64.restype = i32
        lib.or_walk_f64.argtypes = [i32, i64, P, P, P, P, P, i64, P, P]
        lib.or_walk_modp.restype = i32
        lib.or_walk_modp.argtypes = [i32, i64, P, P, P, P, P, i64, P, P]
        lib.or_walk_iv64.restype = i32
        lib.or_walk_iv64.argtypes = [i32, i64, P, P, P, P, P, i64, P, P, P, P]
        lib.or_iv_pow.restype = None
        lib.or_iv_pow.argtypes = [i64, P, P, i64, P, P]
        lib.or_iv_mul.restype = None
        lib.or_iv_mul.argtypes = [i64, P, P, P, P, P, P]
        lib.or_compose_modp_plain.restype = i32
        lib.or_compose_modp_plain.argtypes = [i64, P, i64, P, P]
        lib.or_compose_f64_plain.restype = i32
        lib.or_compose_f64_plain.argtypes = [i64, P, i64, P, P, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _scheme_id(scheme):
    return SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc < 0:
        raise OracleError("oracle error %d" % rc)
    return rc


def scheme_f(scheme, n, ftab=None):
    """f(n) of the function scheme (Sec. 1.1, Sec. 1.2); n = #terms - 1."""
    ft = None if ftab is None else np.ascontiguousarray(ftab, dtype=np.int32)
    return _check(_L().or_scheme_f(_scheme_id(scheme), None if ft is None else _p(ft),
                                   0 if ft is None else len(ft), int(n)))


class Tree:
    """Evaluation tree (Def. 1.1) in node index order <_t (Sec. 1)."""

    def __init__(self, nvars, node_e, term_of_node, parent, pd_var, pd, lh):
        self.nvars = nvars
        self.node_e = node_e
        self.term_of_node = term_of_node
        self.parent = parent
        self.pd_var = pd_var
        self.pd = pd
        self.lh = lh

    @property
    def n(self):
        return len(self.parent)

    def children(self, i):
        return [int(j) for j in np.nonzero(self.parent == i)[0]]

    def node_coeffs(self, coeffs, dtype):
        c = np.zeros(self.n, dtype=dtype)
        real = self.term_of_node >= 0
        c[real] = np.asarray(coeffs, dtype=dtype)[self.term_of_node[real]]
        return c

    def partial_degrees(self):
        """Set of distinct (variable, degree) over non-root nodes with degree > 0."""
        return {(int(v), int(d)) for v, d in zip(self.pd_var[:-1], self.pd[:-1]) if d > 0}


def build_tree(exps, scheme="E", ftab=None, lh_rule=0):
    """Def. 1.2 applied recursively per variable (Remark, Sec. 1.1); lazy
    heights per Def. 1.3 (lh_rule=0: the corrected rule; 1: as printed)."""
    e = np.ascontiguousarray(exps, dtype=np.int32)
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    nterms, nvars = e.shape
    cap = nterms * nvars + 1
    node_e = np.zeros((cap, nvars), dtype=np.int32)
    tnode = np.zeros(cap, dtype=np.int64)
    parent = np.zeros(cap, dtype=np.int64)
    pd_var = np.zeros(cap, dtype=np.int32)
    pd = np.zeros(cap, dtype=np.int64)
    lh = np.zeros(cap, dtype=np.int32)
    ft = None if ftab is None else np.ascontiguousarray(ftab, dtype=np.int32)
    n = _check(_L().or_build_tree(nvars, nterms, _p(e), _scheme_id(scheme),
                                  None if ft is None else _p(ft), 0 if ft is None else len(ft),
                                  lh_rule, cap, _p(node_e), _p(tnode), _p(parent), _p(pd_var),
                                  _p(pd), _p(lh)))
    return Tree(nvars, node_e[:n].copy(), tnode[:n].copy(), parent[:n].copy(), pd_var[:n].copy(),
                pd[:n].copy(), lh[:n].copy())


def _points(points, nvars, dtype):
    x = np.ascontiguousarray(points, dtype=dtype)
    if x.ndim == 1:
        x = x.reshape(1, -1)
    assert x.shape[0] == nvars
    return x


def _drop_zero(exps, coeffs):
    e = np.asarray(exps, dtype=np.int32)
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    c = np.asarray(coeffs)
    keep = c != 0
    return np.ascontiguousarray(e[keep]), np.ascontiguousarray(c[keep])


def eval_f64(exps, coeffs, points):
    """Plain definition p(x) = sum c_e x^e in FP64; returns (p, sum |c_e x^e|)."""
    e = np.ascontiguousarray(exps, dtype=np.int32)
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    x = _points(points, e.shape[1], np.float64)
    out = np.empty(x.shape[1])
    absum = np.empty(x.shape[1])
    _check(_L().or_eval_f64_plain(e.shape[1], e.shape[0], _p(e), _p(c), x.shape[1], _p(x), _p(out), _p(absum)))
    return out, absum


def eval_modp(exps, coeffs, points):
    """Plain definition over Z/pZ, p = 2^64 - 2^32 + 1 (unsigned __int128 % p)."""
    e = np.ascontiguousarray(exps, dtype=np.int32)
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    c = np.ascontiguousarray(coeffs, dtype=np.uint64)
    x = _points(points, e.shape[1], np.uint64)
    out = np.empty(x.shape[1], dtype=np.uint64)
    _check(_L().or_eval_modp_plain(e.shape[1], e.shape[0], _p(e), _p(c), x.shape[1], _p(x), _p(out)))
    return out


def _tree_args(t):
    return (t.nvars, t.n, _p(t.parent), _p(t.pd_var), _p(t.pd), _p(t.lh))


def walk_f64(tree, node_c, points):
    """Coefficient walk of Sec. 2.1 in round-to-nearest FP64."""
    c = np.ascontiguousarray(node_c, dtype=np.float64)
    x = _points(points, tree.nvars, np.float64)
    out = np.empty(x.shape[1])
    _check(_L().or_walk_f64(*_tree_args(tree), _p(c), x.shape[1], _p(x), _p(out)))
    return out


def walk_modp(tree, node_c, points):
    """Coefficient walk of Sec. 2.1 over Z/pZ."""
    c = np.ascontiguousarray(node_c, dtype=np.uint64)
    x = _points(points, tree.nvars, np.uint64)
    out = np.empty(x.shape[1], dtype=np.uint64)
    _check(_L().or_walk_modp(*_tree_args(tree), _p(c), x.shape[1], _p(x), _p(out)))
    return out


def walk_iv64(tree, node_c, lo, hi):
    """Coefficient walk of Sec. 2.1 in directed-rounding interval arithmetic."""
    c = np.ascontiguousarray(node_c, dtype=np.float64)
    lo = _points(lo, tree.nvars, np.float64)
    hi = _points(hi, tree.nvars, np.float64)
    olo = np.empty(lo.shape[1])
    ohi = np.empty(lo.shape[1])
    _check(_L().or_walk_iv64(*_tree_args(tree), _p(c), lo.shape[1], _p(lo), _p(hi), _p(olo), _p(ohi)))
    return olo, ohi


def eval_iv64(exps, coeffs, lo, hi, scheme="E", ftab=None):
    """Interval evaluation: zero terms dropped, tree built, walk run."""
    e, c = _drop_zero(exps, np.asarray(coeffs, dtype=np.float64))
    t = build_tree(e, scheme, ftab)
    return walk_iv64(t, t.node_coeffs(c, np.float64), lo, hi)


def eval_walk_modp(exps, coeffs, points, scheme="E", ftab=None):
    e, c = _drop_zero(exps, np.asarray(coeffs, dtype=np.uint64))
    t = build_tree(e, scheme, ftab)
    return walk_modp(t, t.node_coeffs(c, np.uint64), points)


def eval_walk_f64(exps, coeffs, points, scheme="E", ftab=None):
    e, c = _drop_zero(exps, np.asarray(coeffs, dtype=np.float64))
    t = build_tree(e, scheme, ftab)
    return walk_f64(t, t.node_coeffs(c, np.float64), points)


def iv_pow(lo, hi, d):
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    olo, ohi = np.empty_like(lo), np.empty_like(hi)
    _L().or_iv_pow(len(lo), _p(lo), _p(hi), int(d), _p(olo), _p(ohi))
    return olo, ohi


def iv_mul(alo, ahi, blo, bhi):
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (alo, ahi, blo, bhi)]
    olo, ohi = np.empty_like(a[0]), np.empty_like(a[0])
    _L().or_iv_mul(len(a[0]), *[_p(v) for v in a], _p(olo), _p(ohi))
    return olo, ohi


def compose_modp(pc, qc):
    """r = p o q over Z/pZ by the plain definition sum c_e q^e (schoolbook)."""
    pc = np.ascontiguousarray(pc, dtype=np.uint64)
    qc = np.ascontiguousarray(qc, dtype=np.uint64)
    out = np.empty((len(pc) - 1) * (len(qc) - 1) + 1, dtype=np.uint64)
    _check(_L().or_compose_modp_plain(len(pc), _p(pc), len(qc), _p(qc), _p(out)))
    return out


def compose_f64(pc, qc):
    """r = p o q in FP64 by the plain definition; also returns |p| o |q|."""
    pc = np.ascontiguousarray(pc, dtype=np.float64)
    qc = np.ascontiguousarray(qc, dtype=np.float64)
    n = (len(pc) - 1) * (len(qc) - 1) + 1
    out, absout = np.empty(n), np.empty(n)
    _check(_L().or_compose_f64_plain(len(pc), _p(pc), len(qc), _p(qc), _p(out), _p(absout)))
    return out, absout
