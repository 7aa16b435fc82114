"""Python binding of libfastpoly (GB300 / sm_103a): fast polynomial evaluation
and composition through evaluation trees (Moroz, arXiv:1307.5655).

Argument marshalling only: every step of evaluation runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (PyTorch provides device
memory and streams); the library never falls back to the CPU and importing
fails loudly when the compiled library is missing.

Names mirror the C ABI of ``include/fastpoly.h``.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfastpoly.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libfastpoly.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(or python paper_1307_5655_gb300/build.py)")

_lib = ctypes.CDLL(LIB_PATH)
_P, _I, _I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64

for _name, _args in {
    "fp_compile": [_I, _I64, _P, _P, _I, _I, _P, _I64, ctypes.POINTER(_P)],
    "fp_compile_host": [_I, _I64, _P, _P, _I, _I, _P, _I64, ctypes.POINTER(_P)],
    "fp_eval": [_P, _I, _P, _I64, _P, _P],
    "fp_eval_host": [_P, _I, _P, _I64, _P, _P],
    "fp_eval_ex": [_P, _I, _P, _I64, _P, _P, _P],
    "fp_tune": [_P, _I, _P, _I64, _P, _P, _P],
    "fp_tree_info": [_P, _P, _P, _P, _P, _P],
    "fp_tree_export": [_P, _P, _P, _P, _P, _P, _P],
    "fp_measure_rates": [_P, ctypes.c_int, _P],
    "fp_tune_scheme": [ctypes.c_int, _I64, _P, _P, ctypes.c_int, ctypes.c_int, _P, _I64, _P, _P, _P, _P],
    "fp_rns_primes": [ctypes.c_int, _P],
    "fp_compile_rns": [ctypes.c_int, _I64, _P, ctypes.c_int, _P, ctypes.c_int, _P, _I64, _P],
    "fp_eval_rns": [_P, _P, _I64, _P, _P],
    "fp_crt": [ctypes.c_int, _P, _I64, _P, _P],
    "fp_tree_schedule": [_P] * 12,
    "fp_eval_plain_f64": [_P, _I64, _P, _I64, _P, _P],
    "fp_compose": [_P, _I, _P, _P, _I, _I64, _P, _P],
    "fp_compose_noalloc": [_P, _I, _P, _P, _I, _I64, _P, _P],
    "fp_compose_workspace": [_P, _I, _I, _I, _I64, ctypes.POINTER(ctypes.c_size_t)],
    "fp_set_compose_f64": [_I, _I],
    "fp_resident_create": [_P, ctypes.POINTER(_P)],
    "fp_resident_submit": [_P, _P, ctypes.POINTER(_I64)],
    "fp_resident_query": [_P, _I64],
    "fp_resident_wait": [_P, _I64, ctypes.c_double],
    "fp_resident_state": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I64)],
    "fp_resident_stop": [_P, ctypes.c_double],
}.items():
    getattr(_lib, _name).restype = _I
    getattr(_lib, _name).argtypes = _args
_lib.fp_free.restype = None
_lib.fp_free.argtypes = [_P]
_lib.fp_resident_free.restype = None
_lib.fp_resident_free.argtypes = [_P]
_lib.fp_strerror.restype = ctypes.c_char_p
_lib.fp_strerror.argtypes = [_I]

P_MODP = 0xFFFFFFFF00000001
SCHEMES = {"D": 0, "H": 1, "E": 2, "B": 3, "CUSTOM": 4}
DTYPES = {"f64": 0, "f32c": 1, "iv64": 2, "modp": 3}


class FastPolyError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, _lib.fp_strerror(code).decode(), code))
        self.code = code


def _check(rc, what):
    if rc != 0:
        raise FastPolyError(rc, what)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if isinstance(a, np.ndarray) else ctypes.c_void_p(a.data_ptr())


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Tree:
    """A compiled evaluation tree (owned by the library until freed)."""

    def __init__(self, handle, nvars, coeff_type, nterms=None):
        self._h = handle
        self.nvars = nvars
        self.coeff_type = coeff_type
        self.nterms = nterms  # terms given to the compiler (rows of per-pair coefficients)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            _lib.fp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        n = ctypes.c_int64()
        nv, lh, npw, ct = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.fp_tree_info(self._h, ctypes.byref(n), ctypes.byref(nv), ctypes.byref(lh), ctypes.byref(npw),
                                 ctypes.byref(ct)), "fp_tree_info")
        return {"nnodes": n.value, "nvars": nv.value, "max_lazy_height": lh.value, "npowers": npw.value,
                "coeff_type": ct.value}

    def export(self):
        n = self.info()["nnodes"]
        e = np.zeros((n, self.nvars), dtype=np.int32)
        tn = np.zeros(n, dtype=np.int64)
        par = np.zeros(n, dtype=np.int64)
        pv = np.zeros(n, dtype=np.int32)
        pd = np.zeros(n, dtype=np.int64)
        lh = np.zeros(n, dtype=np.int32)
        _check(_lib.fp_tree_export(self._h, _ptr(e), _ptr(tn), _ptr(par), _ptr(pv), _ptr(pd), _ptr(lh)),
               "fp_tree_export")
        return {"node_e": e, "term_of_node": tn, "parent": par, "pd_var": pv, "pd": pd, "lh": lh}

    def schedule(self):
        """The grouped-op schedule of the fused-type kernels (fp_tree_schedule)."""
        nops, nst, nprog = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.fp_tree_schedule(self._h, ctypes.byref(nops), None, None, None, ctypes.byref(nst), None,
                                     ctypes.byref(nprog), None, None, None, None), "fp_tree_schedule")
        n = self.info()["nnodes"]
        words = np.zeros((nops.value, 4), dtype=np.uint32)
        a = np.zeros(nops.value, dtype=np.int64)
        b = np.zeros(nops.value, dtype=np.int64)
        st = np.zeros(nst.value, dtype=np.int64)
        prog = np.zeros((nprog.value, 2), dtype=np.uint32)
        cp = np.zeros(max(n - 1, 0), dtype=np.uint32)
        bp = np.zeros(17, dtype=np.int32)
        lay = np.zeros(8, dtype=np.int32)
        _check(_lib.fp_tree_schedule(self._h, None, _ptr(words), _ptr(a), _ptr(b), None, _ptr(st), None, _ptr(prog),
                                     _ptr(cp), _ptr(bp), _ptr(lay)), "fp_tree_schedule")
        return {"op_words": words, "op_a_node": a, "op_b_node": b, "stream": st, "prog": prog, "chain_pid": cp,
                "block_pow": bp, "nlive": int(lay[0]), "nslot": int(lay[1]), "entries": int(lay[2]),
                "block_scheme": int(lay[3]), "root_leaf": int(lay[4]), "root_lh": int(lay[5]),
                "root_pid": int(lay[6]), "split": int(lay[7])}


def _compile(fn, exps, coeffs, scheme, ftab, modp):
    e = np.ascontiguousarray(exps, dtype=np.int32)
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    nterms, nvars = e.shape
    c = np.ascontiguousarray(coeffs, dtype=np.uint64 if modp else np.float64)
    if len(c) != nterms:
        raise ValueError("coeffs and exps disagree on the number of terms")
    ft = None if ftab is None else np.ascontiguousarray(ftab, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = fn(nvars, nterms, _ptr(e), _ptr(c), DTYPES["modp"] if modp else DTYPES["f64"],
            SCHEMES[scheme] if isinstance(scheme, str) else int(scheme),
            None if ft is None else _ptr(ft), 0 if ft is None else len(ft), ctypes.byref(h))
    _check(rc, fn.__name__)
    return Tree(h.value, nvars, "modp" if modp else "f64", nterms)


def fp_compile(exps, coeffs, scheme="E", ftab=None, modp=False):
    """Compile terms (exps [nterms, nvars], coeffs [nterms]) under a function
    scheme ('D', 'H', 'E', 'B' or 'CUSTOM' with ftab[n] = f(n)) and upload the
    schedule to the current CUDA device.  modp=True: uint64 coefficients mod p."""
    return _compile(_lib.fp_compile, exps, coeffs, scheme, ftab, modp)


def fp_compile_host(exps, coeffs, scheme="E", ftab=None, modp=False):
    """Host-only compile (no CUDA call): for inspecting the tree."""
    return _compile(_lib.fp_compile_host, exps, coeffs, scheme, ftab, modp)


def out_shape(dtype, npts):
    return (npts,) if dtype in ("f64", "modp") else (2, npts)


def _torch_dtype(dtype):
    import torch
    # residues travel as int64 bit patterns (uint64 tensors have few ops in torch)
    return {"f64": torch.float64, "f32c": torch.float32, "iv64": torch.float64, "modp": torch.int64}[dtype]


def _elem_types(dtype):
    """Element types accepted for a value type's points and results (torch
    dtypes; residues as int64 or uint64 bit patterns)."""
    import torch
    if dtype == "modp":
        return (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())
    return {"f64": (torch.float64,), "f32c": (torch.float32,), "iv64": (torch.float64,)}[dtype]


def _point_elems(dtype, nvars, npts):
    """Elements of a points array in the layout of fp_eval."""
    return nvars * npts * (2 if dtype == "iv64" else 1)


def _out_elems(dtype, npts):
    """Elements of a result array in the layout of fp_eval (out_shape)."""
    return npts * (2 if dtype in ("f32c", "iv64") else 1)


def _check_extent(what, name, etype, numel, types, need):
    if etype not in types:
        raise ValueError("%s: %s has element type %s, expected %s" % (what, name, etype, " or ".join(map(str, types))))
    if numel < need:
        raise ValueError("%s: %s holds %d elements, the call touches %d" % (what, name, numel, need))


def _check_device(what, name, a, types, need, device=None):
    """Refuse, before the C call, a device buffer that would send a kernel
    outside its memory: not a contiguous CUDA tensor, another element type,
    fewer elements than the call touches, or another device than `device`."""
    import torch
    if not isinstance(a, torch.Tensor) or not a.is_cuda or not a.is_contiguous():
        raise ValueError("%s: %s must be a contiguous CUDA tensor" % (what, name))
    _check_extent(what, name, a.dtype, a.numel(), types, need)
    if device is not None and a.device != device:
        raise ValueError("%s: %s is on %s, the points on %s" % (what, name, a.device, device))


def _check_eval_io(what, tree, dtype, points, npts, out):
    """points and out in the layouts of fp_eval for this tree, value type and
    number of points."""
    types = _elem_types(dtype)
    _check_device(what, "points", points, types, _point_elems(dtype, tree.nvars, npts))
    _check_device(what, "out", out, types, _out_elems(dtype, npts), points.device)


def _check_host_io(what, tree, dtype, points, npts, out):
    """The same for host buffers (numpy arrays or CPU tensors), which the
    library copies from and to."""
    import torch
    np_types = {"f64": (np.float64,), "f32c": (np.float32,), "iv64": (np.float64,),
                "modp": (np.uint64, np.int64)}[dtype]
    for name, a, need in (("points", points, _point_elems(dtype, tree.nvars, npts)),
                          ("out", out, _out_elems(dtype, npts))):
        if isinstance(a, np.ndarray):
            if not a.flags.c_contiguous:
                raise ValueError("%s: %s must be a C-contiguous array" % (what, name))
            _check_extent(what, name, a.dtype.type, a.size, np_types, need)
        elif isinstance(a, torch.Tensor) and not a.is_cuda and a.is_contiguous():
            _check_extent(what, name, a.dtype, a.numel(), _elem_types(dtype), need)
        else:
            raise ValueError("%s: %s must be a contiguous host array or CPU tensor" % (what, name))


def fp_eval(tree, dtype, points, npts=None, out=None, stream=None):
    """Evaluate on the GPU.  points: CUDA tensor in the layout of fp_eval
    (f64 [nvars, npts] float64; f32c [nvars, npts] float32; iv64
    [nvars, 2, npts] float64; modp [nvars, npts] uint64).  Returns out."""
    import torch
    _check_device("fp_eval", "points", points, _elem_types(dtype), 0)
    if npts is None:
        npts = points.shape[-1]
    if out is None:
        out = torch.empty(out_shape(dtype, npts), dtype=_torch_dtype(dtype), device=points.device)
    _check_eval_io("fp_eval", tree, dtype, points, npts, out)
    _check(_lib.fp_eval(tree.handle, DTYPES[dtype], _ptr(points), npts, _ptr(out), _stream_handle(stream)), "fp_eval")
    return out


class LaunchCfg(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("points_per_thread", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


KERNELS = {"auto": 0, "ops": 1, "node": 2}


def fp_eval_ex(tree, dtype, points, kernel="auto", npts=None, out=None, stream=None, ppt=0):
    """fp_eval with an explicit kernel choice ('auto', 'ops', 'node') and
    points per thread (0: automatic)."""
    import torch
    _check_device("fp_eval_ex", "points", points, _elem_types(dtype), 0)
    if npts is None:
        npts = points.shape[-1]
    if out is None:
        out = torch.empty(out_shape(dtype, npts), dtype=_torch_dtype(dtype), device=points.device)
    _check_eval_io("fp_eval_ex", tree, dtype, points, npts, out)
    cfg = LaunchCfg(KERNELS[kernel], ppt)
    _check(_lib.fp_eval_ex(tree.handle, DTYPES[dtype], _ptr(points), npts, _ptr(out), _stream_handle(stream),
                           ctypes.byref(cfg)), "fp_eval_ex")
    return out


RNS_MAX_PRIMES = 64
MAX_TERMS = 1 << 24  # FP_MAX_TERMS


def fp_rns_primes(k):
    """The library's first k primes q_i = 2^64 - c_i (largest first), uint64."""
    q = np.zeros(k, dtype=np.uint64)
    _check(_lib.fp_rns_primes(k, _ptr(q)), "fp_rns_primes")
    return q


def fp_compile_rns(exps, residues, scheme="E", ftab=None):
    """Compile integer coefficients given as residues [k][nterms] (uint64,
    residues[i][t] = c_t mod q_i) for fp_eval_rns."""
    e = np.ascontiguousarray(exps, dtype=np.int32)
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    nterms, nvars = e.shape
    r = np.ascontiguousarray(residues, dtype=np.uint64)
    if r.ndim != 2 or r.shape[1] != nterms:
        raise ValueError("residues must be [k][nterms]")
    ft = None if ftab is None else np.ascontiguousarray(ftab, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.fp_compile_rns(nvars, nterms, _ptr(e), r.shape[0], _ptr(r),
                               SCHEMES[scheme] if isinstance(scheme, str) else int(scheme),
                               None if ft is None else _ptr(ft), 0 if ft is None else len(ft), ctypes.byref(h)),
           "fp_compile_rns")
    t = Tree(h.value, nvars, "rns")
    t.rns_k = r.shape[0]
    return t


def fp_eval_rns(tree, points, out=None, stream=None):
    """p(x) mod each prime: points device [k][nvars][npts] (int64 containers of
    uint64 residues), out [k][npts]."""
    import torch
    types = _elem_types("modp")
    _check_device("fp_eval_rns", "points", points, types, 0)
    npts = points.shape[-1]
    k = getattr(tree, "rns_k", 1)
    if out is None:
        out = torch.empty((k, npts), dtype=torch.int64, device=points.device)
    _check_device("fp_eval_rns", "points", points, types, k * tree.nvars * npts)
    _check_device("fp_eval_rns", "out", out, types, k * npts, points.device)
    _check(_lib.fp_eval_rns(tree.handle, _ptr(points), npts, _ptr(out), _stream_handle(stream)), "fp_eval_rns")
    return out


def fp_crt(residues, out=None, stream=None):
    """Integers from residues [k][npts] (device): limbs [npts][k], least
    significant first, two's complement of the value in (-Q/2, Q/2]."""
    import torch
    types = _elem_types("modp")
    _check_device("fp_crt", "residues", residues, types, 0)
    if residues.dim() != 2:
        raise ValueError("fp_crt: residues must be [k][npts]")
    k, npts = residues.shape
    if out is None:
        out = torch.empty((npts, k), dtype=torch.int64, device=residues.device)
    _check_device("fp_crt", "out", out, types, npts * k, residues.device)
    _check(_lib.fp_crt(k, _ptr(residues), npts, _ptr(out), _stream_handle(stream)), "fp_crt")
    return out


def limbs_to_int(limbs):
    """Python integer of k 64-bit limbs (least significant first, two's complement)."""
    v = 0
    for i, w in enumerate(np.asarray(limbs, dtype=np.uint64).tolist()):
        v |= int(w) << (64 * i)
    k = len(limbs)
    return v - (1 << (64 * k)) if v >> (64 * k - 1) else v


RATE_NAMES = ("dfma", "dadd_rd", "dmul_ru", "ffma", "f32c_mad", "f32c_horner", "modp_muladd", "modp_butterfly",
              "imad", "imad_wide")


def fp_measure_rates(stream=None):
    """Sustained rates (G op/s) of the arithmetic the kernels are bound by,
    measured on the current device (fp_measure_rates)."""
    rates = np.zeros(len(RATE_NAMES), dtype=np.float64)
    _check(_lib.fp_measure_rates(_ptr(rates), len(RATE_NAMES), _stream_handle(stream)), "fp_measure_rates")
    return dict(zip(RATE_NAMES, rates.tolist()))


def fp_tune_scheme(exps, coeffs, dtype, points, out=None, stream=None, modp=False):
    """Compile under the fastest combined Estrin/Horner threshold k0 (or the
    Balanced scheme) for these points (fp_tune_scheme); returns (tree, k0),
    k0 = 0 meaning Balanced."""
    import torch
    e = np.ascontiguousarray(exps, dtype=np.int32)
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    nterms, nvars = e.shape
    c = np.ascontiguousarray(coeffs, dtype=np.uint64 if modp else np.float64)
    types = _elem_types(dtype)
    _check_device("fp_tune_scheme", "points", points, types, 0)
    npts = points.shape[-1]
    if out is None:
        out = torch.empty(out_shape(dtype, npts), dtype=_torch_dtype(dtype), device=points.device)
    _check_device("fp_tune_scheme", "points", points, types, _point_elems(dtype, nvars, npts))
    _check_device("fp_tune_scheme", "out", out, types, _out_elems(dtype, npts), points.device)
    h = ctypes.c_void_p()
    k0 = ctypes.c_int64()
    _check(_lib.fp_tune_scheme(nvars, nterms, _ptr(e), _ptr(c), DTYPES["modp"] if modp else DTYPES["f64"],
                               DTYPES[dtype], _ptr(points), npts, _ptr(out), _stream_handle(stream),
                               ctypes.byref(k0), ctypes.byref(h)), "fp_tune_scheme")
    return Tree(h.value, nvars, "modp" if modp else "f64"), k0.value


def fp_tune(tree, dtype, points, out=None, stream=None):
    """Autotune the launch configuration of this tree and value type on these
    points (synchronous); returns (kernel name, points per thread)."""
    import torch
    _check_device("fp_tune", "points", points, _elem_types(dtype), 0)
    npts = points.shape[-1]
    if out is None:
        out = torch.empty(out_shape(dtype, npts), dtype=_torch_dtype(dtype), device=points.device)
    _check_eval_io("fp_tune", tree, dtype, points, npts, out)
    cfg = LaunchCfg()
    _check(_lib.fp_tune(tree.handle, DTYPES[dtype], _ptr(points), npts, _ptr(out), _stream_handle(stream),
                        ctypes.byref(cfg)), "fp_tune")
    names = {v: k for k, v in KERNELS.items()}
    return names[cfg.kernel], cfg.points_per_thread


def fp_eval_host(tree, dtype, points, stream=None):
    """End-to-end: numpy points in host memory -> numpy result (copies inside)."""
    pts = np.ascontiguousarray(points)
    npts = pts.shape[-1]
    npdt = {"f64": np.float64, "f32c": np.float32, "iv64": np.float64, "modp": np.uint64}[dtype]
    out = np.empty(out_shape(dtype, npts), dtype=npdt)
    _check_host_io("fp_eval_host", tree, dtype, pts, npts, out)
    _check(_lib.fp_eval_host(tree.handle, DTYPES[dtype], _ptr(pts), npts, _ptr(out), _stream_handle(stream)),
           "fp_eval_host")
    return out


def fp_eval_plain_f64(coeffs_by_degree, points, out=None, stream=None):
    """Baseline: one thread per point, Horner over dense FP64 coefficients."""
    import torch
    f64 = _elem_types("f64")
    _check_device("fp_eval_plain_f64", "points", points, f64, 0)
    _check_device("fp_eval_plain_f64", "coefficients", coeffs_by_degree, f64, 0, points.device)
    npts = points.shape[-1]
    if out is None:
        out = torch.empty(npts, dtype=torch.float64, device=points.device)
    _check_device("fp_eval_plain_f64", "out", out, f64, npts, points.device)
    _check(_lib.fp_eval_plain_f64(_ptr(coeffs_by_degree), coeffs_by_degree.numel(), _ptr(points), npts, _ptr(out),
                                  _stream_handle(stream)), "fp_eval_plain_f64")
    return out


def _compose_args(tree, dtype, q, pcoeffs, out, degp):
    """Check the tensors of a composition before they reach the C ABI (a host
    pointer or a wrongly shaped buffer there would be a device fault, not an
    error code) and allocate `out` when it is None."""
    import torch
    if dtype not in ("f64", "modp"):
        raise ValueError("composition value types are 'f64' and 'modp'")
    want = _torch_dtype(dtype)

    def dev_tensor(name, a):
        if not isinstance(a, torch.Tensor) or not a.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if a.dim() != 2 or not a.is_contiguous():
            raise ValueError("%s must be a contiguous 2-D tensor" % name)
        if a.dtype != want:
            raise ValueError("%s must have dtype %s for '%s'" % (name, want, dtype))
        if a.device.index != torch.cuda.current_device():
            raise ValueError("%s must be on the current CUDA device (the tree's)" % name)

    dev_tensor("q", q)
    npairs, nq = q.shape
    if nq < 1:
        raise ValueError("q needs at least one coefficient")
    if degp is None:
        degp = int(tree.export()["node_e"][0, 0]) if tree.info()["nnodes"] else 0
    if pcoeffs is not None:
        dev_tensor("pcoeffs", pcoeffs)
        if tree.nterms is not None and tuple(pcoeffs.shape) != (npairs, tree.nterms):
            raise ValueError("pcoeffs must have shape [npairs, nterms] = [%d, %d]" % (npairs, tree.nterms))
        if pcoeffs.shape[0] != npairs:
            raise ValueError("pcoeffs must have one row per pair")
    shape = (npairs, degp * (nq - 1) + 1)
    if out is None:
        out = torch.empty(shape, dtype=want, device=q.device)
    dev_tensor("out", out)
    if tuple(out.shape) != shape:
        raise ValueError("out must have shape [npairs, deg(p) * deg(q) + 1] = [%d, %d]" % shape)
    return npairs, nq - 1, out


def fp_compose(tree, dtype, q, pcoeffs=None, out=None, degp=None, stream=None):
    """Batched composition p_j(q_j(y)): q is a CUDA tensor [npairs, degq + 1]
    (float64, or int64 holding residues for 'modp'); pcoeffs an optional CUDA
    tensor [npairs, nterms] of per-pair coefficients in the compiled term
    order.  Returns out [npairs, deg(p) * degq + 1]."""
    npairs, degq, out = _compose_args(tree, dtype, q, pcoeffs, out, degp)
    pc = None if pcoeffs is None else _ptr(pcoeffs)
    _check(_lib.fp_compose(tree.handle, DTYPES[dtype], pc, _ptr(q), degq, npairs, _ptr(out),
                           _stream_handle(stream)), "fp_compose")
    return out


NOALLOC_SCRATCH_BYTES = 64 << 20


def fp_set_compose_f64(slices=0, min_len=0):
    """Process-wide FP64 composition settings: tensor-core slices per operand
    (6, 7, 8; 0 = 7) and the shortest operand sent to the tensor cores
    (0 = 256; negative = direct convolution only)."""
    _check(_lib.fp_set_compose_f64(slices, min_len), "fp_set_compose_f64")


def fp_compose_workspace(tree, dtype, degq, npairs, per_pair_coeffs=True):
    """Device bytes of work space that fp_compose / fp_compose_noalloc use for
    these sizes (host only: a dry run of the composition driver)."""
    b = ctypes.c_size_t()
    _check(_lib.fp_compose_workspace(tree.handle, DTYPES[dtype], 1 if per_pair_coeffs else 0, degq, npairs,
                                     ctypes.byref(b)), "fp_compose_workspace")
    return b.value


def fp_compose_noalloc(tree, dtype, q, pcoeffs=None, out=None, degp=None, stream=None):
    """fp_compose without any device allocation by the library: the work space
    is a fixed region (NOALLOC_SCRATCH_BYTES per device) shared by all calls,
    so calls must not overlap on the GPU.  The output buffer `out` should be
    provided by the caller (allocating it here would defeat the purpose)."""
    npairs, degq, out = _compose_args(tree, dtype, q, pcoeffs, out, degp)
    pc = None if pcoeffs is None else _ptr(pcoeffs)
    _check(_lib.fp_compose_noalloc(tree.handle, DTYPES[dtype], pc, _ptr(q), degq, npairs, _ptr(out),
                                   _stream_handle(stream)), "fp_compose_noalloc")
    return out


class _Job(ctypes.Structure):
    _fields_ = [("tree", ctypes.c_void_p), ("points", ctypes.c_void_p), ("npts", ctypes.c_int64),
                ("out", ctypes.c_void_p)]


_lib.fp_eval_batch.restype = _I
_lib.fp_eval_batch.argtypes = [_I, _P, _I64, _P]
_lib.fp_batch_create.restype = _I
_lib.fp_batch_create.argtypes = [_I, _P, _I64, ctypes.POINTER(_P)]
_lib.fp_batch_launch.restype = _I
_lib.fp_batch_launch.argtypes = [_P, _P]
_lib.fp_batch_free.restype = None
_lib.fp_batch_free.argtypes = [_P]


def _check_job(what, tree, dtype, points, out):
    """A job (tree, points, out) in the layouts of fp_eval."""
    _check_device(what, "points", points, _elem_types(dtype), 0)
    _check_eval_io(what, tree, dtype, points, points.shape[-1], out)


def _jobs_array(jobs, dtype, what):
    arr = (_Job * max(1, len(jobs)))()
    for i, (tree, pts, out) in enumerate(jobs):
        _check_job(what, tree, dtype, pts, out)
        arr[i] = _Job(tree.handle, pts.data_ptr(), pts.shape[-1], out.data_ptr())
    return arr


def fp_eval_batch(dtype, jobs, stream=None):
    """jobs: list of (tree, points, out) with CUDA tensors in fp_eval layouts."""
    arr = _jobs_array(jobs, dtype, "fp_eval_batch")
    _check(_lib.fp_eval_batch(DTYPES[dtype], ctypes.cast(arr, ctypes.c_void_p), len(jobs), _stream_handle(stream)),
           "fp_eval_batch")


class Batch:
    """A planned batch (fp_batch_create); launch() only enqueues kernels and
    can be captured in a CUDA graph.  Keep the trees and tensors alive."""

    def __init__(self, dtype, jobs):
        self._keep = list(jobs)
        arr = _jobs_array(jobs, dtype, "Batch")
        h = ctypes.c_void_p()
        _check(_lib.fp_batch_create(DTYPES[dtype], ctypes.cast(arr, ctypes.c_void_p), len(jobs), ctypes.byref(h)),
               "fp_batch_create")
        self._h = h.value

    def launch(self, stream=None):
        _check(_lib.fp_batch_launch(self._h, _stream_handle(stream)), "fp_batch_launch")

    def free(self):
        if self._h:
            _lib.fp_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch_jobs", ctypes.c_int), ("streams", ctypes.c_int)]


class _Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("status", ctypes.c_int), ("latency_us", ctypes.c_double)]


_lib.fp_server_create.restype = _I
_lib.fp_server_create.argtypes = [_P, ctypes.POINTER(_P)]
_lib.fp_server_submit.restype = _I
_lib.fp_server_submit.argtypes = [_P, _P, _I, _P, _I64, _P, ctypes.POINTER(ctypes.c_int64)]
_lib.fp_server_poll.restype = _I
_lib.fp_server_poll.argtypes = [_P, _P, _I, ctypes.POINTER(ctypes.c_int)]
_lib.fp_server_drain.restype = _I
_lib.fp_server_drain.argtypes = [_P, ctypes.c_double]
_lib.fp_server_stats.restype = _I
_lib.fp_server_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int64)]
_lib.fp_server_destroy.restype = None
_lib.fp_server_destroy.argtypes = [_P]


class Server:
    """Continuous-batching server (fp_server_*).  Host arrays passed to
    submit() are kept alive until their completion is polled; pinned arrays
    (e.g. torch pinned tensors' .numpy()) let the copies overlap."""

    def __init__(self, hbm_budget_bytes, max_batch_jobs=1024, streams=4):
        import threading
        cfg = _ServerCfg(hbm_budget_bytes, max_batch_jobs, streams)
        h = ctypes.c_void_p()
        _check(_lib.fp_server_create(ctypes.byref(cfg), ctypes.byref(h)), "fp_server_create")
        self._h = h.value
        self._live = {}
        self._lock = threading.Lock()

    def submit(self, tree, dtype, points, out):
        t = ctypes.c_int64()
        npts = points.shape[-1]
        _check_host_io("Server.submit", tree, dtype, points, npts, out)
        with self._lock:
            _check(_lib.fp_server_submit(self._h, tree.handle, DTYPES[dtype], _ptr(points), npts, _ptr(out),
                                         ctypes.byref(t)), "fp_server_submit")
            self._live[t.value] = (tree, points, out)
        return t.value

    def poll(self, max_items=4096):
        buf = (_Completion * max_items)()
        n = ctypes.c_int()
        _check(_lib.fp_server_poll(self._h, ctypes.cast(buf, ctypes.c_void_p), max_items, ctypes.byref(n)),
               "fp_server_poll")
        res = [(buf[i].ticket, buf[i].status, buf[i].latency_us) for i in range(n.value)]
        with self._lock:
            for tk, _, _ in res:
                self._live.pop(tk, None)
        return res

    def drain(self, timeout_s=60.0):
        _check(_lib.fp_server_drain(self._h, timeout_s), "fp_server_drain")

    def stats(self):
        pk, nb = ctypes.c_size_t(), ctypes.c_int64()
        _check(_lib.fp_server_stats(self._h, ctypes.byref(pk), ctypes.byref(nb)), "fp_server_stats")
        return {"peak_bytes": pk.value, "batches": nb.value}

    def close(self):
        if self._h:
            _lib.fp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ResidentCfg(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("max_jobs", ctypes.c_int), ("smem_bytes", ctypes.c_size_t),
                ("blocks_per_sm", ctypes.c_int), ("idle_exit_s", ctypes.c_double), ("max_items", ctypes.c_int64)]


class Resident:
    """A resident evaluation kernel with a device work queue (fp_resident_*):
    jobs submitted while it runs enter the running kernel.  One value type."""

    def __init__(self, dtype, max_jobs=4096, smem_bytes=0, blocks_per_sm=0, idle_exit_s=0.05, max_items=0):
        cfg = _ResidentCfg(DTYPES[dtype], max_jobs, smem_bytes, blocks_per_sm, idle_exit_s, max_items)
        h = ctypes.c_void_p()
        _check(_lib.fp_resident_create(ctypes.byref(cfg), ctypes.byref(h)), "fp_resident_create")
        self._h = h.value
        self.dtype = dtype
        self._keep = {}  # ticket -> (tree, points, out): alive until the job completes

    def submit(self, tree, points, out):
        """points, out: CUDA tensors in fp_eval layouts.  Returns the ticket."""
        _check_job("Resident.submit", tree, self.dtype, points, out)
        job = _Job(tree.handle, points.data_ptr(), points.shape[-1], out.data_ptr())
        t = ctypes.c_int64()
        _check(_lib.fp_resident_submit(self._h, ctypes.byref(job), ctypes.byref(t)), "fp_resident_submit")
        self._keep[t.value] = (tree, points, out)
        return t.value

    def done(self, ticket):
        rc = _lib.fp_resident_query(self._h, ticket)
        if rc < 0:
            _check(rc, "fp_resident_query")
        if rc == 0:
            self._keep.pop(ticket, None)
        return rc == 0

    def wait(self, ticket, timeout_s=60.0):
        _check(_lib.fp_resident_wait(self._h, ticket, timeout_s), "fp_resident_wait")
        self._keep.pop(ticket, None)

    def state(self):
        running, idle, jobs = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(_lib.fp_resident_state(self._h, ctypes.byref(running), ctypes.byref(idle), ctypes.byref(jobs)),
               "fp_resident_state")
        return {"running": bool(running.value), "idle_exits": bool(idle.value), "jobs": jobs.value}

    def stop(self, timeout_s=60.0):
        _check(_lib.fp_resident_stop(self._h, timeout_s), "fp_resident_stop")

    def close(self):
        if self._h:
            _lib.fp_resident_free(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
