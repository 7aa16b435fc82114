"""The compiler's bounds check of every schedule (FP_E_INTERNAL on failure)
accepts the trees of every workload: the benchmark's dense univariate sizes,
the serving stream's extremes (8 to 65536 terms, uni- and bivariate), the
trivariate degree-40 set, the sparse trivariate with virtual roots, the
composition's p, for both coefficient types under every scheme (the mod-p
compile is also the residue path's).  Host only: fp_compile_host runs the same
compiler and check as fp_compile."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_1307_5655_gb300 as fpl
import workloads as W

SCHEMES = ["H", "E", "B"]


def _shapes():
    yield "dense", W.dense_univariate_exps(1024)
    for k in (8, 1000, 3000, 10007, 30000, 65536):
        yield "dense%d" % k, W.dense_univariate_exps(k)
    for k in (8, 5000, 65536):
        yield "graded%d" % k, W.graded_prefix_exps(k, 2)
    yield "trivariate40", W.total_degree_exps(3, 40)
    full = W.total_degree_exps(3, 40)
    yield "sparse_trivariate", full[W.rng(303).random(len(full)) < 0.3]
    yield "compose_p", W.dense_univariate_exps(513)


@pytest.mark.parametrize("modp", [False, True])
def test_every_workload_shape_passes_the_schedule_check(modp):
    for name, e in _shapes():
        c = W.residues(len(e), 1) if modp else W.uniform_f64(len(e), 1)
        for s in SCHEMES:
            t = fpl.fp_compile_host(e, c, s, modp=modp)  # raises FastPolyError(-9) on a failed check
            assert t.info()["nnodes"] >= len(e), (name, s)
            t.free()


def test_direct_and_threshold_schemes_pass_the_schedule_check():
    e = W.dense_univariate_exps(2000)
    c = W.uniform_f64(len(e), 2)
    fpl.fp_compile_host(e, c, "D").free()
    for k0 in (4, 32, 512):
        ft = np.ones(len(e) + 1, dtype=np.int32)
        for n in range(1, len(e) + 1):
            ft[n] = 2 ** int(np.floor(np.log2(n))) if n + 1 > k0 else 1
        fpl.fp_compile_host(e, c, "CUSTOM", ft).free()


def test_planted_schedule_faults_are_refused(tmp_path):
    """The check itself, against planted faults (tests/schedule_check_faults.cpp,
    built with g++ against the compiler's source): one corruption per index the
    kernels take from a schedule -- slots, edge and rebuilt powers, program
    operands, stream offsets and extents, two-part fields, chain powers, the
    split's marks and deferred edges, the table layout -- on Balanced (10007
    terms), bivariate Estrin, Horner and mod-p trees; each is refused with
    FP_E_INTERNAL, and each tree as compiled passes."""
    gxx, nvcc = shutil.which("g++"), shutil.which("nvcc")
    if not gxx or not nvcc:
        pytest.skip("needs g++ and the CUDA headers")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_1307_5655_gb300", "csrc")
    exe = str(tmp_path / "schedule_check_faults")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(root, "include"), "-I", csrc, "-I", cuda_inc,
                    os.path.join(root, "tests", "schedule_check_faults.cpp"), os.path.join(csrc, "compiler.cpp"),
                    "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and "failures: 0" in r.stdout, r.stdout
    assert r.stdout.count(" ok") >= 30, r.stdout
