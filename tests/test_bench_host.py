"""The roofline arithmetic of bench.py's composition line (compose_work), on
CPU, against operation counts worked out by hand for trees small enough to
follow: a transform of length n is (n/2) log2 n radix-2 butterflies, plus n
twiddle multiplications when it takes the four-step form (n > 4096); and
the DRAM traffic figure the benchmark line reports for its FP64 kernel."""
import paper_1307_5655_gb300 as fpl
import workloads as W

import bench


def _tree(k, scheme):
    return fpl.fp_compile_host(W.dense_univariate_exps(k), W.residues(k, 1), scheme, modp=True)


def test_leaf_only():
    # p = c1 x + c0 (Estrin): one leaf c1 * q, no product
    t = _tree(2, "E")
    assert bench.compose_work(t, 64, True) == (0, 65)
    assert bench.compose_work(t, 64, False) == (0, 0)


def test_one_small_product():
    # Horner, p = (c2 x + c1) x + c0: the leaf c2 q (65 multiplications), then
    # (c2 q + c1) * q: lengths 65 and 65, result 129, transform length 256:
    # forward, the cached transform of q (scaled by 1/n once: 256
    # multiplications), pointwise (256), inverse; 3 x 128 x 8 butterflies,
    # less the first stage of the two forward transforms of operands of
    # length <= 128, which is 128 single multiplications each
    t = _tree(3, "H")
    assert bench.compose_work(t, 64, True) == (3 * 128 * 8 - 2 * 128, 65 + 256 + 256 + 2 * 128)
    # FP64: the same product as a direct convolution, 65 x 65 multiply-adds
    assert bench.compose_work(t, 64, False) == (0, 65 * 65)


def test_one_four_step_product():
    # deg q = 3000: the product has 3001 x 3001 coefficients, 6001 long, so
    # length 8192 > 4096: three four-step transforms (forward, cached q,
    # inverse) of 4096 x 13 butterflies and 8192 twiddles each (the two
    # forward ones on operands of length <= 4096: first stage 4096 single
    # multiplications), the pointwise product (8192), no separate scaling,
    # and the leaf c2 q (3001)
    t = _tree(3, "H")
    bfly, mul = bench.compose_work(t, 3000, True)
    assert bfly == 3 * 4096 * 13 - 2 * 4096
    assert mul == 3001 + 3 * 8192 + 8192 + 2 * 4096


def test_f64_traffic_figure_is_a_whole_launch():
    """The committed capture of the FP64 kernel at 10007 terms and 2^24 points
    gives bytes per launch comparable with that launch's point I/O (2^24
    points of 8 bytes in, 8 bytes out): reads at least the points, writes at
    most the results, so between half and 1.1 times the I/O in total."""
    t = bench.f64_traffic_per_launch()
    io = bench.NPTS * 16
    assert t is not None and 0.5 * io <= t <= 1.1 * io, (t, io)
