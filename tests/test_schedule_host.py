"""Host-side replay of the grouped schedule (no GPU).

The FP64 / FP32C / MODP kernels replay the walk of Sec. 2.1 grouped into ops
(single nodes, chains, dense blocks, partial blocks).  This test exports that
schedule through `fp_tree_schedule` and replays it in exact arithmetic modulo
p = 2^64 - 2^32 + 1 with Python integers; the result must equal the plain
definition sum c x^e mod p of the oracle at every point.  A wrong slot, a
wrong power, a dropped or doubled coefficient (e.g. c_N counted both by a
partial block and by the first child's initial value) changes the value.
The block templates are replayed from Def. 1.2 directly: the value of a
dense run is T(b) + T(a) x^f with b its f lowest terms.  A floating-point
block of 17 to 32 nodes is stored as its two parts a and b under the top
split, joined with x^f from the table: the replay checks f, the stored runs
and that power."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1307_5655_gb300 as fpl

P = (1 << 64) - (1 << 32) + 1


def _split(scheme, n):
    if scheme == 2:  # Estrin: the largest power of two <= n
        return 1 << (n.bit_length() - 1)
    return (n + 1) // 2  # Balanced: ceil(n / 2)


def _run_value(scheme, c, xpow):
    """T_f over the dense run c[0..len-1] (c[0] the highest term), relative to
    the exponent of its last (lowest) term."""
    def rec(lo, hi):
        if lo == hi:
            return c[hi]
        f = _split(scheme, hi - lo)
        b = rec(hi - f + 1, hi)
        a = rec(lo, hi - f)
        return (a * xpow(f) + b) % P
    return rec(0, len(c) - 1)


def _replay(t, coeffs, x, counts=None):
    """Run the power program and the ops on one table per point, as the
    kernel does: powers at their positions, slot s at position nlive + s.
    A temporary or a slot that overwrote a power still in use, or a slot
    still in use, would change the value."""
    ex = t.export()
    sc = t.schedule()
    n = len(ex["parent"])
    node_c = [int(coeffs[k]) if k >= 0 else 0 for k in ex["term_of_node"]]
    E, nlive = sc["entries"], sc["nlive"]
    assert nlive + sc["nslot"] <= E
    tab = [None] * E
    for w, dst in sc["prog"]:
        w, dst = int(w), int(dst)
        op, a1, a2 = w & 3, (w >> 2) & 0x7FFF, w >> 17
        assert dst < E
        if op == 0:
            tab[dst] = int(x[a1]) % P
        elif op == 1:
            tab[dst] = tab[a1] * tab[a1] % P
        else:
            tab[dst] = tab[a1] * tab[a2] % P
    x1 = int(x[len(x) - 1])  # blocks run over the innermost variable
    # the block templates read their powers right after the program
    xp = {d: tab[int(q)] for d, q in enumerate(sc["block_pow"]) if q >= 0}
    for d, v in xp.items():
        assert v == pow(x1, d, P), d

    def xpow(d):  # a block longer than 16 (mod-p trees) splits with powers past the table's
        return xp[d] if d in xp else pow(x1, d, P)

    def slot(s_):
        assert 0 <= s_ < sc["nslot"]
        return nlive + s_

    def power(pos, deg, var):  # a walk power: below nlive, and the right one
        assert 0 <= pos < nlive
        assert tab[pos] == pow(int(x[var]), deg, P), (pos, deg, var)
        return tab[pos]

    ops = list(zip(sc["op_words"], sc["op_a_node"], sc["op_b_node"]))

    def run_ops(tab, lo, hi, defer=None):
        for i_op, (rec_, a_node, b_node) in enumerate(ops[lo:hi], start=lo):
            w0, w1, j0, w3 = (int(v) for v in rec_)
            off, root_edge = w3 & 0x7FFFFFFF, w3 >> 31
            kind, S, D = w0 & 3, (w0 >> 2) & 63, (w0 >> 8) & 63
            leaf, first, uniform, pid = (w0 >> 14) & 1, (w0 >> 15) & 1, (w0 >> 16) & 1, w0 >> 17
            ln, fsplit, fpos = (w1 & 255) + 1, (w1 >> 8) & 255, w1 >> 16
            recompute = pid == 0x7FFF  # the edge power is rebuilt from a kept prefix
            if recompute:  # word 2 is the recompute word; the first node is the stream's
                assert kind >= 2 and sc["block_scheme"] in (2, 3)
                ez, j0 = j0, int(sc["stream"][off])
            j1 = j0 + ln - 1
            if counts is not None:
                counts[kind] += 1
            if kind == 0:
                assert ln == 1
                v = node_c[a_node] if leaf else tab[slot(S)]
                if leaf:
                    assert a_node == j0
            else:
                assert off % 4 == 0
                if fsplit:  # two parts: a (ln - f nodes), then b from the next multiple of 4
                    assert kind >= 2 and 16 < ln <= 32 and fsplit == _split(sc["block_scheme"], ln - 1)
                    assert ln - fsplit <= 16 and fsplit <= 16
                    offb = off + (ln - fsplit + 3) // 4 * 4
                    st = [int(s) for s in sc["stream"][off:off + ln - fsplit]] + \
                        [int(s) for s in sc["stream"][offb:offb + fsplit]]
                    assert all(int(s) == -1 for s in sc["stream"][off + ln - fsplit:offb])
                    power(fpos, fsplit, len(x) - 1)  # x^f of the join, kept in the table
                else:
                    st = [int(s) for s in sc["stream"][off:off + ln]]
                assert st == list(range(j0, j1 + 1))
                cs = [node_c[j] for j in st]
                if kind == 1:
                    v = cs[0] if leaf else tab[slot(S)]
                    pids = set()
                    for i in range(1, ln):
                        j = j0 + i - 1
                        assert int(ex["parent"][j]) == j + 1
                        pc = int(sc["chain_pid"][j])
                        pids.add(pc)
                        v = (v * power(pc, int(ex["pd"][j]), int(ex["pd_var"][j])) + cs[i]) % P
                    if uniform:
                        assert len(pids) == 1
                else:
                    # mod-p trees run blocks as a loop: up to 64 nodes (templates:
                    # 16, or 32 as two parts)
                    assert sc["block_scheme"] in (2, 3) and 2 <= ln <= 64
                    run = ex["node_e"][j0:j1 + 1]
                    assert np.array_equal(run[:, -1], np.arange(run[0, -1], run[0, -1] - ln, -1))
                    assert (run[:, :-1] == run[-1, :-1]).all()
                    if kind == 3:  # N's slot (c_N and its earlier children) stands for c_N
                        cs = cs[:-1] + [tab[slot(S)]]
                    v = _run_value(sc["block_scheme"], cs, xpow)
            q = int(ex["parent"][j1])
            # past the split, exactly the edges into the root are marked
            assert root_edge == (sc["split"] > 0 and i_op >= sc["split"] and q == n - 1)
            # the op's outgoing edge is the edge of its last node
            deg, var = int(ex["pd"][j1]), int(ex["pd_var"][j1])
            if recompute:  # x^(d >> m) (kept, or x), then square / times x per bit
                assert var == len(x) - 1
                base, m, bits = ez & 0x7FFF, (ez >> 15) & 15, ez >> 19
                assert bits < (1 << m) and bits == deg % (1 << m)
                xd = x1 if base == 0x7FFF else power(base, deg >> m, var)
                assert base != 0x7FFF or deg >> m == 1
                for i in range(m - 1, -1, -1):
                    xd = xd * xd % P
                    if (bits >> i) & 1:
                        xd = xd * x1 % P
                assert xd == pow(x1, deg, P)
            else:
                xd = power(pid, deg, var)
            if first:
                init = node_c[b_node] if b_node >= 0 else 0
                if b_node >= 0:
                    assert b_node == q
            else:
                init = tab[slot(D)]
            if defer is not None and root_edge:  # kept, applied after the first part
                defer.append((v, xd))
                continue
            tab[slot(D)] = (v * xd + init) % P
    root = n - 1
    split = sc["split"]
    tab0 = list(tab)  # after the power program: the split's halves start here
    run_ops(tab, 0, len(ops))
    r = node_c[root] if sc["root_leaf"] else tab[slot(sc["root_lh"])]
    if split:
        # the small-grid split: ops [0, split) and [split, nops) on separate
        # tables; the second keeps its edges into the root (marked) and
        # applies them, in order, to the first's root slot: the walk's value
        assert 0 < split < len(ops) and not sc["root_leaf"]
        ta, tb = list(tab0), list(tab0)
        run_ops(ta, 0, split)
        kept = []
        run_ops(tb, split, len(ops), kept)
        r2 = ta[slot(sc["root_lh"])]
        for v, xd in kept:
            r2 = (v * xd + r2) % P
        assert r2 == r and len(kept) > 0
    if sc["root_pid"] >= 0:
        r = r * power(sc["root_pid"], int(ex["pd"][root]), 0) % P
    return r


def _check(exps, coeffs, scheme, ftab=None, npts=3, seed=0, counts=None):
    t = fpl.fp_compile_host(exps, coeffs, scheme, ftab, modp=True)
    nvars = 1 if np.ndim(exps) == 1 else np.shape(exps)[1]
    x = W.points_modp(nvars, npts, seed + 77)
    ref = O.eval_modp(exps, coeffs, x)
    for p in range(npts):
        got = _replay(t, coeffs, [int(v) for v in x[:, p]], counts)
        assert got == int(ref[p]), (scheme, p)
    t.free()


@pytest.mark.parametrize("k", [1, 2, 3, 17, 18, 33, 100, 513, 1000, 3000])
@pytest.mark.parametrize("scheme", ["H", "E", "B", "D"])
def test_univariate_schedule_replays_to_the_polynomial(k, scheme):
    e, c, _ = W.univariate_case(k, 1, 1000 + k, "modp")
    _check(e, c, scheme, npts=2, seed=k)


def test_large_univariate_schedules_use_partial_blocks():
    # 10007 terms: every node above the blocks carries a partial block
    for scheme in ("E", "B"):
        counts = [0, 0, 0, 0]
        e, c, _ = W.univariate_case(10007, 1, 4242, "modp")
        _check(e, c, scheme, npts=1, counts=counts)
        assert counts[3] > 0 and counts[2] > 0
        # a partial block absorbs the small children: far fewer ops than nodes
        assert sum(counts) * 6 < 10007, counts
    # the floating-point trees keep blocks of at most 22 nodes, those over 16
    # as two parts under the top split; 10007 terms under B: runs of ~20
    e, c, _ = W.univariate_case(10007, 1, 4243)
    sc = fpl.fp_compile_host(e, c, "B").schedule()
    w1 = sc["op_words"][:, 1][(sc["op_words"][:, 0] & 3) >= 2].astype(np.int64)
    lens, fs = (w1 & 255) + 1, (w1 >> 8) & 255
    assert lens.max() <= 22 and (fs[lens > 16] > 0).all() and (fs[lens <= 16] == 0).all()
    assert lens.mean() > 16
    # 3000 terms: runs of ~23 stay blocks of ~12 (two such parts gain nothing)
    e, c, _ = W.univariate_case(3000, 1, 4244)
    sc = fpl.fp_compile_host(e, c, "B").schedule()
    w1 = sc["op_words"][:, 1][(sc["op_words"][:, 0] & 3) >= 2].astype(np.int64)
    assert ((w1 & 255) + 1 <= 16).all()


def test_sparse_and_hybrid_schedules():
    r = W.rng(5)
    e = np.sort(r.choice(5000, size=700, replace=False))[::-1].astype(np.int32)
    c = W.residues(700, 6)
    for scheme in ("E", "B", "H"):
        _check(e, c, scheme, npts=2, seed=1)
    ft = np.zeros(1001, dtype=np.int32)
    for n in range(1, 1001):
        ft[n] = 2 ** int(math.floor(math.log2(n))) if n > 10 else 1
    e2, c2, _ = W.univariate_case(1000, 1, 9, "modp")
    _check(e2, c2, "CUSTOM", ft, npts=2, seed=2)


@pytest.mark.parametrize("scheme", ["E", "B", "H"])
def test_multivariate_schedule(scheme):
    counts = [0, 0, 0, 0]
    e = W.total_degree_exps(3, 8)
    c = W.residues(len(e), 11)
    _check(e, c, scheme, npts=2, seed=3, counts=counts)
    if scheme != "H":  # the innermost variable's dense runs become blocks
        assert counts[2] > 0


@pytest.mark.parametrize("scheme", ["E", "B"])
def test_trivariate_degree40_schedule(scheme):
    counts = [0, 0, 0, 0]
    e = W.total_degree_exps(3, 40)
    c = W.residues(len(e), 12)
    _check(e, c, scheme, npts=1, seed=4, counts=counts)
    assert counts[2] > 0 and counts[3] > 0
    assert sum(counts) * 4 < len(e), counts


def test_multivariate_with_virtual_roots_and_gaps():
    r = W.rng(8)
    e = W.total_degree_exps(3, 12)
    keep = r.random(len(e)) < 0.7  # gaps in every variable, missing group roots
    e = e[keep]
    c = W.residues(len(e), 13)
    for scheme in ("E", "B"):
        _check(e, c, scheme, npts=2, seed=5)
    e2 = W.total_degree_exps(2, 30)
    c2 = W.residues(len(e2), 14)
    for scheme in ("E", "B"):
        _check(e2, c2, scheme, npts=2, seed=6)


def _random_terms(r, nvars):
    """Exponent sets mixing dense runs with holes in every variable: each
    group (fixed outer exponents) keeps a random prefix and random gaps of
    the innermost variable's run, so blocks, partial blocks, chains, single
    nodes and virtual group roots all occur."""
    deg = int(r.integers(3, 40 if nvars == 1 else 12))
    full = W.total_degree_exps(nvars, deg) if nvars > 1 else np.arange(deg + 1)[::-1].reshape(-1, 1)
    keep = r.random(len(full)) < r.uniform(0.3, 1.0)
    e = full[keep]
    if len(e) == 0:
        e = full[:1]
    return np.ascontiguousarray(e.astype(np.int32))


@pytest.mark.parametrize("seed", range(48))
def test_random_schedules_replay_for_both_coefficient_types(seed):
    """Fuzz: random sparse multivariate term sets under random schemes
    (including random split tables), for the mod-p trees (blocks up to 64
    nodes) and the floating-point trees (up to 32), replayed mod p."""
    r = W.rng(9000 + seed)
    nvars = int(r.integers(1, 4))
    e = _random_terms(r, nvars)
    k = len(e)
    scheme = ["H", "E", "B", "D", "CUSTOM"][int(r.integers(0, 5))]
    ftab = None
    if scheme == "CUSTOM":
        nmax = max(k, int(e.max()) + 1)
        ftab = np.zeros(nmax + 1, dtype=np.int32)
        for n in range(1, nmax + 1):
            ftab[n] = r.integers(1, n + 1)
    res = W.residues(k, 9100 + seed)
    x = W.points_modp(nvars, 1, 9200 + seed)
    ref = int(O.eval_modp(e, res, x)[0])
    xs = [int(v) for v in x[:, 0]]
    for modp in (True, False):
        coeffs = res if modp else W.uniform_f64(k, 9300 + seed)
        t = fpl.fp_compile_host(e, coeffs, scheme, ftab, modp=modp)
        if not modp:  # same tree shape, so the residues go where the floats went
            assert t.info()["nnodes"] >= k
        assert _replay(t, res, xs) == ref, (seed, scheme, nvars, k, modp)
        if not modp:
            sc = t.schedule()
            blk = (sc["op_words"][:, 0] & 3) >= 2
            assert ((sc["op_words"][:, 1][blk].astype(np.int64) & 255) + 1 <= 32).all()
        t.free()


@pytest.mark.parametrize("k", [40, 100, 1000, 3000, 10007])
@pytest.mark.parametrize("scheme", ["E", "B"])
def test_floating_point_schedules_with_two_part_blocks(k, scheme):
    """The floating-point trees' schedules (under B, blocks of 17..22 nodes
    stored as their two parts) replayed mod p with residues in the
    coefficients' places equal the plain definition (and so do the two
    halves of the small-grid split, added); two-part blocks occur, and the
    trees whose first top part holds a quarter of the nodes have a split."""
    e, cf, _ = W.univariate_case(k, 1, 6100 + k)
    res = W.residues(k, 6200 + k)
    t = fpl.fp_compile_host(e, cf, scheme)
    sc = t.schedule()
    kinds = sc["op_words"][:, 0] & 3
    w1 = sc["op_words"][:, 1].astype(np.int64)
    two_part = (kinds >= 2) & (((w1 >> 8) & 255) > 0)
    if scheme == "B" and k == 10007:  # runs of ~20 under the top splits
        assert two_part.any()
    if scheme == "B" and k == 10007:  # the table keeps the powers most ops read
        assert ((sc["op_words"][:, 0] >> 17) == 0x7FFF).any() and sc["entries"] <= 16
    if scheme == "E":  # Estrin keeps blocks of at most 16
        assert not two_part.any() and ((w1[kinds >= 2] & 255) + 1 <= 16).all()
    if k in (1000, 3000):  # top parts of 488 / 952 (E), 500 / 1500 (B) nodes
        assert sc["split"] > 0
    x = W.points_modp(1, 2, 6300 + k)
    ref = O.eval_modp(e, res, x)
    for p in range(2):
        assert _replay(t, res, [int(x[0, p])]) == int(ref[p]), (scheme, k, p)
    t.free()
