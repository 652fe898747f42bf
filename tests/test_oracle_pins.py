"""Pins for the CPU oracle: worked examples printed in the paper, closed forms,
all-pairs brute force of the property definitions (Sec. 2.3, Fig. 5) on small
inputs, library routines for textbook pieces, and invariants the paper states.

Nothing here calls the CUDA library. Each pin is chosen so that a plausible
slip in the oracle (a dropped term, a flipped comparison, an off-by-one, a
swapped operand) breaks at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
I64MIN, I64MAX = oracle.INT64_MIN, oracle.INT64_MAX


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------- worked examples

def test_partition2_demo_fig2():
    g = _gold("partition2_demo.json")
    xs = np.array(g["xs"], np.int32)
    r = oracle.partition(xs, ("lt", 0, g["pred"]["b"]))
    assert r["indices"].tolist() == g["indices"]
    assert int(r["num_true"][0]) == g["num_true"]
    assert r["keys_out"].tolist() == g["ys"]
    # the intermediate scans of the demo, through the oracle's scan
    ft = np.array(g["flagsT"], np.int32)
    assert oracle.scan(ft, inclusive=True)[0].tolist() == g["indicesT"]
    assert oracle.scan(np.array(g["flagsF"], np.int32), inclusive=True)[0].tolist() == g["scan_flagsF"]
    # the demo's indices realise FiltPart ys xs (\_->true) (\i-> p xs[i])
    v = oracle.check_filtpart(r["indices"], xs, part=("lt", 0, 5))
    assert v["ok"] and v["aux0"] == 6
    # any transposition of two destinations breaks it
    for a, b in itertools.combinations(range(6), 2):
        z = np.array(g["indices"], np.int32)
        z[a], z[b] = z[b], z[a]
        assert not oracle.check_filtpart(z, xs, part=("lt", 0, 5))["ok"]


def test_mksgmdescr_example_fig2():
    g = _gold("mksgmdescr_example.json")
    out, off = oracle.flags_from_shape(np.array(g["shape"]), np.array(g["xs"]))
    assert out.tolist() == g["result"]
    assert off.tolist() == [0, 0, 2, 3, 3, 6]


def test_mkii_example_fig2():
    g = _gold("mkii_example.json")
    sct1, _ = oracle.flags_from_shape(np.array(g["shape"]), np.array(g["beg_vs"]))
    assert sct1.tolist() == g["sct_vs1"]
    assert oracle.mkii(np.array(g["shape"])).tolist() == g["II"]
    # the segmented scan with the demo's flags reproduces II from the decremented starts
    dec = np.array([0 if v == 0 else v - 1 for v in g["sct_vs1"]], np.int64)
    assert oracle.sgm_scan(np.array(g["flags"]), dec).tolist() == g["II"]


# ---------------------------------------------------------- brute force (Fig. 5)

def bf_range(x, lo, hi):
    bad = [i for i in range(len(x)) if not (lo <= x[i] <= hi)]
    return bad[0] if bad else -1


OPS = {"le": lambda a, b: a <= b, "lt": lambda a, b: a < b, "ge": lambda a, b: a >= b, "gt": lambda a, b: a > b}


def bf_mono(x, op):
    """Smallest j such that some i < j has not (x[i] op x[j]); -1 when monotone."""
    for j in range(len(x)):
        if any(not OPS[op](x[i], x[j]) for i in range(j)):
            return j
    return -1


def bf_inj(x, lo, hi):
    """Lexicographically smallest pair (i, j), i < j, x[i] = x[j], both in [lo, hi]."""
    n = len(x)
    for i in range(n):
        for j in range(i + 1, n):
            if lo <= x[i] <= hi and lo <= x[j] <= hi and x[i] == x[j]:
                return i, j
    return -1, -1


def bf_bij(x, rlo, rhi, ilo, ihi):
    """Fig. 5 Bij by its definition: (kind, index, value, in-image count, |Img|).
    The position reported is the first one that breaks the property: a value in Rcd
    outside Img, or a value that occurs again; with neither, the smallest image
    value no element takes."""
    n = len(x)
    img = set(range(ilo, ihi + 1))
    in_img = sum(1 for v in x if ilo <= v <= ihi)
    size = ihi - ilo + 1
    for i in range(n):
        if not (rlo <= x[i] <= rhi):
            continue
        if x[i] not in img:
            return "out_of_image", i, x[i], in_img, size
        if any(x[j] == x[i] for j in range(n) if j != i):
            return "duplicate", i, x[i], in_img, size
    s = {v for v in x if rlo <= v <= rhi}
    if s != img:
        return "missing", -1, min(img - s), in_img, size
    return "none", -1, 0, in_img, size


def small_arrays():
    vals = [-1, 0, 1, 2, 3]
    for n in range(0, 6):
        for t in itertools.product(vals, repeat=n):
            yield list(t)


def test_range_brute_force():
    for x in small_arrays():
        a = np.array(x, np.int64)
        for lo, hi in [(0, 2), (-1, 3), (1, 1), (I64MIN, I64MAX), (I64MIN, 0)]:
            v = oracle.check_range(a, lo, hi)
            i = bf_range(x, lo, hi)
            assert v["ok"] == (i < 0) and v["index"] == i
            if i >= 0:
                assert v["kind"] == "out_of_range" and v["value"] == x[i]
            if x:
                assert (v["aux0"], v["aux1"]) == (min(x), max(x))


def test_mono_brute_force():
    for x in small_arrays():
        a = np.array(x, np.int32)
        for op in OPS:
            v = oracle.check_mono(a, op)
            j = bf_mono(x, op)
            assert v["ok"] == (j < 0) and v["index"] == j, (x, op)
            if j >= 0:
                assert v["kind"] == "order" and v["value"] == x[j] and v["aux0"] == x[j - 1]


def test_inj_brute_force():
    for x in small_arrays():
        a = np.array(x, np.int64)
        for lo, hi in [(I64MIN, I64MAX), (0, 2), (0, 0), (1, 3)]:
            v = oracle.check_inj(a, lo, hi)
            i, j = bf_inj(x, lo, hi)
            assert v["ok"] == (i < 0) and v["index"] == i, (x, lo, hi)
            if i >= 0:
                assert v["kind"] == "duplicate" and v["value"] == x[i] and v["aux0"] == j


def test_inj_wide_span_uses_sort_path():
    # values far apart force the (value, index) sort method; brute force must agree
    rng = np.random.default_rng(7)
    for _ in range(300):
        n = int(rng.integers(2, 12))
        base = rng.choice([-(2**62), -5, 0, 2**40, 2**62], size=n)
        x = (base + rng.integers(0, 3, size=n)).astype(np.int64)
        v = oracle.check_inj(x)
        i, j = bf_inj(x.tolist(), I64MIN, I64MAX)
        assert v["index"] == i and v["ok"] == (i < 0)
        if i >= 0:
            assert v["aux0"] == j


def test_bij_brute_force():
    for x in small_arrays():
        a = np.array(x, np.int32)
        for rlo, rhi, ilo, ihi in [(I64MIN, I64MAX, 0, 2), (0, 3, 0, 3), (0, 2, 0, 2), (-1, 3, 0, 1)]:
            v = oracle.check_bij(a, rlo, rhi, ilo, ihi)
            kind, i, val, cnt, size = bf_bij(x, rlo, rhi, ilo, ihi)
            assert v["kind"] == kind and v["index"] == i and v["ok"] == (kind == "none"), (x, rlo, rhi, ilo, ihi)
            if kind != "none":
                assert v["value"] == val
            # aux0 = elements whose value lies in Img, aux1 = |Img| (rule BijF1's two counts)
            assert (v["aux0"], v["aux1"]) == (cnt, size), (x, rlo, rhi, ilo, ihi)


def test_bij_identity_and_permutation():
    n = 1000
    assert oracle.check_bij(synth.identity(n), 0, n - 1, 0, n - 1)["ok"]
    p = synth.permutation(n, 3)
    assert oracle.check_bij(p, I64MIN, I64MAX, 0, n - 1)["ok"]
    assert oracle.check_inj(p)["ok"]
    d, a, b = synth.plant_duplicate(p, 5)
    v = oracle.check_bij(d, I64MIN, I64MAX, 0, n - 1)
    assert v["kind"] == "duplicate" and v["index"] == min(a, b) and v["value"] == p[a]


def test_bij_img_must_lie_in_rcd():
    with pytest.raises(oracle.OracleError):
        oracle.check_bij(np.arange(4, dtype=np.int32), 0, 2, 0, 3)


# ------------------------------------------------------- segmented definitions

def random_segments(rng, n, m):
    cuts = np.sort(rng.integers(0, n + 1, size=m - 1))
    return np.concatenate([[0], cuts, [n]]).astype(np.int64)


def test_segmented_checks_equal_per_segment_checks():
    rng = np.random.default_rng(11)
    for _ in range(300):
        n = int(rng.integers(0, 40))
        m = int(rng.integers(1, 8))
        off = random_segments(rng, n, m)
        x = rng.integers(-2, 6, size=n).astype(np.int32)
        # Mono: per-segment verdicts equal flat verdicts on the slices
        v, so = oracle.check_mono(x, "le", off, seg_ok=True)
        first = -1
        for k in range(m):
            s = x[off[k]:off[k + 1]]
            j = bf_mono(s.tolist(), "le")
            assert bool(so[k]) == (j < 0)
            if j >= 0 and first < 0:
                first = off[k] + j
        assert v["index"] == first
        # Inj per segment
        v, so = oracle.check_inj(x, 0, 4, off, seg_ok=True)
        first = -1
        for k in range(m):
            i, _ = bf_inj(x[off[k]:off[k + 1]].tolist(), 0, 4)
            assert bool(so[k]) == (i < 0)
            if i >= 0 and first < 0:
                first = off[k] + i
        assert v["index"] == first
        # Bij with per-segment image [e_k, e_{k+1})
        y = np.concatenate([rng.permutation(np.arange(off[k], off[k + 1])) for k in range(m)]).astype(np.int32) \
            if n else np.zeros(0, np.int32)
        assert oracle.check_bij(y, I64MIN, I64MAX, seg_img=True, offsets=off)["ok"]
        if n >= 2:
            y2 = y.copy()
            y2[int(rng.integers(0, n))] = int(rng.integers(0, n))
            v = oracle.check_bij(y2, I64MIN, I64MAX, seg_img=True, offsets=off)
            exp_ok = all(sorted(y2[off[k]:off[k + 1]].tolist()) == list(range(off[k], off[k + 1])) for k in range(m))
            assert v["ok"] == exp_ok


def test_segmented_bij_counts_per_segment():
    # Segmented Bij (Fig. 5, Img_k = [e_k, e_{k+1})): the verdict of the first
    # failing segment, with that segment's in-image count and |Img_k| as aux0/aux1;
    # when every segment holds, the counts are summed over the segments.
    rng = np.random.default_rng(13)
    for _ in range(400):
        n = int(rng.integers(0, 14))
        m = int(rng.integers(1, 5))
        off = random_segments(rng, n, m)
        y = np.concatenate([rng.permutation(np.arange(off[k], off[k + 1])) for k in range(m)]).astype(np.int64) \
            if n else np.zeros(0, np.int64)
        for _ in range(int(rng.integers(0, 3))):
            if n:
                y[int(rng.integers(0, n))] = int(rng.integers(-1, n + 1))
        rlo, rhi = (I64MIN, I64MAX) if rng.random() < 0.5 else (0, max(n - 1, 0))
        v = oracle.check_bij(y, rlo, rhi, seg_img=True, offsets=off)
        first = None
        tot_in = tot_size = 0
        for k in range(m):
            a, b = int(off[k]), int(off[k + 1])
            seg = y[a:b].tolist()
            kind, i, val, cnt, size = bf_bij(seg, rlo, rhi, a, b - 1) if b > a else ("none", -1, 0, 0, 0)
            tot_in += cnt
            tot_size += size
            if kind != "none" and first is None:
                first = (kind, a + i if i >= 0 else -1, val, cnt, size)
        if first is None:
            assert v["ok"] and (v["aux0"], v["aux1"]) == (tot_in, tot_size), (y, off)
        else:
            assert not v["ok"], (y, off)
            assert (v["kind"], v["index"], v["value"], v["aux0"], v["aux1"]) == first, (y, off, v, first)


# ------------------------------------------------------------ partition pins

def closed_form_indices(cs, off=None):
    """The printed index functions of partition2 (Sec. 2.3) and partition2L (Sec. 6)."""
    n = len(cs)
    off = [0, n] if off is None else list(off)
    out = [0] * n
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        for i in range(a, b):
            if cs[i]:
                out[i] = a + sum(cs[a:i])          # = -1 + sum_{j=a..i} cs[j] + a
            else:
                out[i] = i + sum(cs[i + 1:b])
    return out


def test_partition_closed_form_flat_and_segmented():
    rng = np.random.default_rng(21)
    for _ in range(200):
        n = int(rng.integers(0, 50))
        keys = rng.integers(-20, 20, size=n).astype(np.int32)
        cs = [int(k % 3 == 0) for k in keys.tolist()]  # Python % is floored
        r = oracle.partition(keys, ("mod_eq", 3, 0))
        assert r["indices"].tolist() == closed_form_indices(cs)
        assert int(r["num_true"][0]) == sum(cs)
        m = int(rng.integers(1, 6))
        off = random_segments(rng, n, m)
        rs = oracle.partition(keys, ("mod_eq", 3, 0), offsets=off)
        assert rs["indices"].tolist() == closed_form_indices(cs, off)
        assert rs["num_true"].tolist() == [sum(cs[off[k]:off[k + 1]]) for k in range(m)]


def test_partition_payload_and_invariants():
    n = 5000
    keys = synth.keys_uniform(n, 1)
    pay = synth.payload_f32(n, 2)
    t = synth.bernoulli_threshold(0.3)
    r = oracle.partition(keys, ("lt", 0, t), payload=pay)
    idx = r["indices"]
    # a partition's index array is a bijection onto [0, n) (Sec. 2.3, InvFiltPart)
    assert oracle.check_bij(idx, I64MIN, I64MAX, 0, n - 1)["ok"]
    # the scattered payload is the stable filter-partition of the input (library stable sort)
    cs = keys < t
    order = np.argsort(~cs, kind="stable")
    assert np.array_equal(r["payload_out"], pay[order])
    assert np.array_equal(r["keys_out"], keys[order])
    assert oracle.check_filtpart_values(r["payload_out"], pay, keys, part=("lt", 0, t))["ok"]


def bf_filtpart_ref(n, kept, cls, off):
    ref = [-1] * n
    pos = 0
    for k in range(len(off) - 1):
        sigma = [i for i in range(off[k], off[k + 1]) if kept[i]]
        for i in sorted(sigma, key=lambda i: cls[i]):  # Python's sort is stable
            ref[i] = pos
            pos += 1
    return ref, pos


def test_filtpart_brute_force_filter_and_classes():
    rng = np.random.default_rng(31)
    for _ in range(300):
        n = int(rng.integers(0, 30))
        v = int(rng.integers(1, 5))
        keys = rng.integers(-9, 9, size=n).astype(np.int64)
        cls = rng.integers(0, v + 1, size=n).astype(np.uint8)
        flags = rng.integers(0, 2, size=n).astype(np.uint8)
        off = random_segments(rng, n, int(rng.integers(1, 5)))
        kept = flags.tolist()
        ref, N = bf_filtpart_ref(n, kept, [min(c, v - 1) for c in cls.tolist()], off.tolist())
        z = np.array([r if r >= 0 else N + 1 + i for i, r in enumerate(ref)], np.int64)
        fl = ("flags", 0, 0, flags)
        vd = oracle.check_filtpart(z, keys, filt=fl, cls=cls, v=v, offsets=off)
        assert vd["ok"] and vd["aux0"] == N and vd["index"] == -1
        z2 = np.array([r if r >= 0 else -1 for r in ref], np.int64)
        assert oracle.check_filtpart(z2, keys, filt=fl, cls=cls, v=v, offsets=off)["ok"]
        if N >= 1:
            # a dropped element aimed inside [0, N), or a kept one moved, must fail at that index
            i = int(rng.integers(0, n))
            z3 = z.copy()
            z3[i] = (ref[i] + 1) % N if ref[i] >= 0 and N > 1 else (0 if ref[i] < 0 else -5)
            vd = oracle.check_filtpart(z3, keys, filt=fl, cls=cls, v=v, offsets=off)
            assert not vd["ok"] and vd["index"] == i and vd["kind"] == "wrong_dest"
            # aux0 = N, aux1 = the destination the definition gives i (-1: dropped)
            assert vd["value"] == z3[i] and vd["aux0"] == N and vd["aux1"] == ref[i]


def test_filtpart_value_mode_brute_force():
    # FiltPart Y X (e_k, p^f, p^p) in value form: Y is X filtered and stably
    # partitioned per segment (built here with Python's stable sort). A swapped pair
    # of rows is reported at the smaller position with that position's source
    # index; a flipped bit at its position; a Y of the wrong length with index -1.
    rng = np.random.default_rng(33)
    for _ in range(300):
        n = int(rng.integers(0, 25))
        v = int(rng.integers(1, 5))
        keys = rng.integers(-9, 9, size=n).astype(np.int64)
        cls = rng.integers(0, v + 1, size=n).astype(np.uint8)
        flags = rng.integers(0, 2, size=n).astype(np.uint8)
        off = random_segments(rng, n, int(rng.integers(1, 4)))
        rows = rng.integers(0, 2**31, size=(n, 3)).astype(np.int32)
        ref, N = bf_filtpart_ref(n, flags.tolist(), [min(c, v - 1) for c in cls.tolist()], off.tolist())
        src = [0] * N
        for i, r in enumerate(ref):
            if r >= 0:
                src[r] = i
        y = rows[src] if N else np.zeros((0, 3), np.int32)
        fl = ("flags", 0, 0, flags)
        vd = oracle.check_filtpart_values(y, rows, keys, filt=fl, cls=cls, v=v, offsets=off)
        assert vd["ok"] and vd["aux0"] == N
        if N >= 2:
            a, b = sorted(rng.choice(N, size=2, replace=False).tolist())
            y2 = y.copy()
            y2[[a, b]] = y2[[b, a]]
            vd = oracle.check_filtpart_values(y2, rows, keys, filt=fl, cls=cls, v=v, offsets=off)
            same = np.array_equal(y[a], y[b])
            assert vd["ok"] == same
            if not same:
                assert (vd["kind"], vd["index"], vd["value"]) == ("wrong_dest", a, src[a])
        if N >= 1:
            p = int(rng.integers(0, N))
            y3 = y.copy()
            y3[p, int(rng.integers(0, 3))] ^= 1 << int(rng.integers(0, 31))
            vd = oracle.check_filtpart_values(y3, rows, keys, filt=fl, cls=cls, v=v, offsets=off)
            assert (vd["ok"], vd["index"], vd["value"]) == (0, p, src[p])
            vd = oracle.check_filtpart_values(y[:-1], rows, keys, filt=fl, cls=cls, v=v, offsets=off)
            assert (vd["ok"], vd["kind"], vd["index"], vd["value"], vd["aux0"]) == (0, "wrong_dest", -1, N - 1, N)


def test_invfiltpart_listed_conditions_are_weaker():
    # n = 2, p^f = [T, F], Z = [5, 0]: the dropped element would land inside [0, N)
    z = np.array([5, 0], np.int32)
    v = oracle.check_filtpart(z, None, filt=("flags", 0, 0, np.array([1, 0], np.uint8)),
                              part=("flags", 0, 0, np.array([1, 1], np.uint8)))
    assert not v["ok"] and v["index"] == 0


# ------------------------------------------------------- scan / scatter / gather

def test_scan_matches_cumsum_with_wrap():
    rng = np.random.default_rng(41)
    for it, ot in [(np.int32, np.int32), (np.int32, np.int64), (np.int64, np.int64)]:
        for n in [0, 1, 2, 33, 1000]:
            x = rng.integers(np.iinfo(it).min // 2, np.iinfo(it).max // 2, size=n).astype(it)
            inc, tot = oracle.scan(x, ot, inclusive=True)
            exc, _ = oracle.scan(x, ot, inclusive=False)
            w = np.iinfo(ot).bits
            ref = [((s + 2**(w - 1)) % 2**w) - 2**(w - 1) for s in itertools.accumulate(int(v) for v in x)]
            assert inc.tolist() == ref
            assert exc.tolist() == ([0] + ref[:-1] if n else [])
            assert int(tot[0]) == (ref[-1] if n else 0)


def test_segmented_scan_restarts():
    rng = np.random.default_rng(43)
    x = rng.integers(0, 5, size=100).astype(np.int32)
    off = random_segments(rng, 100, 7)
    out, tot = oracle.scan(x, np.int64, inclusive=False, offsets=off)
    for k in range(7):
        s = x[off[k]:off[k + 1]].astype(np.int64)
        assert out[off[k]:off[k + 1]].tolist() == (np.cumsum(s) - s).tolist()
        assert int(tot[k]) == int(s.sum())


def test_sgm_scan_pieces():
    rng = np.random.default_rng(45)
    for _ in range(100):
        n = int(rng.integers(1, 30))
        fl = rng.integers(0, 2, size=n).astype(np.uint8)
        x = rng.integers(-5, 5, size=n).astype(np.int64)
        heads = [0] + [i for i in range(1, n) if fl[i]] + [n]
        ref = np.concatenate([np.cumsum(x[a:b]) for a, b in zip(heads[:-1], heads[1:]) if b > a])
        assert oracle.sgm_scan(fl, x).tolist() == ref.tolist()


def test_mkii_matches_repeat_with_empty_segments():
    # mkII (Fig. 2, right) is segment k repeated shape[k] times (numpy's repeat);
    # empty segments contribute nothing, and II[j] = k exactly when
    # offsets[k] <= j < offsets[k + 1]
    rng = np.random.default_rng(46)
    for _ in range(100):
        m = int(rng.integers(1, 20))
        shape = rng.integers(0, 6, size=m).astype(np.int64)
        shape[rng.random(m) < 0.3] = 0
        ii = oracle.mkii(shape)
        assert ii.tolist() == np.repeat(np.arange(m), shape).tolist()
        off = np.concatenate([[0], np.cumsum(shape)])
        for j in range(int(off[-1])):
            k = int(ii[j])
            assert off[k] <= j < off[k + 1]


def test_scatter_gather_library_routines():
    rng = np.random.default_rng(51)
    n, m = 500, 300
    vals = rng.standard_normal((n, 8)).astype(np.float32)
    idx = rng.permutation(n)[:n].astype(np.int64) - 100  # some out of bounds on both sides
    idx[idx >= m] += 1000
    dst = np.zeros((m, 8), np.float32)
    out = oracle.scatter(dst, idx, vals)
    ref = dst.copy()
    ok = (idx >= 0) & (idx < m)
    ref[idx[ok]] = vals[ok]
    assert np.array_equal(out, ref)
    g, oob = oracle.gather(out, np.clip(idx, 0, m - 1))
    assert not oob and np.array_equal(g, out[np.clip(idx, 0, m - 1)])
    g2, oob2 = oracle.gather(out, idx)
    assert oob2 and np.all(g2[~ok] == 0) and np.array_equal(g2[ok], out[idx[ok]])
    # scatter then gather by a bijection is the identity
    p = rng.permutation(n).astype(np.int32)
    y = oracle.scatter(np.zeros_like(vals), p, vals)
    assert np.array_equal(oracle.gather(y, p)[0], vals)


def test_scatter_add_matches_numpy_add_at():
    rng = np.random.default_rng(53)
    idx = synth.zipf_ranks(20000, 64, 1.1, 3)
    vals = rng.standard_normal((20000, 4)).astype(np.float32)
    got = oracle.scatter_add_f64(64, idx, vals)
    ref = np.zeros((64, 4))
    np.add.at(ref, idx, vals.astype(np.float64))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_flags_from_shape_brute_force():
    rng = np.random.default_rng(61)
    for _ in range(200):
        m = int(rng.integers(0, 12))
        shape = rng.integers(0, 5, size=m)
        xs = rng.integers(1, 100, size=m)
        out, off = oracle.flags_from_shape(shape, xs)
        ref = []
        for s, x in zip(shape.tolist(), xs.tolist()):
            ref += ([x] + [0] * (s - 1)) if s > 0 else []
        assert out.tolist() == ref
        assert off.tolist() == [0] + np.cumsum(shape).tolist()
        assert oracle.mkii(shape).tolist() == np.repeat(np.arange(m), shape).tolist()


def test_flags_from_shape_rejects_negative_shape():
    with pytest.raises(oracle.OracleError):
        oracle.flags_from_shape(np.array([1, -1, 2]))


# ------------------------------------------------- reduce-by-index (hist) with min

def test_hist_min_matches_numpy_minimum_at():
    rng = np.random.default_rng(71)
    for dt in (np.int32, np.int64):
        for m in (0, 1, 7, 300):
            n = int(rng.integers(0, 2000))
            idx = rng.integers(-20, m + 20, size=n).astype(dt)  # out of bounds on both sides
            vals = rng.integers(-10**6, 10**6, size=n).astype(dt)
            init = rng.integers(-10**5, 10**6, size=m).astype(dt)
            got = oracle.hist_min(m, idx, vals, init=init, dtype=dt)
            ref = init.copy()
            ok = (idx >= 0) & (idx < m)
            np.minimum.at(ref, idx[ok].astype(np.int64), vals[ok])
            assert got.dtype == dt and np.array_equal(got, ref)


def test_hist_min_of_iota_is_the_first_occurrence():
    rng = np.random.default_rng(72)
    idx = rng.integers(0, 50, size=400).astype(np.int64)
    H = oracle.hist_min(60, idx, init=np.full(60, 400))
    u, first = np.unique(idx, return_index=True)
    ref = np.full(60, 400)
    ref[u] = first
    assert np.array_equal(H, ref)


def test_dynamic_scatter_check_by_hist_decides_inj():
    """The dynamic verification of a scatter (Sec. 6): with H = hist min of iota by
    the indices, Inj on [0, m) holds iff every in-bounds i has H[idx[i]] == i; the
    first occurrence of the earliest repeated value is min H over the violations."""
    rng = np.random.default_rng(73)
    for _ in range(300):
        m = int(rng.integers(1, 40))
        n = int(rng.integers(0, 30))
        idx = rng.integers(-3, m + 3, size=n).astype(np.int64)
        H = oracle.hist_min(m, idx, init=np.full(m, n))
        ok = (idx >= 0) & (idx < m)
        bad = [i for i in range(n) if ok[i] and H[idx[i]] != i]
        v = oracle.check_inj(idx, 0, m - 1)
        assert v["ok"] == (not bad)
        if bad:
            i0 = min(int(H[idx[i]]) for i in bad)
            j0 = min(i for i in bad if H[idx[i]] == i0)
            assert (v["index"], v["aux0"], v["value"]) == (i0, j0, idx[i0])


def _smallest_pairs_brute(nv, n_es, es, is_):
    keep = []
    for i in range(len(es)):
        if not (0 <= es[i] < nv):
            continue
        h = min([n_es] + [int(is_[j]) for j in range(len(es)) if es[j] == es[i]])
        if h == is_[i]:
            keep.append(i)
    return es[keep], is_[keep]


def test_smallest_pairs_brute_force_and_postcondition():
    """get_smallest_pairs (Fig. 16) against its definition written as an all-pairs
    loop, and its postcondition: with is injective, es' and is' are injective and es'
    holds each vertex that occurs in es exactly once."""
    rng = np.random.default_rng(74)
    for dt in (np.int32, np.int64):
        for _ in range(150):
            nv = int(rng.integers(0, 12))
            n = int(rng.integers(0, 40))
            es = rng.integers(-2, nv + 2, size=n).astype(dt)
            is_ = rng.permutation(n * 2)[:n].astype(dt)  # injective
            n_es = int(rng.integers(n, 3 * n + 1))
            oe, oi = oracle.smallest_pairs(nv, n_es, es, is_)
            be, bi = _smallest_pairs_brute(nv, n_es, es, is_)
            assert oe.dtype == dt and np.array_equal(oe, be) and np.array_equal(oi, bi)
            assert oracle.check_inj(oe)["ok"] and oracle.check_inj(oi)["ok"]
            if n_es >= 2 * n:  # every is value is below the neutral element
                inb = es[(es >= 0) & (es < nv)]
                assert np.array_equal(np.sort(oe), np.unique(inb))
    # the neutral element takes part in the min: values at or above it never win
    oe, oi = oracle.smallest_pairs(2, 5, np.array([0, 0, 1], np.int64), np.array([7, 5, 6], np.int64))
    assert oe.tolist() == [0] and oi.tolist() == [5]
