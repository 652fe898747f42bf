"""GPU path vs the CPU oracle, element by element, on seeded inputs of sizes that
span several tiles and ragged tails (tiles are 4096 int32 / 2048 int64 elements,
grid-stride vectors 16 bytes). Verdicts, indices and moved bytes are bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I64MIN, I64MAX = oracle.INT64_MIN, oracle.INT64_MAX
SIZES = [0, 1, 2, 3, 31, 32, 33, 1023, 2047, 2048, 2049, 4095, 4096, 4097, 12289, 65536, 100003]


@pytest.fixture(scope="module")
def ixp():
    import paper_2506_23058_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def same(g, o, what=""):
    g = g.get()
    assert g["status"] == 0, (what, g)
    assert bool(g["ok"]) == o["ok"], (what, g, o)
    for f in ("kind", "index", "value", "aux0", "aux1"):
        assert g[f] == o[f], (what, f, g, o)


def arrays(n, dtype, seed):
    out = {"identity": synth.identity(n, dtype), "perm": synth.permutation(n, seed, dtype),
           "mono": synth.monotone(n, seed, dtype)}
    if n >= 2:
        out["dup"] = synth.plant_duplicate(out["perm"], seed)[0]
        out["oor"] = synth.plant_value(out["perm"], seed, n)[0]
        out["neg"] = synth.plant_value(out["perm"], seed + 1, -1)[0]
        out["brk"] = synth.plant_order_break(out["mono"], seed)[0]
    return out


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", SIZES)
def test_range(ixp, dev, n, dtype):
    for name, a in arrays(n, dtype, 100 + n).items():
        for lo, hi in [(0, max(0, n - 1)), (I64MIN, I64MAX), (1, max(1, n - 2)), (I64MIN, 0)]:
            same(ixp.check_range(T(a, dev), lo, hi), oracle.check_range(a, lo, hi), (name, n, lo, hi))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_range_unaligned_views_and_planted_edges(ixp, dev, dtype):
    n = 20000
    base = synth.permutation(n + 8, 7, dtype)
    for off in range(4):
        a = base[off:off + n]
        same(ixp.check_range(T(base, dev)[off:off + n], 0, n + 7), oracle.check_range(a, 0, n + 7))
    for p in [0, 1, 4095, 4096, 4097, n - 1]:
        a = synth.identity(n, dtype)
        a[p] = -5
        same(ixp.check_range(T(a, dev), 0, n - 1), oracle.check_range(a, 0, n - 1), p)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", SIZES)
def test_mono_flat(ixp, dev, n, dtype):
    for name, a in arrays(n, dtype, 200 + n).items():
        for c in ["le", "lt", "ge", "gt"]:
            same(ixp.check_mono(T(a, dev), c), oracle.check_mono(a, c), (name, n, c))
        r = a[::-1].copy()
        for c in ["ge", "gt"]:
            same(ixp.check_mono(T(r, dev), c), oracle.check_mono(r, c), (name, n, c, "rev"))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_mono_unaligned_and_edges(ixp, dev, dtype):
    n = 30000
    base = synth.identity(n + 8, dtype)
    for p in [1, 2, 3, 4, 5, 127, 128, 129, 4096, 8191, 8192, n - 1]:
        a = base.copy()
        a[p] = a[p - 1] - 1
        t = T(a, dev)
        for off in range(4):
            same(ixp.check_mono(t[off:off + n], "lt"), oracle.check_mono(a[off:off + n], "lt"), (p, off))


def random_offsets(rng, n, m, p_empty=0.2):
    cuts = np.sort(rng.integers(0, n + 1, size=m - 1))
    off = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    return off


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n,m", [(0, 1), (1, 1), (100, 7), (5000, 3), (5000, 900), (70000, 50), (70000, 20000)])
def test_mono_segmented(ixp, dev, n, m, dtype):
    rng = np.random.default_rng(n + m)
    off = random_offsets(rng, n, m)
    # sorted within each segment, resets at segment starts
    a = np.concatenate([np.sort(rng.integers(0, 1000, size=off[k + 1] - off[k])) for k in range(m)]).astype(dtype) \
        if n else np.zeros(0, dtype)
    for trial in range(3):
        b = a.copy()
        if trial and n > 2:
            for p in rng.integers(1, n, size=trial * 3):
                b[p] = b[p - 1] - 1
        for c in ["le", "lt"]:
            so = torch.zeros(m, dtype=torch.uint8, device=dev)
            g = ixp.check_mono(T(b, dev), c, T(off, dev), seg_ok=so)
            o, oso = oracle.check_mono(b, c, off, seg_ok=True)
            same(g, o, (n, m, c, trial))
            assert np.array_equal(so.cpu().numpy(), oso[:m])


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", SIZES)
def test_inj(ixp, dev, n, dtype):
    for name, a in arrays(n, dtype, 300 + n).items():
        for lo, hi in [(I64MIN, I64MAX), (0, max(0, n - 1)), (0, n // 2), (5, 5)]:
            same(ixp.check_inj(T(a, dev), lo, hi), oracle.check_inj(a, lo, hi), (name, n, lo, hi))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_inj_many_duplicates_and_edges(ixp, dev, dtype):
    rng = np.random.default_rng(5)
    for n in [10, 1000, 50000]:
        a = rng.integers(0, n // 2 + 1, size=n).astype(dtype)
        same(ixp.check_inj(T(a, dev)), oracle.check_inj(a), n)
        same(ixp.check_inj(T(a, dev), 3, max(3, n // 4)), oracle.check_inj(a, 3, max(3, n // 4)), n)
    n = 40000
    for p, q in [(0, 1), (0, n - 1), (n - 2, n - 1), (4095, 4096), (17, 30000)]:
        a = synth.permutation(n, 11, dtype)
        a[q] = a[p]
        same(ixp.check_inj(T(a, dev)), oracle.check_inj(a), (p, q))


def test_inj_wide_values_and_span_limit(ixp, dev):
    rng = np.random.default_rng(9)
    n = 5000
    a = (rng.permutation(n).astype(np.int64) * 3 - 7000)
    same(ixp.check_inj(T(a, dev)), oracle.check_inj(a))
    a[100] = a[4000]
    same(ixp.check_inj(T(a, dev)), oracle.check_inj(a))
    # values spread over 2^40: with a bitmap-only workspace the span is too wide
    b = rng.integers(0, 2**40, size=n).astype(np.int64)
    g = ixp.check_inj(T(b, dev), span=4 * n + 4096).get()
    assert g["status"] == -3 and g["ok"] == -1
    # the default workspace holds the hash set, which decides it
    same(ixp.check_inj(T(b, dev)), oracle.check_inj(b))
    # restricting Rcd to a small window makes it a bitmap check again
    same(ixp.check_inj(T(b, dev), 0, 2**20), oracle.check_inj(b, 0, 2**20))


def spread_ids(n, seed, bits=62):
    """Distinct int64 values spread over [0, 2^bits): a permutation in the high bits,
    random low bits."""
    rng = np.random.default_rng(seed)
    hb = max(1, int(n - 1).bit_length())
    low = bits - hb
    return (rng.permutation(n).astype(np.int64) << low) | rng.integers(0, 1 << low, size=n, dtype=np.int64)


@pytest.mark.parametrize("n", [2, 4097, 1 << 20, 3_000_001])
def test_inj_any_span_hash_set(ixp, dev, n):
    """Inj over spans no bitmap covers: int64 ids over [0, 2^62), planted repeats
    (first position at either end, several repeated values), a restricted Rcd, int32
    values over the whole type, and the whole int64 range."""
    x = spread_ids(n, n)
    same(ixp.check_inj(T(x, dev)), oracle.check_inj(x), ("ids", n))
    for p, q in [(0, n - 1), (n - 2, n - 1), (n // 3, n // 2)]:
        if p == q:
            continue
        d = x.copy()
        d[q] = d[p]
        same(ixp.check_inj(T(d, dev)), oracle.check_inj(d), ("ids-dup", n, p, q))
    if n >= 8:
        d = x.copy()
        d[n - 1] = d[3]
        d[n // 2] = d[n // 4]
        d[7] = -1
        d[n - 3] = -1  # the value -1 keeps its pair in the header
        same(ixp.check_inj(T(d, dev)), oracle.check_inj(d), ("ids-several", n))
        lo, hi = int(np.sort(x)[n // 4]), int(np.sort(x)[3 * n // 4])
        same(ixp.check_inj(T(d, dev), lo, hi), oracle.check_inj(d, lo, hi), ("ids-rcd", n))
    rng = np.random.default_rng(n + 1)
    w = rng.integers(-2**31, 2**31, size=n, dtype=np.int64).astype(np.int32)
    same(ixp.check_inj(T(w, dev)), oracle.check_inj(w), ("int32-wide", n))
    e = x.copy()
    e[0] = I64MIN
    e[n - 1] = I64MAX  # the span is all 2^64 values
    same(ixp.check_inj(T(e, dev)), oracle.check_inj(e), ("full-range", n))
    e[n // 2] = I64MAX
    same(ixp.check_inj(T(e, dev)), oracle.check_inj(e), ("full-range-dup", n))


def _mix64(z):
    m = (1 << 64) - 1
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def _unmix64(h):
    """The value whose SplitMix64 finalizer is h (each step of the finalizer is a
    bijection of the 64-bit words)."""
    m = (1 << 64) - 1

    def unxs(y, s):
        x = y
        for _ in range(64 // s + 1):
            x = y ^ (x >> s)
        return x

    z = unxs(h, 31)
    z = (z * pow(0x94D049BB133111EB, -1, 1 << 64)) & m
    z = unxs(z, 27)
    z = (z * pow(0xBF58476D1CE4E5B9, -1, 1 << 64)) & m
    return unxs(z, 30)


def test_inj_any_span_partitioned_paths(ixp, dev):
    """Above 2^21 elements the any-span Inj splits the hash set into parts by the top
    bits of the values' hash; these cases take each of its exits: a part whose pool
    fills up (one value repeated 1.2 M times) and more repeated values than its list
    holds (3000 pairs) both hand the call to the single table; 1500 pairs, and the
    one value whose hash is all ones (counted apart), are decided by the parts."""
    n = 3_000_001
    x = spread_ids(n, 41)
    rng = np.random.default_rng(41)
    a = x.copy()
    a[rng.choice(n, size=1_200_000, replace=False)] = x[12345]
    same(ixp.check_inj(T(a, dev)), oracle.check_inj(a), "pool-full")
    for pairs, what in [(3000, "many-repeats"), (1500, "listed-repeats")]:
        b = x.copy()
        pos = rng.choice(n, size=2 * pairs, replace=False)
        b[pos[pairs:]] = b[pos[:pairs]]
        same(ixp.check_inj(T(b, dev)), oracle.check_inj(b), what)
    top = _unmix64((1 << 64) - 1)
    assert _mix64(top) == (1 << 64) - 1
    top = np.int64(top - (1 << 64) if top >= 1 << 63 else top)
    c = x.copy()
    c[777] = top
    same(ixp.check_inj(T(c, dev)), oracle.check_inj(c), "top-hash-once")
    c[2_500_000] = top
    same(ixp.check_inj(T(c, dev)), oracle.check_inj(c), "top-hash-twice")
    c[100] = c[2_900_000]  # an earlier repeat of another value wins
    same(ixp.check_inj(T(c, dev)), oracle.check_inj(c), "top-hash-and-another")
    # an 8-byte-aligned view (scalar loads in the first grouping pass), clean and with a repeat
    buf = np.concatenate([np.zeros(1, np.int64), x])
    same(ixp.check_inj(T(buf, dev)[1:]), oracle.check_inj(x), "unaligned")
    buf[1 + n - 5] = x[17]
    d = buf[1:].copy()
    same(ixp.check_inj(T(buf, dev)[1:]), oracle.check_inj(d), "unaligned-dup")


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", [1, 2, 33, 4097, 65536, 100003])
def test_bij(ixp, dev, n, dtype):
    seed = 400 + n
    perm = synth.permutation(n, seed, dtype)
    cases = {"perm": perm}
    if n >= 2:
        cases["dup"] = synth.plant_duplicate(perm, seed)[0]
        cases["oor"] = synth.plant_value(perm, seed, n)[0]
        cases["neg"] = synth.plant_value(perm, seed, -1)[0]
        cases["gap"] = synth.plant_value(perm, seed, n + 5)[0]
    for name, a in cases.items():
        for rlo, rhi, ilo, ihi in [(I64MIN, I64MAX, 0, n - 1), (0, n - 1, 0, n - 1), (-1, n + 10, 0, n - 1),
                                   (0, n + 2, 0, n + 2)]:
            same(ixp.check_bij(T(a, dev), rlo, rhi, ilo, ihi), oracle.check_bij(a, rlo, rhi, ilo, ihi),
                 (name, n, rlo, rhi, ilo, ihi))


# ---- large inputs take the value-bucketed Inj/Bij path (n >= 2^18, span >= 2^21)

@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", [1 << 18, (1 << 21) + 12345, 3_000_001])
def test_inj_bij_bucketed(ixp, dev, n, dtype):
    seed = 900 + n
    perm = synth.permutation(n, seed, dtype)
    cases = {"perm": perm, "dup": synth.plant_duplicate(perm, seed)[0], "oor": synth.plant_value(perm, seed, n)[0],
             "neg": synth.plant_value(perm, seed, -1)[0], "far": synth.plant_value(perm, seed, 3 * n)[0]}
    for name, a in cases.items():
        t = T(a, dev)
        for lo, hi in [(I64MIN, I64MAX), (0, n - 1)]:
            same(ixp.check_inj(t, lo, hi), oracle.check_inj(a, lo, hi), (name, n, lo, hi, "inj"))
        for rlo, rhi in [(I64MIN, I64MAX), (0, n - 1), (-1, 2 * n)]:
            same(ixp.check_bij(t, rlo, rhi, 0, n - 1), oracle.check_bij(a, rlo, rhi, 0, n - 1), (name, n, rlo, "bij"))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_inj_bucketed_skewed_overflow(ixp, dev, dtype):
    # most values packed into the first bucket's range of a wide span: the bucket's pool
    # region overflows and the excess takes the L2-atomic path
    rng = np.random.default_rng(17)
    n = 600_000
    dense = rng.permutation(400_000)
    sparse = 400_000 + rng.choice(2**23, size=n - 400_000, replace=False)
    a = rng.permutation(np.concatenate([dense, sparse])).astype(dtype)
    same(ixp.check_inj(T(a, dev)), oracle.check_inj(a), "skew-ok")
    same(ixp.check_inj(T(a, dev), 0, 2**23 + 400_000), oracle.check_inj(a, 0, 2**23 + 400_000), "skew-ok-fixed")
    for p, q in [(3, 500_000), (599_999, 0), (12345, 54321)]:
        b = a.copy()
        b[q] = b[p]
        same(ixp.check_inj(T(b, dev)), oracle.check_inj(b), ("skew-dup", p, q))
    # many repeats inside the dense range
    c = a.copy()
    c[:200_000] = rng.integers(0, 1000, size=200_000)
    same(ixp.check_inj(T(c, dev)), oracle.check_inj(c), "skew-many")
    # Bij over the dense+sparse image with a gap
    img_hi = 2**23 + 400_000 - 1
    same(ixp.check_bij(T(a, dev), I64MIN, I64MAX, 0, img_hi), oracle.check_bij(a, I64MIN, I64MAX, 0, img_hi), "bij-gap")


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_inj_bucketed_pool_overflow_without_row_overflow(ixp, dev, dtype):
    # 512 buckets of 2^15 values over [0, 2^24): every 8192-element tile holds 30
    # values of bucket 0 and about 16 of each other bucket, so no tile overflows a
    # bucket's slot row, but bucket 0 receives more entries in total than its pool
    # region holds; the tiles that come last send them through the L2-atomic path
    rng = np.random.default_rng(23)
    n, tile, k0 = 1 << 20, 8192, 30
    ntile = n // tile
    b0 = rng.permutation(1 << 15)[: ntile * k0]
    rest = (1 << 15) + rng.choice((1 << 24) - (1 << 15), size=n - ntile * k0, replace=False)
    parts = []
    for t in range(ntile):
        chunk = np.concatenate([b0[t * k0:(t + 1) * k0], rest[t * (tile - k0):(t + 1) * (tile - k0)]])
        parts.append(rng.permutation(chunk))
    a = np.concatenate(parts).astype(dtype)
    hi = (1 << 24) - 1
    same(ixp.check_inj(T(a, dev), 0, hi), oracle.check_inj(a, 0, hi), "pool-overflow-ok")
    same(ixp.check_inj(T(a, dev)), oracle.check_inj(a), "pool-overflow-ok-derived")
    pos0 = np.flatnonzero(a < (1 << 15))  # bucket-0 positions, in index order
    for p, q in [(pos0[0], pos0[-1]), (pos0[-2], pos0[-1]), (pos0[5], pos0[ntile * k0 // 2]), (0, n - 1)]:
        b = a.copy()
        b[q] = b[p]
        same(ixp.check_inj(T(b, dev), 0, hi), oracle.check_inj(b, 0, hi), ("pool-overflow-dup", p, q))
        same(ixp.check_bij(T(b, dev), 0, hi, 0, hi), oracle.check_bij(b, 0, hi, 0, hi), ("pool-overflow-bij", p, q))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_inj_bij_bucketed_unaligned_sorted_and_witnesses(ixp, dev, dtype):
    # bucketed path on an unaligned view (scalar loads), on sorted values (each tile
    # lands in one or two buckets, so runs are thousands long), and repeats whose
    # first occurrence sits at either end of the array with the partner far away
    n = 1_500_007
    perm = synth.permutation(n, 77, dtype)
    buf = np.concatenate([np.zeros(1, dtype), perm])
    tv = T(buf, dev)[1:]
    for lo, hi in [(I64MIN, I64MAX), (0, n - 1)]:
        same(ixp.check_inj(tv, lo, hi), oracle.check_inj(perm, lo, hi), ("unaligned", lo))
    same(ixp.check_bij(tv, I64MIN, I64MAX, 0, n - 1), oracle.check_bij(perm, I64MIN, I64MAX, 0, n - 1), "unaligned-bij")
    d = perm.copy()
    d[n - 1] = d[n - 2]
    buf[1:] = d
    tv = T(buf, dev)[1:]
    same(ixp.check_inj(tv), oracle.check_inj(d), "unaligned-dup")
    iota = np.arange(n, dtype=dtype) * 2 + 11
    same(ixp.check_inj(T(iota, dev)), oracle.check_inj(iota), "sorted")
    for p, q in [(0, n - 1), (n - 3, n - 1), (0, 1), (700_000, 700_001)]:
        a = iota.copy()
        a[q] = a[p]
        same(ixp.check_inj(T(a, dev)), oracle.check_inj(a), ("sorted-dup", p, q))
        b = perm.copy()
        b[q] = b[p]
        same(ixp.check_inj(T(b, dev), 0, n - 1), oracle.check_inj(b, 0, n - 1), ("perm-dup", p, q))
        same(ixp.check_bij(T(b, dev), I64MIN, I64MAX, 0, n - 1), oracle.check_bij(b, I64MIN, I64MAX, 0, n - 1),
             ("perm-dup-bij", p, q))
    # several repeated values: the witness is the smallest first occurrence
    c = perm.copy()
    c[1_400_000] = c[5]
    c[900_000] = c[200_000]
    c[1_000_000] = c[1_200_000]
    same(ixp.check_inj(T(c, dev)), oracle.check_inj(c), "several")


def test_inj_bij_both_bucket_paths_launched(ixp, dev):
    # Rcd unbounded and n > 2^26: the bitmap capacity (4n + 4096 bits) exceeds 2^28,
    # so both pass-1 paths are launched and the span found on the device (n) picks
    # the staged one; a planted value far out widens the span past 2^28 and picks the
    # wide one
    n = (1 << 26) + 5
    perm = synth.permutation(n, 91, np.int32)
    t = T(perm, dev)
    same(ixp.check_inj(t), oracle.check_inj(perm), "staged")
    same(ixp.check_bij(t, I64MIN, I64MAX, 0, n - 1), oracle.check_bij(perm, I64MIN, I64MAX, 0, n - 1), "staged-bij")
    d, p, q = synth.plant_duplicate(perm, 92)
    same(ixp.check_inj(T(d, dev)), oracle.check_inj(d), ("staged-dup", p, q))
    w = perm.copy()
    w[12345] = 3 * n + 7  # span 3n + 8 > 2^28, below the 4n + 4096 capacity
    same(ixp.check_inj(T(w, dev)), oracle.check_inj(w), "wide")
    w[777] = w[12345]
    same(ixp.check_inj(T(w, dev)), oracle.check_inj(w), "wide-dup")


# ---- per-segment Inj / Bij

def mixed_segments(rng, m, small_max=300, big=(), empty_p=0.15):
    """Segment lengths: mostly small (warp path), some above 256 (block path), a few big."""
    L = rng.integers(0, small_max, size=m)
    L[rng.random(m) < empty_p] = 0
    for pos, ln in big:
        L[pos] = ln
    return synth.offsets_from_shape(L)


def seg_perm(rng, off, dtype):
    return np.concatenate([rng.permutation(np.arange(off[k], off[k + 1])) for k in range(len(off) - 1)]
                          ).astype(dtype) if off[-1] else np.zeros(0, dtype)


def seg_same(ixp, dev, x, off, g_fn, o_fn, what):
    m = len(off) - 1
    so = torch.full((m,), 7, dtype=torch.uint8, device=dev)
    g = g_fn(T(x, dev), T(off, dev), seg_ok=so)
    o, oso = o_fn(x, off)
    same(g, o, what)
    assert np.array_equal(so.cpu().numpy(), oso[:m]), what


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_bij_seg(ixp, dev, dtype):
    rng = np.random.default_rng(41)
    off = mixed_segments(rng, 2000, big=[(5, 5000), (700, 70000), (1500, 1 << 20)])
    x = seg_perm(rng, off, dtype)
    n = int(off[-1])
    g_fn = lambda t, o, seg_ok: ixp.check_bij_seg(t, o, seg_ok=seg_ok)  # noqa: E731
    o_fn = lambda a, o: oracle.check_bij(a, I64MIN, I64MAX, seg_img=True, offsets=o, seg_ok=True)  # noqa: E731
    seg_same(ixp, dev, x, off, g_fn, o_fn, "ok")
    nonempty = np.flatnonzero(np.diff(off) > 1)
    for trial in range(6):
        y = x.copy()
        k = int(nonempty[rng.integers(0, len(nonempty))]) if trial < 4 else int(nonempty[-1 - trial])
        a, b = int(off[k]), int(off[k + 1])
        i, j = a + int(rng.integers(0, b - a)), a + int(rng.integers(0, b - a))
        if trial % 3 == 0:
            y[j] = y[i] if i != j else y[i]  # duplicate inside the segment (also a missing value)
        elif trial % 3 == 1:
            y[i] = (b + 3) % n  # value of another segment
        else:
            y[i] = n + 10  # outside Rcd [0, n+5]: ignored, leaves a missing value
        for rlo, rhi in [(I64MIN, I64MAX), (0, n + 5)]:
            g_fn2 = lambda t, o, seg_ok: ixp.check_bij_seg(t, o, rlo, rhi, seg_ok=seg_ok)  # noqa: E731
            o_fn2 = lambda a_, o: oracle.check_bij(a_, rlo, rhi, seg_img=True, offsets=o, seg_ok=True)  # noqa: E731
            seg_same(ixp, dev, y, off, g_fn2, o_fn2, (trial, k, rlo))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_inj_seg(ixp, dev, dtype):
    rng = np.random.default_rng(43)
    off = mixed_segments(rng, 3000, big=[(9, 4000), (1000, 50000), (2000, 300000)])
    m = len(off) - 1
    n = int(off[-1])
    g_fn = lambda t, o, seg_ok: ixp.check_inj_seg(t, o, seg_ok=seg_ok)  # noqa: E731
    o_fn = lambda a, o: oracle.check_inj(a, offsets=o, seg_ok=True)  # noqa: E731
    # rows of sorted distinct columns (strict increase), as in CSR
    cols = np.concatenate([np.sort(rng.choice(1 << 24, size=int(off[k + 1] - off[k]), replace=False))
                           for k in range(m)]).astype(dtype)
    seg_same(ixp, dev, cols, off, g_fn, o_fn, "sorted")
    nonempty = np.flatnonzero(np.diff(off) > 2)
    for trial in range(8):
        y = cols.copy()
        k = int(nonempty[rng.integers(0, len(nonempty))]) if trial < 5 else int(nonempty[-1 - trial])
        a, b = int(off[k]), int(off[k + 1])
        p = a + 1 + int(rng.integers(0, b - a - 1))
        if trial % 2 == 0:
            y[p] = y[p - 1]  # planted duplicate
        else:
            y[p], y[p - 1] = y[p - 1], y[p]  # order swap: still injective
        seg_same(ixp, dev, y, off, g_fn, o_fn, (trial, k))
    # unsorted rows with small spans (shared-memory bitmaps) and repeats across rows (allowed)
    z = np.concatenate([rng.permutation(int(off[k + 1] - off[k])) for k in range(m)]).astype(dtype)
    seg_same(ixp, dev, z, off, g_fn, o_fn, "perm-rows")
    z2 = z.copy()
    k = 2000
    z2[int(off[k]) + 7] = z2[int(off[k]) + 100]
    seg_same(ixp, dev, z2, off, g_fn, o_fn, "perm-rows-dup")
    # an unsorted row whose values span more than 2^20 (global-bitmap pass)
    z3 = z.copy()
    a, b = int(off[1000]), int(off[1001])
    z3[a:b] = rng.choice(1 << 23, size=b - a, replace=False)
    seg_same(ixp, dev, z3, off, g_fn, o_fn, "wide-row")
    z3[a + 17] = z3[b - 1]
    seg_same(ixp, dev, z3, off, g_fn, o_fn, "wide-row-dup")
    # Rcd restricts the check
    g_r = lambda t, o, seg_ok: ixp.check_inj_seg(t, o, 0, 100, seg_ok=seg_ok)  # noqa: E731
    o_r = lambda a_, o: oracle.check_inj(a_, 0, 100, offsets=o, seg_ok=True)  # noqa: E731
    seg_same(ixp, dev, z2, off, g_r, o_r, "rcd")


def test_inj_seg_span_limit(ixp, dev):
    rng = np.random.default_rng(47)
    off = np.array([0, 1000, 1300], np.int64)
    x = np.concatenate([np.arange(1000), rng.choice(1 << 40, size=300, replace=False)]).astype(np.int64)
    g = ixp.check_inj_seg(T(x, dev), T(off, dev)).get()
    assert g["status"] == -3 and g["ok"] == -1


@pytest.mark.parametrize("it,ot", [(np.int32, np.int32), (np.int32, np.int64), (np.int64, np.int64)])
@pytest.mark.parametrize("n", SIZES + [300000])
def test_scan_flat(ixp, dev, n, it, ot):
    rng = np.random.default_rng(n)
    info = np.iinfo(it)
    for lo, hi in [(0, 4), (info.min // 4, info.max // 4)]:
        a = rng.integers(lo, hi, size=n).astype(it)
        for inc in (False, True):
            out, tot, st = ixp.scan(T(a, dev), getattr(torch, np.dtype(ot).name), inclusive=inc)
            o, otot = oracle.scan(a, ot, inclusive=inc)
            assert st.item() == 0
            assert np.array_equal(out.cpu().numpy(), o), (n, inc)
            assert int(tot[0].item()) == int(otot[0])


@pytest.mark.parametrize("it,ot", [(np.int32, np.int32), (np.int32, np.int64), (np.int64, np.int64)])
@pytest.mark.parametrize("n,m", [(1, 1), (100, 7), (5000, 3), (5000, 2000), (70000, 50), (70000, 30000),
                                 (300001, 3), (1 << 20, 1)])
def test_scan_segmented(ixp, dev, n, m, it, ot):
    rng = np.random.default_rng(n * 7 + m)
    off = random_offsets(rng, n, m)
    a = rng.integers(-50, 100, size=n).astype(it)
    for inc in (False, True):
        out, tot, st = ixp.scan(T(a, dev), getattr(torch, np.dtype(ot).name), inclusive=inc, offsets=T(off, dev))
        o, otot = oracle.scan(a, ot, inclusive=inc, offsets=off)
        assert st.item() == 0
        assert np.array_equal(out.cpu().numpy(), o), (n, m, inc)
        assert np.array_equal(tot.cpu().numpy(), otot[:m])


def test_scan_segmented_unaligned(ixp, dev):
    # values and outputs off a 16-byte boundary take the register-tiled kernel
    rng = np.random.default_rng(12)
    n = 70001
    off = random_offsets(rng, n, 40)
    a = rng.integers(-50, 100, size=n + 1).astype(np.int32)
    t = T(a, dev)
    o, otot = oracle.scan(a[1:], np.int64, inclusive=True, offsets=off)
    out = torch.empty(n + 1, dtype=torch.int64, device=dev)
    r, tot, st = ixp.scan(t[1:], torch.int64, inclusive=True, offsets=T(off, dev), out=out[1:])
    assert st.item() == 0 and np.array_equal(r.cpu().numpy(), o) and np.array_equal(tot.cpu().numpy(), otot[:40])


def test_scan_unaligned(ixp, dev):
    a = np.arange(50001, dtype=np.int32) % 7
    t = T(a, dev)
    for off in range(4):
        out = torch.empty(50001, dtype=torch.int64, device=dev)
        r, _, _ = ixp.scan(t[off:], torch.int64, out=out[off:], totals=torch.empty(1, dtype=torch.int64, device=dev))
        assert np.array_equal(r.cpu().numpy(), oracle.scan(a[off:], np.int64)[0])


@pytest.mark.parametrize("offset", [0, 1])
def test_scan_timeout_is_reported(ixp, dev, offset):
    # a tile that never publishes makes its successors' bounded waits run out;
    # offset 0 takes the TMA-staged path (16384-element tiles), offset 1 the
    # unaligned register path (4096-element tiles)
    n = 16384 * 12 + 5
    a = np.ones(n + offset, np.int32)
    t = T(a, dev)[offset:]
    try:
        ixp.debug_set_wait(2000, 3)
        _, _, st = ixp.scan(t)
        torch.cuda.synchronize()
        assert st.item() == -6
    finally:
        ixp.debug_set_wait(0, -1)
    out, tot, st = ixp.scan(t)
    assert st.item() == 0 and int(tot.item()) == n


PREDS = [("mod_eq", 3, 0), ("lt", 0, 0), ("lt", 0, synth.bernoulli_threshold(0.01)), ("mod_eq", 5, 2),
         ("lt", 0, (1 << 31) + 5), ("lt", 0, -(1 << 31) - 7), ("lt", 0, -(1 << 31) + 1), ("mod_eq", 4, 7),
         ("mod_eq", 7, 6), ("mod_eq", 1, 0), ("mod_eq", 3, -1)]


@pytest.mark.parametrize("kt", [np.int32, np.int64])
@pytest.mark.parametrize("ot", [np.int32, np.int64])
@pytest.mark.parametrize("n", [0, 1, 5, 2048, 4097, 65536, 100003])
def test_partition_flat(ixp, dev, n, kt, ot):
    keys = synth.keys_uniform(n, 500 + n).astype(kt)
    pay = synth.payload_f32(n, 600 + n)
    for p in PREDS:
        r = ixp.partition(T(keys, dev), p, payload=T(pay, dev), out_dtype=getattr(torch, np.dtype(ot).name))
        o = oracle.partition(keys, p, payload=pay, out_dtype=ot)
        assert r["status"].item() == 0
        assert np.array_equal(r["indices"].cpu().numpy(), o["indices"]), (n, p)
        assert int(r["num_true"][0].item()) == int(o["num_true"][0])
        assert np.array_equal(r["keys_out"].cpu().numpy(), o["keys_out"])
        assert np.array_equal(r["payload_out"].cpu().numpy().view(np.uint32), o["payload_out"].view(np.uint32))


@pytest.mark.parametrize("kt", [np.int32, np.int64])
@pytest.mark.parametrize("shift", [0, 1])
def test_partition_flat_views_and_no_keys(ixp, dev, kt, shift):
    """Keys / payload / outputs at element offsets (unaligned bases take the
    unstaged path) and with keys not requested."""
    n = 3 * 4096 + 777
    keys = synth.keys_uniform(n + 1, 41).astype(kt)
    pay = synth.payload_f32(n + 1, 42)
    p = ("lt", 0, synth.bernoulli_threshold(0.5))
    kd, pd = T(keys, dev)[shift:shift + n], T(pay, dev)[shift:shift + n]
    o = oracle.partition(keys[shift:shift + n], p, payload=pay[shift:shift + n])
    for want in (False, True):
        out_idx = torch.empty(n + 1, dtype=torch.int32, device=dev)[shift:shift + n]
        out_pay = torch.empty(n + 1, dtype=torch.float32, device=dev)[shift:shift + n]
        r = ixp.partition(kd, p, payload=pd, want_keys=want, out=out_idx, out_payload=out_pay)
        assert r["status"].item() == 0
        assert np.array_equal(out_idx.cpu().numpy(), o["indices"])
        assert np.array_equal(out_pay.cpu().numpy().view(np.uint32), o["payload_out"].view(np.uint32))
        if want:
            assert np.array_equal(r["keys_out"].cpu().numpy(), o["keys_out"])


def test_partition_flags_and_wide_rows(ixp, dev):
    n = 30001
    fl = synth.flags_bernoulli(n, 3, 0.3)
    pay = synth.payload_f32(n, 4, cols=8)
    r = ixp.partition(None, ("flags", 0, 0, T(fl, dev)), payload=T(pay, dev), n=n)
    o = oracle.partition(None, ("flags", 0, 0, fl), payload=pay)
    assert np.array_equal(r["indices"].cpu().numpy(), o["indices"])
    assert np.array_equal(r["payload_out"].cpu().numpy(), o["payload_out"])


@pytest.mark.parametrize("kt", [np.int32, np.int64])
@pytest.mark.parametrize("n,m", [(1, 1), (100, 7), (5000, 3), (5000, 2000), (70000, 50), (70000, 30000)])
def test_partition_segmented(ixp, dev, n, m, kt):
    rng = np.random.default_rng(n + 3 * m)
    off = random_offsets(rng, n, m)
    keys = synth.keys_uniform(n, n + m).astype(kt)
    pay = synth.payload_f32(n, n + m + 1)
    p = ("lt", 0, synth.bernoulli_threshold(0.3))
    r = ixp.partition(T(keys, dev), p, payload=T(pay, dev), offsets=T(off, dev))
    o = oracle.partition(keys, p, payload=pay, offsets=off)
    assert np.array_equal(r["indices"].cpu().numpy(), o["indices"])
    assert np.array_equal(r["num_true"].cpu().numpy(), o["num_true"][:m])
    assert np.array_equal(r["keys_out"].cpu().numpy(), o["keys_out"])
    assert np.array_equal(r["payload_out"].cpu().numpy(), o["payload_out"])


def crowded_offsets(rng, n):
    """Segments that stress the per-tile lists of segment starts: a run of size-1
    segments, 10000 empty segments at one position (more starts than a tile holds),
    empty segments at 0 and at n, and a few long segments."""
    cuts = [0, 0, 0]
    cuts += list(range(1, 3000))                        # size-1 segments
    cuts += [5000] * 10000                              # empty segments at one position
    cuts += sorted(rng.integers(5001, n, size=40).tolist())
    cuts += [n, n]
    return np.array(cuts + [n], np.int64)


@pytest.mark.parametrize("kt", [np.int32, np.int64])
def test_partition_and_filtpart_crowded_segments(ixp, dev, kt):
    n = 200_003
    rng = np.random.default_rng(77)
    off = crowded_offsets(rng, n)
    m = off.shape[0] - 1
    keys = synth.keys_uniform(n, 78).astype(kt)
    pay = synth.payload_f32(n, 79)
    p = ("lt", 0, synth.bernoulli_threshold(0.4))
    r = ixp.partition(T(keys, dev), p, payload=T(pay, dev), offsets=T(off, dev))
    o = oracle.partition(keys, p, payload=pay, offsets=off)
    assert np.array_equal(r["indices"].cpu().numpy(), o["indices"])
    assert np.array_equal(r["num_true"].cpu().numpy(), o["num_true"][:m])
    assert np.array_equal(r["keys_out"].cpu().numpy(), o["keys_out"])
    assert np.array_equal(r["payload_out"].cpu().numpy(), o["payload_out"])
    z = o["indices"].astype(np.int64)
    for trial in range(4):
        zz = z.copy()
        if trial == 1:
            zz[4999] += 1
        if trial == 2:
            zz[5000], zz[5001] = zz[5001], zz[5000]
        if trial == 3:
            zz[1500] = -3
        g = ixp.check_filtpart(T(zz, dev), T(keys, dev), part=p, offsets=T(off, dev))
        same(g, oracle.check_filtpart(zz, keys, part=p, offsets=off), ("crowded", trial))


@pytest.mark.parametrize("p", [0.5, 0.01, 0.999])
@pytest.mark.parametrize("n", [1, 5, 4096, 4099, 65536 * 3 + 7, 1_000_003])
def test_filtpart_lt_int32(ixp, dev, n, p):
    """InvFiltPart of a partition by key < b (int32 keys and Z, no filter: the form
    of the partition's own index array) against the oracle: correct, two entries
    swapped, an entry off by one, negative entries and entries that wrap around
    modulo 2^32 (Z - rank computed in 32 bits), a wrong last entry of a ragged tail."""
    rng = np.random.default_rng(n + int(p * 1000))
    keys = synth.keys_uniform(n, 710 + n)
    part = ("lt", 0, synth.bernoulli_threshold(p))
    z = oracle.partition(keys, part, out_dtype=np.int32)["indices"]
    cases = {"ok": z.copy()}
    if n >= 2:
        s = z.copy(); a, b = rng.integers(0, n, size=2); s[a], s[b] = s[b], s[a]; cases["swap"] = s
        s = z.copy(); s[n // 2] += 1; cases["plus1"] = s
        s = z.copy(); s[n // 3] = -1; cases["neg"] = s
        s = z.copy(); s[n // 4] = np.int32(int(s[n // 4]) - 2**31); cases["wrap"] = s
        s = z.copy(); s[rng.integers(0, n)] = np.iinfo(np.int32).min; cases["min"] = s
        s = z.copy(); s[n - 1] = n; cases["last"] = s
    for name, zz in cases.items():
        same(ixp.check_filtpart(T(zz, dev), T(keys, dev), part=part), oracle.check_filtpart(zz, keys, part=part),
             (name, n, p))


@pytest.mark.parametrize("zt", [np.int32, np.int64])
@pytest.mark.parametrize("n", [1, 6, 4097, 65536, 100003])
def test_filtpart(ixp, dev, n, zt):
    rng = np.random.default_rng(n)
    keys = synth.keys_uniform(n, 700 + n)
    part = ("mod_eq", 3, 0)
    z = oracle.partition(keys, part, out_dtype=zt)["indices"]
    cases = {"ok": z.copy()}
    if n >= 2:
        s = z.copy()
        a, b = rng.integers(0, n, size=2)
        s[a], s[b] = s[b], s[a]
        cases["swap"] = s
        s = z.copy()
        s[n - 1] += 1
        cases["last"] = s
    for name, zz in cases.items():
        same(ixp.check_filtpart(T(zz, dev), T(keys, dev), part=part), oracle.check_filtpart(zz, keys, part=part),
             (name, n))


@pytest.mark.parametrize("zt", [np.int32, np.int64])
@pytest.mark.parametrize("n", [4097, 300001])
def test_filtpart_flat_with_filter(ixp, dev, n, zt):
    """Flat InvFiltPart with a filter, over many tiles: planted faults that keep
    every tile's Z - rank constant (a whole tile shifted), a dropped Z inside
    [0, N), negative and extreme values."""
    rng = np.random.default_rng(n + 11)
    keys = synth.keys_uniform(n, 900 + n).astype(np.int64)
    flags = synth.flags_bernoulli(n, 901 + n, 0.6)
    fl_o, fl_g = ("flags", 0, 0, flags), ("flags", 0, 0, T(flags, dev))
    part = ("lt", 0, synth.bernoulli_threshold(0.4))
    kept = flags != 0
    tru = kept & (keys < part[2])
    N, Tn = int(kept.sum()), int(tru.sum())
    z = np.full(n, -1, np.int64)
    z[np.flatnonzero(tru)] = np.arange(Tn)
    z[np.flatnonzero(kept & ~tru)] = Tn + np.arange(N - Tn)
    tile = 2048  # elements per tile for int64 keys
    cases = {"ok": z.copy()}
    s = z.copy(); s[~kept] = N + 3; cases["dropped_above"] = s
    s = z.copy(); s[np.flatnonzero(~kept)[len(np.flatnonzero(~kept)) // 2]] = 0; cases["dropped_inside"] = s
    sel = np.zeros(n, bool); sel[tile:2 * tile] = True
    s = z.copy(); s[sel & tru] += 1; cases["tile_true_shift"] = s
    s = z.copy(); s[sel & kept & ~tru] -= 1; cases["tile_false_shift"] = s
    s = z.copy(); s[np.flatnonzero(tru)[-1]] = -5; cases["true_negative"] = s
    s = z.copy(); s[np.flatnonzero(kept & ~tru)[0]] = np.iinfo(zt).min; cases["false_min"] = s
    s = z.copy(); s[np.flatnonzero(tru)[0]] = np.iinfo(zt).max; cases["true_max"] = s
    a, b = np.flatnonzero(kept)[[3, 10]]
    s = z.copy(); s[a], s[b] = s[b], s[a]; cases["swap"] = s
    for name, zz in cases.items():
        zz = zz.astype(zt)
        same(ixp.check_filtpart(T(zz, dev), T(keys, dev), filt=fl_g, part=part),
             oracle.check_filtpart(zz, keys, filt=fl_o, part=part), (name, n))


@pytest.mark.parametrize("n,m", [(100, 1), (5000, 40), (70000, 30000)])
def test_filtpart_filter_and_segments(ixp, dev, n, m):
    rng = np.random.default_rng(n + m)
    off = random_offsets(rng, n, m)
    keys = synth.keys_uniform(n, n).astype(np.int64)
    flags = synth.flags_bernoulli(n, n + 1, 0.7)
    fl_o = ("flags", 0, 0, flags)
    fl_g = ("flags", 0, 0, T(flags, dev))
    part = ("lt", 0, synth.bernoulli_threshold(0.4))
    # reference destinations from the oracle's definition; dropped elements -> -1
    cls = (keys >= part[2]).astype(np.uint8)
    ref = np.full(n, -1, np.int64)
    pos = 0
    for k in range(m):
        idx = [i for i in range(off[k], off[k + 1]) if flags[i]]
        for i in sorted(idx, key=lambda i: cls[i]):
            ref[i] = pos
            pos += 1
    for trial in range(3):
        z = ref.copy()
        if trial == 1:
            z[rng.integers(0, n)] += 1
        if trial == 2:
            d = np.flatnonzero(ref < 0)
            if len(d):
                z[d[len(d) // 2]] = 0
        g = ixp.check_filtpart(T(z, dev), T(keys, dev), filt=fl_g, part=part, offsets=T(off, dev))
        o = oracle.check_filtpart(z, keys, filt=fl_o, part=part, offsets=off)
        same(g, o, (n, m, trial))


@pytest.mark.parametrize("it", [np.int32, np.int64])
@pytest.mark.parametrize("cols,fdt", [(1, np.float32), (8, np.float32), (3, np.float32), (2, np.float64),
                                      (4, np.float32), (12, np.float32), (40, np.float32), (16, np.float64),
                                      (64, np.float64), (48, np.float64)])
def test_scatter_gather(ixp, dev, it, cols, fdt):
    rng = np.random.default_rng(cols)
    n, m = 50003, 40000
    vals = rng.standard_normal((n, cols)).astype(fdt)
    idx = (rng.permutation(n) - 5000).astype(it)  # injective, some out of bounds on both sides
    dst = np.zeros((m, cols), fdt)
    g = ixp.scatter(T(dst, dev), T(idx, dev), T(vals, dev))
    assert np.array_equal(g.cpu().numpy(), oracle.scatter(dst, idx, vals))
    gi = np.clip(idx, 0, m - 1).astype(it)
    out, st = ixp.gather(g, T(gi, dev))
    assert st.item() == 0 and np.array_equal(out.cpu().numpy(), oracle.gather(g.cpu().numpy(), gi)[0])
    out, st = ixp.gather(g, T(idx, dev))
    o, oob = oracle.gather(g.cpu().numpy(), idx)
    assert st.item() == -7 and oob and np.array_equal(out.cpu().numpy(), o)


def test_scatter_add_f64_zipf(ixp, dev):
    n, m, cols = 200000, 1024, 8
    idx = synth.zipf_ranks(n, m, 1.1, 77)
    vals = synth.payload_f32(n, 78, cols=cols)
    acc = torch.zeros((m, cols), dtype=torch.float64, device=dev)
    ixp.scatter_add_f64(acc, T(idx, dev), T(vals, dev))
    ref = oracle.scatter_add_f64(m, idx, vals)
    absum = oracle.scatter_add_f64(m, idx, np.abs(vals))
    err = np.abs(acc.cpu().numpy() - ref)
    assert np.all(err <= 1e-10 * absum + 1e-300)
    f32 = ixp.f64_to_f32(acc).cpu().numpy()
    assert np.array_equal(f32, ref.astype(np.float32)) or np.all(np.abs(f32 - ref) <= 1e-6 * np.maximum(absum, 1e-30))


@pytest.mark.parametrize("cols", [1, 3, 8])
@pytest.mark.parametrize("it", [np.int32, np.int64])
def test_scatter_add_f64_cache_misses(ixp, dev, cols, it):
    """Most targets outside every block's shared cache (Zipf over 2^18 targets, so
    the missing rows go to the global accumulator, 8 lanes per row), with
    out-of-bounds targets mixed in: against the float64 oracle."""
    rng = np.random.default_rng(cols + 7)
    n, m = 300001, 1 << 18
    idx = synth.zipf_ranks(n, m, 1.1, 79 + cols).astype(it)
    idx[rng.random(n) < 0.01] = -1
    idx[rng.random(n) < 0.01] = m
    vals = synth.payload_f32(n, 80 + cols, cols=cols)
    vals[rng.random(n) < 0.02] = 0.0
    acc = torch.zeros((m, cols) if cols > 1 else (m,), dtype=torch.float64, device=dev)
    ixp.scatter_add_f64(acc, T(idx, dev), T(vals if cols > 1 else vals.reshape(n), dev))
    keep = (idx >= 0) & (idx < m)
    ref = oracle.scatter_add_f64(m, idx[keep], vals[keep])
    absum = oracle.scatter_add_f64(m, idx[keep], np.abs(vals[keep]))
    got = acc.cpu().numpy().reshape(ref.shape)
    assert np.all(np.abs(got - ref) <= 1e-10 * absum + 1e-300)


@pytest.mark.parametrize("m", [0, 1, 5, 1000, 40000])
@pytest.mark.parametrize("ot", [np.int32, np.int64])
def test_flags_from_shape(ixp, dev, m, ot):
    rng = np.random.default_rng(m)
    shape = synth.shapes_with_empties(m, m + 1, 9)
    xs = rng.integers(1, 1000, size=m).astype(np.int64)
    for x in (xs, None):
        out, offs, st = ixp.flags_from_shape(T(shape, dev), None if x is None else T(x, dev),
                                             out_dtype=getattr(torch, np.dtype(ot).name))
        o, ooff = oracle.flags_from_shape(shape, x, out_dtype=ot)
        assert st.item() == 0
        assert np.array_equal(out.cpu().numpy(), o)
        assert np.array_equal(offs.cpu().numpy(), ooff)


def test_flags_from_shape_paper_example(ixp, dev):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mksgmdescr_example.json")))
    out, _, _ = ixp.flags_from_shape(T(np.array(g["shape"], np.int64), dev), T(np.array(g["xs"], np.int64), dev))
    assert out.cpu().tolist() == g["result"]


def test_partition_paper_demo(ixp, dev):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "partition2_demo.json")))
    r = ixp.partition(T(np.array(g["xs"], np.int32), dev), ("lt", 0, 5))
    assert r["indices"].cpu().tolist() == g["indices"]
    assert r["keys_out"].cpu().tolist() == g["ys"]
    assert r["num_true"].item() == g["num_true"]


def classes_dest(cls, v, kept, off):
    """Destinations of the v-class filter-partition: per segment, kept elements by
    class (min(cls, v - 1)), stably; dropped elements get -1."""
    n = cls.shape[0]
    z = np.full(n, -1, np.int64)
    pos = 0
    for k in range(off.shape[0] - 1):
        a, b = int(off[k]), int(off[k + 1])
        idx = np.arange(a, b)[kept[a:b]]
        c = np.minimum(cls[idx], v - 1)
        order = idx[np.argsort(c, kind="stable")]
        z[order] = pos + np.arange(order.shape[0])
        pos += order.shape[0]
    return z


@pytest.mark.parametrize("zt", [np.int32, np.int64])
@pytest.mark.parametrize("v", [1, 2, 3, 7, 256])
@pytest.mark.parametrize("n,m", [(1, 0), (4097, 0), (300001, 0), (5000, 1), (70000, 37), (20000, 3000)])
def test_filtpart_classes(ixp, dev, n, m, v, zt):
    """InvFiltPart with v classes, flat (m = 0) and segmented, with a filter; planted
    faults at a class boundary, inside a class, on a dropped element."""
    rng = np.random.default_rng(n + m + v)
    off = np.array([0, n], np.int64) if m == 0 else random_offsets(rng, n, m)
    keys = synth.keys_uniform(n, n + v).astype(np.int64)
    flags = synth.flags_bernoulli(n, n + v + 1, 0.8)
    cls = rng.integers(0, 256, size=n).astype(np.uint8)
    kept = flags != 0
    z = classes_dest(cls, v, kept, off)
    z[~kept] = -1
    cases = {"ok": z.copy()}
    kidx = np.flatnonzero(kept)
    if kidx.shape[0] >= 2:
        s = z.copy(); a, b = kidx[0], kidx[-1]; s[a], s[b] = s[b], s[a]; cases["swap_ends"] = s
        s = z.copy(); s[kidx[kidx.shape[0] // 2]] += 1; cases["off_by_one"] = s
    if (~kept).any():
        s = z.copy(); s[np.flatnonzero(~kept)[0]] = 0; cases["dropped_inside"] = s
    fl_o, fl_g = ("flags", 0, 0, flags), ("flags", 0, 0, T(flags, dev))
    offs_o = None if m == 0 else off
    offs_g = None if m == 0 else T(off, dev)
    for name, zz in cases.items():
        zz = zz.astype(zt)
        got = ixp.check_filtpart(T(zz, dev), T(keys, dev), filt=fl_g, offsets=offs_g, cls=T(cls, dev), v=v)
        ref = oracle.check_filtpart(zz, keys, filt=fl_o, cls=cls, v=v, offsets=offs_o)
        same(got, ref, (name, n, m, v))


def filtpart_order(kept, cls, off):
    """Source index of every position of FiltPart's Y: per segment, the kept
    elements stably by class (a library stable sort)."""
    n = kept.shape[0]
    seg = np.repeat(np.arange(len(off) - 1), np.diff(off))
    idx = np.flatnonzero(kept)
    return idx[np.lexsort((idx, cls[idx], seg[idx]))] if n else np.zeros(0, np.int64)


@pytest.mark.parametrize("form", ["pred", "classes"])
@pytest.mark.parametrize("cols,dt", [(0, np.float32), (3, np.int32), (8, np.float32)])
@pytest.mark.parametrize("n,m", [(0, 0), (1, 0), (65553, 0), (300001, 0), (70000, 37)])
def test_filtpart_values(ixp, dev, n, m, cols, dt, form):
    """FiltPart in value form against the oracle: the right Y, two rows swapped, one
    bit flipped, a Y one row short and one row long; flat and segmented, with a
    filter, by a predicate (v = 2) or by classes (v = 3)."""
    rng = np.random.default_rng(n + m + cols)
    off = np.array([0, n], np.int64) if m == 0 else random_offsets(rng, n, m)
    keys = synth.keys_uniform(n, n + 3).astype(np.int32)
    flags = synth.flags_bernoulli(n, n + 4, 0.7)
    thr = synth.bernoulli_threshold(0.4)
    shape = (n,) if cols == 0 else (n, cols)
    x = (rng.standard_normal(shape).astype(dt) if dt == np.float32 else
         rng.integers(-2**31, 2**31, size=shape).astype(dt))
    kept = flags != 0
    if form == "pred":
        cls = (keys >= thr).astype(np.uint8)  # class 0 = part true
        v = 2
    else:
        cls = rng.integers(0, 4, size=n).astype(np.uint8)
        v = 3
    order = filtpart_order(kept, np.minimum(cls, v - 1), off)
    y = x[order]
    cases = {"ok": y}
    N = order.shape[0]
    if N >= 2:
        a, b = 0, N - 1
        s2 = y.copy(); s2[[a, b]] = s2[[b, a]]; cases["swap"] = s2
        s3 = y.copy().view(np.int32); s3.reshape(N, -1)[N // 2, 0] ^= 1 << 3; cases["bit"] = s3.view(dt)
    if N >= 1:
        cases["short"] = y[:-1].copy()
    cases["long"] = np.concatenate([y, x[:1] if n else np.zeros((1,) + shape[1:], dt)])
    fl_o, fl_g = ("flags", 0, 0, flags), ("flags", 0, 0, T(flags, dev))
    offs_o = None if m == 0 else off
    offs_g = None if m == 0 else T(off, dev)
    for name, yy in cases.items():
        yy = np.ascontiguousarray(yy)
        if form == "pred":
            got = ixp.check_filtpart_values(T(yy, dev), T(x, dev), T(keys, dev), filt=fl_g, part=("lt", 0, thr),
                                            offsets=offs_g)
            ref = oracle.check_filtpart_values(yy, x, keys, filt=fl_o, part=("lt", 0, thr), offsets=offs_o)
        else:
            got = ixp.check_filtpart_values(T(yy, dev), T(x, dev), T(keys, dev), filt=fl_g, offsets=offs_g,
                                            cls=T(cls, dev), v=v)
            ref = oracle.check_filtpart_values(yy, x, keys, filt=fl_o, cls=cls, v=v, offsets=offs_o)
        same(got, ref, (name, n, m, cols, form))


@pytest.mark.parametrize("ot", [np.int32, np.int64])
@pytest.mark.parametrize("v", [1, 3, 256])
@pytest.mark.parametrize("n,m", [(0, 0), (1, 0), (300001, 0), (70000, 37), (20000, 3000)])
def test_filtpart_classes_index_form(ixp, dev, n, m, v, ot):
    """The filter + v-class partition's destinations (partition3 is v = 3): equal to
    the stable per-segment class order, accepted by the oracle's InvFiltPart, and
    dropped elements marked -1."""
    rng = np.random.default_rng(7 * n + m + v)
    off = np.array([0, n], np.int64) if m == 0 else random_offsets(rng, n, m)
    keys = synth.keys_uniform(n, n + 3).astype(np.int32)
    cls = rng.integers(0, 256, size=n).astype(np.uint8)
    filt = ("mod_eq", 5, 2) if n else ("true", 0, 0)
    kept = np.array([(int(k) % 5) == 2 for k in keys], bool) if n else np.zeros(0, bool)
    ref = classes_dest(cls, v, kept, off)
    got, nk = ixp.filtpart_classes(T(cls, dev), v, T(keys, dev), filt, None if m == 0 else T(off, dev),
                                   out_dtype=getattr(torch, np.dtype(ot).name), n=n)
    assert np.array_equal(got.cpu().numpy(), ref.astype(ot))
    assert int(nk.item()) == int(kept.sum())
    vd = oracle.check_filtpart(ref.astype(ot), keys, filt=filt, cls=cls, v=v, offsets=None if m == 0 else off)
    assert vd["ok"]


@pytest.mark.parametrize("kt,zt", [(np.int32, np.int32), (np.int64, np.int64), (np.int32, np.int64)])
@pytest.mark.parametrize("v", [2, 3, 4])
@pytest.mark.parametrize("n", [4096 * 40, 4096 * 40 + 13])
@pytest.mark.parametrize("shift", [0, 1])
def test_filtpart_classes_tiles(ixp, dev, n, v, kt, zt, shift):
    """The flat v-class check (v <= 4) takes one pass that records each tile's
    Z - rank per class and revisits only the first failing tile: faults planted in
    several tiles (the first one must be reported), a whole class of one tile moved
    by one (every Z - rank agrees inside the tile, only the prefix disagrees), a
    dropped element inside [0, N), a kept Z whose Z - rank wraps around, dropped Z at
    N and below 0 (both fine), against the oracle; arrays at an element offset take
    the unvectorised loads; the index form on the same views."""
    rng = np.random.default_rng(n + 10 * v + shift)
    off = np.array([0, n], np.int64)
    keys = synth.keys_uniform(n + 1, n + v).astype(kt)
    cls = rng.integers(0, 6, size=n + 1).astype(np.uint8)
    thr = synth.bernoulli_threshold(0.85)
    kept = keys[shift:shift + n] < thr
    c = cls[shift:shift + n]
    z = classes_dest(c, v, kept, off)
    N = int(kept.sum())
    kidx, didx = np.flatnonzero(kept), np.flatnonzero(~kept)
    cc = np.minimum(c, v - 1)
    lo = np.iinfo(zt).min
    cases = {"ok": z.copy()}
    s = z.copy(); s[kidx[(kidx >= 30 * 4096)][0]] += 1; s[kidx[(kidx >= 20 * 4096)][5]] -= 1
    cases["two_tiles"] = s
    s = z.copy(); sel = kidx[(kidx // 4096 == 11) & (cc[kidx] == v - 1)]; s[sel] += 1; s[kidx[-1]] = 0
    cases["class_block_shifted"] = s
    s = z.copy(); s[didx[(didx >= 5 * 4096)][0]] = N - 1; s[kidx[(kidx >= 9 * 4096)][0]] += 7
    cases["dropped_inside_first"] = s
    s = z.copy(); s[kidx[(kidx >= 3 * 4096)][2]] = lo
    cases["wrapping_z"] = s
    s = z.copy(); s[didx[0]] = N; s[didx[1]] = -5; s[didx[-1]] = lo
    cases["dropped_outside"] = s
    s = z.copy(); a, b = kidx[(kidx >= 17 * 4096)][:2]; s[a], s[b] = s[b], s[a]
    cases["swap_in_tile"] = s
    filt = ("lt", 0, thr)
    kd = T(keys, dev)[shift:shift + n]
    cd = T(cls, dev)[shift:shift + n]
    for name, zz in cases.items():
        zz = zz.astype(zt)
        zd = torch.empty(n + 1, dtype=getattr(torch, np.dtype(zt).name), device=dev)[shift:shift + n]
        zd.copy_(T(zz, dev))
        got = ixp.check_filtpart(zd, kd, filt=filt, cls=cd, v=v)
        ref = oracle.check_filtpart(zz, keys[shift:shift + n], filt=filt, cls=c, v=v)
        same(got, ref, (name, n, v, shift))
        if name not in ("ok", "dropped_outside"):
            assert not ref["ok"]
    ot = getattr(torch, np.dtype(zt).name)
    out = torch.empty(n + 1, dtype=ot, device=dev)[shift:shift + n]
    got, nk = ixp.filtpart_classes(cd, v, kd, filt, out_dtype=ot, out=out)
    assert np.array_equal(got.cpu().numpy(), z.astype(zt))
    assert int(nk.item()) == N


@pytest.mark.parametrize("it,ot", [(np.int32, np.int32), (np.int32, np.int64), (np.int64, np.int64)])
@pytest.mark.parametrize("n", [0, 1, 33, 4097, 100003, 1 << 20])
def test_sgm_scan_flags(ixp, dev, n, it, ot):
    """sgmSum over a flag array, inclusive (the oracle's literal operator) and
    exclusive (inclusive minus the element), flags at 0, sparse and dense."""
    rng = np.random.default_rng(n + 5)
    x = rng.integers(-1000, 1000, size=n).astype(it)
    tdt = getattr(torch, np.dtype(ot).name)
    for p in (0.0, 0.01, 0.5, 1.0):
        fl = (rng.random(n) < p).astype(np.uint8)
        fl[fl != 0] = rng.integers(1, 256, size=int((fl != 0).sum()))  # any nonzero byte is a head
        inc, st = ixp.sgm_scan(T(fl, dev), T(x, dev), out_dtype=tdt, inclusive=True)
        ref = oracle.sgm_scan(fl, x, out_dtype=ot)
        assert st.item() == 0 and np.array_equal(inc.cpu().numpy(), ref), (n, p)
        exc, _ = ixp.sgm_scan(T(fl, dev), T(x, dev), out_dtype=tdt, inclusive=False)
        assert np.array_equal(exc.cpu().numpy(), (ref - x.astype(ot)).astype(ot)), (n, p)
    # flags one byte off a 16-byte boundary (aligned values), then values off it
    fl = (rng.random(n + 1) < 0.05).astype(np.uint8)
    ref = oracle.sgm_scan(fl[1:], x, out_dtype=ot)
    inc, st = ixp.sgm_scan(T(fl, dev)[1:], T(x, dev), out_dtype=tdt)
    assert st.item() == 0 and np.array_equal(inc.cpu().numpy(), ref)
    xs = np.concatenate([np.zeros(1, it), x])
    inc, st = ixp.sgm_scan(T(fl, dev)[1:], T(xs, dev)[1:], out_dtype=tdt)
    assert st.item() == 0 and np.array_equal(inc.cpu().numpy(), ref)


@pytest.mark.parametrize("form", ["flags", "offsets"])
def test_segmented_scan_timeout_is_reported(ixp, dev, form):
    # a tile that never publishes makes its successors' bounded waits run out, in
    # the TMA-staged segmented scan (16384 int32 elements per tile); no segment head
    # after position 0, so every tile's look-back has to reach the skipped one
    n = 16384 * 12 + 5
    x = T(np.ones(n, np.int32), dev)
    fl = torch.zeros(n, dtype=torch.uint8, device=dev)
    fl[0] = 1
    off = T(np.array([0, n], np.int64), dev)
    run = (lambda: ixp.sgm_scan(fl, x)[1]) if form == "flags" else (lambda: ixp.scan(x, offsets=off)[2])
    try:
        ixp.debug_set_wait(2000, 3)
        st = run()
        torch.cuda.synchronize()
        assert st.item() == -6
    finally:
        ixp.debug_set_wait(0, -1)
    st = run()
    assert st.item() == 0


@pytest.mark.parametrize("ot", [np.int32, np.int64])
@pytest.mark.parametrize("m,maxlen,p_empty", [(1, 5, 0.0), (1000, 40, 0.3), (20000, 300, 0.5), (300, 20000, 0.2)])
def test_mkii(ixp, dev, m, maxlen, p_empty, ot):
    rng = np.random.default_rng(m + maxlen)
    shape = rng.integers(0, maxlen, size=m).astype(np.int64)
    shape[rng.random(m) < p_empty] = 0
    off = synth.offsets_from_shape(shape)
    n = int(off[-1])
    ii, st = ixp.mkii(T(off, dev), n, out_dtype=getattr(torch, np.dtype(ot).name))
    assert st.item() == 0
    assert np.array_equal(ii.cpu().numpy(), oracle.mkii(shape).astype(ot))


def test_scan_totals_take_the_output_dtype(ixp, dev):
    """Totals are written in the output type: an int64 output given without
    out_dtype still gets int64 totals (a sum past 2^31 does not wrap)."""
    x = T(np.full(4099, 2**30, np.int32), dev)
    out = torch.empty(4099, dtype=torch.int64, device=dev)
    _, tot, st = ixp.scan(x, out=out)
    assert st.item() == 0 and tot.dtype == torch.int64 and int(tot[0].item()) == 4099 * 2**30
    assert int(out[-1].item()) == 4098 * 2**30
    with pytest.raises(ValueError):
        ixp.scan(x, out=out, totals=torch.empty(1, dtype=torch.int32, device=dev))


def test_ceiling_microbenchmarks_run_and_check_arguments(ixp, dev):
    """The rate microbenchmarks run (a bitmap OR with and without the returned word
    sets exactly the requested bits) and reject sizes that are not powers of two."""
    import ctypes
    lib = ixp.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sink = torch.empty(lib.ixp_sink_words(), dtype=torch.int32, device=dev)
    pos = T(np.array([3, 35, 64 + 3, 1 << 20, 7, 3, 9, 1023], dtype=np.uint32).view(np.int32), dev)
    for ret in (0, 1):
        bm = torch.zeros(32, dtype=torch.int32, device=dev)  # 1024 bits
        assert lib.ixp_ceiling_atomic_or(bm.data_ptr(), 1024, pos.data_ptr(), 8, ret, sink.data_ptr(), s) == 0
        bits = np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little")
        assert sorted(np.flatnonzero(bits).tolist()) == [0, 3, 7, 9, 35, 67, 1023]
    assert lib.ixp_ceiling_atomic_or(bm.data_ptr(), 1000, pos.data_ptr(), 8, 1, sink.data_ptr(), s) != 0
    rows = torch.zeros(64 * 8, dtype=torch.int32, device=dev)
    assert lib.ixp_ceiling_random_rows(rows.data_ptr(), 64, pos.data_ptr(), 8, sink.data_ptr(), s) == 0
    assert lib.ixp_ceiling_random_rows(rows.data_ptr(), 63, pos.data_ptr(), 8, sink.data_ptr(), s) != 0
    assert lib.ixp_ceiling_stream_read(rows.data_ptr(), rows.numel() * 4, sink.data_ptr(), s) == 0
    torch.cuda.synchronize()


def test_scatter_add_f64_fixed_point_cache_edges(ixp, dev):
    """The shared cache keeps exact fixed-point sums at a scale sampled from each
    block's first rows: rows far below or above that sample, zeros, a long run into
    one target (more rows per block than the sample suggests) and wide dynamic
    ranges must all match the float64 oracle."""
    rng = np.random.default_rng(91)
    n, m = 1 << 20, 512
    idx = synth.zipf_ranks(n, m, 1.1, 92)
    scales = np.where(rng.random(n) < 0.5, 1e-3, 1.0)
    scales[rng.random(n) < 0.01] = 1e-30   # far below any block's sample
    scales[n // 2:][rng.random(n - n // 2) < 0.01] = 1e12  # far above, late in the array
    vals = (rng.uniform(-1, 1, size=(n, 8)) * scales[:, None]).astype(np.float32)
    vals[rng.random(n) < 0.05] = 0.0
    for idx_case in (idx, np.zeros(n, np.int32)):  # the Zipf case, then every row into target 0
        acc = torch.zeros((m, 8), dtype=torch.float64, device=dev)
        ixp.scatter_add_f64(acc, T(idx_case, dev), T(vals, dev))
        ref = oracle.scatter_add_f64(m, idx_case, vals)
        mag = oracle.scatter_add_f64(m, idx_case, np.abs(vals))
        got = acc.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * mag + 1e-300), np.max(np.abs(got - ref) / (mag + 1e-300))
