"""Reduce-by-index with min, the dynamic Inj check built on it, get_smallest_pairs
(maxMatching, Fig. 16) and the partition without its index array, against the
oracle element by element on seeded inputs spanning several tiles (4096 elements
for the filter, 16-byte groups for the streaming kernels) and ragged tails."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [0, 1, 3, 4, 5, 31, 4095, 4096, 4097, 12289, 100003]


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


@pytest.mark.parametrize("it", [np.int32, np.int64])
@pytest.mark.parametrize("ht", [np.int32, np.int64])
@pytest.mark.parametrize("n", SIZES)
def test_hist_min(ixp, dev, n, it, ht):
    rng = np.random.default_rng(n + 7)
    for m in (1, 37, max(1, n // 3), 5000):
        idx = rng.integers(-5, m + 5, size=n).astype(it)  # out of bounds on both sides
        vals = rng.integers(np.iinfo(ht).min, np.iinfo(ht).max, size=n, dtype=np.int64).astype(ht)
        init = rng.integers(np.iinfo(ht).min // 2, np.iinfo(ht).max, size=m, dtype=np.int64).astype(ht)
        H = T(init, dev)
        ixp.hist_min(H, T(idx, dev), T(vals, dev))
        assert np.array_equal(H.cpu().numpy(), oracle.hist_min(m, idx, vals, init=init, dtype=ht)), m
        # iota values (vals = None)
        Hi = T(np.full(m, n, ht), dev)
        ixp.hist_min(Hi, T(idx, dev))
        assert np.array_equal(Hi.cpu().numpy(), oracle.hist_min(m, idx, init=np.full(m, n, ht), dtype=ht))


def test_hist_min_unaligned_views(ixp, dev):
    """Inputs that do not start on a 16-byte boundary take the element-wise path."""
    rng = np.random.default_rng(3)
    n, m = 10007, 999
    idx = rng.integers(0, m, size=n + 1).astype(np.int32)
    vals = rng.integers(-10**9, 10**9, size=n + 1).astype(np.int64)
    H = T(np.full(m, 2**62, np.int64), dev)
    ixp.hist_min(H, T(idx, dev)[1:], T(vals, dev)[1:])
    ref = oracle.hist_min(m, idx[1:], vals[1:], init=np.full(m, 2**62, np.int64))
    assert np.array_equal(H.cpu().numpy(), ref)


def test_hist_min_zipf_contention(ixp, dev):
    """Zipf(1.1) bins: the hottest bin takes about 12% of the updates."""
    n, m = 1 << 20, 1 << 12
    idx = synth.zipf_ranks(n, m, 1.1, 11)
    vals = synth.permutation(n, 12, np.int32)
    H = T(np.full(m, np.iinfo(np.int32).max, np.int32), dev)
    ixp.hist_min(H, T(idx, dev), T(vals, dev))
    assert np.array_equal(H.cpu().numpy(), oracle.hist_min(m, idx, vals, dtype=np.int32))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", SIZES)
def test_check_inj_hist(ixp, dev, n, dtype):
    seed = 300 + n
    perm = synth.permutation(n, seed, dtype)
    cases = {"perm": perm, "identity": synth.identity(n, dtype)}
    if n >= 2:
        cases["dup"] = synth.plant_duplicate(perm, seed)[0]
        cases["oob"] = synth.plant_value(perm, seed, n + 5)[0]
        cases["neg"] = synth.plant_value(perm, seed + 1, -3)[0]
        rng = np.random.default_rng(seed)
        many = perm.copy()
        for _ in range(5):  # several repeated values: the earliest first occurrence wins
            p, q = rng.choice(n, size=2, replace=False)
            many[q] = many[p]
        cases["many"] = many
        cases["small_range"] = rng.integers(0, max(1, n // 2), size=n).astype(dtype)
    for name, x in cases.items():
        for m in (max(1, n), max(1, n // 2), n + 10):
            same(ixp.check_inj_hist(T(x, dev), m), oracle.check_inj(x, 0, m - 1), (name, m))


def test_check_inj_hist_no_bins(ixp, dev):
    x = T(synth.permutation(1000, 1, np.int32), dev)
    v = ixp.check_inj_hist(x, 0).get()
    assert v["ok"] == 1 and v["status"] == 0


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("n", SIZES)
def test_smallest_pairs(ixp, dev, n, dtype):
    for n_verts, zs in ((1, 0.0), (7, 0.0), (max(1, n // 8), 0.0), (max(1, n // 8), 1.1), (4 * n + 1, 0.0)):
        es, is_ = synth.graph_slots(n, n_verts, 500 + n, dtype, zipf_s=zs)
        if n >= 3:
            es[1] = -1  # outside [0, n_verts): no bin, dropped
            es[2] = n_verts
        for n_es in (n, n // 2, 3 * n + 7):
            oe, oi = oracle.smallest_pairs(n_verts, n_es, es, is_)
            ge, gi, cnt = ixp.smallest_pairs(T(es, dev), T(is_, dev), n_verts, n_es)
            c = int(cnt.item())
            assert c == oe.shape[0], (n_verts, zs, n_es)
            assert np.array_equal(ge[:c].cpu().numpy(), oe) and np.array_equal(gi[:c].cpu().numpy(), oi)
            # the paper's postcondition: both outputs are injective
            assert ixp.check_inj(ge[:c]).get()["ok"] == 1 and ixp.check_inj(gi[:c]).get()["ok"] == 1


def test_smallest_pairs_int32_neutral_outside_int32(ixp, dev):
    es, is_ = synth.graph_slots(5000, 300, 9, np.int32)
    is_[7] = np.iinfo(np.int32).max
    es[7] = 299
    for n_es in (2**40, -(2**40), np.iinfo(np.int32).max, np.iinfo(np.int32).min):
        oe, oi = oracle.smallest_pairs(300, n_es, es, is_)
        ge, gi, cnt = ixp.smallest_pairs(T(es, dev), T(is_, dev), 300, n_es)
        c = int(cnt.item())
        assert c == oe.shape[0] and np.array_equal(ge[:c].cpu().numpy(), oe) and \
            np.array_equal(gi[:c].cpu().numpy(), oi), n_es


@pytest.mark.parametrize("n", [1, 4095, 4096, 100003, 1 << 20])
def test_partition_without_indices(ixp, dev, n):
    """partition2 with the index array left out: the keys (and payload) still land
    at the oracle's destinations."""
    x = synth.floats_unit(n, 40 + n)
    bits = x.view(np.int32)  # non-negative floats order like their bit patterns
    thr = int(np.float32(0.5).view(np.int32))
    pred = ("lt", 0, thr)
    o = oracle.partition(bits, pred)
    pay = synth.payload_f32(n, 41 + n)
    o2 = oracle.partition(bits, pred, payload=pay, want_keys=False)
    r = ixp.partition(T(bits, dev), pred, want_indices=False)
    assert r["indices"] is None
    assert np.array_equal(r["keys_out"].cpu().numpy(), o["keys_out"])
    assert int(r["num_true"][0].item()) == int(o["num_true"][0]) == int((x < 0.5).sum())
    r2 = ixp.partition(T(bits, dev), pred, payload=T(pay, dev), want_keys=False, want_indices=False)
    assert np.array_equal(r2["payload_out"].cpu().numpy().view(np.uint32), o2["payload_out"].view(np.uint32))


@pytest.mark.parametrize("n", [1, 2047, 2048, 2049, 100003])
def test_smallest_pairs_int64_priorities_outside_32_bits(ixp, dev, n):
    """int64 priorities reduce in a 32-bit H while they lie in [0, 2^32 - 2]; any
    other priority of an in-range slot, or a negative neutral element, takes the
    64-bit H. Every case against the oracle."""
    es, is_ = synth.graph_slots(n, max(1, n // 6), 900 + n, np.int64)
    cases = {
        "fits": (is_, n),
        "fits_big_neutral": (is_, 2**40),
        "shifted": (is_ + 2**33, 2**33 + n),
        "one_at_2^32-1": (np.where(np.arange(n) == n // 2, 2**32 - 1, is_), 2**32),
        "negative": (is_ - n // 2, n),
        "negative_neutral": (is_, -5),
        "neutral_inside": (is_, n // 3),
    }
    for name, (pr, n_es) in cases.items():
        pr = np.ascontiguousarray(pr, dtype=np.int64)
        oe, oi = oracle.smallest_pairs(max(1, n // 6), n_es, es, pr)
        ge, gi, cnt = ixp.smallest_pairs(T(es, dev), T(pr, dev), max(1, n // 6), n_es)
        c = int(cnt.item())
        assert c == oe.shape[0], name
        assert np.array_equal(ge[:c].cpu().numpy(), oe) and np.array_equal(gi[:c].cpu().numpy(), oi), name
