"""Arrays of more than 2^31 elements (n = 2^31 + 3), where every element index
needs 64 bits: the checks, the scan, the partition (int64 destinations), a gather
and the reduce-by-index, each against positions planted at and beyond 2^31 and
against closed forms that hold at any size (torch's own int64 arithmetic on the
device serves as the reference for the sampled destinations)."""
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I64MIN, I64MAX = oracle.INT64_MIN, oracle.INT64_MAX
N = (1 << 31) + 3
BIG = (1 << 31) + 1  # a position past INT32_MAX


@pytest.fixture(scope="module")
def ixp():
    import paper_2506_23058_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


@pytest.fixture(autouse=True)
def _free_memory():
    yield
    torch.cuda.empty_cache()


def distinct_i32(n, dev):
    """x[i] = (i * 2654435761) mod 2^32 as int32: a bijection of 32-bit words, so
    the n < 2^32 values are distinct."""
    i = torch.arange(n, device=dev, dtype=torch.int64)
    x = (i * 2654435761) & 0xFFFFFFFF
    del i
    x = torch.where(x >= 2**31, x - 2**32, x)
    return x.to(torch.int32)


def test_range_and_mono_past_2_31(ixp, dev):
    x = torch.zeros(N, dtype=torch.int32, device=dev)
    assert ixp.check_range(x, 0, 0).get()["ok"] == 1
    x[BIG] = 7
    v = ixp.check_range(x, 0, 0).get()
    assert v["ok"] == 0 and v["index"] == BIG and v["value"] == 7
    assert v["aux0"] == 0 and v["aux1"] == 7
    x.zero_()
    x[BIG:] = 1  # nondecreasing, the step lies past 2^31
    assert ixp.check_mono(x, "le").get()["ok"] == 1
    x[BIG + 1] = 0
    v = ixp.check_mono(x, "le").get()
    assert v["ok"] == 0 and v["index"] == BIG + 1


def test_inj_past_2_31(ixp, dev):
    x = distinct_i32(N, dev)
    assert ixp.check_inj(x, I64MIN, I64MAX, span=1 << 32).get()["ok"] == 1
    x[BIG] = x[5]
    v = ixp.check_inj(x, I64MIN, I64MAX, span=1 << 32).get()
    assert v["ok"] == 0 and v["index"] == 5 and v["aux0"] == BIG


def test_scan_past_2_31(ixp, dev):
    x = torch.ones(N, dtype=torch.int32, device=dev)
    out = torch.empty(N, dtype=torch.int64, device=dev)
    _, tot, st = ixp.scan(x, out=out)
    assert st.item() == 0 and int(tot[0].item()) == N
    idx = torch.tensor([0, 1, (1 << 31) - 1, 1 << 31, BIG, N - 1], device=dev)
    assert torch.equal(out[idx], idx)


def test_segmented_scan_past_2_31(ixp, dev):
    # ones with segment heads at 0, 2^31 - 5 and 2^31 + 1: the inclusive value at i
    # is i - (last head <= i) + 1, in both forms of the segmentation
    heads = [0, (1 << 31) - 5, BIG]
    x = torch.ones(N, dtype=torch.int32, device=dev)
    out = torch.empty(N, dtype=torch.int64, device=dev)
    fl = torch.zeros(N, dtype=torch.uint8, device=dev)
    fl[torch.tensor(heads, device=dev)] = 1
    pos = [0, 1, (1 << 31) - 6, (1 << 31) - 5, (1 << 31) - 1, 1 << 31, BIG, BIG + 1, N - 1]
    want = torch.tensor([p - max(h for h in heads if h <= p) + 1 for p in pos], device=dev)
    idx = torch.tensor(pos, device=dev)
    _, st = ixp.sgm_scan(fl, x, out=out, inclusive=True)
    assert st.item() == 0 and torch.equal(out[idx], want)
    del fl
    off = torch.tensor(heads + [N], dtype=torch.int64, device=dev)
    out.fill_(-1)
    _, tot, st = ixp.scan(x, inclusive=True, offsets=off, out=out)
    assert st.item() == 0 and torch.equal(out[idx], want)
    assert tot.cpu().tolist() == [(1 << 31) - 5, 6, 2]


def test_partition_past_2_31(ixp, dev):
    x = distinct_i32(N, dev)
    thr = 0
    r = ixp.partition(x, ("lt", 0, thr), out_dtype=torch.int64, want_keys=False)
    assert r["status"].item() == 0
    c = x < thr
    T = int(c.sum().item())
    assert int(r["num_true"][0].item()) == T
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    smp = torch.cat([torch.randint(0, N, (4096,), generator=g, device=dev),
                     torch.tensor([BIG, N - 1], device=dev)])
    before = torch.cumsum(c.to(torch.int64), 0) - c.to(torch.int64)
    exp = torch.where(c[smp], before[smp], T + smp - before[smp])
    assert torch.equal(r["indices"][smp], exp)
    del before
    # the partition's index array is a bijection onto [0, n)
    assert ixp.check_bij(r["indices"], I64MIN, I64MAX, 0, N - 1).get()["ok"] == 1


def test_gather_and_hist_past_2_31(ixp, dev):
    src = torch.arange(1 << 20, dtype=torch.float32, device=dev)
    i = torch.arange(N, device=dev, dtype=torch.int64)
    idx = (i * 7) % (1 << 20)
    del i
    y, st = ixp.gather(src, idx)
    assert st.item() == 0
    smp = torch.tensor([0, 3, (1 << 31) - 1, BIG, N - 1], device=dev)
    assert torch.equal(y[smp], src[idx[smp]])
    del y
    # reduce-by-index of iota: bin k gets the first position whose index is k
    H = torch.full((1 << 20,), I64MAX, dtype=torch.int64, device=dev)
    ixp.hist_min(H, idx)
    assert torch.equal(H, torch.arange(1 << 20, device=dev, dtype=torch.int64).mul(
        pow(7, -1, 1 << 20)).remainder(1 << 20))


@pytest.mark.parametrize("n,zt", [((1 << 30) + 4097, torch.int32), (N, torch.int64)])
def test_classes_past_2_30(ixp, dev, n, zt):
    """The flat 3-class partition and its check past 2^30 elements, where the decide
    pass gives each thread several tiles: the index form against per-class prefix
    counts (torch cumsum) on sampled positions, the check accepting it, and planted
    faults reported at the first one (int32 destinations below 2^31, int64 ones
    past it)."""
    v = 3
    i = torch.arange(n, device=dev, dtype=torch.int64)
    cls = ((i * 2654435761) >> 9).remainder(5).to(torch.uint8)  # classes 3 and 4 fold into 2
    del i
    out, kept = ixp.filtpart_classes(cls, v, None, "true", out_dtype=zt)
    assert int(kept.item()) == n
    cc = torch.clamp(cls, max=v - 1)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    late = n - 5
    early = (1 << 29) + 3
    smp = torch.cat([torch.randint(0, n, (4096,), generator=g, device=dev),
                     torch.tensor([0, early, late, n - 1], device=dev)])
    exp = torch.zeros(smp.numel(), dtype=torch.int64, device=dev)
    base = 0
    for k in range(v):
        m = cc == k
        cs = torch.cumsum(m.to(torch.int64), 0)
        exp = torch.where(cc[smp] == k, base + cs[smp] - m[smp].to(torch.int64), exp)
        base += int(cs[-1].item())
        del cs, m
    del cc
    assert torch.equal(out[smp].to(torch.int64), exp)
    assert ixp.check_filtpart(out, None, cls=cls, v=v).get()["ok"] == 1
    want_late, want_early = int(out[late].item()), int(out[early].item())
    out[late] += 1
    r = ixp.check_filtpart(out, None, cls=cls, v=v).get()
    assert r["ok"] == 0 and r["index"] == late and r["aux1"] == want_late and r["aux0"] == n
    out[early] -= 1
    r = ixp.check_filtpart(out, None, cls=cls, v=v).get()
    assert r["ok"] == 0 and r["index"] == early and r["aux1"] == want_early
