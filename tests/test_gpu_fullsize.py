"""The large plain workload at full size (int32 n = 2^28, int64 n = 2^27, [2^26 x 8]
rows), in the launch configuration bench.py times: verdicts against the planted
violations (positions known by construction) and against the oracle on the whole
array where it finishes in seconds, outputs against properties that hold at any
size and against the oracle's values on sampled positions."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I64MIN, I64MAX = oracle.INT64_MIN, oracle.INT64_MAX


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


@pytest.mark.parametrize("tag,n,dt", [("i32", 1 << 28, torch.int32), ("i64", 1 << 27, torch.int64)])
def test_checks_full_size(ixp, dev, tag, n, dt):
    s = synth.seed_for(1) + 100
    perm = synth.t_permutation(n, s, dev, dt)
    dup, p, q = synth.t_plant_duplicate(perm, s + 1)
    oor, po = synth.t_plant_value(perm, s + 2, n)
    mono = synth.t_monotone(n, s + 3, dev, dt)
    brk, pb = synth.t_plant_order_break(mono, s + 4)
    # Range
    v = ixp.check_range(perm, 0, n - 1).get()
    assert v["ok"] == 1 and v["aux0"] == 0 and v["aux1"] == n - 1
    v = ixp.check_range(oor, 0, n - 1).get()
    assert v["ok"] == 0 and v["index"] == po and v["value"] == n
    # Mono
    assert ixp.check_mono(mono, "le").get()["ok"] == 1
    v = ixp.check_mono(brk, "le").get()
    assert v["ok"] == 0 and v["index"] == pb
    # Inj: the permutation holds; the planted pair (min, max) is the witness
    assert ixp.check_inj(perm, 0, n - 1).get()["ok"] == 1
    v = ixp.check_inj(dup, I64MIN, I64MAX, span=4 * n + 4096).get()
    assert v["ok"] == 0 and v["index"] == min(p, q) and v["aux0"] == max(p, q)
    # Bij onto [0, n): the duplicate pair is reported by its first index, as for Inj
    assert ixp.check_bij(perm, I64MIN, I64MAX, 0, n - 1).get()["ok"] == 1
    v = ixp.check_bij(dup, I64MIN, I64MAX, 0, n - 1).get()
    assert v["ok"] == 0 and v["index"] == min(p, q)
    # the oracle on the whole array agrees (single-threaded C, seconds)
    h = dup.cpu().numpy()
    o = oracle.check_bij(h, I64MIN, I64MAX, 0, n - 1)
    assert (o["kind"], o["index"], o["value"]) == (v["kind"], v["index"], v["value"])


def test_scan_full_size(ixp, dev):
    n = 1 << 28
    g = torch.Generator(device=dev)
    g.manual_seed(synth.seed_for(1) + 106)
    x = torch.randint(0, 4, (n,), generator=g, device=dev, dtype=torch.int32)
    out, tot, st = ixp.scan(x)
    assert st.item() == 0
    xo = x.cpu().numpy()
    ref, rtot = oracle.scan(xo)
    got = out.cpu().numpy()
    assert np.array_equal(got, ref) and int(tot[0].item()) == int(rtot[0])


@pytest.mark.parametrize("p", [0.5, 0.01])
def test_partition_full_size(ixp, dev, p):
    n = 1 << 28
    keys = synth.t_keys_uniform(n, synth.seed_for(1) + 107, dev)
    pay = synth.t_payload_f32(n, synth.seed_for(1) + 108, dev)
    pred = ("lt", 0, synth.bernoulli_threshold(p))
    r = ixp.partition(keys, pred, payload=pay, want_keys=False)
    idx = r["indices"]
    # a partition's index array is a bijection onto [0, n)
    assert ixp.check_bij(idx, I64MIN, I64MAX, 0, n - 1).get()["ok"] == 1
    kh = keys.cpu().numpy()
    c = kh < pred[2]
    T = int(c.sum())
    assert int(r["num_true"][0].item()) == T
    # sampled destinations against the definition (trues first, both sides stable)
    rng = np.random.default_rng(109)
    smp = np.sort(rng.choice(n, size=4096, replace=False))
    before = np.cumsum(c, dtype=np.int64) - c
    ih = idx.cpu().numpy()
    exp = np.where(c[smp], before[smp], T + smp - before[smp])
    assert np.array_equal(ih[smp].astype(np.int64), exp)
    # the payload lands at its destination
    ph, po = pay.cpu().numpy(), r["payload_out"].cpu().numpy()
    assert np.array_equal(po[exp], ph[smp])
    # InvFiltPart accepts the indices and rejects a swap of two of them
    assert ixp.check_filtpart(idx, keys, part=pred).get()["ok"] == 1
    a, b = int(smp[10]), int(smp[-10])
    bad = idx.clone()
    bad[a], bad[b] = idx[b], idx[a]
    v = ixp.check_filtpart(bad, keys, part=pred).get()
    assert v["ok"] == 0 and v["index"] == a and v["aux1"] == exp[10]


def test_scatter_gather_full_size(ixp, dev):
    nr = 1 << 26
    perm = synth.t_permutation(nr, synth.seed_for(1) + 110, dev, torch.int32)
    src = synth.t_payload_f32(nr, synth.seed_for(1) + 111, dev, cols=8)
    y, st = ixp.gather(src, perm)
    assert st.item() == 0
    back = torch.zeros_like(src)
    ixp.scatter(back, perm, y)
    assert torch.equal(back, src)  # scatter by a bijection undoes the gather
    rng = np.random.default_rng(112)
    smp = rng.choice(nr, size=4096, replace=False)
    ph, sh, yh = perm.cpu().numpy(), src.cpu().numpy(), y.cpu().numpy()
    assert np.array_equal(yh[smp], sh[ph[smp]])
