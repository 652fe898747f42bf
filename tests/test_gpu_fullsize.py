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


def test_inj_any_span_full_size(ixp, dev):
    """Inj of 2^27 int64 ids spread over [0, 2^62) (distinct by construction: a
    permutation in the high bits), decided by the hash set: it holds, and a planted
    repeat is reported as the pair (min, max) of its positions."""
    n = 1 << 27
    s = synth.seed_for(1) + 130
    perm = synth.t_permutation(n, s, dev, torch.int64)
    g = torch.Generator(device=dev)
    g.manual_seed(s + 1)
    low = torch.randint(0, 1 << 35, (n,), generator=g, device=dev, dtype=torch.int64)
    ids = (perm << 35) | low
    del perm, low
    v = ixp.check_inj(ids).get()
    assert v["status"] == 0 and v["ok"] == 1
    dup, p, q = synth.t_plant_duplicate(ids, s + 2)
    v = ixp.check_inj(dup).get()
    assert v["status"] == 0 and v["ok"] == 0
    assert v["index"] == min(p, q) and v["aux0"] == max(p, q) and v["value"] == int(dup[min(p, q)].item())


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


def test_segmented_blocks_full_size(ixp, dev):
    """sgmSum under uint8 flags, the offsets form of the segmented scan (with its
    per-segment totals) and mkII over the 4096-segment log-uniform shape that
    bench.py times (2^28 int32 values in [0, 4)), whole arrays against the oracle."""
    s = synth.seed_for(1)
    shape = synth.shapes_log_uniform(4096, s + 11, cap_total=1 << 28)
    off = synth.offsets_from_shape(shape)
    total = int(off[-1])
    g = torch.Generator(device=dev)
    g.manual_seed(s + 6)
    x = torch.randint(0, 4, (total,), generator=g, device=dev, dtype=torch.int32)
    fl = np.zeros(total, np.uint8)
    fl[off[:-1][shape > 0]] = 1
    xo = x.cpu().numpy()
    ref_inc = oracle.sgm_scan(fl, xo)
    got, st = ixp.sgm_scan(torch.from_numpy(fl).to(dev), x, inclusive=True)
    assert st.item() == 0 and np.array_equal(got.cpu().numpy(), ref_inc)
    got, st = ixp.sgm_scan(torch.from_numpy(fl).to(dev), x, inclusive=False)
    assert st.item() == 0 and np.array_equal(got.cpu().numpy(), ref_inc - xo)
    del got
    ref, rtot = oracle.scan(xo, inclusive=True, offsets=off)
    assert np.array_equal(ref, ref_inc)  # the two forms of the same segmentation agree
    got, tot, st = ixp.scan(x, inclusive=True, offsets=torch.from_numpy(off).to(dev))
    assert st.item() == 0 and np.array_equal(got.cpu().numpy(), ref) and np.array_equal(tot.cpu().numpy(), rtot)
    del got, x
    ii, st = ixp.mkii(torch.from_numpy(off).to(dev), total)
    assert st.item() == 0 and np.array_equal(ii.cpu().numpy(), oracle.mkii(shape).astype(np.int32))


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
    del before
    # the whole index array against the oracle (about a second of oracle time)
    o = oracle.partition(kh, pred, want_keys=False)
    assert o["num_true"][0] == T and np.array_equal(ih, o["indices"].astype(ih.dtype))
    del o
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


def test_batched_full_size(ixp, dev):
    """The batched workload at full size (4096 log-uniform segments, 2^28 elements)
    from the graph-captured persistent launch: flags and offsets against the oracle's
    mkSgmDescr, per-segment verdicts against the planted segments, num_true and
    sampled partition destinations against the definition."""
    from paper_2506_23058_gb300 import batched
    s = synth.seed_for(3) + 200
    m = 4096
    shape = synth.shapes_log_uniform(m, s, max_log2=20, cap_total=1 << 28)
    n = int(shape.sum())
    off = synth.offsets_from_shape(shape)
    sh = torch.from_numpy(shape).to(dev)
    seg = torch.repeat_interleave(torch.arange(m, device=dev, dtype=torch.int64), sh)
    g = torch.Generator(device=dev)
    g.manual_seed(s + 1)
    r = torch.randint(0, 2**31, (n,), generator=g, device=dev, dtype=torch.int64)
    chk = torch.argsort(seg * (2**31) + r).to(torch.int32)  # a permutation of each segment's range
    offd = torch.from_numpy(off).to(dev)
    iota = (torch.arange(n, device=dev, dtype=torch.int64) - offd[seg]).to(torch.int32)
    del r, seg
    rng = np.random.default_rng(s + 2)
    planted = np.sort(rng.choice(np.flatnonzero(shape >= 3), size=41, replace=False))
    mono_bad, inj_bad = [], []
    for k in planted:
        i = int(off[k]) + int(rng.integers(1, int(shape[k])))
        if k % 2:
            chk[i] = chk[i - 1]
            inj_bad.append(int(k))
        else:
            iota[i] = iota[i - 1]
            mono_bad.append(int(k))
    keys = synth.t_keys_uniform(n, s + 3, dev)
    thr = synth.bernoulli_threshold(0.3)
    br = batched.BatchRunner(shape, keys, ("lt", 0, thr), chk, iota)
    br.capture()
    br.replay()
    torch.cuda.synchronize()
    res = br.results()
    assert res["status"] == 0
    o_flags, o_off = oracle.flags_from_shape(shape, None, out_dtype=np.int32)
    assert np.array_equal(res["offsets"].cpu().numpy(), o_off)
    assert np.array_equal(res["flags"].cpu().numpy(), o_flags)
    exp_mono = np.ones(m, np.uint8)
    exp_mono[mono_bad] = 0
    exp_inj = np.ones(m, np.uint8)
    exp_inj[inj_bad] = 0
    assert np.array_equal(res["mono_ok"], exp_mono)
    assert np.array_equal(res["inj_ok"], exp_inj)
    assert np.array_equal(res["bij_ok"], exp_inj)  # a repeat inside the segment's own range breaks Bij too
    assert res["first_bad"] == [mono_bad[0], inj_bad[0], inj_bad[0]]
    kh = keys.cpu().numpy()
    c = kh < thr
    segh = np.repeat(np.arange(m), shape)
    T = np.bincount(segh, weights=c, minlength=m).astype(np.int64)
    assert np.array_equal(res["num_true"].cpu().numpy(), T)
    cs = np.cumsum(c, dtype=np.int64) - c  # trues before i overall
    smp = np.sort(rng.choice(n, size=4096, replace=False))
    k = segh[smp]
    tb = cs[smp] - cs[off[k]]  # trues before i in its segment
    exp = np.where(c[smp], off[k] + tb, off[k] + T[k] + (smp - off[k]) - tb)
    assert np.array_equal(res["indices"].cpu().numpy()[smp].astype(np.int64), exp)


def test_differentiation_full_size(ixp, dev):
    """Config 4 at full size: the injective gather's gradient (through the inverse
    index) equals the scatter of the output gradient; the Zipf(1.1) scatter-add over
    2^20 targets against the oracle's float64 sums (relative 1e-6 of the sum of
    magnitudes), on all targets."""
    from paper_2506_23058_gb300 import autograd
    nr, m = 1 << 26, 1 << 20
    perm = synth.t_permutation(nr, synth.seed_for(4) + 1, dev, torch.int32)
    src = synth.t_payload_f32(nr, synth.seed_for(4) + 2, dev, cols=8).requires_grad_(True)
    inv = ixp.invert(perm, nr)
    y = autograd.gather(src, perm, inverse=inv)
    gy = synth.t_payload_f32(nr, synth.seed_for(4) + 3, dev, cols=8)
    (gs,) = torch.autograd.grad(y, src, gy)
    ref = torch.zeros_like(gs)
    ixp.scatter(ref, perm, gy)
    assert torch.equal(gs, ref)
    zipf = synth.zipf_ranks(nr, m, 1.1, synth.seed_for(4) + 4)
    vals = synth.t_payload_f32(nr, synth.seed_for(4) + 5, dev, cols=8)
    dst = torch.zeros((m, 8), dtype=torch.float32, device=dev)
    out = autograd.scatter_add(dst, torch.from_numpy(zipf).to(dev), vals)
    vh = vals.cpu().numpy()
    r64 = oracle.scatter_add_f64(m, zipf, vh)
    a64 = oracle.scatter_add_f64(m, zipf, np.abs(vh))
    got = out.detach().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - r64) <= 1e-6 * np.maximum(np.abs(r64), a64) + 1e-30)


def test_dynamic_inj_check_full_size(ixp, dev):
    """The reduce-by-index Inj check on the 2^28 int32 permutation (a 1 GiB bin
    array): clean, and with a planted duplicate reported at its positions."""
    n = 1 << 28
    s = synth.seed_for(1) + 120
    perm = synth.t_permutation(n, s, dev, torch.int32)
    assert ixp.check_inj_hist(perm, n).get()["ok"] == 1
    dup, p, q = synth.t_plant_duplicate(perm, s + 1)
    del perm
    v = ixp.check_inj_hist(dup, n).get()
    assert v["ok"] == 0 and v["index"] == min(p, q) and v["aux0"] == max(p, q)


def test_partition2_three_ways_200m(ixp, dev):
    """partition2 of 200M float32 in [0, 1) by x < 0.5: the dynamic form (indices,
    reduce-by-index check, scatter) and the fused static form give the oracle's
    output bit for bit."""
    n = 200_000_000
    x = synth.t_floats_unit(n, synth.seed_for(7) + 200, dev)
    bits = x.view(torch.int32)
    pred = ("lt", 0, int(np.float32(0.5).view(np.int32)))
    r = ixp.partition(bits, pred, want_keys=False)
    assert ixp.check_inj_hist(r["indices"], n).get()["ok"] == 1
    ys = torch.zeros_like(x)
    ixp.scatter(ys, r["indices"], x)
    st = ixp.partition(bits, pred, want_indices=False)
    assert torch.equal(st["keys_out"], ys.view(torch.int32))
    o = oracle.partition(bits.cpu().numpy(), pred)
    assert int(st["num_true"][0].item()) == int(o["num_true"][0])
    assert np.array_equal(st["keys_out"].cpu().numpy(), o["keys_out"])


def test_smallest_pairs_full_size(ixp, dev):
    """get_smallest_pairs on 2^26 int64 slots over 2^23 vertices against the oracle
    on the whole arrays, and the postcondition (both outputs injective)."""
    n_verts, n = 1 << 23, 1 << 26
    es, is_ = synth.t_graph_slots(n, n_verts, synth.seed_for(8) + 1, dev, torch.int64)
    ge, gi, cnt = ixp.smallest_pairs(es, is_, n_verts, n)
    c = int(cnt.item())
    oe, oi = oracle.smallest_pairs(n_verts, n, es.cpu().numpy(), is_.cpu().numpy())
    assert c == oe.shape[0]
    assert np.array_equal(ge[:c].cpu().numpy(), oe) and np.array_equal(gi[:c].cpu().numpy(), oi)
    assert ixp.check_inj(ge[:c], 0, n_verts - 1).get()["ok"] == 1
    assert ixp.check_inj(gi[:c], 0, n - 1).get()["ok"] == 1
