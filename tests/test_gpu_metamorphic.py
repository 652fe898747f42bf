"""Property algebra the paper states, checked on the GPU path (Sec. 3 rules and
the invariants of Sec. 2.3): strict Mono implies Inj (rule InjF1); Bij is Range
and Inj and the in-image count (rule BijF1); a filter keeps Mono and Inj; a
partition's index array is Bij onto [0, n) and InvFiltPart; a scan of a
non-negative array is Mono, and a monotone array is its first value plus the scan
of its differences. Also the adjoint identity <J v, w> = <v, J^T w> of the
gather / scatter-add pair at full size."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I64MIN, I64MAX = -(2**63), 2**63 - 1


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


@pytest.mark.parametrize("n", [2, 4097, 300001])
def test_strict_mono_implies_inj(ixp, dev, n):
    rng = np.random.default_rng(n)
    for dt in (np.int32, np.int64):
        x = np.cumsum(rng.integers(1, 5, size=n)).astype(dt) - 7  # strictly increasing
        assert ixp.check_mono(T(x, dev), "lt").get()["ok"] == 1
        assert ixp.check_inj(T(x, dev), I64MIN, I64MAX).get()["ok"] == 1
        y = x.copy()
        y[n // 2] = y[n // 2 - 1]  # a repeat breaks both
        assert ixp.check_mono(T(y, dev), "lt").get()["ok"] == 0
        assert ixp.check_inj(T(y, dev), I64MIN, I64MAX).get()["ok"] == 0


@pytest.mark.parametrize("n", [1000, 65536, 300001])
def test_bij_is_range_inj_and_count(ixp, dev, n):
    rng = np.random.default_rng(n + 1)
    lo, hi = 100, 100 + n - 1
    perm = synth.permutation(n, n + 2, np.int64) + lo
    cases = [perm]
    for kind in range(6):
        x = perm.copy()
        p = int(rng.integers(0, n))
        if kind == 0:
            x[p] = x[(p + 1) % n]  # duplicate (and so a missing value)
        elif kind == 1:
            x[p] = hi + 5  # outside the image, inside Rcd
        elif kind == 2:
            x[p] = lo - 3
        elif kind == 3:
            x = x[: n - 1].copy()  # one value missing
        elif kind == 4:
            x = np.concatenate([x, [hi + 10]])  # an extra value outside the image
        else:
            x[p] = I64MIN  # outside Rcd as well
        cases.append(x)
    rlo, rhi = lo - 50, hi + 50
    for x in cases:
        xd = T(x, dev)
        bij = ixp.check_bij(xd, rlo, rhi, lo, hi).get()["ok"] == 1
        in_rcd = (x >= rlo) & (x <= rhi)
        rng_ok = ixp.check_range(T(x[in_rcd], dev), lo, hi).get()["ok"] == 1  # Rcd values lie in Img
        inj_ok = ixp.check_inj(xd, rlo, rhi).get()["ok"] == 1
        count_ok = int(((x >= lo) & (x <= hi)).sum()) == hi - lo + 1
        assert bij == (rng_ok and inj_ok and count_ok), (bij, rng_ok, inj_ok, count_ok)


@pytest.mark.parametrize("n", [4097, 200003])
def test_filter_keeps_mono_and_inj(ixp, dev, n):
    mono = synth.monotone(n, n + 3, np.int32)
    perm = synth.permutation(n, n + 4, np.int32)
    flags = synth.flags_bernoulli(n, n + 5, 0.4)
    fl = T(flags, dev)
    for x, check in ((mono, lambda y: ixp.check_mono(y, "le")), (perm, lambda y: ixp.check_inj(y))):
        r = ixp.partition(T(x, dev), ("flags", 0, 0, fl))
        k = int(r["num_true"][0].item())
        kept = r["keys_out"][:k]
        assert torch.equal(kept.cpu(), torch.from_numpy(x[flags.astype(bool)]))  # the filter, in order
        assert check(kept).get()["ok"] == 1
        # the partition's index array is Bij onto [0, n) and satisfies InvFiltPart
        assert ixp.check_bij(r["indices"], I64MIN, I64MAX, 0, n - 1).get()["ok"] == 1
        assert ixp.check_filtpart(r["indices"], part=("flags", 0, 0, fl)).get()["ok"] == 1


@pytest.mark.parametrize("n", [1, 4097, 300001])
def test_scan_and_monotone_arrays(ixp, dev, n):
    rng = np.random.default_rng(n + 6)
    d = rng.integers(0, 1000, size=n).astype(np.int32)
    out, tot, st = ixp.scan(T(d, dev), out_dtype=torch.int64)
    assert st.item() == 0 and ixp.check_mono(out, "le").get()["ok"] == 1  # scan of non-negatives is Mono
    x = synth.monotone(n, n + 7, np.int64) + 12345
    diff = np.diff(x, prepend=x[:1])  # x[i] - x[i-1], 0 first: non-negative
    s, _, _ = ixp.scan(T(diff, dev), inclusive=True)
    assert torch.equal(s + int(x[0]), T(x, dev))  # lb plus a prefix sum of a non-negative array


def test_gather_scatter_add_adjoint_full_size(ixp, dev):
    """J v = gather(v, idx) (Zipf indices, many repeats), J^T w = scatter-add of w by
    idx: <J v, w> equals <v, J^T w> in float64 up to rounding."""
    nr, m = 1 << 26, 1 << 20
    idx = torch.from_numpy(synth.zipf_ranks(nr, m, 1.1, synth.seed_for(4) + 7)).to(dev)
    v = synth.t_payload_f32(m, synth.seed_for(4) + 8, dev, cols=8)
    w = synth.t_payload_f32(nr, synth.seed_for(4) + 9, dev, cols=8)
    jv, st = ixp.gather(v, idx)
    assert st.item() == 0
    acc = torch.zeros((m, 8), dtype=torch.float64, device=dev)
    ixp.scatter_add_f64(acc, idx, w)
    lhs = torch.sum(jv.double() * w.double()).item()
    rhs = torch.sum(v.double() * acc).item()
    scale = torch.sum(jv.double().abs() * w.double().abs()).item()
    assert abs(lhs - rhs) <= 1e-9 * scale
