"""Backward of scatter / gather / partition (forward and backward run the library's
kernels): CPU float64 reference gradients from the oracle (relative 1e-6) and
float64 finite differences via torch.autograd.gradcheck (relative 1e-4)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    import paper_2506_23058_gb300 as m
    m.load()
    return m.autograd


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


def T(a, dev, grad=False):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return t.requires_grad_(grad)


def close_to_sum(got, ref, absum, rel=1e-6):
    """|got - ref| <= rel * max(|ref|, sum of |terms|) elementwise."""
    bound = rel * np.maximum(np.abs(ref), absum) + 1e-30
    return np.all(np.abs(got.astype(np.float64) - ref) <= bound)


def test_gather_injective_backward_is_an_exact_scatter(ag, dev):
    n, cols = 50_003, 8
    src = synth.payload_f32(n, 1, cols=cols)
    idx = synth.permutation(n, 2).astype(np.int32)
    w = synth.payload_f32(n, 3, cols=cols)
    s = T(src, dev, True)
    y = ag.gather(s, T(idx, dev), injective=True)
    assert np.array_equal(y.detach().cpu().numpy(), oracle.gather(src, idx)[0])
    (y * T(w, dev)).sum().backward()
    ref = oracle.scatter(np.zeros_like(src), idx, w)  # each target receives exactly one row
    assert np.array_equal(s.grad.cpu().numpy(), ref)


def test_gather_backward_through_the_inverse(ag, dev):
    import paper_2506_23058_gb300 as m
    n, cols, ns = 40_000, 8, 50_000
    src = synth.payload_f32(ns, 31, cols=cols)
    idx = synth.permutation(ns, 32).astype(np.int32)[:n]  # injective, leaves 10000 rows untouched
    w = synth.payload_f32(n, 33, cols=cols)
    inv = m.invert(T(idx, dev), ns)
    ref_inv = np.full(ns, -1, np.int32)
    ref_inv[idx] = np.arange(n, dtype=np.int32)
    assert np.array_equal(inv.cpu().numpy(), ref_inv)
    s = T(src, dev, True)
    y = ag.gather(s, T(idx, dev), inverse=inv)
    (y * T(w, dev)).sum().backward()
    assert np.array_equal(s.grad.cpu().numpy(), oracle.scatter(np.zeros_like(src), idx, w))


@pytest.mark.parametrize("how", ["injective", "inverse"])
def test_gather_claimed_injective_with_duplicates_keeps_every_term(ag, dev, how):
    # idx repeats values although the caller asks for the atomic-free adjoint: the
    # forward pass's Inj check fails, so the backward sums every term per target
    import paper_2506_23058_gb300 as m
    n, cols = 30_011, 8
    idx = synth.permutation(n, 61).astype(np.int32)
    idx[100:400] = idx[5]  # 300 more reads of one row
    idx[7] = idx[9000]
    src = synth.payload_f32(n, 62, cols=cols)
    w = synth.payload_f32(n, 63, cols=cols)
    s = T(src, dev, True)
    ti = T(idx, dev)
    kw = {"injective": True} if how == "injective" else {"inverse": m.invert(ti, n)}
    y = ag.gather(s, ti, **kw)
    (y * T(w, dev)).sum().backward()
    ref = oracle.scatter_add_f64(n, idx, w)
    absum = oracle.scatter_add_f64(n, idx, np.abs(w))
    assert close_to_sum(s.grad.cpu().numpy(), ref, absum)


def test_gather_with_a_failed_proof_keeps_every_term(ag, dev):
    import paper_2506_23058_gb300 as m
    n, cols = 4099, 4
    idx = (np.arange(n) // 2).astype(np.int64)  # every row read twice
    src = synth.payload_f32(n, 64, cols=cols)
    w = synth.payload_f32(n, 65, cols=cols)
    ti = T(idx, dev)
    proof = m.check_inj(ti, 0, n - 1)
    assert proof.get()["ok"] == 0
    s = T(src, dev, True)
    (ag.gather(s, ti, injective=True, proof=proof) * T(w, dev)).sum().backward()
    ref = oracle.scatter_add_f64(n, idx, w)
    assert close_to_sum(s.grad.cpu().numpy(), ref, oracle.scatter_add_f64(n, idx, np.abs(w)))


@pytest.mark.parametrize("it", [np.int32, np.int64])
def test_gather_zipf_backward_matches_fp64_reference(ag, dev, it):
    n, m, cols = 200_000, 4096, 8
    idx = synth.zipf_ranks(n, m, 1.1, 5).astype(it)
    src = synth.payload_f32(m, 6, cols=cols)
    w = synth.payload_f32(n, 7, cols=cols)
    s = T(src, dev, True)
    y = ag.gather(s, T(idx, dev))
    (y * T(w, dev)).sum().backward()
    ref = oracle.scatter_add_f64(m, idx, w)
    absum = oracle.scatter_add_f64(m, idx, np.abs(w))
    assert close_to_sum(s.grad.cpu().numpy(), ref, absum)


def test_scatter_add_forward_and_backward(ag, dev):
    n, m, cols = 300_000, 1 << 14, 8
    idx = synth.zipf_ranks(n, m, 1.1, 9).astype(np.int64)
    idx[::97] = m + 5  # out of bounds: ignored
    vals = synth.payload_f32(n, 10, cols=cols)
    dst = synth.payload_f32(m, 11, cols=cols)
    v = T(vals, dev, True)
    d = T(dst, dev, True)
    out = ag.scatter_add(d, T(idx, dev), v)
    ref = oracle.scatter_add_f64(m, idx, vals, init=dst.astype(np.float64))
    absum = oracle.scatter_add_f64(m, idx, np.abs(vals), init=np.abs(dst).astype(np.float64))
    assert close_to_sum(out.detach().cpu().numpy(), ref, absum)
    g = synth.payload_f32(m, 12, cols=cols)
    out.backward(T(g, dev))
    gv, _ = oracle.gather(g, np.where(idx < m, idx, 0))
    gv[idx >= m] = 0
    assert np.array_equal(v.grad.cpu().numpy(), gv)
    assert np.array_equal(d.grad.cpu().numpy(), g)


def test_scatter_assign_forward_and_backward(ag, dev):
    n, m, cols = 40_000, 30_000, 8
    idx = (synth.permutation(n, 13) - 3000).astype(np.int32)  # injective, some out of bounds
    vals = synth.payload_f32(n, 14, cols=cols)
    dst = synth.payload_f32(m, 15, cols=cols)
    v = T(vals, dev, True)
    d = T(dst, dev, True)
    out = ag.scatter(d, T(idx, dev), v)
    assert np.array_equal(out.detach().cpu().numpy(), oracle.scatter(dst, idx, vals))
    g = synth.payload_f32(m, 16, cols=cols)
    out.backward(T(g, dev))
    inb = (idx >= 0) & (idx < m)
    gv = np.zeros_like(vals)
    gv[inb] = g[idx[inb]]
    gd = g.copy()
    gd[idx[inb]] = 0
    assert np.array_equal(v.grad.cpu().numpy(), gv)
    assert np.array_equal(d.grad.cpu().numpy(), gd)


@pytest.mark.parametrize("seg", [False, True])
def test_partition_backward_is_a_gather(ag, dev, seg):
    cols = 4
    off = synth.offsets_from_shape(synth.shapes_with_empties(300, 19, 400)) if seg else None
    n = int(off[-1]) if seg else 70_001
    keys = synth.keys_uniform(n, 17)
    pay = synth.payload_f32(n, 18, cols=cols)
    p = ("lt", 0, synth.bernoulli_threshold(0.3))
    x = T(pay, dev, True)
    y, ind, nt = ag.partition(x, T(keys, dev), p, None if off is None else T(off, dev))
    o = oracle.partition(keys, p, payload=pay, offsets=off)
    assert np.array_equal(ind.cpu().numpy(), o["indices"])
    assert np.array_equal(y.detach().cpu().numpy(), o["payload_out"])
    g = synth.payload_f32(n, 20, cols=cols)
    y.backward(T(g, dev))
    assert np.array_equal(x.grad.cpu().numpy(), oracle.gather(g, o["indices"])[0])


def test_finite_differences_fp64(ag, dev):
    rng = np.random.default_rng(21)
    kw = dict(eps=1e-6, atol=1e-8, rtol=1e-4, nondet_tol=1e-12)
    src = T(rng.standard_normal((37, 3)), dev, True)
    idx_inj = T(rng.permutation(37)[:29].astype(np.int64), dev)
    idx_rep = T(rng.integers(0, 37, size=53).astype(np.int64), dev)
    assert torch.autograd.gradcheck(lambda s: ag.gather(s, idx_inj, injective=True), (src,), **kw)
    assert torch.autograd.gradcheck(lambda s: ag.gather(s, idx_rep), (src,), **kw)
    import paper_2506_23058_gb300 as m
    inv = m.invert(idx_inj, 37)
    assert torch.autograd.gradcheck(lambda s: ag.gather(s, idx_inj, inverse=inv), (src,), **kw)
    vals = T(rng.standard_normal((53, 3)), dev, True)
    assert torch.autograd.gradcheck(lambda d, v: ag.scatter_add(d, idx_rep, v), (src, vals), **kw)
    sidx = T((rng.permutation(45) - 4).astype(np.int64), dev)  # injective, some out of bounds
    v45 = T(rng.standard_normal((45, 3)), dev, True)
    assert torch.autograd.gradcheck(lambda d, v: ag.scatter(d, sidx, v), (src, v45), **kw)
    keys = T(rng.integers(-50, 50, size=37).astype(np.int32), dev)
    assert torch.autograd.gradcheck(lambda p: ag.partition(p, keys, ("mod_eq", 3, 0))[0], (src,), **kw)
