"""CSR-shaped batch (power-law row lengths, sorted unique columns per row): row
offsets by exclusive scan + Mono check, segmented Inj and strict Mono on the
columns, a partition of the rows by a predicate on their length, the rows' columns
and values moved to the new row order (segment gather) and the values' gradient
through that move, each step against the oracle."""
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


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def same(g, o, what=""):
    g = g.get()
    assert g["status"] == 0, (what, g)
    assert bool(g["ok"]) == o["ok"], (what, g, o)
    for f in ("kind", "index", "value", "aux0", "aux1"):
        assert g[f] == o[f], (what, f, g, o)


def csr(m, seed, max_len, ncols, planted=0.01):
    L = synth.shapes_pareto(m, seed, max_len=max_len)
    cols = synth.sorted_unique_columns(L, ncols, seed + 1)
    off = synth.offsets_from_shape(L)
    rng = np.random.default_rng(seed + 2)
    rows = np.flatnonzero(L >= 2)
    for k in rng.choice(rows, size=min(rows.shape[0], max(1, int(planted * m))), replace=False):
        p = int(off[k]) + int(rng.integers(1, int(L[k])))
        if rng.random() < 0.5:
            cols[p] = cols[p - 1]  # duplicate
        else:
            cols[p - 1], cols[p] = cols[p], cols[p - 1]  # order swap
    vals = synth.payload_f32(int(off[-1]), seed + 3)
    return L.astype(np.int32), cols, vals


def moved_rows_reference(src, off, seg_src, new_off):
    """The row move as a plain gather: idx[j] = off[seg_src[II[j]]] + j - new_off[II[j]]."""
    new_len = np.diff(new_off)
    ii = oracle.mkii(new_len)
    j = np.arange(int(new_off[-1]), dtype=np.int64)
    idx = off[seg_src[ii]] + j - new_off[ii]
    return oracle.gather(src, idx)[0]


@pytest.mark.parametrize("m,max_len", [(1, 8), (37, 16), (4096, 1024), (20000, 65536)])
def test_csr_pipeline_matches_oracle(ixp, dev, m, max_len):
    L, cols, vals = csr(m, 100 + m, max_len, 1 << 20)
    Ld, cd, vd = T(L, dev), T(cols, dev), T(vals, dev)
    # offsets by exclusive scan (int32 lengths -> int64 offsets), total as the last offset
    off_d = torch.empty(m + 1, dtype=torch.int64, device=dev)
    ixp.scan(Ld, out=off_d[:m], totals=off_d[m:])
    o_off, o_tot = oracle.scan(L, out_dtype=np.int64)
    off = np.concatenate([o_off, o_tot[:1]])
    assert np.array_equal(off_d.cpu().numpy(), off)
    same(ixp.check_mono(off_d, "le"), oracle.check_mono(off, "le"), "offsets")
    # segmented checks on the columns
    same(ixp.check_inj_seg(cd, off_d), oracle.check_inj(cols, offsets=off), "seg inj")
    same(ixp.check_mono(cd, "lt", off_d), oracle.check_mono(cols, "lt", off), "seg mono")
    # rows partitioned by length (short rows first), then moved
    p = ("lt", 0, 16)
    r = ixp.partition(Ld, p, want_keys=False)
    o = oracle.partition(L, p, want_keys=False)
    assert np.array_equal(r["indices"].cpu().numpy(), o["indices"])
    src_row = ixp.invert(r["indices"], m)
    o_src = np.empty(m, np.int32)
    o_src[o["indices"]] = np.arange(m, dtype=np.int32)
    assert np.array_equal(src_row.cpu().numpy(), o_src)
    new_len, st = ixp.gather(Ld, src_row)
    assert st.item() == 0 and np.array_equal(new_len.cpu().numpy(), L[o_src])
    new_off = torch.empty(m + 1, dtype=torch.int64, device=dev)
    ixp.scan(new_len, out=new_off[:m], totals=new_off[m:])
    o_new_off = synth.offsets_from_shape(L[o_src].astype(np.int64))
    assert np.array_equal(new_off.cpu().numpy(), o_new_off)
    nnz = int(off[-1])
    for src_h, src_d in ((cols, cd), (vals, vd)):
        out, st = ixp.gather_segments(src_d, off_d, src_row, new_off, nnz)
        assert st.item() == 0
        ref = moved_rows_reference(src_h, off, o_src, o_new_off)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    # gradient of the values through the move: the move back (the inverse row map)
    x = vd.clone().requires_grad_(True)
    y = ixp.autograd.gather_segments(x, off_d, src_row, new_off, r["indices"])
    g = synth.payload_f32(nnz, 7 + m)
    y.backward(T(g, dev))
    ref = moved_rows_reference(g, o_new_off, o["indices"], off)
    assert np.array_equal(x.grad.cpu().numpy(), ref)


def test_gather_segments_with_empty_segments_and_bad_map(ixp, dev):
    shape = np.array([0, 3, 0, 0, 5, 1, 0, 4097, 2, 0], np.int64)
    off = synth.offsets_from_shape(shape)
    src = synth.payload_f32(int(off[-1]), 3)
    perm = synth.permutation(shape.shape[0], 4).astype(np.int64)
    new_shape = shape[perm]
    new_off = synth.offsets_from_shape(new_shape)
    out, st = ixp.gather_segments(T(src, dev), T(off, dev), T(perm, dev), T(new_off, dev), int(off[-1]))
    assert st.item() == 0
    assert np.array_equal(out.cpu().numpy(), moved_rows_reference(src, off, perm, new_off))
    bad = perm.copy()
    bad[np.flatnonzero(new_shape == 5)[0]] = np.flatnonzero(shape == 4097)[0]  # lengths differ
    out, st = ixp.gather_segments(T(src, dev), T(off, dev), T(bad, dev), T(new_off, dev), int(off[-1]))
    assert st.item() == -1


def test_csr_full_size_properties(ixp, dev):
    """2^24 rows (Pareto lengths up to 2^16, about 2^28 nonzeros): checked against
    the planted rows, by invariants, and on sampled rows."""
    m, ncols = 1 << 24, 1 << 24
    L = synth.t_shapes_pareto(m, 500, dev)
    off = torch.zeros(m + 1, dtype=torch.int64, device=dev)
    torch.cumsum(L, 0, out=off[1:])
    cols = synth.t_stratified_columns(L, off, ncols, 501)
    cols, planted = synth.t_plant_rows(cols, off, L, 502)
    L32 = L.to(torch.int32)
    del L
    off_d = torch.empty(m + 1, dtype=torch.int64, device=dev)
    ixp.scan(L32, out=off_d[:m], totals=off_d[m:])
    assert torch.equal(off_d, off)
    assert ixp.check_mono(off_d, "le").get()["ok"] == 1
    vi = ixp.check_inj_seg(cols, off_d).get()
    vm = ixp.check_mono(cols, "lt", off_d).get()
    # a planted duplicate breaks Inj and strict Mono, a planted swap only strict Mono; every
    # other row is strictly increasing, so strict Mono fails first in the first planted row
    offh = off.cpu().numpy()
    assert vm["ok"] == 0 and offh[planted[0]] < vm["index"] < offh[planted[0] + 1]
    assert vi["ok"] == 0
    assert int(np.searchsorted(offh, vi["index"], side="right") - 1) in set(planted.tolist())
    r = ixp.partition(L32, ("lt", 0, 16), want_keys=False)
    idx = r["indices"]
    assert ixp.check_bij(idx, I64MIN, I64MAX, 0, m - 1).get()["ok"] == 1
    src_row = ixp.invert(idx, m)
    new_len, _ = ixp.gather(L32, src_row)
    new_off = torch.empty(m + 1, dtype=torch.int64, device=dev)
    ixp.scan(new_len, out=new_off[:m], totals=new_off[m:])
    nnz = int(off[-1].item())
    moved, st = ixp.gather_segments(cols, off_d, src_row, new_off, nnz)
    assert st.item() == 0
    nt = int(r["num_true"][0].item())
    nl = new_len.cpu().numpy()
    assert np.all(nl[:nt] < 16) and np.all(nl[nt:] >= 16)
    rng = np.random.default_rng(503)
    srch, newh, colh, movh = (src_row.cpu().numpy(), new_off.cpu().numpy(), cols.cpu().numpy(),
                              moved.cpu().numpy())
    for k in rng.choice(m, size=2000, replace=False):
        s = srch[k]
        assert np.array_equal(movh[newh[k]:newh[k + 1]], colh[offh[s]:offh[s + 1]])
