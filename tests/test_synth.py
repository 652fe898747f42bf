"""The seeded input generators (host side): each one has the structure its workload
recipe states, and the same seed gives the same draw. These are inputs, not
results: nothing here is the method's arithmetic."""
import numpy as np
import pytest

import synth


def test_seeded_draws_repeat_and_differ():
    a, b = synth.permutation(1000, 5), synth.permutation(1000, 5)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.permutation(1000, 6))
    assert np.array_equal(synth.keys_uniform(100, 3), synth.keys_uniform(100, 3))


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_permutation_is_a_permutation(dtype):
    for n in (1, 2, 17, 4096):
        x = synth.permutation(n, n, dtype)
        assert x.dtype == dtype and np.array_equal(np.sort(x), np.arange(n))


def test_monotone_steps():
    x = synth.monotone(10000, 1)
    d = np.diff(x.astype(np.int64))
    assert x[0] == 0 and d.min() >= 0 and d.max() <= 3


def test_planted_duplicate_value_and_order_break():
    perm = synth.permutation(5000, 2)
    dup, p, q = synth.plant_duplicate(perm, 9)
    assert p != q and dup[p] == dup[q]
    assert np.unique(dup).shape[0] == perm.shape[0] - 1  # exactly one value repeated
    assert np.count_nonzero(dup != perm) == 1
    oor, po = synth.plant_value(perm, 9, 5000)
    assert oor[po] == 5000 and np.count_nonzero(oor != perm) == 1
    mono = synth.monotone(5000, 3)
    brk, pb = synth.plant_order_break(mono, 9)
    assert pb >= 1 and brk[pb] < brk[pb - 1]
    assert np.all(np.diff(brk[:pb].astype(np.int64)) >= 0) and np.all(np.diff(brk[pb:].astype(np.int64)) >= 0)


def test_bernoulli_threshold_fraction():
    keys = synth.keys_uniform(1 << 20, 4)
    for p in (0.01, 0.5, 0.9):
        frac = np.count_nonzero(keys < synth.bernoulli_threshold(p)) / keys.shape[0]
        assert abs(frac - p) < 5e-3, (p, frac)
    assert synth.bernoulli_threshold(0.0) == -(2**31) and synth.bernoulli_threshold(1.0) == 2**31


def test_segment_shapes():
    s = synth.shapes_log_uniform(4096, 11, max_log2=20, cap_total=1 << 40)
    assert s.min() >= 1 and s.max() <= 1 << 20
    # the cap rounds each size down and keeps it >= 1: at most one element per segment over
    for cap in (1 << 16, 1 << 20):
        c = synth.shapes_log_uniform(4096, 11, max_log2=20, cap_total=cap)
        assert c.min() >= 1 and int(c.sum()) <= cap + c.shape[0]
    # the bench's shapes stay within their element counts
    for cap in (1 << 26, 1 << 28):
        assert int(synth.shapes_log_uniform(4096, synth.seed_for(1) + 11, cap_total=cap).sum()) <= cap
    e = synth.shapes_with_empties(1000, 5, 40, p_empty=0.3)
    assert e.min() == 0 and e.max() <= 40
    r = synth.shapes_pareto(10000, 6)
    assert r.min() >= 1 and r.max() <= 1 << 16
    off = synth.offsets_from_shape(e)
    assert off[0] == 0 and np.array_equal(np.diff(off), e)


def test_graph_slots_and_columns():
    es, is_ = synth.graph_slots(4096, 512, 7)
    assert es.min() >= 0 and es.max() < 512
    assert np.array_equal(np.sort(is_), np.arange(4096))  # injective priorities
    ez, _ = synth.graph_slots(4096, 512, 7, zipf_s=1.1)
    assert ez.min() >= 0 and ez.max() < 512 and np.count_nonzero(ez == 0) > np.count_nonzero(ez == 511)
    lengths = np.array([0, 3, 1, 5], np.int64)
    cols = synth.sorted_unique_columns(lengths, 16, 8)
    off = synth.offsets_from_shape(lengths)
    for k in range(lengths.shape[0]):
        row = cols[off[k]:off[k + 1]]
        assert np.all(np.diff(row) > 0) and (row.shape[0] == 0 or (row.min() >= 0 and row.max() < 16))
