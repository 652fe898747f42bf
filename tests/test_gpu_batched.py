"""Batched pipeline (one persistent launch, CUDA graph, autotuned shape) against the
oracle: flag array, per-segment partition, per-segment Mono / Inj / Bij."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I64MIN, I64MAX = oracle.INT64_MIN, oracle.INT64_MAX


@pytest.fixture(scope="module")
def mod():
    import paper_2506_23058_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def workload(m, max_log2, seed, p_bad=0.05):
    """Log-uniform segment sizes, keys, a segmented partition output as `chk` and a
    segmented iota as `iota`, with violations planted in a few segments."""
    rng = np.random.default_rng(seed)
    shape = synth.shapes_log_uniform(m, seed, max_log2=max_log2, cap_total=1 << 40)
    shape[rng.random(m) < 0.05] = 0  # some empty segments
    off = synth.offsets_from_shape(shape)
    n = int(off[-1])
    keys = synth.keys_uniform(n, seed + 1)
    chk = np.concatenate([rng.permutation(np.arange(off[k], off[k + 1])) for k in range(m)]).astype(np.int32)
    iota = np.concatenate([np.arange(off[k + 1] - off[k]) for k in range(m)]).astype(np.int32)
    for k in np.flatnonzero((rng.random(m) < p_bad) & (shape >= 3)):
        a, b = int(off[k]), int(off[k + 1])
        kind = int(rng.integers(0, 3))
        i = a + int(rng.integers(1, b - a))
        if kind == 0:
            chk[i] = chk[i - 1]  # duplicate: breaks Inj and Bij
        elif kind == 1:
            chk[i] = (b + 5) % n  # value of another segment: breaks Bij only
        else:
            iota[i] = iota[i - 1]  # breaks strict Mono
    return shape, off, keys, chk, iota


def check_against_oracle(r, shape, off, keys, chk, iota, p):
    m = len(shape)
    assert r["status"] == 0
    o_flags, o_off = oracle.flags_from_shape(shape, None, out_dtype=np.int32)
    assert np.array_equal(r["flags"].cpu().numpy(), o_flags)
    assert np.array_equal(r["offsets"].cpu().numpy(), o_off)
    op = oracle.partition(keys, p, offsets=off)
    assert np.array_equal(r["indices"].cpu().numpy(), op["indices"])
    assert np.array_equal(r["num_true"].cpu().numpy(), op["num_true"][:m])
    _, mono = oracle.check_mono(iota, "lt", off, seg_ok=True)
    _, inj = oracle.check_inj(chk, offsets=off, seg_ok=True)
    _, bij = oracle.check_bij(chk, I64MIN, I64MAX, seg_img=True, offsets=off, seg_ok=True)
    for got, ref, name in ((r["mono_ok"], mono, "mono"), (r["inj_ok"], inj, "inj"), (r["bij_ok"], bij, "bij")):
        assert np.array_equal(got, ref[:m]), name
    fb = [int(np.flatnonzero(ref[:m] == 0)[0]) if (ref[:m] == 0).any() else -1 for ref in (mono, inj, bij)]
    assert r["first_bad"] == fb


@pytest.mark.parametrize("tuning", [(256, 2, 16, 4), (256, 4, 14, 8), (512, 1, 18, 8), (512, 2, 14, 4)])
def test_batch_matches_oracle(mod, dev, tuning):
    shape, off, keys, chk, iota = workload(700, 16, 5)
    p = ("lt", 0, synth.bernoulli_threshold(0.3))
    br = mod.batched.BatchRunner(shape, T(keys, dev), p, T(chk, dev), T(iota, dev), tuning=tuning)
    br.run()
    torch.cuda.synchronize()
    check_against_oracle(br.results(), shape, off, keys, chk, iota, p)


def test_batch_graph_replay_and_autotune(mod, dev, tmp_path, monkeypatch):
    monkeypatch.setenv("IXP_TUNE_CACHE", str(tmp_path / "tune.json"))
    shape, off, keys, chk, iota = workload(400, 15, 9)
    p = ("mod_eq", 3, 0)
    br = mod.batched.BatchRunner(shape, T(keys, dev), p, T(chk, dev), T(iota, dev))
    entry = mod.tune.autotune(br, reps=1, candidates=mod.tune.CANDIDATES[:6])
    assert tuple(entry["tuning"]) == mod.tune.lookup(br.n, br.m)
    br.capture()
    for _ in range(2):
        br.indices.fill_(-1)
        br.flags.fill_(-1)
        br.replay()
        torch.cuda.synchronize()
        check_against_oracle(br.results(), shape, off, keys, chk, iota, p)


def test_batch_rejects_bad_shapes(mod, dev):
    shape = np.array([3, -1, 2], np.int64)
    keys = T(np.zeros(4, np.int32), dev)
    br = mod.batched.BatchRunner(np.array([3, 1, 0], np.int64), keys, "true", keys, keys)
    br.shape.copy_(T(shape, dev))  # a negative size reaches the device
    br.run()
    assert br.results()["status"] == -1
