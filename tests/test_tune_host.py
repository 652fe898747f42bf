"""The batched autotuner's host logic on CPU: candidate selection and the JSON
cache, with CUDA events replaced by a fake clock that each run advances by the
candidate's cost (no GPU, no kernel)."""
import pytest

torch = pytest.importorskip("torch")


class _Clock:
    t = 0.0


class _Event:
    def __init__(self, enable_timing=False):
        self.at = None

    def record(self, stream=None):
        self.at = _Clock.t

    def elapsed_time(self, other):
        return other.at - self.at


class _Runner:
    """Stands in for a BatchRunner: each run costs cost(tuning) milliseconds."""

    def __init__(self, cost, n=1 << 20, m=64):
        self.cost, self.n, self.m, self.tuning, self.runs = cost, n, m, None, 0

    def set_tuning(self, t):
        self.tuning = tuple(t)

    def run(self):
        self.runs += 1
        _Clock.t += self.cost(self.tuning)


@pytest.fixture
def tune(monkeypatch, tmp_path):
    from paper_2506_23058_gb300 import tune as m
    monkeypatch.setenv("IXP_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(m.torch.cuda, "Event", _Event)
    monkeypatch.setattr(m.torch.cuda, "synchronize", lambda *a, **k: None)
    return m


def test_candidates_respect_the_thread_and_shared_memory_limits(tune):
    assert len(tune.CANDIDATES) == len(set(tune.CANDIDATES))
    for t, c, s, ch in tune.CANDIDATES:
        assert t * c <= 1024 and t in (256, 512) and ch in (4, 8) and 14 <= s <= 20
        assert (1 << s) // 8 * c <= 200 * 1024  # the CTAs' shared bitmaps fit one SM
    # a 2^20-element segment can be checked in shared memory by some candidate
    assert any(s == 20 for _, _, s, _ in tune.CANDIDATES)


def test_fastest_candidate_is_kept_and_cached(tune):
    want = (512, 2, 16, 8)
    cost = lambda c: 1.0 if c == want else 2.0 + 0.01 * sum(c)  # noqa: E731
    r = _Runner(cost)
    entry = tune.autotune(r, reps=2)
    assert tuple(entry["tuning"]) == want and entry["ms"] == pytest.approx(1.0)
    assert r.tuning == want  # the runner is left on the winner
    assert r.runs == len(tune.CANDIDATES) * 3  # one warm-up and two timed runs each
    assert [row[0] for row in entry["tried"]] == sorted(row[0] for row in entry["tried"])
    assert tune.lookup(r.n, r.m) == want
    # another size bucket has no entry; the same bucket shares it
    assert tune.lookup(r.n * 4, r.m) is None
    assert tune.lookup(r.n + 1, r.m) == want


def test_restricted_candidates_and_no_store(tune):
    cands = [(256, 1, 14, 4), (256, 2, 14, 4)]
    r = _Runner(lambda c: 3.0 if c[1] == 1 else 1.5)
    entry = tune.autotune(r, reps=1, candidates=cands, store=False)
    assert tuple(entry["tuning"]) == (256, 2, 14, 4) and len(entry["tried"]) == 2
    assert tune.lookup(r.n, r.m) is None
