"""Autotuner for the batched launch shape.

Times every candidate (threads per CTA, CTAs per SM, shared bitmap size, chunk) on
the caller's runner with CUDA events and stores the fastest in a JSON cache keyed
by GPU name and power-of-two buckets of n and m. The cache lives at
$IXP_TUNE_CACHE, or next to the built library.
"""
from __future__ import annotations

import json
import os

import torch

from . import build as _build

# shared bitmaps up to 2^20 bits (128 KB) let every segment of up to 2^20 elements
# be checked in shared memory; a launch shape is kept only while its CTAs' bitmaps
# fit in 200 KB of one SM's shared memory
CANDIDATES = [(t, c, s, ch) for t in (256, 512) for c in (1, 2, 3, 4) for s in (14, 16, 18, 19, 20) for ch in (4, 8)
              if not (t == 512 and c > 2) and (1 << s) // 8 * c <= 200 * 1024]


def cache_path() -> str:
    return os.environ.get("IXP_TUNE_CACHE") or os.path.join(_build.BUILD, "tune.json")


def _key(n: int, m: int) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{name}|n2^{max(n, 1).bit_length()}|m2^{max(m, 1).bit_length()}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(n: int, m: int):
    t = _load().get(_key(n, m))
    return tuple(t["tuning"]) if t else None


def autotune(runner, reps: int = 3, candidates=None, store: bool = True) -> dict:
    """Times each candidate on `runner` (a BatchRunner) and keeps the fastest."""
    results = []
    for cand in candidates or CANDIDATES:
        runner.set_tuning(cand)
        runner.run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(reps):
            a.record()
            runner.run()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        results.append((best, cand))
    results.sort()
    best_ms, best = results[0]
    runner.set_tuning(best)
    entry = {"tuning": list(best), "ms": best_ms, "tried": [[ms, list(c)] for ms, c in results]}
    if store:
        data = _load()
        data[_key(runner.n, runner.m)] = entry
        os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
        with open(cache_path(), "w") as f:
            json.dump(data, f, indent=1)
    return entry
