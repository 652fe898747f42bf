"""Seeded synthetic inputs for the index-array workloads.

This module only draws random numbers and lays them out; it holds none of the
arithmetic of the checks, scans or partitions themselves. Both the CPU oracle
tests and the CUDA-path tests/bench take their inputs from here, so the two sides
see byte-identical data.

Small inputs are drawn on the host with NumPy's PCG64 generator (its
``shuffle`` is a Fisher-Yates shuffle); large inputs are drawn with torch's own
generator on the target device, which keeps a 2^28-element workload's set-up in
seconds. Every function is a pure function of its arguments.

Workload recipes (the paper measures partition2 on "random floats", Sec. 6; the
other workloads are synthetic stand-ins with the shapes the paper's programs
use):
  * permutation         - uniform random permutation of [0, n)
  * monotone            - x[i] = sum_{j<i} u[j], u ~ uniform{0..3}
  * planted variants    - one entry overwritten at a seeded uniform position
  * keys                - uniform int32 over the full range
  * Bernoulli(p) predicate - ``key < INT32_MIN + round(p * 2^32)``
  * payload             - float32 uniform in [-1, 1)
  * segment shapes      - log-uniform in [1, 2^20] (batched), Pareto rows (CSR)
  * Zipf(s) targets     - inverse-CDF draw of ranks over m targets
  * unit floats         - float32 uniform in [0, 1) (partition2's "random floats")
  * graph slots         - edge endpoints es uniform over [0, n_verts) (or Zipf
                          ranks for a skewed degree law), priorities is a uniform
                          random permutation of [0, n) (injective)
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x1DA2506
INT32_MIN = -(2**31)


def seed_for(config_index: int, salt: int = 0) -> int:
    return SEED_BASE + 1000 * config_index + salt


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


# ---------------------------------------------------------------- host (NumPy)

def identity(n: int, dtype=np.int32) -> np.ndarray:
    return np.arange(n, dtype=dtype)


def permutation(n: int, seed: int, dtype=np.int32) -> np.ndarray:
    """Fisher-Yates shuffle of [0, n) (NumPy's Generator.shuffle)."""
    x = np.arange(n, dtype=dtype)
    _rng(seed).shuffle(x)
    return x


def monotone(n: int, seed: int, dtype=np.int32) -> np.ndarray:
    """Nondecreasing array starting at 0 with steps drawn from uniform{0..3}."""
    steps = _rng(seed).integers(0, 4, size=n, dtype=np.int64)
    x = np.zeros(n, dtype=np.int64)
    if n > 1:
        np.cumsum(steps[:-1], out=x[1:])
    return x.astype(dtype)


def planted_position(n: int, seed: int, lo: int = 0) -> int:
    return int(_rng(seed ^ 0x5EED).integers(lo, n))


def plant_duplicate(x: np.ndarray, seed: int) -> tuple[np.ndarray, int, int]:
    """Copy of x with x[q] := x[p] for two distinct seeded positions p, q."""
    n = x.shape[0]
    r = _rng(seed ^ 0xD0B)
    p = int(r.integers(0, n))
    q = int(r.integers(0, n - 1))
    if q >= p:
        q += 1
    y = x.copy()
    y[q] = y[p]
    return y, p, q


def plant_value(x: np.ndarray, seed: int, value: int) -> tuple[np.ndarray, int]:
    p = planted_position(x.shape[0], seed)
    y = x.copy()
    y[p] = value
    return y, p


def plant_order_break(x: np.ndarray, seed: int) -> tuple[np.ndarray, int]:
    """x[p] := x[p-1] - 1 at a seeded p >= 1 (breaks nondecreasing order)."""
    p = planted_position(x.shape[0], seed, lo=1)
    y = x.copy()
    y[p] = y[p - 1] - 1
    return y, p


def keys_uniform(n: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(INT32_MIN, 2**31, size=n, dtype=np.int64).astype(np.int32)


def bernoulli_threshold(p: float) -> int:
    """Threshold t such that ``key < t`` holds with probability p for uniform int32 keys."""
    return INT32_MIN + int(round(p * 2.0**32))


def payload_f32(n: int, seed: int, cols: int = 1) -> np.ndarray:
    shape = (n,) if cols == 1 else (n, cols)
    return _rng(seed).uniform(-1.0, 1.0, size=shape).astype(np.float32)


def floats_unit(n: int, seed: int) -> np.ndarray:
    return _rng(seed).random(n, dtype=np.float32)


def graph_slots(n: int, n_verts: int, seed: int, dtype=np.int64, zipf_s: float = 0.0):
    """(es, is): n edge-endpoint slots over n_verts vertices and injective priorities."""
    if zipf_s > 0.0:
        es = zipf_ranks(n, max(n_verts, 1), zipf_s, seed).astype(dtype)
    else:
        es = _rng(seed).integers(0, max(n_verts, 1), size=n, dtype=np.int64).astype(dtype)
    return es, permutation(n, seed + 1, dtype)


def class_ids(n: int, seed: int, v: int) -> np.ndarray:
    return _rng(seed).integers(0, v, size=n, dtype=np.int64).astype(np.uint8)


def flags_bernoulli(n: int, seed: int, p: float) -> np.ndarray:
    return (_rng(seed).random(n) < p).astype(np.uint8)


def shapes_log_uniform(m: int, seed: int, max_log2: int = 20, cap_total: int = 2**28) -> np.ndarray:
    """Segment sizes s_k = clamp(floor(2^(max_log2 * U)), 1, 2^max_log2), total capped."""
    u = _rng(seed).random(m)
    s = np.clip(np.floor(np.exp2(max_log2 * u)), 1, 2**max_log2).astype(np.int64)
    tot = int(s.sum())
    if tot > cap_total:
        s = np.maximum(1, (s * cap_total) // tot)
    return s


def shapes_with_empties(m: int, seed: int, max_len: int, p_empty: float = 0.2) -> np.ndarray:
    r = _rng(seed)
    s = r.integers(0, max_len + 1, size=m, dtype=np.int64)
    s[r.random(m) < p_empty] = 0
    return s


def shapes_pareto(m: int, seed: int, alpha: float = 2.0, xmin: float = 1.5, max_len: int = 2**16) -> np.ndarray:
    """Row lengths L = clamp(floor(X), 1, max_len), X ~ Pareto(alpha, xmin)."""
    u = _rng(seed).random(m)
    x = xmin / np.power(1.0 - u, 1.0 / (alpha - 1.0))  # inverse CDF of pdf ~ x^-alpha on [xmin, inf)
    return np.clip(np.floor(x), 1, max_len).astype(np.int64)


def sorted_unique_columns(lengths: np.ndarray, ncols: int, seed: int) -> np.ndarray:
    """For each row, `len` distinct sorted column ids in [0, ncols) (selection sampling)."""
    r = _rng(seed)
    out = np.empty(int(lengths.sum()), dtype=np.int32)
    pos = 0
    for L in lengths.tolist():
        cols = np.sort(r.choice(ncols, size=L, replace=False)) if L > 0 else np.empty(0)
        out[pos:pos + L] = cols
        pos += L
    return out


def zipf_ranks(n: int, m: int, s: float, seed: int) -> np.ndarray:
    """Ranks in [0, m) with P(rank = k) proportional to (k+1)^-s (inverse-CDF table)."""
    w = np.power(np.arange(1, m + 1, dtype=np.float64), -s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = _rng(seed).random(n)
    return np.minimum(np.searchsorted(cdf, u, side="right"), m - 1).astype(np.int32)


def offsets_from_shape(shape: np.ndarray) -> np.ndarray:
    """Segment offsets e_0 = 0, e_{k+1} = e_k + shape_k (input layout, not a result)."""
    off = np.zeros(shape.shape[0] + 1, dtype=np.int64)
    np.cumsum(shape, out=off[1:])
    return off


# ---------------------------------------------------------- device (torch)

def _torch_gen(seed: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def t_permutation(n: int, seed: int, device, dtype=None):
    import torch
    dtype = dtype or torch.int32
    return torch.randperm(n, generator=_torch_gen(seed, device), device=device, dtype=torch.int64).to(dtype)


def t_monotone(n: int, seed: int, device, dtype=None):
    import torch
    dtype = dtype or torch.int32
    steps = torch.randint(0, 4, (n,), generator=_torch_gen(seed, device), device=device, dtype=torch.int64)
    x = torch.zeros(n, dtype=torch.int64, device=device)
    if n > 1:
        torch.cumsum(steps[:-1], 0, out=x[1:])
    return x.to(dtype)


def t_keys_uniform(n: int, seed: int, device):
    import torch
    return torch.randint(INT32_MIN, 2**31, (n,), generator=_torch_gen(seed, device),
                         device=device, dtype=torch.int64).to(torch.int32)


def t_payload_f32(n: int, seed: int, device, cols: int = 1):
    import torch
    shape = (n,) if cols == 1 else (n, cols)
    return torch.rand(shape, generator=_torch_gen(seed, device), device=device, dtype=torch.float32) * 2.0 - 1.0


def t_floats_unit(n: int, seed: int, device):
    import torch
    return torch.rand(n, generator=_torch_gen(seed, device), device=device, dtype=torch.float32)


def t_graph_slots(n: int, n_verts: int, seed: int, device, dtype=None):
    """Device version of graph_slots (uniform endpoints, torch's generator)."""
    import torch
    dtype = dtype or torch.int64
    es = torch.randint(0, max(n_verts, 1), (n,), generator=_torch_gen(seed, device), device=device,
                       dtype=torch.int64).to(dtype)
    return es, t_permutation(n, seed + 1, device, dtype)


def t_shapes_pareto(m: int, seed: int, device, alpha: float = 2.0, xmin: float = 1.5, max_len: int = 2**16):
    """Device version of shapes_pareto (same law, torch's generator)."""
    import torch
    u = torch.rand(m, generator=_torch_gen(seed, device), device=device, dtype=torch.float64)
    x = xmin / torch.pow(1.0 - u, 1.0 / (alpha - 1.0))
    return torch.clamp(torch.floor(x), 1, max_len).to(torch.int64)


def t_stratified_columns(lengths, offsets, ncols: int, seed: int):
    """Device CSR columns: for a row of length L, element t takes a uniform column in
    [t * s, (t + 1) * s) with s = ncols // L, so every row is sorted, unique and
    inside [0, ncols) (a stratified sample; needs L <= ncols)."""
    import torch
    device = lengths.device
    m = lengths.shape[0]
    nnz = int(offsets[-1].item())
    row = torch.repeat_interleave(torch.arange(m, device=device), lengths, output_size=nnz)
    t = torch.arange(nnz, device=device, dtype=torch.int64) - offsets[:-1][row]
    stride = (ncols // lengths)[row]
    del row
    u = torch.rand(nnz, generator=_torch_gen(seed, device), device=device, dtype=torch.float64)
    jitter = torch.minimum((u * stride).to(torch.int64), stride - 1)
    return (t * stride + jitter).to(torch.int32)


def t_plant_rows(cols, offsets, lengths, seed: int, frac: float = 0.001):
    """In a fraction of the rows of length >= 2, make the element at a uniform
    position p >= 1 of the row equal its predecessor (a duplicate) or swap it with
    its predecessor (an order break). Returns (cols, planted row ids ascending)."""
    import torch
    r = _rng(seed)
    L = lengths.cpu().numpy()
    cand = np.flatnonzero(L >= 2)
    k = max(1, int(round(frac * L.shape[0])))
    rows = np.sort(r.choice(cand, size=min(k, cand.shape[0]), replace=False))
    off = offsets.cpu().numpy()
    pos = off[rows] + 1 + (r.random(rows.shape[0]) * (L[rows] - 1)).astype(np.int64)
    dup = r.random(rows.shape[0]) < 0.5
    y = cols.clone()
    p = torch.from_numpy(pos).to(cols.device)
    prev = y[p - 1].clone()
    cur = y[p].clone()
    d = torch.from_numpy(dup).to(cols.device)
    y[p] = prev
    y[p - 1] = torch.where(d, prev, cur)
    return y, rows


def t_position(n: int, seed: int, lo: int = 0) -> int:
    return planted_position(n, seed, lo)


def t_plant_duplicate(x, seed: int):
    n = x.shape[0]
    r = _rng(seed ^ 0xD0B)
    p = int(r.integers(0, n))
    q = int(r.integers(0, n - 1))
    if q >= p:
        q += 1
    y = x.clone()
    y[q] = y[p]
    return y, p, q


def t_plant_value(x, seed: int, value: int):
    p = planted_position(x.shape[0], seed)
    y = x.clone()
    y[p] = value
    return y, p


def t_plant_order_break(x, seed: int):
    p = planted_position(x.shape[0], seed, lo=1)
    y = x.clone()
    y[p] = y[p - 1] - 1
    return y, p

