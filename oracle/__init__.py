"""CPU oracle for the index-array checks and combinators (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
import this package. It wraps ``ixo.c`` (plain single-threaded C, compiled with
gcc into ``oracle/_build/libixo.so``) with NumPy-in/NumPy-out functions. It
shares nothing with the CUDA library and never imports it.

Verdicts come back as dicts with the fields ok, kind, index, value, aux0, aux1
(kinds: none, out_of_range, order, duplicate, out_of_image, missing, wrong_dest).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libixo.so")
_SRC = os.path.join(_HERE, "ixo.c")

KINDS = ["none", "out_of_range", "order", "duplicate", "out_of_image", "missing", "wrong_dest"]
CMPS = {"le": 0, "lt": 1, "ge": 2, "gt": 3}
INT64_MIN = -(2**63)
INT64_MAX = 2**63 - 1


class OracleError(RuntimeError):
    pass


class _Verdict(C.Structure):
    _fields_ = [("ok", C.c_int32), ("kind", C.c_int32), ("index", C.c_int64), ("value", C.c_int64),
                ("aux0", C.c_int64), ("aux1", C.c_int64)]


class _Pred(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_int32), ("b", C.c_int64), ("flags", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile ixo.c with gcc (no vendor-specific flags; same code on x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _itype(a) -> int:
    if a.dtype == np.int32:
        return 0
    if a.dtype == np.int64:
        return 1
    raise OracleError(f"index arrays are int32 or int64, not {a.dtype}")


def _segs(offsets):
    if offsets is None:
        return None, 0
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    return off, off.shape[0] - 1


def _verdict(v: _Verdict) -> dict:
    return {"ok": bool(v.ok), "kind": KINDS[v.kind], "index": v.index, "value": v.value,
            "aux0": v.aux0, "aux1": v.aux1}


def _check(rc: int):
    if rc != 0:
        raise OracleError(f"oracle returned {rc}")


def pred(kind: str = "true", a: int = 0, b: int = 0, flags=None):
    """Predicate spec: 'true', 'mod_eq' (key mod a == b, floored), 'lt' (key < b), 'flags'."""
    k = {"true": 0, "mod_eq": 1, "lt": 2, "flags": 3}[kind]
    fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
    return (k, a, b, fl)


def _pred(p):
    k, a, b, fl = p
    return _Pred(k, a, b, None if fl is None else fl.ctypes.data)


def check_range(x, lo=INT64_MIN, hi=INT64_MAX) -> dict:
    x = np.ascontiguousarray(x)
    v = _Verdict()
    _check(lib().ixo_check_range(_ptr(x), _itype(x), C.c_int64(x.shape[0]), C.c_int64(lo), C.c_int64(hi),
                                 C.byref(v)))
    return _verdict(v)


def check_mono(x, cmp="le", offsets=None, seg_ok=False):
    x = np.ascontiguousarray(x)
    off, nseg = _segs(offsets)
    v = _Verdict()
    so = np.zeros(max(nseg, 1), np.uint8) if seg_ok else None
    _check(lib().ixo_check_mono(_ptr(x), _itype(x), C.c_int64(x.shape[0]), CMPS[cmp], _ptr(off),
                                C.c_int64(nseg), C.byref(v), _ptr(so)))
    return (_verdict(v), so) if seg_ok else _verdict(v)


def check_inj(x, rcd_lo=INT64_MIN, rcd_hi=INT64_MAX, offsets=None, seg_ok=False):
    x = np.ascontiguousarray(x)
    off, nseg = _segs(offsets)
    v = _Verdict()
    so = np.zeros(max(nseg, 1), np.uint8) if seg_ok else None
    _check(lib().ixo_check_inj(_ptr(x), _itype(x), C.c_int64(x.shape[0]), C.c_int64(rcd_lo), C.c_int64(rcd_hi),
                               _ptr(off), C.c_int64(nseg), C.byref(v), _ptr(so)))
    return (_verdict(v), so) if seg_ok else _verdict(v)


def check_bij(x, rcd_lo, rcd_hi, img_lo=0, img_hi=0, seg_img=False, offsets=None, seg_ok=False):
    x = np.ascontiguousarray(x)
    off, nseg = _segs(offsets)
    v = _Verdict()
    so = np.zeros(max(nseg, 1), np.uint8) if seg_ok else None
    _check(lib().ixo_check_bij(_ptr(x), _itype(x), C.c_int64(x.shape[0]), C.c_int64(rcd_lo), C.c_int64(rcd_hi),
                               C.c_int64(img_lo), C.c_int64(img_hi), int(seg_img), _ptr(off), C.c_int64(nseg),
                               C.byref(v), _ptr(so)))
    return (_verdict(v), so) if seg_ok else _verdict(v)


def _keys(keys):
    if keys is None:
        return None, 0
    k = np.ascontiguousarray(keys)
    return k, _itype(k)


def check_filtpart(z, keys=None, filt=("true", 0, 0, None), part=("true", 0, 0, None), cls=None, v=2,
                   offsets=None) -> dict:
    z = np.ascontiguousarray(z)
    k, kt = _keys(keys)
    off, nseg = _segs(offsets)
    cl = None if cls is None else np.ascontiguousarray(cls, dtype=np.uint8)
    vd = _Verdict()
    _check(lib().ixo_check_filtpart(_ptr(z), _itype(z), C.c_int64(z.shape[0]), _ptr(k), kt, _pred(_p(filt)),
                                    _ptr(cl), _pred(_p(part)), int(v), _ptr(off), C.c_int64(nseg), C.byref(vd)))
    return _verdict(vd)


def check_filtpart_values(y, x, keys=None, filt=("true", 0, 0, None), part=("true", 0, 0, None), cls=None, v=2,
                          offsets=None) -> dict:
    y = np.ascontiguousarray(y)
    x = np.ascontiguousarray(x)
    row_bytes = x.dtype.itemsize * (int(np.prod(x.shape[1:])) if x.ndim > 1 else 1)
    k, kt = _keys(keys)
    off, nseg = _segs(offsets)
    cl = None if cls is None else np.ascontiguousarray(cls, dtype=np.uint8)
    vd = _Verdict()
    _check(lib().ixo_check_filtpart_values(_ptr(y), C.c_int64(y.shape[0]), _ptr(x), C.c_int64(x.shape[0]),
                                           row_bytes, _ptr(k), kt, _pred(_p(filt)), _ptr(cl), _pred(_p(part)),
                                           int(v), _ptr(off), C.c_int64(nseg), C.byref(vd)))
    return _verdict(vd)


def _p(p):
    """Accept either the tuple from pred() or a (kind, a, b[, flags]) shorthand."""
    if isinstance(p, str):
        return pred(p)
    if len(p) == 3:
        return pred(p[0], p[1], p[2])
    k, a, b, fl = p
    if isinstance(k, str):
        return pred(k, a, b, fl)
    return p


def scan(x, out_dtype=None, inclusive=False, offsets=None):
    x = np.ascontiguousarray(x)
    out_dtype = np.dtype(out_dtype or x.dtype)
    out = np.empty(x.shape[0], dtype=out_dtype)
    off, nseg = _segs(offsets)
    tot = np.zeros(max(nseg, 1) if offsets is not None else 1, dtype=out_dtype)
    _check(lib().ixo_scan(_ptr(x), _itype(x), _ptr(out), _itype(out), C.c_int64(x.shape[0]), int(inclusive),
                          _ptr(off), C.c_int64(nseg), _ptr(tot)))
    return out, tot


def sgm_scan(flags, x, out_dtype=None):
    x = np.ascontiguousarray(x)
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    out = np.empty(x.shape[0], dtype=np.dtype(out_dtype or x.dtype))
    _check(lib().ixo_sgm_scan(_ptr(fl), _ptr(x), _itype(x), _ptr(out), _itype(out), C.c_int64(x.shape[0])))
    return out


def _row_bytes(a):
    return a.dtype.itemsize * (int(np.prod(a.shape[1:])) if a.ndim > 1 else 1)


def scatter(dst, idx, vals):
    """Returns a copy of dst with the scatter applied (dst is not modified)."""
    out = np.array(dst, copy=True, order="C")
    idx = np.ascontiguousarray(idx)
    vals = np.ascontiguousarray(vals)
    _check(lib().ixo_scatter(_ptr(out), C.c_int64(out.shape[0]), _ptr(idx), _itype(idx), _ptr(vals),
                             C.c_int64(idx.shape[0]), _row_bytes(vals)))
    return out


def scatter_add_f64(dst_len, idx, vals, init=None):
    """dst (float64, shape [dst_len, cols]) = init + sum of vals rows per in-bounds index."""
    idx = np.ascontiguousarray(idx)
    vals = np.ascontiguousarray(vals)
    cols = int(np.prod(vals.shape[1:])) if vals.ndim > 1 else 1
    out = np.zeros((dst_len,) + tuple(vals.shape[1:]), dtype=np.float64) if init is None else \
        np.array(init, dtype=np.float64, copy=True, order="C")
    _check(lib().ixo_scatter_add_f64(_ptr(out), C.c_int64(dst_len), _ptr(idx), _itype(idx), _ptr(vals),
                                     vals.dtype.itemsize, C.c_int64(idx.shape[0]), cols))
    return out


def gather(src, idx):
    """Returns (out, oob) where oob is True when some index was outside [0, len(src))."""
    src = np.ascontiguousarray(src)
    idx = np.ascontiguousarray(idx)
    out = np.empty((idx.shape[0],) + src.shape[1:], dtype=src.dtype)
    rc = lib().ixo_gather(_ptr(out), _ptr(src), C.c_int64(src.shape[0]), _ptr(idx), _itype(idx),
                          C.c_int64(idx.shape[0]), _row_bytes(src))
    if rc not in (0, -7):
        _check(rc)
    return out, rc == -7


def partition(keys, p, payload=None, out_dtype=np.int32, offsets=None, want_keys=True):
    """Stable 2-way partition; returns dict(indices, num_true, keys_out, payload_out)."""
    k = None if keys is None else np.ascontiguousarray(keys)
    kt = 0 if k is None else _itype(k)
    n = (k.shape[0] if k is not None else np.asarray(_p(p)[3]).shape[0])
    off, nseg = _segs(offsets)
    idx = np.empty(n, dtype=np.dtype(out_dtype))
    nt = np.zeros(max(nseg, 1) if offsets is not None else 1, dtype=np.int64)
    ko = np.empty_like(k) if (want_keys and k is not None) else None
    pl = None if payload is None else np.ascontiguousarray(payload)
    po = None if pl is None else np.empty_like(pl)
    _check(lib().ixo_partition(_ptr(k), kt, C.c_int64(n), _pred(_p(p)), _ptr(pl),
                               0 if pl is None else _row_bytes(pl), _ptr(idx), _itype(idx), _ptr(ko), _ptr(po),
                               _ptr(nt), _ptr(off), C.c_int64(nseg)))
    return {"indices": idx, "num_true": nt, "keys_out": ko, "payload_out": po}


def flags_from_shape(shape, xs=None, out_dtype=np.int64):
    shape = np.ascontiguousarray(shape, dtype=np.int64)
    m = shape.shape[0]
    total = int(shape[shape > 0].sum()) if m else 0
    out = np.empty(total, dtype=np.dtype(out_dtype))
    offs = np.empty(m + 1, dtype=np.int64)
    x = None if xs is None else np.ascontiguousarray(xs, dtype=np.int64)
    _check(lib().ixo_flags_from_shape(_ptr(shape), C.c_int64(m), _ptr(x), _ptr(out), _itype(out),
                                      C.c_int64(total), _ptr(offs)))
    return out, offs


def mkii(shape):
    shape = np.ascontiguousarray(shape, dtype=np.int64)
    total = int(shape[shape > 0].sum()) if shape.shape[0] else 0
    out = np.empty(total, dtype=np.int64)
    _check(lib().ixo_mkii(_ptr(shape), C.c_int64(shape.shape[0]), _ptr(out), C.c_int64(total)))
    return out


def hist_min(m, idx, vals=None, init=None, dtype=np.int64):
    """Reduce-by-index with min: H = init (default: the dtype's maximum) lowered by
    vals[i] at idx[i] for in-bounds indices; vals None means vals[i] = i."""
    idx = np.ascontiguousarray(idx)
    if init is None:
        H = np.full(m, np.iinfo(np.dtype(dtype)).max, dtype=np.dtype(dtype))
    else:
        H = np.array(init, dtype=np.dtype(dtype), copy=True, order="C")
    v = None if vals is None else np.ascontiguousarray(vals, dtype=H.dtype)
    _check(lib().ixo_hist_min(_ptr(H), _itype(H), C.c_int64(m), _ptr(idx), _itype(idx), _ptr(v),
                              C.c_int64(idx.shape[0])))
    return H


def smallest_pairs(n_verts, n_es, es, is_):
    """get_smallest_pairs of maxMatching: returns (es', is') kept in input order."""
    es = np.ascontiguousarray(es)
    is_ = np.ascontiguousarray(is_, dtype=es.dtype)
    n = es.shape[0]
    oe, oi = np.empty(n, es.dtype), np.empty(n, es.dtype)
    cnt = C.c_int64(0)
    _check(lib().ixo_smallest_pairs(C.c_int64(n_verts), C.c_int64(n_es), _ptr(es), _ptr(is_), _itype(es),
                                    C.c_int64(n), _ptr(oe), _ptr(oi), C.byref(cnt)))
    return oe[:cnt.value].copy(), oi[:cnt.value].copy()
