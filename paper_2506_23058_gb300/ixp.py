"""Python binding of the C ABI in include/ixp.h (ctypes; argument marshalling only).

Every function here takes torch CUDA tensors, passes their device pointers, sizes
and the current CUDA stream to the library, and returns device tensors. All work
runs in the library's kernels; if the library cannot be loaded the call raises.
torch supplies device memory (workspaces come from its caching allocator) and
streams, nothing else.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import torch

from . import build as _build

I64MIN = -(2**63)
I64MAX = 2**63 - 1

KINDS = ["none", "out_of_range", "order", "duplicate", "out_of_image", "missing", "wrong_dest"]
CMPS = {"le": 0, "lt": 1, "ge": 2, "gt": 3}
PREDS = {"true": 0, "mod_eq": 1, "lt": 2, "flags": 3}
OPS = {"range": 0, "mono": 1, "inj": 2, "bij": 3, "filtpart": 4, "scan": 5, "partition": 6, "flags": 7,
       "inj_seg": 8, "bij_seg": 9, "gather_segments": 10, "filtpart_classes": 11, "inj_hist": 12,
       "smallest_pairs": 13, "filtpart_values": 14}
ERRORS = {0: "ok", -1: "invalid argument", -2: "unsupported element type", -3: "value span exceeds the workspace",
          -4: "workspace too small", -5: "CUDA launch failed", -6: "bounded device wait gave up",
          -7: "index out of bounds"}


class IxpError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({code})")
        self.code = code


class Pred(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_int32), ("b", C.c_int64), ("flags", C.c_void_p)]


class Segs(C.Structure):
    _fields_ = [("offsets", C.c_void_p), ("nseg", C.c_int64)]


class BatchTuning(C.Structure):
    _fields_ = [("threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("smem_bits_log2", C.c_int32),
                ("chunk", C.c_int32)]


_P = C.c_void_p
_I = C.c_int
_L = C.c_int64
_Z = C.c_size_t

_SIGS = {
    "ixp_workspace_size": (_Z, [_I, _I, _L, _L]),
    "ixp_strerror": (C.c_char_p, [_I]),
    "ixp_version": (_I, []),
    "ixp_check_range": (_I, [_P, _I, _L, _L, _L, _P, _P, _Z, _P]),
    "ixp_check_mono": (_I, [_P, _I, _L, _I, Segs, _P, _P, _P, _Z, _P]),
    "ixp_check_inj": (_I, [_P, _I, _L, _L, _L, _P, _P, _Z, _P]),
    "ixp_check_bij": (_I, [_P, _I, _L, _L, _L, _L, _L, _P, _P, _Z, _P]),
    "ixp_check_filtpart": (_I, [_P, _I, _L, _P, _I, Pred, Pred, Segs, _P, _P, _Z, _P]),
    "ixp_check_inj_seg": (_I, [_P, _I, _L, _L, _L, Segs, _P, _P, _P, _Z, _P]),
    "ixp_check_bij_seg": (_I, [_P, _I, _L, _L, _L, Segs, _P, _P, _P, _Z, _P]),
    "ixp_scan": (_I, [_P, _I, _P, _I, _L, _I, Segs, _P, _P, _P, _Z, _P]),
    "ixp_partition": (_I, [_P, _I, _L, Pred, _P, C.c_int32, _P, _I, _P, _P, _P, Segs, _P, _P, _Z, _P]),
    "ixp_scatter": (_I, [_P, _L, _P, _I, _P, _L, C.c_int32, C.c_int32, C.c_int32, _P]),
    "ixp_scatter_add_f32_to_f64": (_I, [_P, _L, _P, _I, _P, _L, C.c_int32, _P]),
    "ixp_f64_to_f32": (_I, [_P, _P, _L, _P]),
    "ixp_f32_to_f64": (_I, [_P, _P, _L, _P]),
    "ixp_invert": (_I, [_P, _I, _L, _P, _I, _L, _P]),
    "ixp_gather": (_I, [_P, _P, _L, _P, _I, _L, C.c_int32, C.c_int32, _P, _P]),
    "ixp_gather_segments": (_I, [_P, _L, _P, _L, _P, _L, _P, _L, _P, _I, C.c_int32, _P, _P, _Z, _P]),
    "ixp_check_filtpart_classes": (_I, [_P, _I, _L, _P, _I, Pred, _P, C.c_int32, Segs, _P, _P, _Z, _P]),
    "ixp_filtpart_classes": (_I, [_P, _I, _L, Pred, _P, C.c_int32, Segs, _P, _I, _P, _P, _Z, _P]),
    "ixp_check_filtpart_values": (_I, [_P, _L, _P, _L, C.c_int32, _P, _I, Pred, Pred, _P, C.c_int32, Segs, _P, _P,
                                       _Z, _P]),
    "ixp_sgm_scan": (_I, [_P, _P, _I, _P, _I, _L, _I, _P, _P, _Z, _P]),
    "ixp_mkii": (_I, [_P, _L, _P, _I, _L, _P, _P, _Z, _P]),
    "ixp_flags_from_shape": (_I, [_P, _L, _P, _P, _I, _L, _P, _P, _P, _Z, _P]),
    "ixp_hist_min": (_I, [_P, _I, _L, _P, _I, _P, _L, _P]),
    "ixp_check_inj_hist": (_I, [_P, _I, _L, _L, _P, _P, _Z, _P]),
    "ixp_smallest_pairs": (_I, [_P, _P, _I, _L, _L, _L, _P, _P, _P, _P, _Z, _P]),
    "ixp_sink_words": (_I, []),
    "ixp_ceiling_atomic_or": (_I, [_P, _L, _P, _L, _I, _P, _P]),
    "ixp_ceiling_random_rows": (_I, [_P, _L, _P, _L, _P, _P]),
    "ixp_ceiling_stream_read": (_I, [_P, _L, _P, _P]),
    "ixp_debug_set_wait": (_I, [C.c_longlong, C.c_longlong]),
    "ixp_kernel_launches": (C.c_ulonglong, []),
    "ixp_batch_workspace_size": (_Z, [_P]),
    "ixp_batch_run": (_I, [_P, _L, _P, Pred, _P, _P, _L, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _Z, _P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libixp.so (building it first if asked). Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is missing or stale; call paper_2506_23058_gb300.build.build()")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ck(code: int, what: str):
    if code != 0:
        raise IxpError(code, what)


def _itype(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return 0
    if t.dtype == torch.int64:
        return 1
    raise IxpError(-2, f"index arrays are int32 or int64, not {t.dtype}")


def _dev(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _need(t: torch.Tensor, name: str, n: int, dtypes=None, rows: bool = False):
    """Checks a buffer the library reads or writes n entries (rows with rows=True) of."""
    if dtypes is not None and t.dtype not in dtypes:
        raise ValueError(f"{name} must be one of {dtypes}, not {t.dtype}")
    have = (t.shape[0] if t.dim() else 1) if rows else t.numel()
    if have < n:
        raise ValueError(f"{name} has {have} {'rows' if rows else 'entries'}, {n} needed")


def _row_elems(t: torch.Tensor) -> int:
    per = 1
    for d in t.shape[1:]:
        per *= d
    return per


def _pred_flags_ok(pred, n: int):
    p = make_pred(pred)
    if p.kind == PREDS["flags"]:
        fl = pred[3] if isinstance(pred, (tuple, list)) and len(pred) > 3 else None
        if fl is not None:
            _need(fl, "flags", n, (torch.uint8,))


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _segs(offsets):
    if offsets is None:
        return Segs(None, 0)
    return Segs(_dev(offsets, "offsets"), offsets.numel() - 1)


def make_pred(kind="true", a=0, b=0, flags=None) -> Pred:
    """Predicate: 'true', 'mod_eq' (floored key mod a == b), 'lt' (key < b), 'flags' (flags[i] != 0)."""
    if isinstance(kind, Pred):
        return kind
    if isinstance(kind, (tuple, list)):
        return make_pred(*kind)
    fp = None
    if kind == "flags":
        if flags is None or flags.dtype != torch.uint8:
            raise ValueError("flags predicate needs a uint8 CUDA tensor")
        fp = _dev(flags, "flags")
    return Pred(PREDS[kind], int(a), int(b), fp)


def workspace_size(op: str, itype: int, n: int, extra: int = 0) -> int:
    return int(load().ixp_workspace_size(OPS[op], itype, n, extra))


_WS_CACHE: dict = {}


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A reusable uint8 device buffer of at least nbytes (one per device and stream)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = (dev, torch.cuda.current_stream(dev).cuda_stream)
    buf = _WS_CACHE.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        _WS_CACHE[key] = buf
    return buf


@dataclass
class Verdict:
    """A verdict in device memory (48 bytes). `.get()` copies it to the host."""
    buf: torch.Tensor  # int64[6]

    def get(self) -> dict:
        w = self.buf.cpu().tolist()
        lo, hi = w[0] & 0xFFFFFFFF, (w[0] >> 32) & 0xFFFFFFFF
        ok = lo - (1 << 32) if lo >= (1 << 31) else lo
        st = w[5] & 0xFFFFFFFF
        st = st - (1 << 32) if st >= (1 << 31) else st
        return {"ok": ok, "kind": KINDS[hi] if hi < len(KINDS) else hi, "index": w[1], "value": w[2],
                "aux0": w[3], "aux1": w[4], "status": st}


def _verdict_buf(device, out=None):
    if out is not None:
        _need(out, "verdict buffer", 6, (torch.int64,))
        return out
    return torch.empty(6, dtype=torch.int64, device=device)


# ------------------------------------------------------------------- checks

def check_range(x, lo=I64MIN, hi=I64MAX, *, out=None, ws=None, stream=None) -> Verdict:
    v = _verdict_buf(x.device, out)
    need = workspace_size("range", _itype(x), x.numel())
    ws = ws if ws is not None else workspace(need, x.device)
    _ck(load().ixp_check_range(_dev(x, "x"), _itype(x), x.numel(), lo, hi, v.data_ptr(), ws.data_ptr(),
                               ws.numel(), _stream(stream)), "check_range")
    return Verdict(v)


def check_mono(x, cmp="le", offsets=None, *, seg_ok=None, out=None, ws=None, stream=None) -> Verdict:
    v = _verdict_buf(x.device, out)
    segs = _segs(offsets)
    need = workspace_size("mono", _itype(x), x.numel(), segs.nseg)
    ws = ws if ws is not None else workspace(need, x.device)
    so = None if seg_ok is None else _dev(seg_ok, "seg_ok")
    _ck(load().ixp_check_mono(_dev(x, "x"), _itype(x), x.numel(), CMPS[cmp], segs, v.data_ptr(), so, ws.data_ptr(),
                              ws.numel(), _stream(stream)), "check_mono")
    return Verdict(v)


HASH_SET_MAX_BYTES = 1 << 34  # the default workspace holds a hash set up to this size
RCD_BITMAP_MAX_BITS = 1 << 30  # a finite Rcd up to this width gets a bitmap over all of it


def check_inj(x, rcd_lo=I64MIN, rcd_hi=I64MAX, *, span=None, out=None, ws=None, stream=None) -> Verdict:
    """`span`: the largest value span the bitmap must cover (a wider span found in the
    data reports IXP_E_SPAN). Default: the Rcd width when it is at most
    max(4n + 4096, RCD_BITMAP_MAX_BITS); otherwise any span: bitmaps for 4n + 4096
    bits plus a hash set of 16 bytes per slot (the power of two >= 2n slots) that
    decides wider spans, while that set stays within HASH_SET_MAX_BYTES
    (n <= 2^29), else 4n + 4096 bits."""
    v = _verdict_buf(x.device, out)
    n = x.numel()
    extra = span
    if span is None:
        extra = 4 * n + 4096
        if rcd_hi - rcd_lo + 1 <= max(extra, RCD_BITMAP_MAX_BITS):
            extra = rcd_hi - rcd_lo + 1
        elif 16 * max(2, 1 << max(0, (2 * n - 1).bit_length())) <= HASH_SET_MAX_BYTES:
            extra = -1
    need = workspace_size("inj", _itype(x), n, extra if extra < 0 else max(1, extra))
    # exactly the bytes asked for: the library reads its capacities (and whether a
    # hash set is there) from the size it is given
    ws = ws if ws is not None else workspace(need, x.device)[:need]
    _ck(load().ixp_check_inj(_dev(x, "x"), _itype(x), n, rcd_lo, rcd_hi, v.data_ptr(), ws.data_ptr(), ws.numel(),
                             _stream(stream)), "check_inj")
    return Verdict(v)


def check_inj_hist(x, m, *, out=None, ws=None, stream=None) -> Verdict:
    """Inj on [0, m) by reduce-by-index with min (the dynamic verification of scatter);
    same verdict as check_inj(x, 0, m - 1)."""
    v = _verdict_buf(x.device, out)
    need = workspace_size("inj_hist", _itype(x), x.numel(), m)
    ws = ws if ws is not None else workspace(need, x.device)
    _ck(load().ixp_check_inj_hist(_dev(x, "x"), _itype(x), x.numel(), m, v.data_ptr(), ws.data_ptr(), ws.numel(),
                                  _stream(stream)), "check_inj_hist")
    return Verdict(v)


def check_bij(x, rcd_lo, rcd_hi, img_lo, img_hi, *, out=None, ws=None, stream=None) -> Verdict:
    v = _verdict_buf(x.device, out)
    need = workspace_size("bij", _itype(x), x.numel(), img_hi - img_lo + 1)
    ws = ws if ws is not None else workspace(need, x.device)
    _ck(load().ixp_check_bij(_dev(x, "x"), _itype(x), x.numel(), rcd_lo, rcd_hi, img_lo, img_hi, v.data_ptr(),
                             ws.data_ptr(), ws.numel(), _stream(stream)), "check_bij")
    return Verdict(v)


def check_inj_seg(x, offsets, rcd_lo=I64MIN, rcd_hi=I64MAX, *, seg_ok=None, out=None, ws=None, stream=None):
    """Inj of every segment [offsets[k], offsets[k+1])."""
    v = _verdict_buf(x.device, out)
    segs = _segs(offsets)
    need = workspace_size("inj_seg", _itype(x), x.numel(), segs.nseg)
    ws = ws if ws is not None else workspace(need, x.device)
    if seg_ok is not None:
        _need(seg_ok, "seg_ok", segs.nseg, (torch.uint8,))
    so = None if seg_ok is None else _dev(seg_ok, "seg_ok")
    _ck(load().ixp_check_inj_seg(_dev(x, "x"), _itype(x), x.numel(), rcd_lo, rcd_hi, segs, v.data_ptr(), so,
                                 ws.data_ptr(), ws.numel(), _stream(stream)), "check_inj_seg")
    return Verdict(v)


def check_bij_seg(x, offsets, rcd_lo=I64MIN, rcd_hi=I64MAX, *, seg_ok=None, out=None, ws=None, stream=None):
    """Bij of every segment onto its own index range [offsets[k], offsets[k+1])."""
    v = _verdict_buf(x.device, out)
    segs = _segs(offsets)
    need = workspace_size("bij_seg", _itype(x), x.numel(), segs.nseg)
    ws = ws if ws is not None else workspace(need, x.device)
    if seg_ok is not None:
        _need(seg_ok, "seg_ok", segs.nseg, (torch.uint8,))
    so = None if seg_ok is None else _dev(seg_ok, "seg_ok")
    _ck(load().ixp_check_bij_seg(_dev(x, "x"), _itype(x), x.numel(), rcd_lo, rcd_hi, segs, v.data_ptr(), so,
                                 ws.data_ptr(), ws.numel(), _stream(stream)), "check_bij_seg")
    return Verdict(v)


def check_filtpart(z, keys=None, filt="true", part="true", offsets=None, *, cls=None, v=2, out=None, ws=None,
                   stream=None) -> Verdict:
    """InvFiltPart. With `cls` (uint8 per element) the kept elements are placed by
    class min(cls, v - 1) instead of by the `part` predicate."""
    if cls is not None:
        return _check_filtpart_classes(z, keys, filt, cls, v, offsets, out=out, ws=ws, stream=stream)
    v = _verdict_buf(z.device, out)
    segs = _segs(offsets)
    if keys is not None:
        _need(keys, "keys", z.numel())
    _pred_flags_ok(filt, z.numel())
    _pred_flags_ok(part, z.numel())
    kt = _itype(keys) if keys is not None else 0
    need = workspace_size("filtpart", kt, z.numel(), segs.nseg)
    ws = ws if ws is not None else workspace(need, z.device)
    kp = None if keys is None else _dev(keys, "keys")
    _ck(load().ixp_check_filtpart(_dev(z, "z"), _itype(z), z.numel(), kp, kt, make_pred(filt), make_pred(part), segs,
                                  v.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "check_filtpart")
    return Verdict(v)


def _check_filtpart_classes(z, keys, filt, cls, v, offsets, *, out=None, ws=None, stream=None) -> Verdict:
    vb = _verdict_buf(z.device, out)
    segs = _segs(offsets)
    _need(cls, "cls", z.numel(), (torch.uint8,))
    if keys is not None:
        _need(keys, "keys", z.numel())
    _pred_flags_ok(filt, z.numel())
    kt = _itype(keys) if keys is not None else 0
    need = workspace_size("filtpart_classes", int(v), z.numel(), segs.nseg)
    ws = ws if ws is not None else workspace(need, z.device)
    kp = None if keys is None else _dev(keys, "keys")
    _ck(load().ixp_check_filtpart_classes(_dev(z, "z"), _itype(z), z.numel(), kp, kt, make_pred(filt),
                                          _dev(cls, "cls"), int(v), segs, vb.data_ptr(), ws.data_ptr(), ws.numel(),
                                          _stream(stream)), "check_filtpart_classes")
    return Verdict(vb)


def filtpart_classes(cls, v, keys=None, filt="true", offsets=None, out_dtype=torch.int32, *, n=None, out=None,
                     kept=None, ws=None, stream=None):
    """Destinations of the filter + v-class partition (-1 for dropped elements).
    Returns (out_idx, kept) with kept = N as a 1-element int64 device tensor."""
    n = cls.numel() if n is None else n
    segs = _segs(offsets)
    _need(cls, "cls", n, (torch.uint8,))
    if keys is not None:
        _need(keys, "keys", n)
    _pred_flags_ok(filt, n)
    out = out if out is not None else torch.empty(n, dtype=out_dtype, device=cls.device)
    _need(out, "out", n, (torch.int32, torch.int64))
    kept = kept if kept is not None else torch.empty(1, dtype=torch.int64, device=cls.device)
    _need(kept, "kept", 1, (torch.int64,))
    kt = _itype(keys) if keys is not None else 0
    need = workspace_size("filtpart_classes", int(v), n, segs.nseg)
    ws = ws if ws is not None else workspace(need, cls.device)
    _ck(load().ixp_filtpart_classes(None if keys is None else _dev(keys, "keys"), kt, n, make_pred(filt),
                                    _dev(cls, "cls"), int(v), segs, out.data_ptr(), _itype(out), kept.data_ptr(),
                                    ws.data_ptr(), ws.numel(), _stream(stream)), "filtpart_classes")
    return out, kept


def check_filtpart_values(y, x, keys=None, filt="true", part="true", offsets=None, *, cls=None, v=2, out=None,
                          ws=None, stream=None) -> Verdict:
    """FiltPart in value form: Y (rows) equals X filtered and stably partitioned (by
    `part`, or by class min(cls, v - 1) when `cls` is given), bitwise, with length N."""
    vb = _verdict_buf(x.device, out)
    n, ny = x.shape[0], y.shape[0]
    segs = _segs(offsets)
    if x.dtype != y.dtype or tuple(x.shape[1:]) != tuple(y.shape[1:]):
        raise ValueError("y rows must have the type and shape of x rows")
    row_bytes = x.element_size() * math.prod(x.shape[1:])
    if row_bytes % 4:
        raise ValueError("rows must be a multiple of 4 bytes")
    for t, nm in ((x, "x"), (y, "y")):
        if not t.is_contiguous():
            raise ValueError(f"{nm} must be contiguous")
    if keys is not None:
        _need(keys, "keys", n)
    _pred_flags_ok(filt, n)
    if cls is not None:
        _need(cls, "cls", n, (torch.uint8,))
    else:
        _pred_flags_ok(part, n)
    kt = _itype(keys) if keys is not None else 0
    need = workspace_size("filtpart_values", int(v) if cls is not None else 0, n, segs.nseg)
    ws = ws if ws is not None else workspace(need, x.device)
    _ck(load().ixp_check_filtpart_values(y.data_ptr() if ny else None, ny, x.data_ptr() if n else None, n,
                                         row_bytes, None if keys is None else _dev(keys, "keys"), kt,
                                         make_pred(filt), make_pred(part),
                                         None if cls is None else _dev(cls, "cls"), int(v), segs, vb.data_ptr(),
                                         ws.data_ptr(), ws.numel(), _stream(stream)), "check_filtpart_values")
    return Verdict(vb)


# ---------------------------------------------------------------- combinators

def scan(x, out_dtype=None, inclusive=False, offsets=None, *, out=None, totals=None, status=None, ws=None,
         stream=None):
    """Returns (out, totals, status) as device tensors. The totals have the output's
    dtype (the library writes them in the output type)."""
    out_dtype = out.dtype if out is not None else (out_dtype or x.dtype)
    n = x.numel()
    out = out if out is not None else torch.empty(n, dtype=out_dtype, device=x.device)
    _need(out, "out", n, (torch.int32, torch.int64))
    segs = _segs(offsets)
    if totals is None:
        totals = torch.empty(max(1, segs.nseg), dtype=out_dtype, device=x.device)
    elif totals.dtype != out.dtype or totals.numel() < max(1, segs.nseg):
        raise ValueError("totals must have the output's dtype and one entry per segment")
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=x.device)
    _need(status, "status", 1, (torch.int32,))
    need = workspace_size("scan", _itype(x), n, segs.nseg)
    ws = ws if ws is not None else workspace(need, x.device)
    _ck(load().ixp_scan(_dev(x, "x"), _itype(x), out.data_ptr(), _itype(out), n, int(inclusive), segs,
                        totals.data_ptr(), status.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "scan")
    return out, totals, status


def partition(keys, pred, payload=None, out_dtype=torch.int32, offsets=None, *, want_keys=True, want_indices=True,
              n=None, out=None, out_keys=None, out_payload=None, num_true=None, status=None, ws=None, stream=None):
    """Stable two-way partition. Returns dict(indices, num_true, keys_out, payload_out, status);
    indices is None when want_indices is False (keys / payload moved without the index array)."""
    p = make_pred(pred)
    if keys is not None:
        n = keys.numel()
        device = keys.device
    else:
        device = pred[3].device if isinstance(pred, (tuple, list)) else torch.device("cuda")
    segs = _segs(offsets)
    _pred_flags_ok(pred, n)
    if want_indices:
        out = out if out is not None else torch.empty(n, dtype=out_dtype, device=device)
        _need(out, "out", n, (torch.int32, torch.int64))
    else:
        out = None
    if want_keys and keys is not None and out_keys is None:
        out_keys = torch.empty_like(keys)
    if want_keys and out_keys is not None:
        _need(out_keys, "out_keys", n, (keys.dtype,))
    if payload is not None:
        _need(payload, "payload", n, rows=True)
        if out_payload is None:
            out_payload = torch.empty_like(payload)
        _need(out_payload, "out_payload", n, (payload.dtype,), rows=True)
        if _row_elems(out_payload) != _row_elems(payload):
            raise ValueError("out_payload rows must match payload rows")
    num_true = num_true if num_true is not None else torch.empty(max(1, segs.nseg), dtype=torch.int64, device=device)
    _need(num_true, "num_true", max(1, segs.nseg), (torch.int64,))
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=device)
    _need(status, "status", 1, (torch.int32,))
    kt = _itype(keys) if keys is not None else 0
    need = workspace_size("partition", kt, n, segs.nseg)
    ws = ws if ws is not None else workspace(need, device)
    row_bytes = 0
    if payload is not None:
        row_bytes = payload.element_size()
        for d in payload.shape[1:]:
            row_bytes *= d
    ot = _itype(out) if out is not None else (0 if out_dtype == torch.int32 else 1)
    _ck(load().ixp_partition(None if keys is None else _dev(keys, "keys"), kt, n, p,
                             None if payload is None else _dev(payload, "payload"), row_bytes,
                             None if out is None else out.data_ptr(), ot,
                             None if out_keys is None or not want_keys else out_keys.data_ptr(),
                             None if out_payload is None else out_payload.data_ptr(), num_true.data_ptr(), segs,
                             status.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "partition")
    return {"indices": out, "num_true": num_true, "keys_out": out_keys if want_keys else None,
            "payload_out": out_payload, "status": status}


def _rows(t: torch.Tensor, n: int):
    per = 1
    for d in t.shape[1:]:
        per *= d
    return per, t.element_size()


def scatter(dst, idx, vals, mode="assign", *, stream=None):
    """In place: dst[idx[i]] = vals[i] (or += for mode='add'); out-of-bounds indices are ignored."""
    n = idx.numel()
    row_elems, eb = _rows(vals, n)
    _need(vals, "vals", n, rows=True)
    if dst.element_size() != eb or _row_elems(dst) != row_elems:
        raise ValueError("dst rows must have the element size and width of vals rows")
    _ck(load().ixp_scatter(_dev(dst, "dst"), dst.shape[0], _dev(idx, "idx"), _itype(idx), _dev(vals, "vals"), n,
                           row_elems, eb, 0 if mode == "assign" else 1, _stream(stream)), "scatter")
    return dst


def scatter_add_f64(acc, idx, vals, *, stream=None):
    """In place: acc (float64) [idx[i]] += vals[i] (float32 rows)."""
    n = idx.numel()
    row_elems = _rows(vals, n)[0]
    _need(vals, "vals", n, (torch.float32,), rows=True)
    _need(acc, "acc", 0, (torch.float64,))
    if _row_elems(acc) != row_elems:
        raise ValueError("acc rows must have the width of vals rows")
    _ck(load().ixp_scatter_add_f32_to_f64(_dev(acc, "acc"), acc.shape[0], _dev(idx, "idx"), _itype(idx),
                                          _dev(vals, "vals"), n, row_elems, _stream(stream)), "scatter_add_f64")
    return acc


def f64_to_f32(acc, out=None, *, stream=None):
    out = out if out is not None else torch.empty(acc.shape, dtype=torch.float32, device=acc.device)
    _need(out, "out", acc.numel(), (torch.float32,))
    _ck(load().ixp_f64_to_f32(_dev(out, "out"), _dev(acc, "acc"), acc.numel(), _stream(stream)), "f64_to_f32")
    return out


def invert(idx, inv_len, out_dtype=None, *, out=None, stream=None):
    """inv[idx[i]] = i for in-bounds idx[i] (idx injective), -1 where nothing lands."""
    out_dtype = out_dtype or idx.dtype
    out = out if out is not None else torch.empty(inv_len, dtype=out_dtype, device=idx.device)
    _need(out, "out", inv_len, (torch.int32, torch.int64))
    _ck(load().ixp_invert(_dev(idx, "idx"), _itype(idx), idx.numel(), out.data_ptr() if inv_len else None,
                          _itype(out), inv_len, _stream(stream)), "invert")
    return out


def f32_to_f64(x, out=None, *, stream=None):
    out = out if out is not None else torch.empty(x.shape, dtype=torch.float64, device=x.device)
    _need(out, "out", x.numel(), (torch.float64,))
    _ck(load().ixp_f32_to_f64(_dev(out, "out"), _dev(x, "x"), x.numel(), _stream(stream)), "f32_to_f64")
    return out


def gather(src, idx, *, out=None, status=None, stream=None):
    """out[i] = src[idx[i]]; an out-of-range index zero-fills its row and sets status to -7."""
    n = idx.numel()
    shape = (n,) + tuple(src.shape[1:])
    out = out if out is not None else torch.empty(shape, dtype=src.dtype, device=src.device)
    row_elems = _row_elems(src)
    _need(out, "out", n, (src.dtype,), rows=True)
    if _row_elems(out) != row_elems:
        raise ValueError("out rows must have the width of src rows")
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=src.device)
    _need(status, "status", 1, (torch.int32,))
    _ck(load().ixp_gather(_dev(out, "out"), _dev(src, "src"), src.shape[0], _dev(idx, "idx"), _itype(idx), n,
                          row_elems, src.element_size(), status.data_ptr(), _stream(stream)), "gather")
    return out, status


def gather_segments(src, src_off, seg_src, out_off, n_out, *, out=None, status=None, ws=None, stream=None):
    """Output segment k = source segment seg_src[k] (CSR rows moved to a new order).
    src/out: 1-D tensors of 4- or 8-byte elements; offsets int64 [m + 1]; n_out = out_off[-1]."""
    m = seg_src.numel()
    _need(out_off, "out_off", m + 1, (torch.int64,))
    _need(src_off, "src_off", 1, (torch.int64,))
    out = out if out is not None else torch.empty(n_out, dtype=src.dtype, device=src.device)
    _need(out, "out", n_out, (src.dtype,))
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=src.device)
    _need(status, "status", 1, (torch.int32,))
    need = workspace_size("gather_segments", 0, n_out)
    ws = ws if ws is not None else workspace(need, src.device)
    _ck(load().ixp_gather_segments(_dev(out, "out"), n_out, _dev(out_off, "out_off"), m, _dev(src, "src"),
                                   src.numel(), _dev(src_off, "src_off"), src_off.numel() - 1,
                                   _dev(seg_src, "seg_src"), _itype(seg_src), src.element_size(), status.data_ptr(),
                                   ws.data_ptr() if ws.numel() else None, ws.numel(), _stream(stream)),
        "gather_segments")
    return out, status


def sgm_scan(flags, x, out_dtype=None, inclusive=True, *, out=None, status=None, ws=None, stream=None):
    """sgmSum: scan that restarts at every flagged position. Returns (out, status)."""
    out_dtype = out_dtype or x.dtype
    n = x.numel()
    out = out if out is not None else torch.empty(n, dtype=out_dtype, device=x.device)
    _need(flags, "flags", n, (torch.uint8, torch.bool))
    _need(out, "out", n, (torch.int32, torch.int64))
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=x.device)
    _need(status, "status", 1, (torch.int32,))
    need = workspace_size("scan", _itype(x), n, 0)
    ws = ws if ws is not None else workspace(need, x.device)
    _ck(load().ixp_sgm_scan(_dev(flags, "flags"), _dev(x, "x"), _itype(x), out.data_ptr(), _itype(out), n,
                            int(inclusive), status.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "sgm_scan")
    return out, status


def hist_min(H, idx, vals=None, *, stream=None):
    """In place: H[idx[i]] = min(H[idx[i]], vals[i]) for in-bounds idx[i] (vals None: i)."""
    if vals is not None and vals.dtype != H.dtype:
        raise ValueError("vals must have H's dtype")
    if vals is not None:
        _need(vals, "vals", idx.numel())
    _ck(load().ixp_hist_min(_dev(H, "H") if H.numel() else None, _itype(H), H.numel(),
                            _dev(idx, "idx") if idx.numel() else None, _itype(idx),
                            None if vals is None else _dev(vals, "vals"), idx.numel(), _stream(stream)), "hist_min")
    return H


def smallest_pairs(es, is_, n_verts, n_es, *, out_es=None, out_is=None, count=None, ws=None, stream=None):
    """get_smallest_pairs of maxMatching. Returns (out_es, out_is, count): the first
    count entries of the outputs are the kept pairs in input order (count stays on
    the device)."""
    if is_.dtype != es.dtype or is_.numel() != es.numel():
        raise ValueError("es and is must have one dtype and one length")
    n = es.numel()
    out_es = out_es if out_es is not None else torch.empty_like(es)
    out_is = out_is if out_is is not None else torch.empty_like(is_)
    _need(out_es, "out_es", n, (es.dtype,))  # room for every slot: the kept count is known on the device only
    _need(out_is, "out_is", n, (es.dtype,))
    count = count if count is not None else torch.empty(1, dtype=torch.int64, device=es.device)
    _need(count, "count", 1, (torch.int64,))
    need = workspace_size("smallest_pairs", _itype(es), n, n_verts)
    ws = ws if ws is not None else workspace(need, es.device)
    _ck(load().ixp_smallest_pairs(_dev(es, "es") if n else None, _dev(is_, "is") if n else None, _itype(es), n,
                                  n_verts, n_es, out_es.data_ptr() if n else None, out_is.data_ptr() if n else None,
                                  count.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "smallest_pairs")
    return out_es, out_is, count


def mkii(offsets, n, out_dtype=torch.int32, *, out=None, status=None, ws=None, stream=None):
    """Segment index of every position: out[j] = k for offsets[k] <= j < offsets[k+1]."""
    m = offsets.numel() - 1
    _need(offsets, "offsets", 1, (torch.int64,))
    out = out if out is not None else torch.empty(n, dtype=out_dtype, device=offsets.device)
    _need(out, "out", n, (torch.int32, torch.int64))
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=offsets.device)
    _need(status, "status", 1, (torch.int32,))
    need = workspace_size("gather_segments", 0, n)
    ws = ws if ws is not None else workspace(need, offsets.device)
    _ck(load().ixp_mkii(_dev(offsets, "offsets"), m, out.data_ptr() if n else None, _itype(out), n, status.data_ptr(),
                        ws.data_ptr(), ws.numel(), _stream(stream)), "mkii")
    return out, status


def flags_from_shape(shape, xs=None, out_dtype=torch.int64, out_len=None, *, out=None, offsets=None, status=None,
                     ws=None, stream=None):
    """mkSgmDescr. Returns (flags, offsets, status). out_len=None reads sum(shape) (one sync)."""
    m = shape.numel()
    offs = offsets if offsets is not None else torch.empty(m + 1, dtype=torch.int64, device=shape.device)
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=shape.device)
    _need(status, "status", 1, (torch.int32,))
    need = workspace_size("flags", 1, m)
    ws = ws if ws is not None else workspace(need, shape.device)
    xp = None if xs is None else _dev(xs, "xs")
    if out_len is None:
        _ck(load().ixp_flags_from_shape(_dev(shape, "shape"), m, xp, None, 1, 0, offs.data_ptr(), status.data_ptr(),
                                        ws.data_ptr(), ws.numel(), _stream(stream)), "flags_from_shape")
        out_len = int(offs[m].item()) if m else 0
        if status.item() != 0:
            raise IxpError(int(status.item()), "flags_from_shape")
    if out is None:
        out = torch.empty(out_len, dtype=out_dtype, device=shape.device)
    _ck(load().ixp_flags_from_shape(_dev(shape, "shape"), m, xp, out.data_ptr() if out_len else None,
                                    _itype(out), out_len, offs.data_ptr(), status.data_ptr(), ws.data_ptr(),
                                    ws.numel(), _stream(stream)), "flags_from_shape")
    return out, offs, status


def debug_set_wait(spin_limit: int, skip_tile: int = -1):
    """Testing hook: bound on device waits (polls) and a tile that never publishes."""
    _ck(load().ixp_debug_set_wait(spin_limit, skip_tile), "debug_set_wait")
