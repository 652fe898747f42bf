"""Differentiable scatter, gather and partition over float payloads.

Forward and backward both run the library's kernels (this module only allocates
outputs and marshals arguments):

* ``gather``   y[i] = src[idx[i]].  Adjoint: grad_src[t] = sum of grad_y[i] over
  idx[i] = t. When idx is injective on [0, len(src)) that sum has at most one
  term: with the inverse index array (``invert``; the paper's scatter rule Sc1
  builds the same is^-1 for a bijective index) the adjoint is a gather,
  grad_src[t] = grad_y[inv[t]], with sequential writes and no atomics; without it,
  a plain atomic-free scatter. That path is taken only on a proven Inj: asking for
  it (``injective=True`` or an ``inverse``) runs ``check_inj(idx, 0, len(src) - 1)``
  in the forward pass, unless the caller hands in the verdict of that same check
  (``proof``, e.g. kept beside a cached inverse); the backward reads the verdict
  and, when Inj does not hold, takes the general path below, so duplicate indices
  never lose gradient terms. In the general path float32 gradients accumulate in
  float64 and are rounded once; float64 gradients use float64 atomics.
* ``scatter``  out = dst with rows idx[i] replaced by vals[i] (indices outside
  dst are ignored, Sec. 2.1). Requires injective in-bounds indices (the paper's
  condition for a deterministic scatter). Adjoint: grad_vals = gather of grad_out
  (zero for ignored indices); grad_dst = grad_out with the overwritten rows zeroed.
* ``scatter_add``  out = dst + sum of vals rows per index. Indexing is exact and
  needs no injectivity; adjoint: grad_vals = gather of grad_out, grad_dst = grad_out.
* ``partition``  the payload rows moved to the stable two-way partition order
  (partition2, Fig. 2). Adjoint: grad_payload = gather of grad_out by ``indices``
  (every element goes to exactly one destination).
* ``gather_segments``  whole segments (CSR rows) moved to a new segment order
  ``seg_src``, a permutation of the segments. Adjoint: the same move with the
  inverse permutation (each element has exactly one destination).
"""
from __future__ import annotations

import torch

from . import ixp


def _zeros(shape, dtype, device):
    return torch.zeros(shape, dtype=dtype, device=device)


def _scatter_add_into(grad, idx, g):
    """grad (zeroed, float32 or float64) += rows of g grouped by idx."""
    if g.dtype == torch.float32:
        acc = _zeros(grad.shape, torch.float64, g.device)
        ixp.scatter_add_f64(acc, idx, g)
        ixp.f64_to_f32(acc, out=grad)
    else:
        ixp.scatter(grad, idx, g, mode="add")
    return grad


class GatherFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, src, idx, injective=False, inverse=None, proof=None):
        out, status = ixp.gather(src.contiguous(), idx)
        ctx.src_shape = src.shape
        ctx.fast = bool(injective) or inverse is not None
        ctx.has_inverse = inverse is not None
        if ctx.fast and proof is None:
            proof = ixp.check_inj(idx, 0, max(src.shape[0] - 1, 0))  # device work only; read in backward
        ctx.proof = proof
        ctx.save_for_backward(idx, inverse if inverse is not None else idx)
        ctx.mark_non_differentiable(status)
        return out, status

    @staticmethod
    def backward(ctx, g, _g_status):
        idx, inv = ctx.saved_tensors
        g = g.contiguous()
        proven = False
        if ctx.fast:
            v = ctx.proof.get()
            proven = v["ok"] == 1 and v["status"] == 0
        if proven and ctx.has_inverse:
            grad, _ = ixp.gather(g, inv)  # rows no index reaches read as zero
            return grad, None, None, None, None
        grad = _zeros(ctx.src_shape, g.dtype, g.device)
        if proven:
            ixp.scatter(grad, idx, g)  # one term per target: no atomics
        else:
            _scatter_add_into(grad, idx, g)
        return grad, None, None, None, None


class ScatterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dst, idx, vals):
        out = dst.contiguous().clone()
        ixp.scatter(out, idx, vals.contiguous())
        ctx.save_for_backward(idx)
        ctx.vals_shape = vals.shape
        return out

    @staticmethod
    def backward(ctx, g):
        (idx,) = ctx.saved_tensors
        g = g.contiguous()
        grad_vals, _ = ixp.gather(g, idx)  # out-of-bounds indices give zero rows
        grad_dst = g.clone()
        ixp.scatter(grad_dst, idx, _zeros(ctx.vals_shape, g.dtype, g.device))
        return grad_dst, None, grad_vals


class ScatterAddFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dst, idx, vals):
        dst = dst.contiguous()
        vals = vals.contiguous()
        if vals.dtype == torch.float32:
            acc = ixp.f32_to_f64(dst)
            ixp.scatter_add_f64(acc, idx, vals)
            out = ixp.f64_to_f32(acc)
        else:
            out = dst.clone()
            ixp.scatter(out, idx, vals, mode="add")
        ctx.save_for_backward(idx)
        return out

    @staticmethod
    def backward(ctx, g):
        (idx,) = ctx.saved_tensors
        g = g.contiguous()
        grad_vals, _ = ixp.gather(g, idx)
        return g, None, grad_vals


class PartitionFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, payload, keys, pred, offsets=None, out_dtype=torch.int32):
        r = ixp.partition(keys, pred, payload=payload.contiguous(), out_dtype=out_dtype, offsets=offsets,
                          want_keys=False, n=payload.shape[0])
        ctx.save_for_backward(r["indices"])
        ctx.mark_non_differentiable(r["indices"], r["num_true"])
        return r["payload_out"], r["indices"], r["num_true"]

    @staticmethod
    def backward(ctx, g, _gi, _gn):
        (indices,) = ctx.saved_tensors
        grad, _ = ixp.gather(g.contiguous(), indices)
        return grad, None, None, None, None


class GatherSegmentsFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, src, src_off, seg_src, out_off, inv_seg):
        out, status = ixp.gather_segments(src.contiguous(), src_off, seg_src, out_off, src.numel())
        ctx.save_for_backward(src_off, out_off, inv_seg)
        ctx.mark_non_differentiable(status)
        return out, status

    @staticmethod
    def backward(ctx, g, _g_status):
        src_off, out_off, inv_seg = ctx.saved_tensors
        grad, _ = ixp.gather_segments(g.contiguous(), out_off, inv_seg, src_off, g.numel())
        return grad, None, None, None, None


def gather(src, idx, injective=False, inverse=None, proof=None):
    """Differentiable gather. ``injective=True`` or ``inverse`` (``invert(idx,
    src.shape[0])``) ask for the atomic-free adjoint, which is used only when Inj of
    idx on [0, src.shape[0]) holds; ``proof`` is the Verdict of
    ``check_inj(idx, 0, src.shape[0] - 1)`` when the caller already ran it (cache it
    with the inverse when idx is fixed), else the forward pass runs that check."""
    return GatherFn.apply(src, idx, injective, inverse, proof)[0]


def scatter(dst, idx, vals):
    return ScatterFn.apply(dst, idx, vals)


def scatter_add(dst, idx, vals):
    return ScatterAddFn.apply(dst, idx, vals)


def gather_segments(src, src_off, seg_src, out_off, inv_seg):
    """Segments of src (offsets src_off) in the order seg_src (a permutation of the
    segments; out_off the offsets of the result, inv_seg its inverse, e.g. the
    partition ``indices`` of the rows)."""
    return GatherSegmentsFn.apply(src, src_off, seg_src, out_off, inv_seg)[0]


def partition(payload, keys, pred, offsets=None, out_dtype=torch.int32):
    """Returns (payload_out, indices, num_true); only payload_out carries gradients."""
    return PartitionFn.apply(payload, keys, pred, offsets, out_dtype)
