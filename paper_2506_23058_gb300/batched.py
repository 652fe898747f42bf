"""Batched pipeline over a jagged array: one persistent launch (ixp_batch_run) per
step, captured in a CUDA graph and replayed.

For shape[m] (segment sizes, n = sum(shape) int32 elements) one launch computes the
flag array (mkSgmDescr), the stable per-segment partition of the keys
(partition2L), and per-segment Mono< of `iota`, Inj and Bij of `chk`. The work list
is the segments in decreasing length (longest-processing-time order), built once on
the host from the shape. The launch shape comes from the autotuner's cache when one
exists for this GPU and workload size.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import ixp, tune

DEFAULT_TUNING = (256, 2, 16, 4)


class BatchRunner:
    def __init__(self, shape, keys, pred, chk, iota, tuning=None, device=None):
        dev = torch.device(device) if device is not None else keys.device
        shape_np = shape.cpu().numpy() if isinstance(shape, torch.Tensor) else np.asarray(shape, dtype=np.int64)
        self.m = int(shape_np.shape[0])
        self.n = int(shape_np.sum())
        if keys.numel() != self.n or chk.numel() != self.n or iota.numel() != self.n:
            raise ValueError("keys, chk and iota must each hold sum(shape) elements")
        self.device = dev
        self.shape = torch.as_tensor(shape_np, dtype=torch.int64).to(dev)
        self.order = torch.as_tensor(np.argsort(-shape_np, kind="stable").astype(np.int32)).to(dev)
        self.keys, self.chk, self.iota = keys, chk, iota
        self.pred = ixp.make_pred(pred)
        self.flags = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.indices = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.num_true = torch.empty(self.m, dtype=torch.int64, device=dev)
        self.offsets = torch.empty(self.m + 1, dtype=torch.int64, device=dev)
        self.seg_ok = torch.empty(3 * self.m, dtype=torch.uint8, device=dev)
        self.first_bad = torch.empty(3, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        if tuning is None:
            tuning = tune.lookup(self.n, self.m) or DEFAULT_TUNING
        self.set_tuning(tuning)
        self.graph = None

    def set_tuning(self, tuning):
        self.tuning = ixp.BatchTuning(*tuning)
        need = int(ixp.load().ixp_batch_workspace_size(C.byref(self.tuning)))
        self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        self.graph = None

    def run(self, stream=None):
        rc = ixp.load().ixp_batch_run(
            self.shape.data_ptr(), self.m, self.keys.data_ptr(), self.pred, self.chk.data_ptr(),
            self.iota.data_ptr(), self.n, self.order.data_ptr(), self.flags.data_ptr(), self.indices.data_ptr(),
            self.num_true.data_ptr(), self.offsets.data_ptr(), self.seg_ok.data_ptr(), self.first_bad.data_ptr(),
            self.status.data_ptr(), C.byref(self.tuning), self.ws.data_ptr(), self.ws.numel(),
            ixp._stream(stream))
        if rc != 0:
            raise ixp.IxpError(rc, "batch_run")

    def capture(self):
        """Records one step in a CUDA graph (warm-up on a side stream first)."""
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.run(s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def results(self):
        m = self.m
        ok = self.seg_ok.cpu().numpy()
        return {"flags": self.flags, "indices": self.indices, "num_true": self.num_true, "offsets": self.offsets,
                "mono_ok": ok[:m], "inj_ok": ok[m:2 * m], "bij_ok": ok[2 * m:],
                "first_bad": self.first_bad.cpu().tolist(), "status": int(self.status.item())}

    def algorithmic_bytes(self):
        # keys, iota, chk read; flags, indices written; shape read, offsets and counts written
        return 20 * self.n + 8 * self.m + 8 * (self.m + 1) + 8 * self.m
