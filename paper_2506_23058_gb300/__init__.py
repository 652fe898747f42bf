"""GB300 (sm_103a) runtime checks of the index-array properties of arXiv 2506.23058
(Range, Monotonic, Inj, Bij, FiltPart/InvFiltPart) and the scan / scatter /
gather / partition / mkSgmDescr combinators that build and use such arrays.

The compute path is the CUDA library built from ``csrc/`` (C ABI: include/ixp.h);
this package only marshals torch tensors into it. There is no CPU fallback.
"""
from . import autograd, batched, tune  # noqa: F401
from .ixp import (I64MAX, I64MIN, IxpError, Verdict, check_bij, check_bij_seg, check_filtpart,
                  check_filtpart_values, check_inj,
                  check_inj_hist, check_inj_seg, check_mono,  # noqa: F401
                  check_range, debug_set_wait, f32_to_f64, f64_to_f32, filtpart_classes, flags_from_shape, gather,
                  gather_segments, hist_min, invert, mkii, sgm_scan, smallest_pairs,
                  lib_path, load,
                  make_pred,
                  partition, scan, scatter, scatter_add_f64, workspace, workspace_size)

__all__ = ["check_range", "check_mono", "check_inj", "check_inj_hist", "hist_min", "smallest_pairs", "check_bij", "check_inj_seg", "check_bij_seg", "check_filtpart", "check_filtpart_values", "filtpart_classes", "scan", "partition", "scatter",
           "scatter_add_f64", "f64_to_f32", "f32_to_f64", "invert", "gather", "gather_segments", "mkii", "sgm_scan", "flags_from_shape", "Verdict", "IxpError", "load", "lib_path",
           "workspace", "workspace_size", "make_pred", "debug_set_wait", "I64MIN", "I64MAX"]
