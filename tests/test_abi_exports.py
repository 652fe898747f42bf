"""The C ABI library builds (nvcc cross-compiles for sm_103a without a GPU), loads,
and exports every function that include/ixp.h declares. No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ixp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ixp_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["ixp_check_range", "ixp_check_mono", "ixp_check_inj", "ixp_check_bij", "ixp_check_filtpart",
                 "ixp_scan", "ixp_partition", "ixp_scatter", "ixp_gather", "ixp_flags_from_shape",
                 "ixp_workspace_size", "ixp_strerror"]:
        assert want in names


@pytest.fixture(scope="module")
def lib():
    from paper_2506_23058_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_helpers(lib):
    lib.ixp_strerror.restype = ctypes.c_char_p
    assert lib.ixp_strerror(0) == b"ok"
    assert b"span" in lib.ixp_strerror(-3)
    lib.ixp_workspace_size.restype = ctypes.c_size_t
    lib.ixp_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64]
    assert lib.ixp_workspace_size(0, 0, 1 << 20, 0) == 256
    # Inj: header + two bitmaps of span bits
    assert lib.ixp_workspace_size(2, 0, 1 << 20, 1 << 20) >= 256 + 2 * (1 << 17)
    assert lib.ixp_workspace_size(99, 0, 10, 0) == 0
    assert lib.ixp_version() >= 100


def test_invalid_arguments_are_rejected_on_the_host(lib):
    # argument checks run before any CUDA call, so they work without a GPU
    v = ctypes.c_void_p(16)
    lib.ixp_check_range.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    assert lib.ixp_check_range(v, 7, 10, 0, 1, v, v, 256, None) == -2      # bad dtype
    assert lib.ixp_check_range(v, 0, -1, 0, 1, v, v, 256, None) == -1      # n < 0
    assert lib.ixp_check_range(v, 0, 10, 5, 1, v, v, 256, None) == -1      # lo > hi
    assert lib.ixp_check_range(v, 0, 10, 0, 1, v, None, 256, None) == -4   # no workspace
    assert lib.ixp_check_range(v, 0, 10, 0, 1, v, ctypes.c_void_p(512), 8, None) == -4  # too small


def test_segmented_and_hist_arguments_rejected_on_the_host(lib):
    v, odd = ctypes.c_void_p(256), ctypes.c_void_p(258)  # 258: not 4-byte aligned
    I64, SZ, P = ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
    lib.ixp_sgm_scan.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, I64, ctypes.c_int, P, P, SZ, P]
    assert lib.ixp_sgm_scan(v, v, 7, v, 0, 10, 1, None, v, 1 << 20, None) == -2    # bad input type
    assert lib.ixp_sgm_scan(v, v, 1, v, 0, 10, 1, None, v, 1 << 20, None) == -2    # int64 into int32
    assert lib.ixp_sgm_scan(v, v, 0, v, 0, -1, 1, None, v, 1 << 20, None) == -1    # n < 0
    assert lib.ixp_sgm_scan(None, v, 0, v, 0, 10, 1, None, v, 1 << 20, None) == -1  # no flags
    assert lib.ixp_sgm_scan(v, odd, 0, v, 0, 10, 1, None, v, 1 << 20, None) == -1  # misaligned values
    assert lib.ixp_sgm_scan(v, v, 0, v, 0, 10, 1, None, v, 8, None) == -4          # workspace too small
    lib.ixp_mkii.argtypes = [P, I64, P, ctypes.c_int, I64, P, P, SZ, P]
    assert lib.ixp_mkii(v, 4, v, 7, 10, None, v, 1 << 20, None) == -2   # bad output type
    assert lib.ixp_mkii(v, -1, v, 0, 10, None, v, 1 << 20, None) == -1  # m < 0
    assert lib.ixp_mkii(v, 0, v, 0, 10, None, v, 1 << 20, None) == -1   # positions but no segment
    assert lib.ixp_mkii(v, 4, odd, 0, 10, None, v, 1 << 20, None) == -1  # misaligned output
    assert lib.ixp_mkii(v, 4, v, 0, 0, None, None, 0, None) == 0        # nothing to do
    assert lib.ixp_mkii(v, 4, v, 0, 10, None, v, 8, None) == -4         # workspace too small
    lib.ixp_hist_min.argtypes = [P, ctypes.c_int, I64, P, ctypes.c_int, P, I64, P]
    assert lib.ixp_hist_min(v, 7, 4, v, 0, None, 10, None) == -2   # bad H type
    assert lib.ixp_hist_min(v, 0, 4, v, 9, None, 10, None) == -2   # bad index type
    assert lib.ixp_hist_min(v, 0, -1, v, 0, None, 10, None) == -1  # m < 0
    assert lib.ixp_hist_min(v, 0, 4, None, 0, None, 10, None) == -1  # no indices
    assert lib.ixp_hist_min(odd, 0, 4, v, 0, None, 10, None) == -1  # misaligned H
    assert lib.ixp_hist_min(v, 0, 0, v, 0, None, 10, None) == 0    # empty H: nothing lands
    lib.ixp_smallest_pairs.argtypes = [P, P, ctypes.c_int, I64, I64, I64, P, P, P, P, SZ, P]
    assert lib.ixp_smallest_pairs(v, v, 7, 10, 4, 10, v, v, v, v, 1 << 20, None) == -2    # bad type
    assert lib.ixp_smallest_pairs(v, v, 0, -1, 4, 10, v, v, v, v, 1 << 20, None) == -1    # n < 0
    assert lib.ixp_smallest_pairs(v, v, 0, 10, 4, 10, v, v, None, v, 1 << 20, None) == -1  # no count
    assert lib.ixp_smallest_pairs(v, odd, 0, 10, 4, 10, v, v, v, v, 1 << 20, None) == -1   # misaligned
