"""The allocation-free scan, for callers that cannot allocate device memory.

ixp_scan_noalloc keeps its scratch in a fixed array inside the library instead of
a caller-supplied workspace. Called through the C ABI, it must return exactly
what the workspace-based ixp_scan returns, and what the CPU oracle's scan returns,
on two calls in a row: the second call finds the first call's leftovers in the
shared array and must clear what it needs. The cases reach the largest size the
array holds, an empty input, and 4-byte-offset views (the scalar-load kernel).
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fn(lib):
    f = lib.ixp_scan_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    m = lib.ixp_scan_noalloc_max_n
    m.restype = ctypes.c_int64
    m.argtypes = [ctypes.c_int]
    return f, m


MAX_I32 = 2**26  # ixp_scan_noalloc_max_n(IXP_I32), checked below

CASES = [  # (input dtype, output dtype, n, inclusive, element offset of the views)
    (torch.int32, torch.int32, 1_000_003, False, 0),
    (torch.int32, torch.int64, 777_777, True, 0),
    (torch.int64, torch.int64, 300_001, False, 0),
    (torch.int32, torch.int32, 4096 * 37, True, 0),
    (torch.int32, torch.int32, MAX_I32, False, 0),
    (torch.int32, torch.int32, 0, False, 0),
    (torch.int32, torch.int32, 500_001, True, 1),
    (torch.int32, torch.int64, 123_457, False, 1),
]


def test_noalloc_scan_matches_workspace_scan_and_oracle_on_two_calls():
    import oracle
    import paper_2506_23058_gb300 as ixp
    lib = ixp.load()
    fn, max_n = _fn(lib)
    assert max_n(0) == MAX_I32
    dev = torch.device("cuda:0")
    code = {torch.int32: 0, torch.int64: 1}
    npt = {torch.int32: "int32", torch.int64: "int64"}
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        for case, (it, ot, n, inc, k) in enumerate(CASES):
            g = torch.Generator(device=dev)
            g.manual_seed(1000 * call + case)
            xb = torch.randint(-(2**20), 2**20, (n + k,), generator=g, device=dev, dtype=torch.int64).to(it)
            x = xb[k:]
            ref_out, ref_tot, ref_st = ixp.scan(x, ot, inclusive=inc)
            ob = torch.full((n + k,), -7, dtype=ot, device=dev)
            out = ob[k:]
            tot = torch.full((1,), -7, dtype=ot, device=dev)
            st = torch.full((1,), 99, dtype=torch.int32, device=dev)
            rc = fn(x.data_ptr() if n else xb.data_ptr(), code[it], out.data_ptr() if n else ob.data_ptr(), code[ot],
                    n, int(inc), tot.data_ptr(), st.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, (call, case)
            torch.cuda.synchronize(dev)
            assert int(st.item()) == 0 and int(ref_st.item()) == 0
            assert torch.equal(out, ref_out), (call, case)
            assert int(tot.item()) == int(ref_tot[0].item()), (call, case)
            o_out, o_tot = oracle.scan(x.cpu().numpy(), npt[ot], inclusive=bool(inc))
            assert (out.cpu().numpy() == o_out).all(), (call, case)
            assert int(tot.item()) == int(o_tot[0]), (call, case)


def test_noalloc_scan_rejects_sizes_beyond_its_array():
    import paper_2506_23058_gb300 as ixp
    fn, max_n = _fn(ixp.load())
    assert max_n(0) == 2**26 and max_n(1) == 2**25
    dev = torch.device("cuda:0")
    x = torch.zeros(8, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    # argument checks run before the pointers are used
    assert fn(x.data_ptr(), 0, x.data_ptr(), 0, max_n(0) + 1, 0, None, st.data_ptr(), None) == -1
    assert fn(x.data_ptr(), 1, x.data_ptr(), 1, max_n(1) + 1, 0, None, st.data_ptr(), None) == -1
    assert fn(x.data_ptr(), 1, x.data_ptr(), 0, 8, 0, None, st.data_ptr(), None) == -2
