"""bench.py's host-side bookkeeping on CPU: the algorithmic bytes each op of the
step is credited with (the per-element figures the roofline uses), the kernel
named for each op, the workload description and the peak it divides by."""
import json
import os

import pytest

bench = pytest.importorskip("bench")

N32, N64 = 1 << 28, 1 << 27


def test_algorithmic_bytes_per_op():
    ops = {name: (kind, inputs, nbytes) for name, kind, inputs, nbytes in bench.make_ops(N32, N64)}
    for tag, n, es in (("i32", N32, 4), ("i64", N64, 8)):
        # the checks read the index array once
        for op in ("range_perm", "range_oor", "mono_le", "mono_brk"):
            assert ops[f"{op}_{tag}"][2] == es * n
        # Inj / Bij also clear and count a bitmap of span bits (span = n here)
        for op in ("inj_perm", "inj_dup", "bij_perm", "bij_dup"):
            assert ops[f"{op}_{tag}"][2] == es * n + 2 * (n // 8)
    assert ops["scan_i32"][2] == 8 * N32  # 4 in + 4 out
    assert ops["partition_p50"][2] == ops["partition_p01"][2] == 16 * N32  # key + payload in and out
    assert ops["filtpart_p50"][2] == 8 * N32  # Z + key
    # 2^26 rows of 32 bytes by a 4-byte index: index + row read + row write
    assert ops["scatter_rows8"][2] == ops["gather_rows8"][2] == (4 + 32 + 32) * (N32 // 4)
    assert ops["flags_from_shape"][2] is None  # filled in from the drawn shape
    assert bench.flags_bytes(4096, 1000) == 8 * 4096 + 8 * 4097 + 4 * 1000
    assert len(ops) == 23


def test_inj_bij_design_traffic():
    # the bucketed design reads the elements once and writes and reads a 4-byte pool
    # entry per element; other ops carry no design figure
    assert bench.inj_design_bytes("inj_perm_i32", N32, N64) == 12 * N32
    assert bench.inj_design_bytes("bij_dup_i64", N32, N64) == 16 * N64
    assert bench.inj_design_bytes("range_perm_i32", N32, N64) is None
    assert bench.inj_design_bytes("scan_i32", N32, N64) is None


def test_every_op_names_its_kernel():
    for name, _, _, _ in bench.make_ops(N32, N64):
        assert bench.OP_KERNELS.get(name), name


def test_workload_and_peak():
    c = bench.arm_config(N32, N64, False, 1)
    assert c["n_i32"] == N32 and c["n_i64"] == N64 and c["parallelism"] == "replicas x1"
    assert "larger than L2" in c["l2"]
    peak, source = bench.peaks()
    path = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert source == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert source == "fallback" and peak == 6800.0


def test_per_op_record_and_elements():
    assert bench.op_elements("range_perm_i32", N32, N64, 7) == N32
    assert bench.op_elements("inj_dup_i64", N32, N64, 7) == N64
    assert bench.op_elements("scatter_rows8", N32, N64, 7) == N32 // 4
    assert bench.op_elements("flags_from_shape", N32, N64, 7) == 7
    r = bench.op_record(2.0, 4 * 10**9, 10**9, 8000.0)  # 4 GB and 1 G elements in 2 ms
    assert r["gbs"] == 2000.0 and r["gelem_s"] == 500.0 and r["frac"] == 0.25
    assert r["frac_nominal"] == round(2000.0 / bench.NOMINAL_HBM_GBS, 4)


def test_host_info():
    h = bench.host_info()
    assert h["nproc"] == os.cpu_count() and isinstance(h["cpu_model"], str) and h["cpu_model"]


def test_host_info_names_arm_parts(tmp_path):
    f = tmp_path / "cpuinfo"
    f.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n\n"
                 "processor\t: 1\nCPU part\t: 0xd4f\n")
    assert "Neoverse V2" in bench.host_info(str(f))["cpu_model"]
    f.write_text("processor\t: 0\nmodel name\t: Example CPU @ 2.0GHz\n")
    assert bench.host_info(str(f))["cpu_model"] == "Example CPU @ 2.0GHz"


def test_roofline_takes_the_slowest_op_and_reports_families(tmp_path):
    peak = 8000.0
    per_op = {"range_perm_i32": bench.op_record(0.2, 4 * 10**9 // 5, 1, peak),
              "inj_perm_i32": bench.op_record(1.0, 10**9, 1, peak),
              "bij_dup_i32": bench.op_record(3.0, 10**9, 1, peak),
              "scatter_rows8": bench.op_record(2.0, 4 * 10**9, 1, peak)}
    tf = tmp_path / "traffic.json"
    tf.write_text(json.dumps({"ops": {"bij_dup_i32": {"bytes": 1234}}}))
    r = bench.roofline_of(per_op, peak, "measured", traffic_file=str(tf))
    assert r["op"] == "bij_dup_i32" and r["traffic"] == 1234 and r["achieved"] == per_op["bij_dup_i32"]["gbs"]
    assert r["frac"] == round(per_op["bij_dup_i32"]["gbs"] / peak, 4)
    fam = r["families"]["inj_bij"]
    assert fam["ops"] == 2 and fam["ms"] == 4.0 and fam["gbs"] == 500.0 and fam["frac"] == 0.0625
    assert r["families"]["range_mono"]["ops"] == 1
    # no summary for the op: traffic unknown
    r = bench.roofline_of(per_op, peak, "measured", traffic_file=str(tmp_path / "none.json"))
    assert r["traffic"] is None
