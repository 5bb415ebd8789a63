"""The committed ncu counters that bench.py turns into the raster backward's
roofline (executed instructions and FP32 flops per walked pair, DRAM bytes)
were taken on the kernel source as it stands: bench.py uses them only while
the source hash they record matches, and otherwise falls back to a nominal
flop model, so a stale file would silently change what the benchmark
reports."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _entry(name):
    with open(os.path.join(ROOT, "profiles", name)) as f:
        return json.load(f)["raster_backward"]


def test_counters_match_the_kernel_source():
    h = bench.kernel_source_hash()
    for name in ("flops_raster_backward.json", "traffic.json"):
        assert _entry(name)["source_hash"] == h, name


def test_counters_are_consistent():
    fl = _entry("flops_raster_backward.json")
    c = fl["counters"]
    flops = (2 * c["sm__sass_thread_inst_executed_op_ffma_pred_on.sum"]
             + c["sm__sass_thread_inst_executed_op_fadd_pred_on.sum"]
             + c["sm__sass_thread_inst_executed_op_fmul_pred_on.sum"]
             + 4 * c["sm__sass_thread_inst_executed_op_ffma2_pred_on.sum"]
             + 2 * c["sm__sass_thread_inst_executed_op_fadd2_pred_on.sum"]
             + 2 * c["sm__sass_thread_inst_executed_op_fmul2_pred_on.sum"])
    assert abs(fl["executed_fp32_flops"] - flops) <= 1e-9 * flops
    assert abs(fl["flops_per_pair"] - flops / fl["pairs_walked"]) <= 1e-9 * fl["flops_per_pair"]
    assert abs(fl["warp_inst_per_pair"] - c["smsp__inst_executed.sum"] / fl["pairs_walked"]) <= 1e-9
    tr = _entry("traffic.json")
    assert tr["dram_read_bytes"] == c["dram__bytes_read.sum"]
    assert tr["dram_write_bytes"] == c["dram__bytes_write.sum"]
    # the roofline's traffic at full size scales these bytes by the ratio of algorithmic bytes
    assert bench.ncu_traffic("raster_backward", tr["algorithmic_bytes"]) == \
        tr["dram_read_bytes"] + tr["dram_write_bytes"]
    assert bench.ncu_flops("raster_backward")["flops_per_pair"] == fl["flops_per_pair"]
