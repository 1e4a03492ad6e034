"""The DRAM-traffic records that bench.py reports beside its rooflines belong
to the kernel sources in the tree: every record's fingerprint is the current
source's, so a kernel changed after its ncu capture cannot keep reporting
the old traffic, and each record's bytes per row sit within 10 % of the
kernel's algorithmic plus fused bytes."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# algorithmic + fused bytes per row (k = 28 slots): FP32 pressure SpMV
# 28 (4 + 4) + 2 * 4 + 3 * 4, FP64 pressure SpMV 28 (4 + 8) + 2 * 8 + 3 * 8,
# FP64 viscous SpMV with two right sides 28 (4 + 8) + 2 (8 + 8) + 2 * 8
EXPECTED = {"k_spmv_pc_fp32": 244, "k_spmv_pc_fp64": 376, "k_spmv_p_fp64_2rhs": 384}


def records():
    out = {}
    for line in open(os.path.join(ROOT, "profiles", "dram_traffic.txt")):
        f = line.split("#")[0].split()
        if len(f) >= 4:
            out[f[0]] = (float(f[1]), float(f[2]), f[3])
    return out


def test_every_reported_kernel_has_a_current_record():
    rec = records()
    assert set(EXPECTED) <= set(rec)
    for key in EXPECTED:
        assert rec[key][2] == bench.spmv_source_sha(key), key
        assert bench.profiled_traffic(key, 1000) is not None


def test_recorded_traffic_matches_the_algorithmic_bytes():
    for key, (nbytes, rows, _) in records().items():
        per_row = nbytes / rows
        assert abs(per_row - EXPECTED[key]) < 0.1 * EXPECTED[key], (key, per_row)


def test_viscous_roofline_arithmetic():
    """bench.py's roofline of the viscous SpMV: 4 (k + 1) flops per row against
    the measured FP64 FMA rate, 12 k + 32 algorithmic bytes per row against
    HBM; absent without the profiled timing."""
    r = {"vspmv_batch_launches": 20, "vspmv_batch_ms": 20 * 0.25}
    v = bench.viscous_roofline(r, 1_000_000, 28, 5000.0, "measured", 1000.0, {"p": 1})
    assert v["bound"] == "alu" and v["unit"] == "TFLOP/s"
    assert abs(v["achieved"] - 1e6 * 116 / 0.25e-3 / 1e12) < 1e-12
    assert abs(v["frac"] - v["achieved"] / 1.0) < 1e-12
    assert v["hbm"]["bytes_per_row"] == 368
    assert abs(v["hbm"]["achieved"] - 1e6 * 368 / 0.25e-3 / 1e9) < 1e-9
    assert v["pressure_spmv"] == {"p": 1}
    assert bench.viscous_roofline({}, 1, 28, 1.0, "m", 1.0, None) is None
    assert bench.viscous_roofline(r, 1, 28, 1.0, "m", 0.0, None) is None
