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
