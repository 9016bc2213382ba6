"""Host-side arithmetic of the benchmark line (CPU): throughput, the paper
ratio, and the DRAM-traffic lookup that goes null when a kernel changed."""
import json
import os

import pytest

import bench


def test_job_throughput_counts_every_rank_over_the_slowest_time():
    assert bench.job_throughput(1_000_000, 4, 20.0) == pytest.approx(4 * 1e6 / 0.02)


def test_paper_ratio_only_for_the_papers_exact_workloads():
    # Table 5: N = 1e9 in 121 s on the paper's desktop
    v = 3.5e9
    assert bench.paper_ratio("matern2d_table5", 1_000_000_000, v) == pytest.approx(v / (1e9 / 121.0))
    assert bench.paper_ratio("matern2d_table5", 10_000_000, v) is None      # not the paper's N
    assert bench.paper_ratio("matern2d_1e9", 1_000_000_000, v) is None      # no paper number


def test_traffic_lookup_is_null_for_a_changed_kernel():
    from paper_2210_10210_gb300 import build as B
    os.makedirs(B.OUT_DIR, exist_ok=True)
    path = os.path.join(B.OUT_DIR, "traffic_check.json")
    good = bench.kernel_fingerprint("spread")
    with open(path, "w") as f:
        json.dump({"kernels": {"spread": {"dram_bytes_per_point": 12.5, "src_sha1": good},
                               "bin_count": {"dram_bytes_per_point": 8.0, "src_sha1": "0" * 40}}}, f)
    assert bench.traffic_for("spread", 1000, path) == pytest.approx(12500.0)
    assert bench.traffic_for("bin_count", 1000, path) is None          # stale fingerprint
    assert bench.traffic_for("bin_scatter", 1000, path) is None        # absent
    assert bench.kernel_fingerprint("spread") != bench.kernel_fingerprint("bin_scatter")
