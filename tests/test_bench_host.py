"""Host-side arithmetic of bench.py's roofline report (no GPU)."""
import pytest

import bench

S = 8 * 16384 ** 2  # one complex64 plane of the benchmark workload


def test_stage_bytes_of_the_benchmark_design():
    n_vis = 100_000_000
    assert bench.stage_bytes("sort", 16384, 32, 1, 1, n_vis, n_vis) == 52 * n_vis
    assert bench.stage_bytes("grid", 16384, 32, 1, 1, n_vis, n_vis) == 32 * S + 32 * n_vis
    assert bench.stage_bytes("cols_a", 16384, 32, 1, 1, n_vis, n_vis) == 64 * S
    assert bench.stage_bytes("cols_b", 16384, 32, 1, 1, n_vis, n_vis) == 33 * S
    # planes streamed in 4 chunks: per launch a quarter of the planes, the image once over the chunks
    assert bench.stage_bytes("cols_b", 16384, 32, 4, 1, n_vis, n_vis) == 8 * S + S / 4
    # oversampled grid: planes of (2n)^2, the image n^2
    assert bench.stage_bytes("cols_b", 4096, 32, 1, 1, 0, 0, 2) == 32 * 4 * 8 * 4096 ** 2 + 8 * 4096 ** 2


def test_step_roofline_sums_the_stages_and_states_the_all_resident_floor():
    n_vis = 100_000_000
    ms = {"sort": 3.9, "grid": 20.0, "rows": 0.0, "cols_a": 19.7, "cols_b": 20.2}
    r = bench.step_roofline(ms, 16384, 32, 1, 1, n_vis, n_vis, 1, 63.8, 6769.4)
    total = 52 * n_vis + (32 * S + 32 * n_vis) + 64 * S + 33 * S
    assert r["bytes"] == total == 285_425_390_592
    assert r["all_resident_floor_bytes"] == 129 * S == 277_025_390_592  # 4 S per plane + S
    assert r["achieved"] == pytest.approx(total / 63.8e-3 / 1e9, abs=0.1)
    assert r["frac"] == pytest.approx(total / 63.8e-3 / 1e9 / 6769.4, abs=1e-4)
    assert r["frac_of_all_resident_floor"] == pytest.approx(129 * S / 63.8e-3 / 1e9 / 6769.4, abs=1e-4)
