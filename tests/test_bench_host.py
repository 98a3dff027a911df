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


def test_synthetic_workloads_follow_their_stated_recipes():
    """The shapes the bench lines and the design notes quote: the array workload is
    60 stations (1770 baselines) x 144 dumps x 16 channels; the benchmark's 1e8
    visibilities need 35 dumps of 300 stations (44,850 baselines) x 64 channels; the
    64 batched images hold 1e5 to 2e6 visibilities each, 37.7M in all."""
    from paper_2301_06061_gb300 import synth

    a = synth.array()
    assert a.n_vis == 1770 * 144 * 16 == 4_078_080 and (a.n, a.n_w, a.fov) == (4096, 32, 0.2)
    assert a.rows_m.shape == (1770 * 144, 3) and a.chan_scale.size == 16
    assert -(-100_000_000 // (44_850 * 64)) == 35
    small = synth.large(n_vis=3_000_000)
    assert small.n_vis == 3_000_000 and small.rows_m.shape[1] == 3 and small.chan_scale.size == 64
    assert small.rows_m.shape[0] % 44_850 == 0
    c = synth.batched_counts()
    assert c.size == 64 and c.min() >= 100_000 and c.max() <= 2_000_000
    assert round(c.sum() / 1e6, 1) == 37.7


def test_oracle_extrapolation_scales_gridding_by_visibilities_and_the_rest_by_planes():
    """A sample plane of 4M of the job's 1e8 visibilities: gridding 2 s, the plane's image
    10 s (8 s of FFT, screen and correction).  The job grids all 1e8 visibilities (25x the
    sample) and transforms 32 planes."""
    job = bench.oracle_job_seconds(2.0, 10.0, 4_000_000, 100_000_000, 32)
    assert job == pytest.approx(25 * 2.0 + 32 * 8.0)
    # a sample with every visibility of the job: gridding is billed once
    assert bench.oracle_job_seconds(2.0, 10.0, 100, 100, 1) == pytest.approx(10.0)


def test_launch_traffic_scales_the_design_bytes_by_the_measured_ratios():
    r = {"grid_read": 1.13, "grid_write": 1.0, "cols_a_read": 1.02, "cols_a_write": 0.99, "cols_b_read": 1.0,
         "cols_b_write": 0.99}
    n, rows, kept = 16384, 224_000, 100_000_000
    row = 8.0 * n
    assert bench.launch_traffic("grid", n, 32, rows, kept, 1, ratios=r) == pytest.approx(1.13 * 32 * kept + rows * row)
    assert bench.launch_traffic("cols_a", n, 32, rows, kept, 1, ratios=r) == pytest.approx(
        1.02 * rows * row + 0.99 * 32 * S)
    assert bench.launch_traffic("cols_b", n, 32, rows, kept, 1, ratios=r) == pytest.approx(32 * S + 0.99 * S)
    assert bench.launch_traffic("sort", n, 32, rows, kept, 1, ratios=r) is None
