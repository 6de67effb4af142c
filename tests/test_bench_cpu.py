"""Host logic of bench.py (CPU): clock-sample parsing, the algorithmic flop
counts and the roofline arithmetic of the dominant kernel."""
import bench


def test_clock_samples_median_max_and_reasons():
    lines = [
        "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active\n",
        "1980, 2070, 1390.0, Not Active, Not Active, Not Active, Active\n",
        "2010, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active\n",
        "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active\n",   # unreadable sample
        "garbage\n",
    ]
    out = bench.parse_clock_samples(lines)
    assert out == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.parse_clock_samples([]) is None
    hot = bench.parse_clock_samples(["1500, 2070, 1400, Active, Not Active, Active, Not Active\n"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_flop_counts_two_and_three_fluids():
    # two fluids in 3-D: cons->prim 22, WENO5 107 x 7 fields, HLLC 122, divergence 18
    assert bench.flops_cell_dir(2, 3, 5) == 22 + 107 * 7 + 122 + 18 == 911
    assert bench.flops_cell_dir(2, 3, 3) == 22 + 38 * 7 + 122 + 18 == 428
    # last sweep: accumulate 7 + stage update 28 + a third of the wave speed 45
    assert bench.flops_cell_dir() + bench.flops_last_sweep_extra() == 961
    # each added fluid adds two fields (partial density and volume fraction)
    assert bench.flops_cell_dir(3, 3, 5) - bench.flops_cell_dir(2, 3, 5) == 6 + 107 * 2 + 19 + 2 * 2 + 4
    assert bench.flops_cell_dir(3, 3, 5) == 1158


def test_roofline_of_the_dominant_kernel():
    ncell = 256 ** 3
    res = {"kernels": {"sweep_x": (3 * 38.0, 3), "sweep_y": (3 * 38.5, 3), "sweep_z": (3 * 40.0, 3),
                       "step_begin": (0.03, 1)},
           "ncell": ncell, "neq": 7, "grind": 1.0}
    r = bench.roofline_for("fp64", res, 1.23, "measured", 6782.1, "measured")
    # FP64 forms: algorithmic operations per second against the FP64
    # instruction rate, i.e. the FMA probe's TFLOP/s over 2 flops per FMA
    assert r["kernel"] == "sweep_z" and r["bound"] == "alu" and r["unit"] == "Top/s"
    achieved = 961 * ncell / 40.0e-3 / 1e12
    assert abs(r["peak"] - 0.615) < 1e-4
    assert abs(r["achieved"] - achieved) < 1e-4 and abs(r["frac"] - achieved / 0.615) < 1e-4
    assert abs(r["share_of_step"] - 120.0 / (114.0 + 115.5 + 120.0 + 0.03)) < 1e-3
    # algorithmic HBM bytes: 8/3 state arrays of FP64 per cell, equation and RHS
    assert abs(r["hbm"]["achieved_gbs"] - 21.3) < 0.06
    # three fluids: 9 equations, the N-fluid count
    res3 = dict(res, neq=9)
    r3 = bench.roofline_for("fp64_3fluid", res3, 1.23, "measured", 6782.1, "measured")
    assert r3["algorithmic_flops_per_cell"] == 1220.0
    assert r3["traffic"] is None and r3["pipe_busy_ncu"] is None   # only the base forms carry ncu figures
    # the reorganised FP64 form contracts FMAs: TFLOP/s at 2 flops per FMA
    rf = bench.roofline_for("fp64_fast", res, 1.23, "measured", 6782.1, "measured")
    assert rf["unit"] == "TFLOP/s" and rf["peak"] == 1.23
    # FP32 forms: TFLOP/s against the FP32 probe at 2 flops per FMA
    rm = bench.roofline_for("mixed", res, 77.5, "measured", 6782.1, "measured")
    assert rm["unit"] == "TFLOP/s" and rm["peak"] == 77.5
    assert abs(rm["frac"] - achieved / 77.5) < 1e-4
    # algorithmic HBM bytes of the mixed form: 16 B per cell, equation and RHS
    assert abs(rm["hbm"]["achieved_gbs"] - 16.0) < 1e-9


def test_timed_steps_split_into_regions():
    assert bench.split_steps(20) == [4, 4, 4, 4, 4]
    assert bench.split_steps(12) == [3, 3, 2, 2, 2]
    assert bench.split_steps(3) == [1, 1, 1]
    assert bench.split_steps(1) == [1]
    for k in range(1, 40):
        parts = bench.split_steps(k)
        assert sum(parts) == k and min(parts) >= 1 and len(parts) == min(5, k)


def test_cpu_baseline_entry_states_the_host():
    b = bench.baseline_entry(100.0, "a sample")
    n = b["host"]["nproc"]
    assert n >= 1 and b["cores"] == 1 and b["kind"] == "oracle"
    assert abs(b["ideal_scaling_all_cores"]["value"] - 100.0 / n) < 1e-3
    assert b["ideal_scaling_all_cores"]["cores"] == n


def test_both_arms_quote_the_same_config():
    assert bench.headline_config(n_gpus=2) == bench.headline_config(256 ** 3, 7, 2)
