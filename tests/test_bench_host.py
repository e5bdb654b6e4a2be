"""Host-side logic of bench.py that needs no GPU: the clock and throttle-reason
summary parsed from nvidia-smi samples, and the per-rank pair seeds."""
import bench


def test_clock_summary_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.lines = [
        "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
        "2040, 2070, 1350.0, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1200.5, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 1.0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_clock_summary_reports_thermal_slowdown():
    c = bench.ClockSampler(0)
    c.lines = ["1500, 2070, 1400.0, Active, Not Active, Active, Not Active"]
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_pair_ids_disjoint_across_ranks_and_steps():
    seen = set()
    for rank in range(4):
        for step in range(6):
            ids = bench.pair_ids(rank, step, 128)
            assert len(ids) == 128 and not (seen & set(ids))
            seen |= set(ids)


def test_bench_schedule_is_the_library_calibrated_schedule():
    """The oracle arm needs the benchmark's tolerance schedule without a GPU, so
    bench.py keeps its own copy; it must equal the library's
    w1_options.schedule = 1 table (a host-only call)."""
    from paper_1810_00118_gb300 import w1
    for norm in bench.NORMS:
        scale, alpha, theta, ratio = w1.calibrated_schedule(norm)
        assert scale == bench.TOL_SCALE[norm] and alpha == bench.ALPHA[norm] and theta == bench.THETA[norm]
        assert ratio == bench.RATIO[norm]
