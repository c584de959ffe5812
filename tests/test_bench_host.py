"""Host-side pieces of the benchmark: clock-sample parsing and the peak source."""
import json
import os

import bench


def test_clock_rows_median_max_and_reasons():
    text = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1300.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, 1980, 2070, 1390.0, 0x8, Active, Not Active, Not Active, Active",
    ])
    c = bench.parse_clock_rows(text)
    assert c["samples"] == 3 and c["sm_mhz"] == 2055 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_rows_empty():
    assert bench.parse_clock_rows("") is None
    assert bench.parse_clock_rows("0, N/A, N/A, N/A, N/A, N/A, N/A, N/A, N/A") is None


def test_peak_is_the_measured_copy_bandwidth():
    peak, kind = bench._peaks()
    p = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        assert kind == "measured" and peak == float(json.load(open(p))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6800.0


def test_traffic_record_sources_exist_and_hash_is_stable():
    """The DRAM-traffic record is tied to the step kernel's own sources."""
    import os
    import bench
    for src in bench.TRAFFIC_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, src)), src
    h = bench.traffic_sources_sha256()
    assert len(h) == 64 and h == bench.traffic_sources_sha256()


def test_nvml_clock_samples_inside_or_bracketing_the_timed_region():
    """The NVML poller keeps the samples taken inside the timed region; when the
    region is shorter than one poll it keeps the polls on either side, and it
    names the active slowdown reasons."""
    import threading
    import time
    import bench

    def fake(rows, t_in):
        c = bench.Clocks.__new__(bench.Clocks)
        c.nv, c.rows, c.t_in, c.max_mhz = object(), rows, t_in, 2070.0
        c.stop_flag, c.th = threading.Event(), threading.Thread(target=lambda: None)
        c.th.start()
        return c

    now = time.perf_counter()
    c = fake([(now - 1.0, 1800.0, 0), (now - 0.4, 2070.0, 0x4), (now - 0.3, 2070.0, 0), (now + 10.0, 900.0, 0x40)],
             now - 0.5)
    r = c.stop()
    assert r["sm_mhz"] == 2070.0 and r["samples"] == 2 and r["reasons"] == ["sw_power_cap"]
    assert r["source"].endswith("inside the timed region")
    c = fake([(now - 2.0, 2000.0, 0), (now + 5.0, 2060.0, 0x8)], time.perf_counter())
    r = c.stop()
    assert r["samples"] == 2 and r["sm_mhz"] == 2030.0 and r["reasons"] == ["hw_slowdown"]
    assert "bracketing" in r["source"]
