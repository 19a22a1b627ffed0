"""Host-side pieces of bench.py that need no GPU: the clock-record parser that decides
whether a run saw throttling, and the peak lookup."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_parser_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1995, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
    ]
    out = bench.parse_clock_lines(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    hot = bench.parse_clock_lines(["0, 1500, 2070, 1, 0x8, Not Active, Active, Not Active, Not Active\n"])
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert bench.parse_clock_lines([])["sm_mhz"] is None


def test_peak_lookup_returns_a_bandwidth():
    gbs, src = bench.peaks()
    assert gbs > 1000 and src in ("measured", "fallback")


def test_extras_section_records_an_error_and_goes_on():
    """A failing block of the extras leaves its error under its key; the line is kept."""
    import bench
    out = {}
    with bench._section(out, "a"):
        raise RuntimeError("boom")
    with bench._section(out, "b"):
        out["b"] = 1
    assert out == {"a": {"error": "RuntimeError: boom"}, "b": 1}
