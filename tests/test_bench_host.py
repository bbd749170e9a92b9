"""Host-side helpers of the benchmark: the clock record and the CPU-baseline row sample."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_median_and_reasons():
    na = "Not Active"
    lines = [f"0, {mhz}, 2070, 900.5, 0x0, {na}, {na}, {na}, {cap}"
             for mhz, cap in ((2070, na), (2055, "Active"), (1980, na), (2070, na), (2040, na))]
    lines.append("garbage line")
    lines.append("0, [N/A], 2070, 1.0, 0x0, a, b, c, d")           # unparsable clock: skipped
    s = _sampler(lines)
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 5
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_thermal_reasons_and_empty_record():
    na = "Not Active"
    s = _sampler([f"0, 1500, 2070, 1400, 0x0, Active, {na}, Active, {na}"])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    e = _sampler([])
    assert e["sm_mhz"] is None and e["reasons"] == ["unsampled"] and e["samples"] == 0


def test_spread_rows_cover_edges_evenly():
    assert bench.spread_rows(128, 8) == [0, 16, 32, 48, 64, 80, 96, 112]
    assert bench.spread_rows(5, 99) == [0, 1, 2, 3, 4]              # capped at bd
    assert bench.spread_rows(10, 0) == [0]                           # at least one row
    r = bench.spread_rows(128, 8, offset=5)
    assert len(r) == 8 and all(0 <= x < 128 for x in r) and r == sorted(set(r))


def test_job_throughput_sums_ranks():
    assert bench.job_throughput(2.0e12, 1000.0, 4) == 8.0e12


def test_blas_threads_reads_the_pins(monkeypatch):
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.setenv(k, "1")
    assert bench.blas_threads() == 1
    monkeypatch.setenv("OMP_NUM_THREADS", "8")
    monkeypatch.setenv("MKL_NUM_THREADS", "junk")
    assert bench.blas_threads() == 8
