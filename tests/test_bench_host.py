"""Host logic of bench.py (CPU): the roofline entry, the DRAM figures it
takes from the committed ncu summaries, and the clock record."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_picks_the_level_that_serves_the_blocks():
    ceil = {"stream_gbs": 30_000.0, "chase_gbs": 10_000.0, "bytes": 28e6}
    # 10^6 crossings of 334 B in 1 ms: 334 GB/s
    r = bench.roofline(1_000_000, 334.0, 1.0, 28_000_000, ceil, traffic=1.5e8)
    assert r["achieved"] == pytest.approx(334.0)
    assert r["bound"] == "l2" and r["peak"] == 30_000.0
    assert r["frac"] == pytest.approx(334.0 / 30_000.0)
    assert r["frac_of_l2_chase"] == pytest.approx(334.0 / 10_000.0)
    assert r["traffic"] == 1.5e8 and r["unit"] == "GB/s"
    hbm, _ = bench.measured_peaks()
    assert r["frac_of_hbm"] == pytest.approx(334.0 / hbm)
    # blocks larger than half of L2 stream from HBM
    r = bench.roofline(1_000_000, 334.0, 1.0, int(bench.L2_BYTES), ceil)
    assert r["bound"] == "hbm" and r["peak"] == hbm and r["frac"] == pytest.approx(334.0 / hbm)
    assert r["traffic"] is None


def test_committed_traversal_summaries_match_the_kernel_source():
    """The DRAM bytes the bench reports come from ncu summaries keyed by a
    hash of the traversal's sources; both summaries must be current."""
    for name in ("trace_kernel_disk1e5.md", "trace_kernel_clumpy1e6.md"):
        v = bench.profiled(name, "dram bytes per full launch")
        assert v is not None and v > 0, name


def test_profiled_ignores_a_summary_of_another_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "x.md").write_text("kernel source hash: 0000000000000000\ndram bytes per full launch: 5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "1111111111111111")
    assert bench.profiled("x.md", "dram bytes per full launch") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.profiled("x.md", "dram bytes per full launch") == 5.0


class _FakeSmi:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _row(sm, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ", ".join("Active" if n in reasons else "Not Active" for n in names)
    return f"0, {sm}, 2070, 1000.0, 0x0, {flags}"


def test_clock_record_takes_the_loaded_median_and_the_reasons(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    cs = bench.ClockSampler(0)
    cs.p = _FakeSmi("\n".join([_row(1500)] * 2 + [_row(2070)] * 5 + [_row(2055, ("sw_power_cap",))]))
    r = cs.stop()
    # the lowest quarter of the samples (idle before the load) is left out
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 8}
    cs.p = _FakeSmi("\n".join([_row(2070)] * 3 + [_row(1800, ("hw_thermal_slowdown", "hw_slowdown"))]))
    r = cs.stop()
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    cs.p = _FakeSmi("")
    assert cs.stop() is None
