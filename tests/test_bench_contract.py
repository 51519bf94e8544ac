"""Host-side pieces of bench.py: the measured-traffic lookup and the clock-sample parser."""
import dataclasses
import os

import pytest

import bench
import scenegen


def test_traffic_is_null_for_other_sizes_or_changed_sources(tmp_path, monkeypatch):
    cfg = scenegen.CONFIGS["frame800_bf16"]
    assert bench.measured_traffic(dataclasses.replace(cfg, width=400)) is None
    stale = tmp_path / "traffic.txt"
    stale.write_text("# header\nprecision=bf16 kernel=render_bf16_kernel source_sha256=00 bytes_per_launch=7\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(stale))
    assert bench.measured_traffic(cfg) is None
    fresh = tmp_path / "traffic2.txt"
    fresh.write_text(f"precision=bf16 kernel=render_bf16_kernel source_sha256={bench.kernel_source_hash('bf16')} "
                     "bytes_per_launch=7\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(fresh))
    assert bench.measured_traffic(cfg) == 7
    monkeypatch.setattr(bench, "TRAFFIC_FILE", os.path.join(str(tmp_path), "missing.txt"))
    assert bench.measured_traffic(cfg) is None


def test_kernel_source_hash_covers_every_listed_file():
    for precision, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2409_10327_gb300", "csrc", f)), f
        assert len(bench.kernel_source_hash(precision)) == 64


def test_clock_sampler_parses_clocks_and_throttle_reasons():
    class _Done:
        def terminate(self):
            pass

        def wait(self):
            return 0

    cs = bench.ClockSampler(0)
    cs.f.write("0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
               "0, 2055, 2070, 1390.1, 0x4, Not Active, Not Active, Not Active, Active\n"
               "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    cs.p = _Done()
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
