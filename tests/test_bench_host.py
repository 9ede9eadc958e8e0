"""Host-side pieces of bench.py, without a GPU: the clock samples' parsing
(the median SM clock under load and the throttle reasons that reject a
run), the whole-job rate, the roofline arithmetic and the hash that ties
the ncu traffic record to the compositing kernel's sources."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(uuid, sm, smax, active=("Not Active",) * 4):
    return ", ".join(["0", uuid, str(sm), str(smax), "900.5", "0x0", *active])


def _sampler(tmp_path, lines, uuid):
    s = bench.ClockSampler(uuid)
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    s.path, s.proc = str(p), _Done()
    return s.stop()


def test_clock_samples_median_under_load_and_reasons(tmp_path):
    lines = [_row("GPU-a", 345, 2070)] + [_row("GPU-a", f, 2070) for f in (2070, 2055, 2070)]
    lines += [_row("GPU-b", 900, 2070)]                          # another GPU: ignored
    lines += [_row("GPU-a", 2040, 2070, ("Not Active", "Not Active", "Not Active", "Active"))]
    c = _sampler(tmp_path, lines, "GPU-a")
    assert c["samples"] == 5
    assert c["sm_max_mhz"] == 2070.0
    assert c["sm_mhz"] == 2062.5              # idle sample (345 MHz) left out of the median
    assert c["reasons"] == ["sw_power_cap"]
    thermal = [_row("GPU-a", 1800, 2070, ("Not Active", "Active", "Not Active", "Not Active"))]
    assert _sampler(tmp_path, thermal, "GPU-a")["reasons"] == ["hw_thermal_slowdown"]
    assert _sampler(tmp_path, [], "GPU-a")["reasons"] == ["no samples"]


def test_job_rate_counts_every_rank_over_the_slowest_time():
    assert bench.job_rate(4_531_200, 1, 1.0) == pytest.approx(4531.2)
    assert bench.job_rate(4_531_200, 4, 2.0) == pytest.approx(4 * 4531.2 / 2)


def test_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "sm_count", lambda: 152)
    monkeypatch.setattr(bench, "peaks", lambda: {"sm_max_mhz": 2070.0, "hbm_gbs": 6780.0})
    seq = np.array([[0.1, 0.12, 0.13, 0.36], [0.09, 0.12, 0.15, 0.51]])
    r = bench.roofline(seq, 0.85, seq, {})
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["peak"] == pytest.approx(peak) and r["bound"] == "alu"
    work = json.load(open(os.path.join(ROOT, "tests", "golden", "bench_work.json")))
    pairs = [work["views"][v]["evaluated_pairs"] for v in ("fisheye", "pinhole")]
    tflops = sum(pairs) * bench.FLOP_PER_PAIR / 0.85e-3 / 1e12
    assert r["achieved"] == pytest.approx(tflops) and r["frac"] == pytest.approx(tflops / peak)
    assert r["per_view_achieved_alone"][1] == pytest.approx(
        pairs[1] * bench.FLOP_PER_PAIR / 0.51e-3 / 1e12)
    # the traffic record counts only for the kernel sources it was taken on
    monkeypatch.setattr(bench, "kernel_source_hash", lambda read=None: "not the recorded one")
    assert bench.roofline(seq, 0.85, seq, {})["traffic"] is None
    s = bench.stage_rooflines(seq, pairs, 1_000_000)
    assert s["per_view"][0]["project_gbs"] == pytest.approx(336e6 / 0.1e-3 / 1e9)
    assert s["per_view"][1]["bin_tile_sort_frac"] == pytest.approx(
        36 * pairs[1] / 0.15e-3 / 1e9 / 6780.0)


def test_kernel_source_hash_follows_the_kernel_and_the_record_layout():
    files = {n: open(os.path.join(ROOT, "paper_2510_12901_gb300", "csrc", n), "rb").read()
             for n in bench.KERNEL_SOURCES + ("internal.h",)}
    base = bench.kernel_source_hash(lambda n: files[n])
    assert base == bench.kernel_source_hash()
    for n in bench.KERNEL_SOURCES:
        changed = dict(files)
        changed[n] = files[n] + b"\n"
        assert bench.kernel_source_hash(lambda k: changed[k]) != base, n
    inc = files["internal.h"]
    rec = inc.index(b"struct __align__(16) GRec")
    elsewhere = dict(files, **{"internal.h": b"// note\n" + inc})
    assert bench.kernel_source_hash(lambda k: elsewhere[k]) == base
    layout = dict(files, **{"internal.h": inc[:rec] + inc[rec:].replace(b"float4 rect;",
                                                                         b"float4 box;", 1)})
    assert bench.kernel_source_hash(lambda k: layout[k]) != base
