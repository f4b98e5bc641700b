"""Host logic of bench.py that decides what its JSON line reports (no GPU).

The clock record of the timed region (parsed from nvidia-smi samples) voids a
number that saw a hardware or thermal slowdown, or SM clocks stuck well below
their maximum with no reason active; power capping is kept. The roofline block
divides the pair's algorithmic bytes by its measured time and scales the ncu
traffic ratio by the same bytes. The defaults keep at least 3 warm-up steps.
"""
from types import SimpleNamespace

import pytest

import bench

NA = "Not Active"


def _line(sm, smax=2070, power=700.0, hw=NA, hw_th=NA, sw_th=NA, cap=NA):
    return f"{sm}, {smax}, {power}, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {cap}"


def test_clock_samples_are_summarised():
    lines = [_line(2070, power=650.5), _line(2055, power=720.25), _line(2070, cap="Active"),
             "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]", "garbage"]
    c = bench.ClockSampler.summarize(lines)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["power_w_max"] == 720.25
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler.summarize([])["sm_mhz"] is None


@pytest.mark.parametrize("field", ["hw", "hw_th", "sw_th"])
def test_a_slowdown_voids_the_timed_region(field):
    c = bench.ClockSampler.summarize([_line(2070), _line(1500, **{field: "Active"})])
    why = bench.clocks_rejected(c)
    assert why.startswith("slowdown")


def test_power_capping_is_kept():
    c = bench.ClockSampler.summarize([_line(1455, cap="Active")] * 5)
    assert bench.clocks_rejected(c) == ""


def test_clocks_stuck_low_with_no_reason_void_the_timed_region():
    c = bench.ClockSampler.summarize([_line(1200)] * 5)
    assert "no reason" in bench.clocks_rejected(c)
    assert bench.clocks_rejected(bench.ClockSampler.summarize([_line(2000)] * 5)) == ""


def test_no_clock_record_is_not_a_rejection():
    assert bench.clocks_rejected(None) == ""
    assert bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}) == ""


def test_one_rank_decides_alone():
    assert bench.agree_remeasure("", None) is False
    assert bench.agree_remeasure("slowdown: hw_slowdown", None) is True


def test_pair_roofline_arithmetic():
    # two LM steps, each with 9 pairs of 1e9 algorithmic bytes in 2 + 3 + 4 + 1 ms of pair phases
    st = SimpleNamespace(ms_phase=[100.0, 50.0, 2.0, 3.0, 4.0, 1.0, 7.0, 8.0], pair_bytes=9e9, n_pairs=9)
    peak = {"hbm_gbs": 5000.0, "source": "measured"}
    r = bench.pair_roofline([st, st], peak, 1)
    assert r["achieved"] == pytest.approx(18e9 / 20e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert r["bytes_per_pair"] == pytest.approx(1e9)
    assert r["ms_per_pair"] == pytest.approx(20.0 / 18)
    assert r["traffic"] == pytest.approx(bench.PAIR_DRAM_PER_ALG_BYTE[1] * 1e9)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert bench.pair_roofline([st], peak, 2)["traffic"] is None      # no capture for that format


def test_default_invocation_warms_up_at_least_three_steps():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.impl == "ours" and a.workload == "paper"
    assert a.warmup >= 3 and a.steps >= 1
