"""Host-side helpers of bench.py, without a GPU: the clock record taken
during the timed region (a run with thermal or hardware slowdown is rejected
on these fields), the algorithmic flop count of the roofline, and the
parameter selection (autotuned entry, then command-line overrides)."""
import argparse

import pytest

pytest.importorskip("torch")

import bench  # noqa: E402


def _line(sm, smax, hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 950.00, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {cap}"


def test_clock_record_median_max_and_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = [_line(2070, 2070), _line(2055, 2070, cap="Active"), "garbage", _line(2070, 2070),
                _line(1980, 2070, sw_th="Active"), "0, N/A, 2070, 1, 2, 3, 4, 5, 6"]
    rec = cs.stop()
    assert rec["samples"] == 4
    assert rec["sm_mhz"] == pytest.approx(2062.5)
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_clock_record_without_samples():
    rec = bench.ClockSampler(0).stop()
    assert rec == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_sweep_flops_counts_steps_and_unknowns():
    assert bench.sweep_flops(0, 0) == 0
    assert bench.sweep_flops(1000, 10) == 15 * 1000 + 9 * 10


def _args(**kw):
    base = dict(no_tuned=False, block=None, overlap=None, k=None, robin=None, levels=None, coarse_tol=None,
                final_rtol=None, device_loop=1)
    base.update(kw)
    return argparse.Namespace(**base)


def test_solver_params_tuned_then_overrides():
    prm, src = bench.solver_params(_args(), "fp32")
    assert "autotuned" in src and prm["overlap"] < prm["block"]
    prm2, src2 = bench.solver_params(_args(overlap=5, k=12, device_loop=0), "fp32")
    assert prm2["overlap"] == 5 and prm2["local_cg_iters"] == 12 and prm2["device_loop"] == 0
    assert "overlap overridden" in src2 and "device loops off" in src2
    prm4, src4 = bench.solver_params(_args(final_rtol=0.0), "fp32")
    assert prm4["final_local_rtol"] == 0.0 and "final_local_rtol overridden" in src4
    prm5, src5 = bench.solver_params(_args(ml_mode="correction", trigger=0.9, correction_cg=300, local_atol=0.5,
                                           local_rtol=0.02), "fp32")
    assert (prm5["ml_mode"], prm5["correction_trigger"], prm5["correction_cg"]) == ("correction", 0.9, 300)
    assert prm5["local_atol"] == 0.5 and prm5["local_rtol"] == 0.02 and "correction_cg overridden" in src5
    prm3, src3 = bench.solver_params(_args(no_tuned=True), "fp32")
    assert prm3 == bench.PAPER_DEFAULTS and src3.startswith("defaults")
