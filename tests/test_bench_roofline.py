"""bench.py's roofline arithmetic for the tensor-core apply (CPU): algorithmic flops per solve,
the measured-peak denominator, the DRAM traffic reported only for the workload it was captured
on, and the issued rate of the hi/lo launches."""
import numpy as np
import pytest

import bench


def test_algorithmic_work_is_two_applies_per_iteration_plus_the_first_source_apply():
    n = 4096
    iters = np.array([19, 19, 18])
    r = bench.tc_apply_roofline(bench.TC_APPLY_TRAFFIC_WORKLOAD, n, iters, (10.0, 40),
                                {"bf16_tflops_sustained": 1700.0})
    flops = 2.0 * n * n * ((2 * 19 + 1) + (2 * 19 + 1) + (2 * 18 + 1))
    assert r["achieved"] == pytest.approx(flops / 10.0e-3 / 1e12)
    assert r["peak"] == 1700.0 and r["frac"] == pytest.approx(r["achieved"] / 1700.0)
    assert r["unit"] == "TFLOP/s" and r["bound"] == "tensor"
    assert r["launch_ms_avg"] == pytest.approx(0.25)
    assert r["traffic"] == bench.TC_APPLY_TRAFFIC
    # no hi/lo-throughout solve: every launch counted as three products
    assert r["issued_tensor_tflops_hilo"] == pytest.approx(3 * r["achieved"])


def test_traffic_is_reported_only_for_the_captured_workload_and_issued_rate_comes_from_the_hilo_solve():
    r = bench.tc_apply_roofline("batch1024_n1024_kl_l1", 1024, np.array([100]), (1.0, 201), {},
                                np.array([100]), (3.0, 201))
    assert r["traffic"] is None and "no DRAM capture" in r["traffic_note"]
    assert r["peak"] == 1700.0 and "fallback" in r["peak_basis"]
    flops = 2.0 * 1024 * 1024 * 201
    assert r["issued_tensor_tflops_hilo"] == pytest.approx(3 * flops / 3.0e-3 / 1e12)
    assert r["issued_frac_hilo"] == pytest.approx(r["issued_tensor_tflops_hilo"] / 1700.0)
