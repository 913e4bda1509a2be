"""bench.step_rates: whole-step tangent traffic and flop rate from the measured throughput."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_step_rates_by_hand():
    # two kernels: 3 GB + 1 GB and 2 + 6 TFLOP per step of N = 4 trajectories; 8 traj-steps/s
    # is one step of all four in 0.5 s: 8 GB/s, 16 TFLOP/s
    work = {"a": (2e12, 3e9), "b": (6e12, 1e9)}
    r = bench.step_rates(work, 8.0, 4, hbm_gbs=16.0, fp64_tflops=32.0, bf16_tflops=1600.0)
    assert r["tangent_bytes_per_step"] == 4e9 and r["tangent_flops_per_step"] == 8e12
    assert r["hbm_gbs"] == pytest.approx(8.0) and r["hbm_frac"] == pytest.approx(0.5)
    assert r["tflops"] == pytest.approx(16.0)
    assert r["vs_fp64_peak"] == pytest.approx(0.5) and r["vs_bf16_peak"] == pytest.approx(0.01)
    assert bench.step_rates(work, 8.0, 4, 16.0)["vs_fp64_peak"] is None


def test_step_rates_of_the_shell_workload():
    # the benchmark's tangent traffic: 10 n P words per trajectory-step (rhs 3, fwd 2, bwd 5)
    from paper_2508_06302_gb300 import inputs as I
    wl = I.workload_shell1872()
    m = wl.model
    work = bench.step_work(m, wl.N, 86, 0, 4)
    P = 2 * m.n + 1
    r = bench.step_rates(work, 8000.0, wl.N, hbm_gbs=6757.9)
    assert r["tangent_bytes_per_step"] == pytest.approx(10 * m.n * P * 4 * wl.N)
    assert 0.0 < r["hbm_frac"] < 1.0
