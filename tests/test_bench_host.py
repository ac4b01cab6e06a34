"""bench.py host logic on CPU: the clock / throttle sampler reads the sampling
tool's CSV from a pipe and summarises it (a fake tool stands in for nvidia-smi)."""
import sys
import time

import bench

FAKE = ("import sys, time\n"
        "rows = ['0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active',\n"
        "        '0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active',\n"
        "        '0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active']\n"
        "for r in rows:\n"
        "    print(r, flush=True)\n"
        "    time.sleep(0.05)\n"
        "time.sleep(30)\n")


def test_clock_sampler_reads_the_pipe_and_reports_reasons():
    s = bench.ClockSampler(0, cmd=[sys.executable, "-c", FAKE])
    s.start()
    t0 = time.time()
    while len(s.lines) < 3 and time.time() - t0 < 20:
        time.sleep(0.05)
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_of_throttled_and_malformed_lines():
    lines = ["0, 1400, 2070, 1400, 0x8, Active, Not Active, Active, Not Active",
             "garbage", "0, N/A, 2070, 1, 0, Not Active, Not Active, Not Active, Not Active",
             "0, 1500, 2070, 1400, 0x8, Not Active, Active, Not Active, Not Active"]
    out = bench.ClockSampler.summarise(lines)
    assert out["samples"] == 2 and out["sm_mhz"] == 1450.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_the_tool():
    s = bench.ClockSampler(0, cmd=["/nonexistent/sampler-tool"])
    s.start()
    out = s.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_cpu_baseline_leg_on_the_tiny_workload():
    """The CPU-baseline leg: one-thread and all-thread rates of the oracle, and the
    shrunk image against the unshrunk oracle (here the oracle's own shrunk image, so the
    error is that of shrinking alone)."""
    import math

    import numpy as np

    import oracle
    tree, cams, tau_R, _ = bench.workload("tiny")
    tau = 0.1
    ln_tau = float(np.float32(math.log(tau)))
    p = oracle.Params(tau_R=tau_R, shrink=True, tau=tau, ln_tau=ln_tau)
    img = {0: oracle.frame(tree, cams[0], p).rgb.astype(np.float32)}
    out = bench.cpu_baseline(tree, cams, tau_R, tau, ln_tau, img)
    assert out["value"] > 0 and out["single_core"]["value"] > 0
    assert out["cores"] >= 1 and out["single_core"]["cores"] == 1
    e = out["shrink_vs_unshrunk_oracle"]["poses"][0]
    assert e["pose"] == 0 and e["max_abs"] > 0 and 10 < e["psnr_db"] < 200
    assert "1 whole frames" in out["sample"]


def test_cpu_sample_pose_order():
    """The CPU-baseline sample takes the compared poses first, then spreads over the
    flythrough; every pose appears once."""
    order = bench.cpu_sample_poses(64, [0, 32])
    assert order[:8] == [0, 32, 8, 16, 24, 40, 48, 56]
    assert sorted(order) == list(range(64))
    assert bench.cpu_sample_poses(1, [0]) == [0]
    assert sorted(bench.cpu_sample_poses(8, [0, 4])) == list(range(8))


def test_hold_stream_lengths():
    """The timed loops' stream hold: at least the minimum, 10 ms a step, at most 5 s,
    passed to torch's spin helper as clock cycles; nothing without the helper."""
    calls = []

    class Cuda:
        @staticmethod
        def _sleep(c):
            calls.append(c)

    class Torch:
        cuda = Cuda

    assert bench.hold_stream(Torch, 20) == 0.5
    assert bench.hold_stream(Torch, 64) == 0.64
    assert bench.hold_stream(Torch, 10_000) == 5.0
    assert bench.hold_stream(Torch, 1, min_s=0.01) == 0.01
    assert calls == [int(s * 2.07e9) for s in (0.5, 0.64, 5.0, 0.01)]

    class NoSpin:
        class cuda:
            pass

    assert bench.hold_stream(NoSpin, 20) == 0.0
