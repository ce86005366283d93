"""CPU checks of bench.py's output contract on its reference arm (the oracle timed on the
host cores), which runs without a GPU: one JSON line with every key the contract names,
the same workload description as the native arm, and a bounded oracle sample."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

REQUIRED = ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"]


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in REQUIRED:
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["unit"] == "s"
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "sample" in cb
    # one labelled extrapolation shared with the native line's cpu_baseline: ms_per_step is
    # the measured time of the sampled step, value that time scaled by (n / n_sample)^2
    sys.path.insert(0, ROOT)
    import bench
    assert d["value_extrapolated"] is True and cb["extrapolated"] is True
    assert cb["n_sample"] == bench.CPU_SAMPLE and abs(cb["measured_s"] * 1e3 - d["ms_per_step"]) <= 1e-6
    scale = (d["config"]["n"] / bench.CPU_SAMPLE) ** 2
    assert abs(d["value"] - cb["measured_s"] * scale) <= 1e-9 * d["value"]
    # the native arm builds its config with the same function; the keys describe the workload
    cfg = d["config"]
    assert cfg["workload"] == bench.WORKLOAD and cfg["n"] == 1_048_576 and cfg["fmm_order"] == bench.default_fmm_order()
    assert cfg["alpha_normalised"] == bench.ALPHA and cfg["nu"] == bench.NU and cfg["leaf_cap"] == 96


def test_cpu_record_is_shared_by_both_legs():
    """The native line's cpu_baseline and the reference arm describe the oracle time with
    the same function, sample size and labels."""
    sys.path.insert(0, ROOT)
    import bench
    rec = bench.cpu_record(2.0, 8, 1_048_576, 3)
    assert rec["extrapolated"] is True and rec["n_sample"] == bench.CPU_SAMPLE and rec["measured_s"] == 2.0
    assert rec["value"] == 2.0 * (1_048_576 / bench.CPU_SAMPLE) ** 2
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert src.count("cpu_record(") >= 3  # definition, native leg, reference arm


def test_default_fmm_order_rule():
    """The library's order rule for fmm_order <= 0 (ceil(log eps / log 0.55), clamped to
    4..60), as the bench restates it for the reference arm's config."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.default_fmm_order(1e-11) == 43
    assert bench.default_fmm_order(0.9) == 4 and bench.default_fmm_order(1e-40) == 60
    src = open(os.path.join(ROOT, "paper_2608_11462_b300", "csrc", "abi.cu")).read()
    assert "std::log(o.fmm_eps) / std::log(0.55)" in src and "std::max(4, std::min(p, 60))" in src


def test_fifo_latencies_of_the_sequential_serving_arm():
    """The serving case's one-at-a-time latencies at Poisson rates come from the single
    FIFO server recursion over measured service times.  Checked on a hand-worked case, on
    simultaneous arrivals (latency i = s_0 + ... + s_i), and against a discrete-event
    simulation that tracks the server's state between events."""
    import heapq

    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    # a = 0, 1, 1.5, 10 with s = 2, 2, 1, 1: ends 2, 4, 5, 11
    lat = bench.fifo_latencies([0.0, 1.0, 1.5, 10.0], [2.0, 2.0, 1.0, 1.0])
    assert np.array_equal(lat, [2.0, 3.0, 3.5, 1.0])
    svc = np.array([0.5, 0.25, 2.0, 1.0])
    assert np.allclose(bench.fifo_latencies(np.zeros(4), svc), np.cumsum(svc), rtol=0, atol=1e-15)

    def simulate(arr, svc_):
        # events (time, kind, request): kind 0 = a request ends, kind 1 = a request arrives
        ev = [(a_, 1, i) for i, a_ in enumerate(arr)]
        heapq.heapify(ev)
        queue, busy, end = [], False, [0.0] * len(arr)
        while ev:
            t, kind, i = heapq.heappop(ev)
            if kind == 0:
                end[i] = t
                busy = False
            else:
                queue.append(i)
            if not busy and queue:
                j = queue.pop(0)
                busy = True
                heapq.heappush(ev, (t + svc_[j], 0, j))
        return np.asarray(end) - np.asarray(arr)

    rng = np.random.default_rng(5)
    for rate in (0.5, 2.0, 8.0):
        arr = np.cumsum(rng.exponential(1.0 / rate, 300))
        s_ = rng.lognormal(-1.0, 1.0, 300)
        assert np.allclose(bench.fifo_latencies(arr, s_), simulate(arr, s_), rtol=1e-12, atol=1e-12)
