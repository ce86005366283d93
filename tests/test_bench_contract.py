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
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * d["value"]) <= 1e-9 * d["ms_per_step"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "sample" in cb
    # the native arm builds its config with the same function; the keys describe the workload
    sys.path.insert(0, ROOT)
    import bench
    cfg = d["config"]
    assert cfg["workload"] == bench.WORKLOAD and cfg["n"] == 1_048_576 and cfg["fmm_order"] == bench.default_fmm_order()
    assert cfg["alpha_normalised"] == bench.ALPHA and cfg["nu"] == bench.NU and cfg["leaf_cap"] == 96


def test_default_fmm_order_rule():
    """The library's order rule for fmm_order <= 0 (ceil(log eps / log 0.55), clamped to
    4..60), as the bench restates it for the reference arm's config."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.default_fmm_order(1e-11) == 43
    assert bench.default_fmm_order(0.9) == 4 and bench.default_fmm_order(1e-40) == 60
    src = open(os.path.join(ROOT, "paper_2608_11462_b300", "csrc", "abi.cu")).read()
    assert "std::log(o.fmm_eps) / std::log(0.55)" in src and "std::max(4, std::min(p, 60))" in src
