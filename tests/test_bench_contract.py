"""The bench's JSON line (reference arm, on the CPU) and its refusal to run the
GPU arm without a GPU: the product path has no CPU fallback."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args,
                          capture_output=True, text=True, timeout=timeout, cwd=ROOT)


def test_reference_arm_prints_one_json_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "DOF-stage/s" and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and "sample" in cb
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_gpu_arm_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run(["--steps", "1", "--warmup", "0", "--no-cpu-baseline", "--no-ensemble", "--no-fp32",
              "--no-stab"], timeout=300)
    assert r.returncode != 0
    assert not any(ln.startswith("{") for ln in r.stdout.splitlines())


def test_algorithmic_bytes_per_node():
    sys.path.insert(0, ROOT)
    import importlib
    bench = importlib.import_module("bench")
    # (2.25 n_f + 6) words: read U_s, write U_{s+1}, U^n on one stage in four,
    # write + read T, rho_v, p'
    assert bench.algorithmic_bytes_per_node(7, 8) == pytest.approx(174.0)
    assert bench.algorithmic_bytes_per_node(7, 4) == pytest.approx(87.0)


def test_roofline_arithmetic():
    """frac = achieved / peak with achieved = algorithmic bytes per launch over
    the mean launch time; traffic is the profiled bytes per node scaled to the
    mesh, and null for a configuration without a capture."""
    sys.path.insert(0, ROOT)
    import importlib
    import types
    bench = importlib.import_module("bench")
    info = types.SimpleNamespace(n_fields=7, n_nodes=16_384_000, launches_per_stage=2)
    t_total, steps, peak = 0.5, 10, 6705.5
    r = bench._roofline(info, 8, t_total, steps, peak, "measured",
                        bench._traffic({"dim": 3, "order": 4}, "fp64", info))
    launch_s = t_total / (bench.STAGES * steps)
    assert r["avg_launch_ms"] == pytest.approx(1000.0 * launch_s)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(174.0 * info.n_nodes)
    assert r["achieved"] == pytest.approx(174.0 * info.n_nodes / launch_s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] == pytest.approx(bench.PROFILED_TRAFFIC[(3, 4, "fp64")][0] * info.n_nodes)
    # every traffic figure names the profile summary it comes from
    assert r["traffic_source"].startswith("ncu capture, profiles/")
    src = r["traffic_source"].split(", ", 1)[1].split(":")[0]
    assert os.path.exists(os.path.join(ROOT, src)), src
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    # no capture for this configuration, or the inline / column schedule: traffic null
    assert bench._traffic({"dim": 2, "order": 3}, "fp64", info) == (None, None)
    inline = types.SimpleNamespace(n_fields=7, n_nodes=10, launches_per_stage=1)
    assert bench._traffic({"dim": 3, "order": 4}, "fp64", inline) == (None, None)


def test_fp64_alu_roofline():
    """The float64 form's roofline: algorithmic flops per node (the items sum
    to the total) x nodes over the mean stage time, against 152 SMs x 2 FP64
    FMA per clock x 2 flop x the sampled clock."""
    sys.path.insert(0, ROOT)
    import importlib
    import types
    bench = importlib.import_module("bench")
    fpn, items = bench.fp64_flops_per_node(3, 4, 7, 1)
    assert fpn == pytest.approx(sum(items.values()))
    assert items["volume"] == 2 * 3 * 7 * 5 and items["lift"] == 4 * 3 * 7
    info = types.SimpleNamespace(n_fields=7, n_nodes=16_384_000, launches_per_stage=2)
    hbm = bench._roofline(info, 8, 0.5, 10, 6705.5, "measured", (None, None))
    r = bench.fp64_alu_roofline(info, {"dim": 3, "order": 4, "rain": 1}, 0.5, 10, 152, 2070.0, 1.25, hbm)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert r["achieved"] == pytest.approx(fpn * info.n_nodes / (0.5 / 40) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["hbm"]["frac"] == pytest.approx(hbm["frac"])
    assert r["fp64_fma_probe"]["frac_of_probe"] == pytest.approx(r["achieved"] / 1.25)


def test_whole_job_rate_is_weak_scaling():
    sys.path.insert(0, ROOT)
    import importlib
    bench = importlib.import_module("bench")
    # every rank steps a full replica: twice the ranks, twice the work per time
    assert bench.whole_job_rate(2, 100.0, 1.0) == 2 * bench.whole_job_rate(1, 100.0, 1.0)
