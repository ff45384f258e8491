"""bench.py's JSON line on CPU: the keys and values main() assembles from a
run's result, the CPU-baseline leg, and the reference arm.

The GPU leg (run_gpu) and the oracle subprocess are replaced by fixed results,
so nothing here needs a GPU or takes the oracle's time; what is checked is the
line the driver parses."""
import json
import sys

import pytest

import bench

FAKE_RUN = dict(
    ms=846.6, e2e_ms=83.7, systems=10, h2d=133431296, d2h=16777216, launches=21368,
    agg=dict(steps=3646, checks=41, cycles=40, svd=0),
    roofline=dict(bound="hbm", achieved=2207.0, peak=6660.3, unit="GB/s", frac=2207.0 / 6660.3, traffic=2.6e8,
                  kernel="spmv_dots", peak_kind="measured", bytes_per_launch=2.09e8, ms_per_launch=0.0946),
    clocks=dict(sm_mhz=2070.0, sm_max_mhz=2070.0, reasons=[], samples=5),
    cycle_hbm=dict(achieved=1554.7, unit="GB/s"), prof={}, workload="cd3d_128_seq20", N=2097152, nnz=14581760)

COMMON_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
               "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"}


def fake_oracle(steps=bench.ORACLE_SAMPLE_STEPS):
    return {"per_step": 0.2, "info": {"steps": steps, "seconds": 0.2 * (steps + 1)}}


def run_main(monkeypatch, capsys, argv, env=None):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    for k, v in dict(WORLD_SIZE="1", RANK="0", **(env or {})).items():
        monkeypatch.setenv(k, v)
    bench.main()
    out = capsys.readouterr().out.strip().splitlines()
    return json.loads(out[-1]) if out else None


def test_bench_line_keys_and_values(monkeypatch, capsys):
    monkeypatch.setattr(bench, "run_gpu", lambda args, rank, world: FAKE_RUN)
    monkeypatch.setattr(bench, "run_oracle_subprocess", fake_oracle)
    line = run_main(monkeypatch, capsys, ["--steps", "10", "--warmup", "3"])
    assert COMMON_KEYS | {"roofline", "clocks", "gpu_launches"} <= set(line)
    assert line["value"] == pytest.approx(84.66) and line["unit"] == "ms/system"
    assert line["higher_is_better"] is False and line["n_gpus"] == 1 and line["scaling"] == "weak"
    assert line["steps"] == 10 and line["warmup"] == 3 and line["dtype"] == "f64"
    assert line["config"]["workload"] == "cd3d_128_seq20"
    rf = line["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(rf)
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert line["e2e"] == {"value": 83.7, "unit": "ms/system", "h2d_bytes_per_step": 133431296,
                           "d2h_bytes_per_step": 16777216}
    assert line["gpu_launches"] == 21368 and line["clocks"]["sm_mhz"] == 2070.0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == "ms/system" and cb["sample"]
    # per-step time x Arnoldi-step equivalents per system (steps + checks + k recycled SpMVs)
    equiv = (3646 + 41 + 20 * 10) / 10
    assert cb["value"] == pytest.approx(0.2 * equiv * 1e3)


def test_reference_arm_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "run_oracle_subprocess", fake_oracle)
    line = run_main(monkeypatch, capsys, ["--impl", "reference", "--steps", "2", "--warmup", "3"])
    assert COMMON_KEYS | {"impl"} <= set(line)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is False
    assert line["value"] == pytest.approx(0.2 * bench.STEP_EQUIV_PER_SYSTEM * 1e3)
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
