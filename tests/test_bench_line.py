"""The benchmark's JSON line, assembled on the CPU from stubbed GPU arms:
every key of the line's contract, the derived rates, the roofline object
(achieved = algorithmic bytes per launch / average launch time, frac against
the peak, the stored DRAM traffic used only while its source hash matches),
the end-to-end object and the launch count."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CATS = ["apply64", "residual64", "smooth64", "smooth_first64", "apply32", "residual32", "smooth32",
        "smooth_first32", "transfer", "p1", "krylov", "rhs", "recover", "layout", "condense"]


def _arm(ms_total, steps, smooth_ms, cold_factor=1.25):
    prof = {c: (0.0, 0) for c in CATS}
    prof.update({"smooth32": (smooth_ms, 22 * steps), "apply32": (0.5, 11 * steps), "residual32": (0.4, 11 * steps),
                 "smooth_first32": (0.3, 11 * steps),
                 "p1": (2.0, 100 * steps), "krylov": (1.0, 60 * steps), "rhs": (0.3, 2 * steps),
                 "recover": (0.7, steps), "layout": (0.05, 2 * steps)})
    cold = {c: (ms * cold_factor, n) for c, (ms, n) in prof.items()}
    return {"ms": ms_total, "infos": [{"iters": 11, "true_rel_res": 3.4e-9}] * steps, "n_cells": 131072,
            "NF": 196608, "pp": 4, "n_p": 10, "coarse": "stub", "data_gb": 1.82, "prof": prof, "prof_cold": cold,
            "prof_steps": steps, "levels_nv": [65536, 16384, 4096, 1024, 256, 64, 16],
            "condense_ms": 28.0, "launches": 43400, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
            "e2e_s": ms_total * 1.07e-3, "h2d": 31457280, "d2h": 37748736}


def test_bench_line_contract(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    steps = 4
    arms = {"mixed": _arm(7.7, steps, 1.2), "mixed_bf16": _arm(8.3, steps, 1.0),
            "fgmres64": _arm(10.6, steps, 1.2), "fp64": _arm(19.1, steps, 2.0)}
    fma = {"fp64_tflops": 1.2, "fp32_tflops": 75.0, "how": "stub"}
    monkeypatch.setattr(bench, "gpu_arm", lambda args, rank, world: (arms, fma))
    cpu = {"value": 0.11, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": "stub"}
    monkeypatch.setattr(bench, "oracle_start", lambda *a, **k: "started")
    monkeypatch.setattr(bench, "oracle_wait", lambda h: {"stub": h})
    monkeypatch.setattr(bench, "cpu_baseline_entry", lambda r, *a, **k: cpu if r == {"stub": "started"} else None)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", str(steps), "--warmup", "3"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main()
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == steps and line["warmup"] == 3 and line["higher_is_better"]
    assert line["value"] == pytest.approx(steps / 7.7e-3) and line["ms_per_step"] == pytest.approx(7.7 / steps)
    assert line["speedup_vs_plain_fp64"] == pytest.approx(19.1 / 7.7)
    assert "workload" in line["config"] and line["cpu_baseline"] == cpu and line["gpu_launches"] == 43400
    e2e = line["e2e"]
    assert e2e["value"] == pytest.approx(steps / (7.7 * 1.07e-3)) and e2e["unit"] == "solves/s"
    assert e2e["h2d_bytes_per_step"] == 31457280 and e2e["d2h_bytes_per_step"] == 37748736
    r = line["roofline"]
    assert r["bound"] == "hbm" and r["kernel"] == "smooth32" and r["unit"] == "GB/s"
    per_launch = bench.trace_bytes("smooth32", 196608, 4)
    assert r["algorithmic_bytes_per_launch"] == per_launch
    # the headline figure is the cold (L2-evicted) timing, the warm one beside it
    assert r["achieved"] == pytest.approx(per_launch / (1.25 * 1.2e-3 / (22 * steps)) / 1e9)
    assert r["warm"]["achieved"] == pytest.approx(per_launch / (1.2e-3 / (22 * steps)) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get("smooth32_fp32_p3")
    expect = tr["bytes_per_launch"] if tr and tr["source_sha"] == bench.source_sha() else None
    assert r["traffic"] == expect
    names = [o["kernel"] for o in r["others"]]
    assert any(n.startswith("P1") for n in names) and "recover" in names
    for o in r["others"]:
        assert 0 <= o["share_of_kernel_time"] <= 1
    # the BF16-operator smoother never borrows the FP32 capture
    rb = line["mixed_bf16_smoother"]["roofline"]
    assert rb["algorithmic_bytes_per_launch"] == bench.trace_bytes("smooth32", 196608, 4, 2)
    tb = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get("smooth32_bf16_p3")
    assert rb["traffic"] == (tb["bytes_per_launch"] if tb and tb["source_sha"] == bench.source_sha() else None)
    # the FP64 arm's sweep against the measured FP64 FMA rate
    fp = line["plain_fp64"]["roofline"]
    assert fp["kernel"] == "smooth32"          # the stub arms all run FP32 sweeps
    assert line["condense_fp64_pipe"]["peak_tflops"] == 1.2 and line["measured_fma"] == fma
    assert 0 < line["whole_solve"]["frac"] < 2
