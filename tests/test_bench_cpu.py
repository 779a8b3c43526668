"""The benchmark's reference arm (the FP64 CPU oracle on a bounded sample of
the workload) runs without a GPU and prints one JSON line with the contract's
keys; its cells/s is the sample's cells over the measured time per step."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                        "--ref-sample", "8"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "cells/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["sample_grid"] == [8, 8, 8] and "workload" in d["config"]
    assert d["value"] == pytest.approx(8 ** 3 / (d["ms_per_step"] / 1e3), rel=1e-2)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert isinstance(d["cpu_baseline"]["cpu_model"], str) and d["cpu_baseline"]["cpu_model"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_pass_bytes_and_flop_estimate():
    """The roofline bytes of the 256^3 step (padded 512^3): 349 B per cell
    with the energy (x R2C 36, y 72, z 120.6 with the octant tensor, y inverse
    72, x C2R + energy 48), and the FFT flop estimate grows as L log2 L."""
    sys.path.insert(0, ROOT)
    import bench
    n, P = (256, 256, 256), (512, 512, 512)
    pb = bench.pass_bytes(n, P, 4)
    cells = 256 ** 3
    assert pb["x_fwd"] == 3 * cells * 4 + 3 * 256 * 256 * 257 * 8
    assert pb["y_fwd"] == pb["y_inv"] == 3 * 256 * 256 * 257 * 8 + 3 * 256 * 512 * 257 * 8
    assert pb["z_conv"] == 2 * 3 * 256 * 512 * 257 * 8 + 6 * 257 * 257 * 257 * 4
    assert pb["x_inv"] - bench.pass_bytes(n, P, 4, energy=False)["x_inv"] == 3 * cells * 4
    assert 345 < sum(pb.values()) / cells < 352
    assert bench.fft_flops(1) == 0 and bench.fft_flops(8) == 5 * 8 * 3
    assert bench.step_flops(n, P) > 2 * 3 * 512 * 257 * bench.fft_flops(512)
