"""bench.py pieces that need no GPU: the reference arm's JSON line (the FP64 oracle on
the host, warm-up steps untimed, every timed step a bounded sample) and the roofline
arithmetic of the training-pass kernels."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--cpu-seconds", "0.4"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("dd8")


def test_oracle_steps_are_separate_samples_after_warmup():
    rate, per_step, sample = bench.oracle_rate(0.2, steps=3, warmup=1)
    assert len(per_step) == 3 and all(r > 0 for r in per_step)
    assert min(per_step) <= rate <= max(per_step)
    assert "1 thread" in sample


def test_roofline_entries_are_consistent():
    wl = bench.workload_of("dd8")
    n = 2653469
    kt = {"query": 2.8, "k_enc": 0.8, "k_mlp": 0.6, "k_scat": 1.4}
    rl = bench.kernel_rooflines(wl, n, kt, 6800.0, 1700.0, "measured")
    assert set(rl) == {"k_enc", "k_mlp", "k_scat"}
    # k_scat: xyz and bf16 dL/dy per point, every FP32 gradient grid read and written
    m, r, c, b = 64, 32, 2, 8
    assert rl["k_scat"]["algorithmic_per_launch"] == n * (12 + 2 * m * c) + 2 * 4 * b * m * r ** 3 * c
    for k, v in rl.items():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])
        assert v["kernel_ms"] == kt[k]
    assert rl["k_scat"]["bound"] == "hbm" and rl["k_mlp"]["bound"] == "tensor"
    on = bench.onchip_rooflines(wl, n, kt, 152, 2070.0)
    # 8 corners x 2 channels per (point, grid), 32 lanes per warp instruction
    assert on["k_scat"]["algorithmic_per_launch"] == n * m * 16 / 32
    assert on["k_scat"]["peak"] == pytest.approx(0.94 * 152 * 2.07)
    for v in on.values():
        assert 0 < v["frac"] == pytest.approx(v["achieved"] / v["peak"])
