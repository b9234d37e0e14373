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
    # labelled with what it times (one FP64 model on the host), and what that stands for
    assert d["config"]["workload"].startswith("FP64 oracle on the host")
    assert d["config"]["stands_for"].startswith("dd8")


def test_oracle_steps_are_separate_samples_after_warmup():
    rate, per_step, sample = bench.oracle_rate(0.2, steps=3, warmup=1)
    assert len(per_step) == 3 and all(r > 0 for r in per_step)
    assert min(per_step) <= rate <= max(per_step)
    assert "1 thread" in sample


def test_roofline_entries_are_consistent():
    wl = bench.workload_of("dd8")
    n = 2653469
    kt = {"query": 2.8, "k_enc": 0.8, "k_mlp": 0.6, "k_scat": 1.4}
    rl = bench.kernel_rooflines(wl, n, kt, 6800.0, 1700.0, 152, 2070.0, "measured")
    assert set(rl) == {"k_enc", "k_mlp", "k_scat"}
    m, r, c, b = 64, 32, 2, 8
    # k_scat against its shared-memory reductions: 8 corners x 2 channels per (point, grid)
    assert rl["k_scat"]["bound"] == "smem" and rl["k_mlp"]["bound"] == "tensor"
    assert rl["k_scat"]["algorithmic_per_launch"] == n * m * 16 / 32
    assert rl["k_scat"]["peak"] == pytest.approx(0.94 * 152 * 2.07)
    # the method's own HBM bytes only: xyz, and each FP32 gradient grid written once
    assert rl["k_scat"]["hbm"]["algorithmic_bytes"] == n * 12 + 4 * b * m * r ** 3 * c
    assert rl["k_enc"]["hbm"]["algorithmic_bytes"] == n * 12 + 2 * b * m * r ** 3 * c
    # dL/dy and Y are reported as intermediates, never as algorithmic bytes
    assert rl["k_scat"]["intermediates"]["bytes"] == n * m * c * 2
    for k, v in rl.items():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])
        assert v["hbm"]["frac"] == pytest.approx(v["hbm"]["achieved"] / v["hbm"]["peak"])
        assert v["kernel_ms"] == kt[k]
    # recomputed by hand: 84.9 M warp reductions in 1.4 ms against 295.8 G/s
    assert rl["k_scat"]["frac"] == pytest.approx(n * 64 * 16 / 32 / 1.4e-3 / 1e9 / (0.94 * 152 * 2.07), rel=1e-12)


def test_step_floors_follow_the_method_work():
    wl = bench.workload_of("dd8")
    n = 2653469
    w = bench.method_work(wl, n)
    # per step: 48 B per point plus, per brick, the BF16 grids (8.4 MB), one FP32 gradient
    # write (16.8 MB), Adam over 4.2 M parameters (28 B each) and the BF16 shadow (8.4 MB)
    grid = 64 * 32 ** 3 * 2
    params = grid + 64 * 128 + 64 * 64 + 64 + 64 * 12
    per_brick = 2 * grid + 4 * grid + 28 * params + 2 * (grid + 64 * 128 + 64 * 64 + 64)
    assert w["hbm_bytes"] == n * 48 + 8 * per_brick
    assert 1.33e9 < w["hbm_bytes"] < 1.35e9
    assert w["tensor_flop"] == n * bench.FLOP_PER_POINT
    f = bench.step_floors(wl, n, 3.389, 6757.9, 1727.4, 152, 2070.0, "measured")
    assert f["binding"] == "smem"
    assert f["smem_ms"] == pytest.approx(0.287 + 0.135, abs=0.002)
    assert f["hbm_ms"] == pytest.approx(0.198, abs=0.002)
    assert f["frac"] == pytest.approx(f["floor_ms"] / 3.389)
    assert f["floor_ms"] == max(f["hbm_ms"], f["tensor_ms"], f["smem_ms"], f["alu_ms"])


def test_render_roofline_names_its_binder():
    wl = bench.workload_of("dd8")
    rr = bench.render_roofline(2.3e9, wl, 1760.0, 152, 2070.0, "measured")
    assert rr["tensor"]["achieved"] == pytest.approx(2.3e9 * 2 * bench.MLP_MACS_FWD / 1e12)
    assert rr["gather"]["achieved"] == pytest.approx(2.3e9 * 64 * 8 * 2 * 2 / 1e9)
    assert rr["bound"] in ("tensor", "gather")
    assert rr[rr["bound"]]["frac"] == max(rr["tensor"]["frac"], rr["gather"]["frac"])


def test_step_spread():
    s = bench.spread([3.0, 3.1, 3.2, 3.3, 10.0])
    assert s["median_ms"] == 3.2 and s["min_ms"] == 3.0 and s["max_ms"] == 10.0 and s["steps"] == 5
    assert s["p10_ms"] <= s["median_ms"] <= s["p90_ms"]
