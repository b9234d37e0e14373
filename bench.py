#!/usr/bin/env python3
"""Training-step throughput of the batched APMGSRN hot path on one GB300.

Workload (default "dd8"): a synthetic 1024^3 float32 turbulence volume split into
2x2x2 bricks of 512^3 (+2 ghost voxels), one APMGSRN per brick (M=64 grids of
32^3 x 2 channels, MLP 128->64->64->1, BF16 grids/decoder with FP32 masters),
uneven per-brick batches drawn from U[2^16, 2^19].  One step = sample the batch
(Philox + Morton counting sort) -> ground truth lookup -> forward/backward of
L_rec -> feature-density loss and its transform gradient -> Adam on every
parameter, replayed from a CUDA graph.  Throughput = points of all bricks per
second.

Roofline accounting follows the method's own work per point and per step (Eq. 1-9,
the decoder, Adam): the HBM bytes the method must move (points, targets, the volume
corners, grids, gradients and Adam state), the decoder's tensor flops, the corner
reads and reductions that live in shared memory, and the FP32 arithmetic of the map,
the blend and the density.  Intermediates that this implementation keeps in HBM (the
features Y and dL/dy between its kernels) are reported beside that, never counted
as algorithmic.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "train fwd+bwd points/s (BF16 batched vs FP32 plain) at stated err; % roofline"
UNIT = "points/s"
# MACs per point of the 128->64->64->1 decoder: forward, and backward (dX of the two
# hidden layers and of the first layer's input, dW of all three)
MLP_MACS_FWD = 128 * 64 + 64 * 64 + 64
MLP_MACS_BWD = 64 * 64 + 64 * 64 + 64 * 128 + 64 * 128 + 64
FLOP_PER_POINT = 2 * (MLP_MACS_FWD + MLP_MACS_BWD)
# kernels of one training step: sampler (3), target lookup, the query pass (BF16: tile
# list (the unit starts come from the sampler), encoder, decoder, scatter; FP32: 1 fused
# kernel), density passes (BF16: 3 on the second stream; FP32: 2), finalisation, step
# counter, Adam (BF16 density steps: F and the decoder, then G)
KERNELS_PER_STEP = {"bf16": 15, "fp32": 10}


# DRAM bytes (read + write) per launch of each training-pass kernel, from an ncu capture
# of the 8-brick step (profiles/).  They hold only for the kernel sources they were
# taken on: any change to those files makes bench report traffic as null.
NCU_TRAFFIC = {"sources_sha1": "73322001601b1f903f64ee9a83c237cd246f79fe",
               "k_scat": 1082.62e6, "k_enc": 715.19e6, "k_mlp": 1336.33e6}
TRAFFIC_SOURCES = ("k_train_bf16.cu", "k_mlp_tc.cu", "common.cuh", "bf16_ops.cuh", "tc_ops.cuh", "enc_ops.cuh")


def sources_sha1():
    """SHA-1 of the kernel sources' code: line comments and blank lines are left out, so
    that a comment edit keeps the measured traffic (the sources hold no block comments
    and no "//" inside a string)."""
    import hashlib
    h = hashlib.sha1()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2308_02494_gb300", "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def measured_traffic(name):
    return NCU_TRAFFIC.get(name) if sources_sha1() == NCU_TRAFFIC["sources_sha1"] else None


# On-chip rates for the gather and the scatter, whose per-(point, grid) corner work
# lives in shared memory: the scatter adds 8 x C contributions with conflict-free
# red.shared.add.u32 (measured on this GB300 with a probe of 16 warps per SM,
# conflict-free addresses: 0.94 warp instructions per SM clock); the encoder reads 8
# corners of C bf16 values (4 bytes per lane for C = 2; the kernel stages them as
# float32, 8 bytes) at the nominal rate of one warp instruction of 32 x 4 B per SM clock.
SMEM_RED_PER_CLK = 0.94
SMEM_LDS_PER_CLK = 1.0
FP32_LANES_PER_SM = 128


def method_work(wl, n_total):
    """Algorithmic work of one training step (density phase) of the workload: what the
    method must do, independent of how it is implemented.  Per point: the map (M x 12
    FMA), the gather (8 corners x C reads and FMAs per grid), the decoder (fwd + bwd
    flops), the scatter (8 corners x C adds per grid), the density (per grid: map,
    flat top, exp, its gradient ~ 30 flop + 12 FMA) and the HBM bytes xyz (12 B),
    target (4 B) and the 8 volume corners (32 B).  Per brick: the BF16 grids read once,
    the FP32 feature gradient written once, Adam over every parameter (FP32 p, g, m, v
    read, p, m, v written, the BF16 shadow of F and the decoder written)."""
    m, r, c, b = wl["grids"], wl["res"], wl["channels"], wl["bricks"]
    k = m * c
    grid_vals = m * r ** 3 * c
    dec = 64 * k + 64 * 64 + 64
    params = grid_vals + dec + m * 12
    feat_bytes = 2 if wl["precision"] == "bf16" else 4
    per_brick = (grid_vals * feat_bytes                  # grids read
                 + grid_vals * 4                         # feature gradient written once
                 + params * (4 * 4 + 3 * 4)              # Adam: p, g, m, v read; p, m, v written
                 + (grid_vals + dec) * (2 if wl["precision"] == "bf16" else 0))   # BF16 shadow written
    return {
        "hbm_bytes": n_total * (12 + 4 + 32) + b * per_brick,
        "tensor_flop": n_total * FLOP_PER_POINT,
        "smem_scatter_warp_red": n_total * m * 8 * c / 32,
        "smem_gather_warp_lds": n_total * m * 8 / 32,
        "alu_flop": n_total * (m * (2 * 12 + 2 * 8 * c + 8 * c + 30 + 2 * 12)),
        "per_point": {"hbm_bytes": 48, "tensor_flop": FLOP_PER_POINT, "shared_corner_reads": m * 8 * c,
                      "shared_corner_adds": m * 8 * c, "alu_flop": m * (2 * 12 + 2 * 8 * c + 8 * c + 30 + 2 * 12)},
        "per_brick_hbm_bytes": per_brick,
    }


def step_floors(wl, n_total, step_ms, hbm, tf_sus, sms, sm_mhz, src):
    """The step's roofline time per resource (each resource's algorithmic work at its
    peak) and the binding one; frac = binding floor / measured step time."""
    w = method_work(wl, n_total)
    clk = sm_mhz * 1e6
    fl = {
        "hbm_ms": w["hbm_bytes"] / (hbm * 1e9) * 1e3,
        "tensor_ms": w["tensor_flop"] / (tf_sus * 1e12) * 1e3,
        "smem_ms": (w["smem_scatter_warp_red"] / (SMEM_RED_PER_CLK * sms * clk)
                    + w["smem_gather_warp_lds"] / (SMEM_LDS_PER_CLK * sms * clk)) * 1e3,
        "alu_ms": w["alu_flop"] / (2 * FP32_LANES_PER_SM * sms * clk) * 1e3,
    }
    bind = max(fl, key=fl.get)
    return dict(fl, binding=bind[:-3], floor_ms=fl[bind], step_ms=step_ms, frac=fl[bind] / step_ms,
                algorithmic={k: w[k] for k in ("hbm_bytes", "tensor_flop", "smem_scatter_warp_red",
                                                "smem_gather_warp_lds", "alu_flop")},
                peaks=f"HBM {hbm} GB/s ({src} copy); bf16 {tf_sus} TFLOP/s ({src}, sustained); shared-memory "
                      f"reductions {SMEM_RED_PER_CLK} and loads {SMEM_LDS_PER_CLK} warp instructions per SM clock; "
                      f"FP32 {FP32_LANES_PER_SM} FMA lanes per SM; {sms} SMs at {sm_mhz:.0f} MHz")


def kernel_rooflines(wl, n_total, kt, hbm, tf_sus, sms, sm_mhz, src):
    """Each training-pass kernel against its binding resource, from its measured mean
    time (ms): the scatter and the encoder against their shared-memory instruction rate,
    the decoder against the tensor pipe.  'hbm' gives the method's own HBM bytes that the
    kernel moves (no intermediates) against the measured copy bandwidth; 'intermediates'
    the bytes of Y / dL/dy that this implementation stores between kernels."""
    m, r, c, b = wl["grids"], wl["res"], wl["channels"], wl["bricks"]
    k = m * c
    grid_vals = b * m * r ** 3 * c
    clk = sm_mhz * 1e6
    spec = {
        "k_scat": ("smem", n_total * m * 8 * c / 32, SMEM_RED_PER_CLK * sms * clk / 1e9, "G warp instructions/s",
                   "8 corners x C channels per (point, grid) added in shared memory, 32 lanes per warp instruction",
                   f"measured conflict-free red.shared.add.u32 rate, {SMEM_RED_PER_CLK} per SM clock x {sms} SMs x "
                   f"{sm_mhz:.0f} MHz",
                   n_total * 12 + grid_vals * 4, "xyz (12 B per point) + every FP32 feature-gradient grid written once",
                   n_total * k * 2, "dL/dy (K bf16 per point) read"),
        "k_enc": ("smem", n_total * m * 8 / 32, SMEM_LDS_PER_CLK * sms * clk / 1e9, "G warp instructions/s",
                  "8 corners per (point, grid) read from shared memory (C bf16 in one word), 32 lanes per warp "
                  "instruction",
                  f"nominal conflict-free shared-load issue rate, {SMEM_LDS_PER_CLK} per SM clock x {sms} SMs x "
                  f"{sm_mhz:.0f} MHz",
                  n_total * 12 + grid_vals * 2, "xyz (12 B per point) + every BF16 feature grid read once",
                  n_total * k * 2, "Y (K bf16 per point) written"),
        "k_mlp": ("tensor", n_total * FLOP_PER_POINT / 1e12, tf_sus, "TFLOP/s",
                  f"{FLOP_PER_POINT} decoder flop per point (forward + backward MACs x 2)",
                  f"{src} bf16 sustained (cuBLAS)",
                  n_total * 4, "target (4 B per point)",
                  n_total * k * 2 * 2, "Y (K bf16 per point) read + dL/dy (K bf16 per point) written"),
    }
    out = {}
    for name, ms in kt.items():
        if name not in spec or not ms:
            continue
        bound, amount, peak, unit, per, psrc, hb, hper, ib, iper = spec[name]
        ach = amount / (ms / 1e3) / (1e9 if bound == "smem" else 1.0)   # G warp instructions/s
        hach = hb / (ms / 1e3) / 1e9
        tr = measured_traffic(name) if b == 8 else None
        out[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                     "traffic": tr, "kernel_ms": ms, "peak_source": psrc, "algorithmic": per,
                     "algorithmic_per_launch": amount,
                     "hbm": {"algorithmic_bytes": hb, "algorithmic": hper, "achieved": hach, "peak": hbm,
                             "unit": "GB/s", "frac": hach / hbm},
                     "intermediates": {"bytes": ib, "what": iper},
                     "traffic_over_algorithmic_hbm": (tr / hb) if tr else None}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--workload", choices=["dd8", "single-bf16", "single-fp32"], default="dd8")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the render, decode, e2e, single-model and CPU legs")
    ap.add_argument("--tiles", choices=["auto", "default"], default="auto",
                    help="BF16 tile shape: picked by srn_autotune on one batch before warm-up, or the "
                         "library default")
    ap.add_argument("--volume", type=int, default=None,
                    help="voxels per axis of the synthetic volume (default: the workload's); a smaller "
                         "volume keeps the same batch and model with a small device footprint, for profilers")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


# ----------------------------------------------------------------------------- oracle legs
# The reference arm: the FP64 oracle training one model on the host (one thread).
REF_WORKLOAD = ("FP64 oracle on the host, 1 thread: one model (M=64 R=32 C=2, MLP 128-64-64-1, Sec. 4.3.3 "
                "init), 2048-point uniform batches over a 64^3 Gaussian-sum volume; each iteration = target "
                "lookup + forward + L_rec backward + density backward + Adam over all 4.2M parameters")
ORACLE_SNIPPET = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, %(root)r)
from oracle import apmgsrn as ap
from paper_2308_02494_gb300 import synth
shape = synth.ModelShape(64, 32, 2, 64)
p = synth.init_model(shape, 0)
n = %(n)d
x = synth.uniform_points(n, 1).astype(np.float64)
vol, _ = synth.gaussian_volume(64, 16, seed=0)
keys = ("F", "W1", "W2", "w3", "G")
mom = {k: (np.zeros_like(p[k]), np.zeros_like(p[k])) for k in keys}
it = 0
out = []
for step in range(%(steps)d):   # each step: whole iterations until its time budget is spent
    t0 = time.perf_counter(); done = 0; reps = 0
    while True:
        v = ap.volume_sample(vol, x)
        g = ap.grad_rec(p, x, v)
        d = ap.grad_density(p["G"], x, g["h"])
        grads = {"F": g["dF"], "W1": g["dW1"], "W2": g["dW2"], "w3": g["dw3"], "G": d["dG"]}
        it += 1
        for k in keys:
            lr = 1e-3 if k == "G" else 1e-2
            p[k], m1, m2 = ap.adam_update(p[k], grads[k], mom[k][0], mom[k][1], it, lr)
            mom[k] = (m1, m2)
        done += n; reps += 1
        if time.perf_counter() - t0 >= %(budget)f:
            break
    out.append({"points": done, "seconds": time.perf_counter() - t0, "reps": reps})
print(json.dumps(out))
"""


def oracle_rate(budget_s: float, n: int = 2048, steps: int = 1, warmup: int = 0):
    """The FP64 oracle's training-iteration rate on one host thread, in one subprocess:
    `warmup` untimed then `steps` timed steps of at least budget_s seconds each (whole
    iterations).  Returns (points/s over the timed steps, per-step points/s, a
    description of the sample)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET % {"root": ROOT, "n": n, "budget": budget_s, "steps": warmup + steps}
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=600 + 2 * (warmup + steps) * budget_s)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])[warmup:]
    points, seconds, reps = (sum(q[k] for q in r) for k in ("points", "seconds", "reps"))
    sample = (f"FP64 oracle, 1 thread: one model (M=64, R=32, C=2, 128->64->64->1), "
              f"{n}-point batches x {reps} reps: target lookup + fwd + L_rec bwd + density bwd + "
              f"Adam over all 4.2M parameters, {seconds:.1f} s")
    return points / seconds, [q["points"] / q["seconds"] for q in r], sample


def oracle_rate_all_cores(budget_s: float, n: int = 2048):
    """The same oracle on every host core at once: one single-threaded process per core,
    each timing its own budget_s seconds of whole iterations; the rate is the sum of
    theirs.  Returns (points/s, cores) or raises."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET % {"root": ROOT, "n": n, "budget": budget_s, "steps": 1}
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=env) for _ in range(cores)]
    rate = 0.0
    try:
        for p in procs:
            out, err = p.communicate(timeout=600 + 2 * budget_s)
            if p.returncode != 0:
                raise RuntimeError(err[-2000:])
            q = json.loads(out.strip().splitlines()[-1])[0]
            rate += q["points"] / q["seconds"]
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    return rate, cores


# The CPU-baseline leg of the own arm: the oracle on a sample of the timed workload
# (one brick's parameters as the kernels read them, a strided sample of that brick's
# points from a timed batch, the GPU's targets as inputs).  The same subprocess compares
# the library's outputs on that sample (forward f, the training pass's losses and
# gradients) with the oracle's, exact and with the BF16 operand rounding, then times
# whole oracle iterations (forward + L_rec backward + density backward + Adam).
SAMPLE_SNIPPET = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, %(root)r)
from oracle import apmgsrn as ap
z = np.load(%(path)r)
p = {k: z[k].astype(np.float64) for k in ("F", "W1", "W2", "w3", "G")}
p["vmin"], p["vmax"] = float(z["vmin"]), float(z["vmax"])
x, v = z["x"].astype(np.float64), z["v"].astype(np.float64)
def rel(a, b):
    a, b = np.ravel(np.asarray(a, np.float64)), np.ravel(np.asarray(b, np.float64))
    d = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (d if d > 0 else 1.0))
errors = {}
readings = [("fp64_exact", None)] + ([("bf16_operands", ap.bf16)] if %(bf16)r else [])
for name, rnd in readings:
    g = ap.grad_rec(p, x, v, rnd=rnd)
    d = ap.grad_density(p["G"], x, g["h"])
    errors[name] = {"f": rel(z["f"], g["f"]), "L_rec": abs(float(z["L_rec"]) - g["L_rec"]) / abs(g["L_rec"]),
                    "L_den": abs(float(z["L_den"]) - d["L_den"]) / abs(d["L_den"]),
                    "dF": rel(z["dF"], g["dF"]), "dW1": rel(z["dW1"], g["dW1"]), "dW2": rel(z["dW2"], g["dW2"]),
                    "dw3": rel(z["dw3"], g["dw3"]), "dG": rel(z["dG"], d["dG"])}
keys = ("F", "W1", "W2", "w3", "G")
mom = {k: (np.zeros_like(p[k]), np.zeros_like(p[k])) for k in keys}
it = 0; done = 0; reps = 0
t0 = time.perf_counter()
while True:
    g = ap.grad_rec(p, x, v)
    d = ap.grad_density(p["G"], x, g["h"])
    grads = {"F": g["dF"], "W1": g["dW1"], "W2": g["dW2"], "w3": g["dw3"], "G": d["dG"]}
    it += 1
    for k in keys:
        lr = 1e-3 if k == "G" else 1e-2
        p[k], m1, m2 = ap.adam_update(p[k], grads[k], mom[k][0], mom[k][1], it, lr)
        mom[k] = (m1, m2)
    done += len(x); reps += 1
    if time.perf_counter() - t0 >= %(budget)f:
        break
print(json.dumps({"errors": errors, "points": done, "seconds": time.perf_counter() - t0, "reps": reps}))
"""


def gpu_sample(m, xyz, tgt, off, wl, n_sample=4096):
    """The library's outputs on a strided sample of brick 0's points of the last batch:
    f from srn_forward, and L_rec, L_den and every gradient from srn_backward with the
    density loss, through a one-brick model holding brick 0's parameters (same kernels,
    same precision).  Returns the arrays the oracle leg compares."""
    import numpy as np
    import torch
    from paper_2308_02494_gb300 import synth
    from paper_2308_02494_gb300.model import SRN
    b0, b1 = int(off[0]), int(off[1])
    stride = max(1, (b1 - b0) // n_sample)
    idx = torch.arange(b0, b1, stride, device="cuda")[:n_sample]
    xs, vs = xyz[idx].contiguous(), tgt[idx].contiguous()
    n = int(idx.numel())
    prm = m.get("params")[0]
    shape = synth.ModelShape(wl["grids"], wl["res"], wl["channels"], 64)
    one = SRN(shape, 1, precision=wl["precision"], max_points=n)
    one.set_params([prm])
    f = one.forward(xs, [0, n]).cpu().numpy()
    losses = one.backward(xs, vs, [0, n], density=True).cpu().numpy()
    g = one.get("grads")[0]
    torch.cuda.synchronize()
    stored = {k: np.asarray(prm[k], dtype=np.float32).astype(np.float64) for k in ("F", "W1", "W2", "w3", "G")}
    if wl["precision"] == "bf16":   # the kernels read the BF16 shadow of F and the decoder's matrices
        for k in ("F", "W1", "W2"):
            stored[k] = synth.round_bf16(stored[k])
    out = dict(stored, vmin=prm["vmin"], vmax=prm["vmax"], x=xs.cpu().numpy(), v=vs.cpu().numpy(), f=f,
               L_rec=losses[0, 0], L_den=losses[0, 1], dF=g["F"], dW1=g["W1"], dW2=g["W2"], dw3=g["w3"], dG=g["G"])
    del one
    return out, (f"brick 0's model ({'BF16 shadow of F, W1, W2' if wl['precision'] == 'bf16' else 'FP32'}) and "
                 f"{n} of its points (every {stride}th of a timed batch; targets from the GPU lookup)")


def oracle_sample_leg(sample, desc, budget_s, bf16):
    """Runs SAMPLE_SNIPPET on one host thread; returns (cpu_baseline dict, errors)."""
    import numpy as np
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "sample.npz")
        np.savez(path, **sample)
        code = SAMPLE_SNIPPET % {"root": ROOT, "path": path, "budget": budget_s, "bf16": bool(bf16)}
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                             timeout=900 + 2 * budget_s)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    cpu = {"value": r["points"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"FP64 oracle, 1 thread, {r['reps']} whole iterations (fwd + L_rec bwd + density bwd + Adam "
                     f"over all parameters) in {r['seconds']:.1f} s on {desc}"}
    return cpu, dict(r["errors"], sample=desc)


def run_reference(args, workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # every step a bounded sample (at least one whole iteration), all in one process
    steps = max(1, args.steps)
    value, _, sample = oracle_rate(max(0.2, args.cpu_seconds / steps), steps=steps, warmup=max(0, args.warmup))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": REF_WORKLOAD, "stands_for": workload["workload"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 8:
                continue
            for nm, val in zip(names, r[4:8]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- own leg
VOLUME_LAYOUT = "4^3-voxel tiles (srn_tile_volume, made once before any timing)"


def workload_of(name, n_points=1 << 18):
    if name == "dd8":
        return {"workload": "dd8: 8 bricks (2x2x2 of a 1024^3 Fourier volume, ghost 2), per-brick "
                            "batches U[2^16,2^19], M=64 R=32 C=2, MLP 128-64-64-1, BF16, density phase",
                "bricks": 8, "volume": 1024, "grids": 64, "res": 32, "channels": 2, "precision": "bf16",
                "l2": "inputs larger than L2 (4 GiB volume; 1.1 GB of parameters and Adam state streamed per step)",
                "volume_layout": VOLUME_LAYOUT}
    prec = "bf16" if name == "single-bf16" else "fp32"
    return {"workload": f"single model, 512^3 Fourier volume, N=2^{n_points.bit_length() - 1}, M=64 R=32 C=2, "
                        f"{prec.upper()}, density phase",
            "bricks": 1, "volume": 512, "grids": 64, "res": 32, "channels": 2, "precision": prec,
            "points": n_points, "l2": "inputs larger than L2 (512 MiB volume)", "volume_layout": VOLUME_LAYOUT}


def setup(wl, seed_offset=0):
    import numpy as np
    import torch
    from paper_2308_02494_gb300 import synth
    from paper_2308_02494_gb300.model import SRN, TiledVolume

    shape = synth.ModelShape(wl["grids"], wl["res"], wl["channels"], 64)
    vox = wl["volume"]
    modes = synth.fourier_modes(256, 1, 64, seed=0)
    lin, _, _ = synth.fourier_volume(vox, modes, device="cuda")
    # the volume in the library's tiled layout (srn_tile_volume), made once here, before
    # any timing, like the volume's upload; the ground-truth lookup reads it every step
    vol = TiledVolume(lin)
    del lin
    if wl["bricks"] == 8:
        boxes = synth.brick_boxes(vox, (2, 2, 2), ghost=2)
        counts = synth.uneven_counts(8, 1 << 16, 1 << 19, seed=1 + seed_offset)
    else:
        boxes = np.array([[0, 0, 0, vox - 1, vox - 1, vox - 1]], dtype=np.int64)
        counts = np.array([wl.get("points", 1 << 18)], dtype=np.int64)
    n_total = int(counts.sum())
    m = SRN(shape, n_bricks=wl["bricks"], precision=wl["precision"], max_points=n_total)
    m.set_params([synth.init_model(shape, 100 + b + seed_offset) for b in range(wl["bricks"])])
    off = SRN.offsets_of(counts)
    xyz = torch.empty((n_total, 3), dtype=torch.float32, device="cuda")
    tgt = torch.empty(n_total, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    return m, vol, boxes, off, xyz, tgt, n_total


def time_steps(m, vol, boxes, off, xyz, tgt, steps, warmup, stream, sync_all, per_step=False):
    """Warm-up steps, then `steps` timed steps between CUDA events on the launching
    stream.  Returns the total ms, and with per_step the ms of every step (an event
    pair around each replay)."""
    import torch
    with torch.cuda.stream(stream):
        for i in range(warmup):
            m.train_step(7, vol, boxes, off, True, xyz, tgt, stream=stream)
        stream.synchronize()
        sync_all()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1 if per_step else 2)]
        evs[0].record(stream)
        for i in range(steps):
            m.train_step(7, vol, boxes, off, True, xyz, tgt, stream=stream)
            if per_step:
                evs[i + 1].record(stream)
        if not per_step:
            evs[1].record(stream)
        stream.synchronize()
    sync_all()
    total = evs[0].elapsed_time(evs[-1])
    if not per_step:
        return total
    return total, [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]


def spread(ms_list):
    import numpy as np
    a = np.asarray(ms_list, dtype=np.float64)
    return {"median_ms": float(np.median(a)), "p10_ms": float(np.percentile(a, 10)),
            "p90_ms": float(np.percentile(a, 90)), "min_ms": float(a.min()), "max_ms": float(a.max()),
            "steps": int(a.size)}


def reduce_over_ranks(points, ms, world, device):
    """Whole-job totals for the JSON line: points summed over the ranks, time of the
    slowest rank (ranks train disjoint bricks; no other data crosses ranks)."""
    if world == 1:
        return points, ms
    import torch
    import torch.distributed as dist
    p = torch.tensor([float(points)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return int(round(p.item())), float(t.item())


def render_roofline(queries_per_s, wl, tf_sus, sms, sm_mhz, src):
    """Forward queries of the renderer against the tensor pipe (decoder forward flops)
    and against the shared-memory/L1 data path (8 corners x C features per grid)."""
    m, c = wl["grids"], wl["channels"]
    flop = 2 * MLP_MACS_FWD
    gather_bytes = m * 8 * c * 2
    l1 = 128 * sms * sm_mhz * 1e6 / 1e9   # 128 B per SM clock
    t = queries_per_s * flop / 1e12
    g = queries_per_s * gather_bytes / 1e9
    tens = {"achieved": t, "peak": tf_sus, "unit": "TFLOP/s", "frac": t / tf_sus,
            "algorithmic": f"{flop} decoder forward flop per query", "peak_source": f"{src} bf16 sustained"}
    gath = {"achieved": g, "peak": l1, "unit": "GB/s", "frac": g / l1,
            "algorithmic": f"{gather_bytes} B of BF16 corner features per query (M x 8 x C)",
            "peak_source": f"nominal shared-memory/L1 data path, 128 B per SM clock x {sms} SMs x {sm_mhz:.0f} MHz"}
    bind = "gather" if gath["frac"] >= tens["frac"] else "tensor"
    return {"bound": bind, "tensor": tens, "gather": gath}


def render_rate(m, boxes, vox, width=1024, height=1024, samples=512):
    """Frames/s of the headless renderer over the 8-brick model: one orthographic and one
    perspective view, CUDA events around each frame on its stream."""
    import torch
    from paper_2308_02494_gb300 import synth
    lut = torch.as_tensor(synth.random_lut(3), device="cuda")
    views = synth.random_views(2, 5)
    cams = [synth.orbit_camera(views[0][0], views[0][1], True), synth.orbit_camera(views[1][0], views[1][1], False)]
    rgba = torch.empty((height, width, 4), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m.render(cams[0], lut, 0.0, 1.0, 64, 64, samples, (2, 2, 2), boxes, vox, stream=s)   # warm-up
        s.synchronize()
        times = []
        for cam in cams:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            m.render(cam, lut, 0.0, 1.0, width, height, samples, (2, 2, 2), boxes, vox, rgba=rgba, stream=s)
            e1.record(s)
            s.synchronize()
            times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    return {"frames_per_s": 1e3 / ms, "ms_per_frame": ms, "queries_per_s": width * height * samples / (ms / 1e3),
            "width": width, "height": height, "samples": samples,
            "views": "orthographic + perspective, random angles (seed 5), random 8-knot LUT (seed 3)",
            "ms_per_view": times}


def decode_rate(m, boxes, vox):
    """Points/s of the full-volume decode (srn_decode) of the 8-brick model over the
    whole vox^3 lattice, CUDA events around the call on its stream."""
    import torch
    out = torch.empty((vox, vox, vox), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        from paper_2308_02494_gb300 import synth
        m.decode((2, 2, 2), synth.brick_boxes(64, (2, 2, 2), ghost=2), 64, stream=s)   # warm-up
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        m.decode((2, 2, 2), boxes, vox, out=out, stream=s)
        e1.record(s)
        s.synchronize()
    ms = e0.elapsed_time(e1)
    return {"points_per_s": vox ** 3 / (ms / 1e3), "ms": ms, "volume": vox,
            "note": "every voxel of the lattice through its brick's model (BF16 forward), output written to HBM"}


def single_model_leg(name, n_points, steps, sync_all, errors=False):
    """Throughput of one single-model workload (512^3 volume, 2^k points, density phase)
    and, with errors, its library outputs on a sample for the oracle leg."""
    import torch
    wl = workload_of(name, n_points)
    m, vol, boxes, off, xyz, tgt, n = setup(wl)
    s = torch.cuda.Stream()
    time_steps(m, vol, boxes, off, xyz, tgt, 0, 3, s, sync_all)
    ms = time_steps(m, vol, boxes, off, xyz, tgt, steps, 0, s, sync_all)
    leg = {"value": n * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "workload": wl["workload"]}
    smp = gpu_sample(m, xyz, tgt, off, wl) if errors else None
    del m, vol, xyz, tgt
    torch.cuda.empty_cache()
    return leg, smp


def run_own(args, workload):
    if args.volume:
        workload = dict(workload, volume=args.volume,
                        workload=workload["workload"] + f" [volume {args.volume}^3]",
                        l2=f"volume {args.volume}^3 ({4 * args.volume ** 3 / 2 ** 20:.0f} MiB); 1.1 GB of "
                           "parameters and Adam state streamed per step")
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2308_02494_gb300 import srn as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    wl = workload
    # every rank trains its own bricks: different models and uneven batch sizes per rank
    m, vol, boxes, off, xyz, tgt, n_total = setup(wl, seed_offset=rank)
    stream = torch.cuda.Stream()
    tiles = None
    if wl["precision"] == "bf16":
        if args.tiles == "auto":   # the library's tuner on one batch of the workload, before any timing
            m.sample_points(5, 0, off, xyz)
            m.sample_target(vol, boxes, xyz, off, tgt)
            tiles = dict(m.autotune(xyz, tgt, off, density=True, reps=3), picked_by="srn_autotune")
        else:
            tiles = dict(m.tuning, picked_by="library default")
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    # warm up (first call eager, second captures the CUDA graph, the rest replay it)
    time_steps(m, vol, boxes, off, xyz, tgt, 0, max(3, args.warmup), stream, sync_all)
    clocks.start()
    ms, per_step = time_steps(m, vol, boxes, off, xyz, tgt, args.steps, 0, stream, sync_all, per_step=True)
    clk = clocks.stop()
    m.status(stream)
    points_all, ms = reduce_over_ranks(n_total * args.steps, ms, world, "cuda")
    value = points_all / (ms / 1e3)
    losses = m.losses.cpu().numpy()

    # per-kernel times: the library's CUDA-event hook (events on the launching stream)
    # over eager steps of the same workload, one kernel at a time
    bf16 = wl["precision"] == "bf16"
    k_steps = min(args.steps, 30)
    dflt = torch.cuda.default_stream()
    targets = [("query", S.SRN_TIME_QUERY)]
    if bf16:
        targets += [("k_enc", S.SRN_TIME_ENCODER), ("k_mlp", S.SRN_TIME_DECODER), ("k_scat", S.SRN_TIME_SCATTER)]
    kt = {}
    for name, which in targets:
        S.srn_set_timing(m.handle, which)
        for _ in range(k_steps):
            m.train_step(7, vol, boxes, off, True, xyz, tgt, stream=dflt)
        torch.cuda.synchronize()
        k_ms, k_n = S.srn_read_timing(m.handle)
        kt[name] = k_ms / max(1, k_n)
    S.srn_set_timing(m.handle, S.SRN_TIME_OFF)
    hbm, tf_burst, tf_sus, src = peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or 2070.0   # the median SM clock under load (nominal max without a record)
    step_ms = ms / args.steps
    floors = step_floors(wl, n_total, step_ms, hbm, tf_sus, sms, sm_mhz, src)
    if bf16:
        rl = kernel_rooflines(wl, n_total, kt, hbm, tf_sus, sms, sm_mhz, src)
        dom = max(rl, key=lambda k: rl[k]["kernel_ms"])
        roof = dict(rl[dom], kernel=dom, query_pass_ms=kt["query"],
                    others={k: v for k, v in rl.items() if k != dom}, step=floors)
    else:
        fp32_peak = 2 * FP32_LANES_PER_SM * sms * sm_mhz * 1e6 / 1e12
        ach = FLOP_PER_POINT * n_total / (kt["query"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": None, "kernel": "k_query_f32 (fused)", "kernel_ms": kt["query"],
                "peak_source": f"nominal FP32 FMA rate, {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 flop at "
                               f"{sm_mhz:.0f} MHz",
                "algorithmic": f"{FLOP_PER_POINT} decoder flop per point", "step": floors}

    e2e = None
    render = None
    decode = None
    legs = {}
    samples = {}
    if not args.no_extras and wl["bricks"] == 8:
        render = render_rate(m, boxes, wl["volume"])
        render["roofline"] = render_roofline(render["queries_per_s"], wl, tf_sus, sms, sm_mhz, src)
        decode = decode_rate(m, boxes, wl["volume"])
    if not args.no_extras:
        if rank == 0 and world == 1:   # a sample of the timed workload for the oracle leg
            samples["main"] = gpu_sample(m, xyz, tgt, off, wl)
        # end to end through the C ABI: pinned host points/targets -> device, backward+step, losses -> host
        m.sample_points(11, 0, off, xyz)
        m.sample_target(vol, boxes, xyz, off, tgt)
        torch.cuda.synchronize()
        hx = xyz.cpu().pin_memory()
        ht = tgt.cpu().pin_memory()
        hl = torch.empty_like(m.losses, device="cpu").pin_memory()
        e_steps = min(args.steps, 50)
        with torch.cuda.stream(stream):
            for it in range(3 + e_steps):
                if it == 3:
                    stream.synchronize()
                    t0 = time.perf_counter()
                xyz.copy_(hx, non_blocking=True)
                tgt.copy_(ht, non_blocking=True)
                m.backward(xyz, tgt, off, density=True, stream=stream)
                m.step(density=True, stream=stream)
                hl.copy_(m.losses, non_blocking=True)
            stream.synchronize()
            el = time.perf_counter() - t0
        e_points, e_ms = reduce_over_ranks(n_total * e_steps, el * 1e3, world, "cuda")
        e2e = {"value": e_points / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(hx.numel() * 4 + ht.numel() * 4),
               "d2h_bytes_per_step": int(hl.numel() * 8),
               "path": "srn_backward(SRN_DENSITY) + srn_step with host-pinned points/targets, losses read back"}
        # single-model legs on the same GPU: the FP32 plain path (the speedup's denominator)
        # and the BF16 path on the same model and batch, then the BF16 path at 2^20 points
        del m, vol
        torch.cuda.empty_cache()
        one = rank == 0 and world == 1
        n_leg = min(args.steps, 40)
        legs["fp32_plain_2^18"], samples["fp32"] = single_model_leg("single-fp32", 1 << 18, n_leg, sync_all, one)
        legs["bf16_single_2^18"], _ = single_model_leg("single-bf16", 1 << 18, n_leg, sync_all)
        legs["bf16_single_2^20"], _ = single_model_leg("single-bf16", 1 << 20, n_leg, sync_all)

    if rank != 0:
        return
    cpu = None
    errors = None
    if world == 1:
        if "main" in samples:
            cpu, err_main = oracle_sample_leg(*samples["main"], budget_s=args.cpu_seconds, bf16=bf16)
            errors = {wl["precision"] + "_batched": err_main}
            if samples.get("fp32"):
                _, err32 = oracle_sample_leg(*samples["fp32"], budget_s=0.0, bf16=False)
                errors["fp32_plain"] = err32
        else:
            rate, _, sample = oracle_rate(args.cpu_seconds)
            cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
        try:   # the same oracle on all host cores, one process per core (reported beside)
            r_all, n_all = oracle_rate_all_cores(min(args.cpu_seconds, 12.0))
            cpu["all_cores"] = {"value": r_all, "unit": UNIT, "cores": n_all,
                                "sample": f"{n_all} concurrent single-threaded oracle processes, each training "
                                          "one model on 2048-point batches of a 64^3 volume"}
        except Exception as exc:   # never let the extra figure cost the bench line
            cpu["all_cores"] = {"error": str(exc)[-300:]}
    cfg = dict(wl)
    cfg["points_per_step"] = points_all // args.steps
    cfg["parallelism"] = f"{world} GPUs, each training its own 8 bricks (no collective)" if world > 1 else "1 GPU"
    if tiles:
        cfg["tiles"] = tiles
    if render:
        cfg["render"] = render
    if decode:
        cfg["decode"] = decode
    if legs:
        cfg["single_model_legs"] = legs
        f32 = legs["fp32_plain_2^18"]["value"]
        cfg["speedup_vs_fp32_plain"] = {
            "batched_bf16_vs_fp32_plain": value / world / f32,
            "same_model_and_batch_bf16_vs_fp32": legs["bf16_single_2^18"]["value"] / f32,
            "note": "BF16 operands carry the errors in 'errors' (rel L2 against the FP64 oracle); the FP32 "
                    "path's are in errors.fp32_plain"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "step_spread": spread(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": wl["precision"],
            "data": "synthetic", "config": cfg, "clocks": clk, "e2e": e2e,
            "gpu_launches": KERNELS_PER_STEP[wl["precision"]] * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "errors": errors,
            "last_losses": {"L_rec_mean": float(np.mean(losses[:, 0])), "L_den_mean": float(np.mean(losses[:, 1]))}}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    wl = workload_of(args.workload)
    if args.impl == "reference":
        run_reference(args, wl)
        return
    run_own(args, wl)


if __name__ == "__main__":
    main()
