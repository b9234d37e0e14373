#!/usr/bin/env python3
"""Training-step throughput of the batched APMGSRN hot path on one GB300.

Workload (default "dd8"): a synthetic 1024^3 float32 turbulence volume split into
2x2x2 bricks of 512^3 (+2 ghost voxels), one APMGSRN per brick (M=64 grids of
32^3 x 2 channels, MLP 128->64->64->1, BF16 grids/decoder with FP32 masters),
uneven per-brick batches drawn from U[2^16, 2^19].  One step = sample the batch
(Philox + Morton counting sort) -> ground truth lookup -> fused forward/backward
of L_rec -> feature-density loss and its transform gradient -> Adam on every
parameter, replayed from a CUDA graph.  Throughput = points of all bricks per
second.  The roofline line is the slowest kernel of the training pass, timed with the
library's CUDA-event hook on eager steps of the same workload, against its
algorithmic bytes (HBM-bound kernels) or decoder flops (the tensor-core kernel).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "train fwd+bwd points/s (BF16 batched vs FP32 plain) at stated err; % roofline"
UNIT = "points/s"
# fused kernel: MACs per point of the 128->64->64->1 decoder, forward + backward
MLP_MACS_FWD = 128 * 64 + 64 * 64 + 64
MLP_MACS_BWD = 64 * 64 + 64 * 64 + 64 * 128 + 64 * 128 + 64
FLOP_PER_POINT = 2 * (MLP_MACS_FWD + MLP_MACS_BWD)
# kernels of one training step: sampler (3), target lookup, the query pass (BF16: scatter
# tile list (the unit starts come from the sampler), encoder, decoder, scatter; FP32: 1
# fused kernel), density passes (BF16: 3 on the second stream; FP32: 2), finalisation,
# step counter, Adam (BF16 density steps: F and the decoder, then G)
KERNELS_PER_STEP = {"bf16": 15, "fp32": 10}


# DRAM bytes (read + write) per launch of each training-pass kernel, from the ncu
# capture summarised in profiles/train_kernels_dd8.txt (the same 8-brick batch and
# model).  They hold only for the kernel sources they were taken on: any change to those
# files makes bench report traffic as null until a new capture.
NCU_TRAFFIC = {"sources_sha1": "7c156c05bdf0292936912669e94681a5df21ff4b",
               "k_scat": 1037.7e6, "k_enc": 716.1e6, "k_mlp": 1333.7e6}
TRAFFIC_SOURCES = ("k_train_bf16.cu", "k_mlp_tc.cu", "common.cuh", "bf16_ops.cuh", "tc_ops.cuh")


def measured_traffic(name):
    import hashlib
    h = hashlib.sha1()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2308_02494_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return NCU_TRAFFIC.get(name) if h.hexdigest() == NCU_TRAFFIC["sources_sha1"] else None


# On-chip rates for the gather and the scatter, whose per-(point, grid) corner work
# lives in shared memory: the scatter adds 8 x C contributions with conflict-free
# red.shared.add.u32 (measured on this GB300 with a probe of 16 warps per SM,
# conflict-free addresses: 0.94 warp instructions per SM clock); the encoder reads 8
# corners of C bf16 (one 4-byte word for C = 2) with conflict-free shared loads
# (nominal: one warp instruction of 32 x 4 B per SM clock).
SMEM_RED_PER_CLK = 0.94
SMEM_LDS_PER_CLK = 1.0


def onchip_rooflines(wl, n_total, kt, sms, sm_mhz):
    """Shared-memory instruction rooflines of k_scat and k_enc (warp instructions/s)."""
    m, c = wl["grids"], wl["channels"]
    work = {"k_scat": (n_total * m * 8 * c / 32, SMEM_RED_PER_CLK,
                       "8 corners x C channels per (point, grid), one lane each: shared integer reductions",
                       "measured red.shared.add.u32 rate, conflict-free"),
            "k_enc": (n_total * m * 8 / 32, SMEM_LDS_PER_CLK,
                      "8 corners per (point, grid), one lane each: shared loads of C bf16",
                      "nominal shared-load issue rate, conflict-free")}
    out = {}
    for name, (inst, per_clk, per, psrc) in work.items():
        ms = kt.get(name)
        if not ms:
            continue
        ach = inst / (ms / 1e3) / 1e9
        peak = per_clk * sms * sm_mhz * 1e6 / 1e9
        out[name] = {"bound": "smem", "achieved": ach, "peak": peak, "unit": "G warp instructions/s",
                     "frac": ach / peak, "algorithmic": per, "algorithmic_per_launch": inst,
                     "peak_source": f"{psrc}, {per_clk} per SM clock x {sms} SMs x {sm_mhz:.0f} MHz"}
    return out


def kernel_rooflines(wl, n_total, kt, hbm, tf_sus, src):
    """Roofline entries of the training-pass kernels from their measured mean times (ms)."""
    m, r, c = wl["grids"], wl["res"], wl["channels"]
    nb, k = wl["bricks"], wl["grids"] * wl["channels"]
    grid_vals = nb * m * r ** 3 * c
    algo = {
        "k_scat": ("hbm", n_total * (12 + m * c * 2) + 2 * 4 * grid_vals,
                   "xyz (12 B) + dL/dy (M*C bf16) per point; read+write of every FP32 feature-gradient grid"),
        "k_enc": ("hbm", n_total * (12 + k * 2) + 2 * grid_vals,
                  "xyz (12 B) + features y (K bf16) per point; every BF16 feature grid once"),
        "k_mlp": ("tensor", n_total * FLOP_PER_POINT, f"{FLOP_PER_POINT} flop per point (decoder fwd+bwd MACs x2)"),
    }
    out = {}
    for name, ms in kt.items():
        if name not in algo or not ms:
            continue
        bound, amount, per = algo[name]
        if bound == "hbm":
            ach, peak, unit, psrc = amount / (ms / 1e3) / 1e9, hbm, "GB/s", f"{src} HBM copy"
        else:
            ach, peak, unit, psrc = amount / (ms / 1e3) / 1e12, tf_sus, "TFLOP/s", f"{src} bf16 sustained"
        out[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                     "traffic": measured_traffic(name) if wl["bricks"] == 8 else None, "kernel_ms": ms, "peak_source": psrc, "algorithmic": per,
                     "algorithmic_per_launch": amount}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--workload", choices=["dd8", "single-bf16", "single-fp32"], default="dd8")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP32-plain and e2e legs")
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


# ----------------------------------------------------------------------------- oracle leg
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
    sample = (f"FP64 oracle, 1 thread: one brick's model (M=64, R=32, C=2, 128->64->64->1), "
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
            "data": "synthetic", "config": workload,
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
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
def workload_of(name):
    if name == "dd8":
        return {"workload": "dd8: 8 bricks (2x2x2 of a 1024^3 Fourier volume, ghost 2), per-brick "
                            "batches U[2^16,2^19], M=64 R=32 C=2, MLP 128-64-64-1, BF16, density phase",
                "bricks": 8, "volume": 1024, "grids": 64, "res": 32, "channels": 2, "precision": "bf16",
                "l2": "inputs larger than L2 (4 GiB volume; 1.1 GB of parameters and Adam state streamed per step)"}
    if name == "single-bf16":
        return {"workload": "single model, 512^3 Fourier volume, N=2^18, M=64 R=32 C=2, BF16, density phase",
                "bricks": 1, "volume": 512, "grids": 64, "res": 32, "channels": 2, "precision": "bf16",
                "l2": "inputs larger than L2 (512 MiB volume)"}
    return {"workload": "single model, 512^3 Fourier volume, N=2^18, M=64 R=32 C=2, FP32, density phase",
            "bricks": 1, "volume": 512, "grids": 64, "res": 32, "channels": 2, "precision": "fp32",
            "l2": "inputs larger than L2 (512 MiB volume)"}


def setup(wl, seed_offset=0):
    import numpy as np
    import torch
    from paper_2308_02494_gb300 import synth
    from paper_2308_02494_gb300.model import SRN

    shape = synth.ModelShape(wl["grids"], wl["res"], wl["channels"], 64)
    vox = wl["volume"]
    modes = synth.fourier_modes(256, 1, 64, seed=0)
    vol, _, _ = synth.fourier_volume(vox, modes, device="cuda")
    if wl["bricks"] == 8:
        boxes = synth.brick_boxes(vox, (2, 2, 2), ghost=2)
        counts = synth.uneven_counts(8, 1 << 16, 1 << 19, seed=1 + seed_offset)
    else:
        boxes = np.array([[0, 0, 0, vox - 1, vox - 1, vox - 1]], dtype=np.int64)
        counts = np.array([1 << 18], dtype=np.int64)
    n_total = int(counts.sum())
    m = SRN(shape, n_bricks=wl["bricks"], precision=wl["precision"], max_points=n_total)
    m.set_params([synth.init_model(shape, 100 + b + seed_offset) for b in range(wl["bricks"])])
    off = SRN.offsets_of(counts)
    xyz = torch.empty((n_total, 3), dtype=torch.float32, device="cuda")
    tgt = torch.empty(n_total, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    return m, vol, boxes, off, xyz, tgt, n_total


def time_steps(m, vol, boxes, off, xyz, tgt, steps, warmup, stream, sync_all):
    import torch
    with torch.cuda.stream(stream):
        for i in range(warmup):
            m.train_step(7, vol, boxes, off, True, xyz, tgt, stream=stream)
        stream.synchronize()
        sync_all()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(steps):
            m.train_step(7, vol, boxes, off, True, xyz, tgt, stream=stream)
        ev1.record(stream)
        stream.synchronize()
    sync_all()
    return ev0.elapsed_time(ev1)


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
    ms = time_steps(m, vol, boxes, off, xyz, tgt, args.steps, 0, stream, sync_all)
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
    if bf16:
        rl = kernel_rooflines(wl, n_total, kt, hbm, tf_sus, src)
        dom = max(rl, key=lambda k: rl[k]["kernel_ms"])
        roof = dict(rl[dom], kernel=dom, query_pass_ms=kt["query"],
                    others={k: {f: v[f] for f in ("bound", "achieved", "unit", "frac", "kernel_ms")}
                            for k, v in rl.items() if k != dom})
        # the gather's and the scatter's shared-memory work against its instruction rate,
        # at the highest SM clock seen (nominal 2070 MHz without a clock record)
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        roof["onchip"] = onchip_rooflines(wl, n_total, kt, sms, clk.get("sm_max_mhz") or 2070.0)
    else:
        fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 FMA lanes x 2 flop x max SM clock
        ach = FLOP_PER_POINT * n_total / (kt["query"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": None, "kernel": "k_query_f32 (fused)", "kernel_ms": kt["query"],
                "peak_source": "nominal FP32 FMA rate, 152 SMs x 128 lanes at 2.07 GHz",
                "algorithmic": f"{FLOP_PER_POINT} decoder flop per point"}

    # end to end through the C ABI: pinned host points/targets -> device, backward+step, losses -> host
    e2e = None
    fp32_plain = None
    render = None
    decode = None
    if not args.no_extras and wl["bricks"] == 8:
        render = render_rate(m, boxes, wl["volume"])
        decode = decode_rate(m, boxes, wl["volume"])
    if not args.no_extras:
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
        # the plain FP32 single-model path (the speedup denominator)
        del m, vol
        torch.cuda.empty_cache()
        wl32 = workload_of("single-fp32")
        m2, vol2, boxes2, off2, xyz2, tgt2, n2 = setup(wl32)
        s2 = torch.cuda.Stream()
        time_steps(m2, vol2, boxes2, off2, xyz2, tgt2, 0, 3, s2, sync_all)
        ms2 = time_steps(m2, vol2, boxes2, off2, xyz2, tgt2, min(args.steps, 40), 0, s2, sync_all)
        fp32_plain = {"value": n2 * min(args.steps, 40) / (ms2 / 1e3), "unit": UNIT,
                      "workload": wl32["workload"]}

    if rank != 0:
        return
    cpu = None
    if world == 1:
        rate, _, sample = oracle_rate(args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
        try:   # the same oracle on all host cores, one process per core (reported beside)
            r_all, n_all = oracle_rate_all_cores(min(args.cpu_seconds, 12.0))
            cpu["all_cores"] = {"value": r_all, "unit": UNIT, "cores": n_all,
                                "sample": f"{n_all} concurrent single-threaded oracle processes, each as above"}
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
    if fp32_plain:
        cfg["fp32_plain"] = fp32_plain
        cfg["speedup_vs_fp32_plain"] = value / world / fp32_plain["value"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl["precision"], "data": "synthetic",
            "config": cfg, "clocks": clk, "e2e": e2e, "gpu_launches": KERNELS_PER_STEP[wl["precision"]] * args.steps,
            "roofline": roof, "cpu_baseline": cpu,
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
