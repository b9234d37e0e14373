"""Helpers shared by the GPU parity tests: library build, model set-up from the
seeded generators, oracle-side parameter rounding, point filtering and error norms."""
import os

import numpy as np

from oracle import apmgsrn as ap
from paper_2308_02494_gb300 import synth

TOL = {"fp32": 1e-5, "bf16": 2e-3}   # rel L2 bars per output (FP32 path, BF16 path)


def ensure_built():
    from paper_2308_02494_gb300 import build as pb
    pb.build()


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def as_stored(params: dict, precision: str) -> dict:
    """The parameters exactly as the kernels read them: float32 masters, and for the
    BF16 path the bfloat16 (RNE) shadow of F, W1 and W2."""
    out = {}
    for k in ("F", "W1", "W2", "w3", "G"):
        out[k] = np.asarray(params[k], dtype=np.float32).astype(np.float64)
    if precision == "bf16":
        for k in ("F", "W1", "W2"):
            out[k] = synth.round_bf16(out[k])
    out["vmin"], out["vmax"] = params["vmin"], params["vmax"]
    return out


def points_off_faces(G, n, seed, margin=1e-5, lo=-1.0, hi=1.0):
    """n points uniform in [lo, hi)^3 whose local coordinates stay `margin` away from
    every grid's faces (the inside/outside decision of Eq. 2 is then the same in
    float32 and float64)."""
    r = np.random.default_rng(seed)
    keep = []
    total = 0
    while total < n:
        x = r.uniform(lo, hi, size=(2 * n + 64, 3)).astype(np.float32)
        u = ap.local_coords(G, x.astype(np.float64))
        ok = np.all(np.abs(np.abs(u) - 1.0) > margin, axis=(1, 2))
        keep.append(x[ok])
        total += int(ok.sum())
    return np.concatenate(keep)[:n]


def make_model(shape, n_bricks, precision, max_points, seed, shrink=0.4):
    import torch
    from paper_2308_02494_gb300.model import SRN
    models = [synth.parity_model(shape, seed + 101 * b, shrink=shrink) for b in range(n_bricks)]
    m = SRN(shape, n_bricks=n_bricks, precision=precision, max_points=max_points)
    m.set_params(models)
    torch.cuda.synchronize()
    return m, [as_stored(p, precision) for p in models]
