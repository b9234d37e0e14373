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


def density_grad_scale(G, x, h, p=10, eps=1e-8):
    """Per-entry magnitude of the sum behind dL_den/dG: the same chain as the
    oracle's gradient with every summand replaced by its absolute value.  Float
    summation of N terms errs by at most ~N u sum|terms| (u the unit roundoff), so
    where the terms nearly cancel (all points deep inside every flat top, so that
    sum q E ~ 0) the error is bounded by this scale, not by |dL/dG| itself."""
    G = np.asarray(G, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    E, det, u = ap.flat_top_terms(G, x, p)
    t = ap.density_terms(E @ det, h, eps)
    g = -t["rho_star"] / (n * (t["rho_s"] + eps))
    q = np.abs(g - np.sum(g * t["rho_s"])) / t["S"]
    out = np.zeros_like(G)
    for i in range(G.shape[0]):
        inv_t = np.abs(np.linalg.inv(G[i, :, :3]).T)
        up = np.abs(2 * p * u[:, i, :] ** (2 * p - 1))
        wq = q * E[:, i] * abs(det[i])
        out[i, :, :3] = np.sum(wq) * inv_t + (wq[:, None] * up).T @ np.abs(x)
        out[i, :, 3] = (wq[:, None] * up).sum(axis=0)
    return out


def dG_error(got, want, scale) -> float:
    """Max over entries of |got - want| relative to the entry's summation scale."""
    return float(np.max(np.abs(np.asarray(got) - want) / (scale + 1e-300)))


def morton_order(x, bits=5):
    """Permutation that orders x by the Morton code of its 2^bits-per-axis bin (the
    order the library's sampler produces), stable inside a bin."""
    x = np.asarray(x)
    cell = np.minimum(((x.astype(np.float64) + 1.0) * (1 << bits) / 2.0).astype(np.int64), (1 << bits) - 1)
    cell = np.maximum(cell, 0)
    code = np.zeros(len(x), dtype=np.int64)
    for bit in range(bits):
        for a in range(3):
            code |= ((cell[:, a] >> bit) & 1) << (3 * bit + a)
    return np.argsort(code, kind="stable")


def morton_sorted(x, bits=5):
    """x in the order of morton_order."""
    x = np.asarray(x)
    return x[morton_order(x, bits)]


def near_bf16_midpoint(a, eps, min_ulp=3e-5):
    """Entries of a within eps (absolute, broadcast) of a bfloat16 rounding midpoint,
    among those whose bfloat16 spacing is at least min_ulp (a one-step change of a
    smaller entry moves nothing downstream by more than min_ulp times its weight)."""
    a = np.abs(np.asarray(a, dtype=np.float64))
    e = np.floor(np.log2(np.maximum(a, 1e-300)))
    ulp = np.exp2(e - 7)                      # 8 significant bits
    q = a / ulp
    dist = np.abs(q - np.floor(q) - 0.5) * ulp
    return (dist < eps) & (ulp >= min_ulp) & (a > 0)


def points_off_kinks(params, x, rnd, margin=2e-3):
    """Keep the points whose decoder pre-activations (oracle, with the path's operand
    rounding) all stay `margin` x their layer's RMS away from zero: the ReLU mask is an
    FP-decided switch, and BF16 operand rounding ties decided differently in float32 and
    float64 (about 2^-15 of operands) would otherwise flip a handful of masks, each
    moving one gradient entry by its own size."""
    y = ap.encode(params["F"], params["G"], np.asarray(x, dtype=np.float64))
    _, c = ap.mlp_forward(params["W1"], params["W2"], params["w3"], y, rnd)
    ok = np.ones(len(x), dtype=bool)
    for z in (c["z1"], c["z2"]):
        rms = np.sqrt(np.mean(z * z)) + 1e-30
        ok &= np.all(np.abs(z) > margin * rms, axis=1)
    return np.asarray(x)[ok]


def points_off_bf16_midpoints(params, x):
    """Keep the points whose BF16 operand roundings are the same in float32 and float64:
    no feature y and no ReLU(z1) lies within the float32 error of its computation (the
    8-corner blend, ~2^-22 of the largest feature; the K-term dot product, ~4e-7 of its
    absolute terms) of a bfloat16 rounding midpoint, where the kernel (rounding a float32
    value) and the oracle (rounding a float64 value) would pick neighbouring bfloat16
    numbers.  Such a one-step change of an operand of 2^-8 relative size moves f by up
    to ~1e-3 and, through dL/dm, that point's whole gradient."""
    x = np.asarray(x)
    y = ap.encode(params["F"], params["G"], x.astype(np.float64))
    _, c = ap.mlp_forward(params["W1"], params["W2"], params["w3"], y, ap.bf16)
    fmax = float(np.max(np.abs(params["F"])))
    ok = ~np.any(near_bf16_midpoint(y, 2.5e-7 * fmax, 3e-5), axis=1)
    scale = np.abs(c["yq"]) @ np.abs(np.asarray(params["W1"], dtype=np.float64)).T
    ok &= ~np.any(near_bf16_midpoint(c["h1"], 4e-7 * scale, 3e-5), axis=1)
    return x[ok]


def make_model(shape, n_bricks, precision, max_points, seed, shrink=0.4):
    import torch
    from paper_2308_02494_gb300.model import SRN
    models = [synth.parity_model(shape, seed + 101 * b, shrink=shrink) for b in range(n_bricks)]
    m = SRN(shape, n_bricks=n_bricks, precision=precision, max_points=max_points)
    m.set_params(models)
    torch.cuda.synchronize()
    return m, [as_stored(p, precision) for p in models]

# Operand rounding of the decoder's matrix products in each path (the kernel's
# precision, in which the ReLU masks are decided), and the looser bounds against the
# exact FP64 oracle: BF16 operands perturb pre-activations by ~2^-9 relative, which
# flips the ReLU mask of near-zero units and moves each such gradient entry by its
# own size (measured: forward ~3e-3, gradients up to ~5e-2 rel L2).
RND = {"fp32": None, "bf16": ap.bf16}
EXACT = {"fp32": {"value": 1e-5, "grad": 1e-5}, "bf16": {"value": 1e-2, "grad": 1e-1}}
