"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds random draws and workload recipes only: point batches, the
parameter initialisation of Sec. 4.3.3, synthetic volumes standing in for the
paper's datasets (Table 1), cameras and transfer functions.  None of the
model's arithmetic (Eq. 1-9, the decoder, Adam, compositing) lives here, so the
oracle and the CUDA path can both consume these inputs without sharing code.

Everything is deterministic in its ``seed`` (numpy PCG64 via ``default_rng``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class ModelShape:
    """Shape of one APMGSRN (Sec. 4.1): M grids of R^3 nodes with C channels,
    and a bias-free MLP K -> H -> H -> 1 with K = M*C."""

    n_grids: int = 64
    res: int = 32
    channels: int = 2
    hidden: int = 64

    @property
    def feat(self) -> int:
        return self.n_grids * self.channels


# --------------------------------------------------------------------------- points
def uniform_points(n: int, seed: int) -> np.ndarray:
    """n points uniform in [-1, 1)^3 as float32 [n, 3] (the batch of Sec. 6 "Training")."""
    r = np.random.default_rng(seed)
    return (r.random((n, 3)) * 2.0 - 1.0).astype(np.float32)


# --------------------------------------------------------------------------- parameters
def init_transforms(m: int, rng: np.random.Generator, std: float = 0.05) -> np.ndarray:
    """[m, 3, 4] first three rows of each G_i (Sec. 4.3.3): diagonal ~ N(1, std),
    every other entry of the first three rows (translation included) ~ N(0, std)."""
    g = rng.normal(0.0, std, size=(m, 3, 4))
    for d in range(3):
        g[:, d, d] += 1.0
    return g


def kaiming_uniform(fan_out: int, fan_in: int, rng: np.random.Generator) -> np.ndarray:
    """Kaiming-uniform draw for a ReLU layer: U(-b, b) with b = sqrt(6 / fan_in)."""
    b = math.sqrt(6.0 / fan_in)
    return rng.uniform(-b, b, size=(fan_out, fan_in))


def init_model(shape: ModelShape, seed: int, feat_amp: float = 1e-4,
               xform_std: float = 0.05, vmin: float = 0.0, vmax: float = 1.0) -> dict:
    """One model's parameters in float64 (callers round to their storage type).

    F  [M, R, R, R, C]  features, z-major, channel innermost, ~ U(-feat_amp, feat_amp)
    G  [M, 3, 4]        transforms (see init_transforms)
    W1 [H, K], W2 [H, H], w3 [H]   decoder weights, Kaiming-uniform
    vmin, vmax          the saved data range of Sec. 4.1.2 "Scaling"
    """
    r = np.random.default_rng(seed)
    m, res, c, h = shape.n_grids, shape.res, shape.channels, shape.hidden
    return {
        "F": r.uniform(-feat_amp, feat_amp, size=(m, res, res, res, c)),
        "G": init_transforms(m, r, xform_std),
        "W1": kaiming_uniform(h, shape.feat, r),
        "W2": kaiming_uniform(h, h, r),
        "w3": kaiming_uniform(1, h, r)[0],
        "vmin": float(vmin),
        "vmax": float(vmax),
    }


def parity_model(shape: ModelShape, seed: int, shrink: float = 0.0) -> dict:
    """A "trained-looking" model for parity tests: O(1) features so that every
    term of the decoder matters, and transforms that may zoom grids in by up to
    (1 + shrink) so that some points fall outside some grids."""
    r = np.random.default_rng(seed)
    p = init_model(shape, seed, feat_amp=1.0)
    if shrink > 0.0:
        s = 1.0 + shrink * r.random(shape.n_grids)
        p["G"][:, :, :3] *= s[:, None, None]
        p["G"][:, :, 3] += r.uniform(-0.3, 0.3, size=(shape.n_grids, 3))
    p["vmin"], p["vmax"] = -0.5, 1.5
    return p


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round float64/float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# --------------------------------------------------------------------------- volumes
def voxel_coords(v: int) -> np.ndarray:
    """Global coordinate of voxel j on a corner-aligned axis of v voxels: -1 + 2j/(v-1)."""
    return -1.0 + 2.0 * np.arange(v) / (v - 1)


def gaussian_volume(v: int = 64, n_gauss: int = 16, seed: int = 0):
    """v^3 float32 volume [z, y, x] = sum of n_gauss isotropic Gaussians with centres
    U[-1,1]^3, sigma U[0.05, 0.3], amplitude U[-1, 1].  Returns (volume, params)."""
    r = np.random.default_rng(seed)
    cen = r.uniform(-1, 1, size=(n_gauss, 3))
    sig = r.uniform(0.05, 0.3, size=n_gauss)
    amp = r.uniform(-1, 1, size=n_gauss)
    ax = voxel_coords(v)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    vol = np.zeros((v, v, v))
    for g in range(n_gauss):
        d2 = (x - cen[g, 0]) ** 2 + (y - cen[g, 1]) ** 2 + (z - cen[g, 2]) ** 2
        vol += amp[g] * np.exp(-d2 / (2 * sig[g] ** 2))
    return vol.astype(np.float32), {"centre": cen, "sigma": sig, "amp": amp}


def fourier_modes(n_modes: int = 256, kmin: float = 1.0, kmax: float = 64.0, seed: int = 0):
    """n_modes integer wave vectors with kmin <= |k| <= kmax (rejection sampled from
    the cube [-kmax, kmax]^3), amplitude |k|^(-5/3), phase U[0, 2pi)."""
    r = np.random.default_rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = r.integers(-int(kmax), int(kmax) + 1, size=3)
        n = float(np.linalg.norm(k))
        if kmin <= n <= kmax:
            ks.append(k)
    k = np.array(ks, dtype=np.float64)
    amp = np.linalg.norm(k, axis=1) ** (-5.0 / 3.0)
    phase = r.uniform(0, 2 * np.pi, size=n_modes)
    return {"k": k, "amp": amp, "phase": phase}


def fourier_value(modes: dict, x: np.ndarray) -> np.ndarray:
    """Unnormalised turbulence field phi(x) = sum_m a_m cos(pi k_m.(x+1) + phase_m), float64."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    arg = np.pi * (x + 1.0) @ modes["k"].T + modes["phase"][None, :]
    return (np.cos(arg) * modes["amp"][None, :]).sum(axis=1)


def fourier_volume(v: int, modes: dict, device="cpu", z_chunk: int = 64):
    """v^3 float32 torch tensor [z, y, x] of the Fourier field at voxel centres,
    normalised to [0, 1] by its own voxel min/max.  Evaluated as a rank-n_modes
    separable sum (one real matmul per z-chunk).  Returns (volume, lo, hi) where
    lo/hi are the raw min/max used for the normalisation."""
    import torch

    ax = torch.as_tensor(voxel_coords(v), dtype=torch.float64, device=device)
    k = torch.as_tensor(modes["k"], dtype=torch.float64, device=device)
    amp = torch.as_tensor(modes["amp"], dtype=torch.float64, device=device)
    ph = torch.as_tensor(modes["phase"], dtype=torch.float64, device=device)
    th = torch.pi * (ax[None, :] + 1.0)                      # [1, v]
    ex = torch.polar(torch.ones_like(th * k[:, 0:1]), th * k[:, 0:1])  # [m, v]
    ey = torch.polar(torch.ones_like(th * k[:, 1:2]), th * k[:, 1:2])
    ez = torch.polar(torch.ones_like(th * k[:, 2:3]), th * k[:, 2:3])
    wz = (amp * torch.polar(torch.ones_like(ph), ph))[:, None] * ez   # [m, v]
    q = torch.cat([ex.real, ex.imag], 0).to(torch.float32)            # [2m, v]
    vol = torch.empty((v, v, v), dtype=torch.float32, device=device)
    for z0 in range(0, v, z_chunk):
        z1 = min(v, z0 + z_chunk)
        p = ey.T[None, :, :] * wz.T[z0:z1, None, :]                    # [zc, v(y), m]
        pr = torch.cat([p.real, -p.imag], 2).to(torch.float32)         # [zc, v, 2m]
        vol[z0:z1] = torch.matmul(pr, q)
    lo, hi = float(vol.min()), float(vol.max())
    vol.sub_(lo).div_(hi - lo)
    return vol, lo, hi


# --------------------------------------------------------------------------- bricks
def brick_boxes(v: int, grid=(2, 2, 2), ghost: int = 2) -> np.ndarray:
    """Voxel boxes of an I x J x K domain decomposition (Sec. 5.1) of a v^3 volume.

    Brick (i, j, k) covers, per axis, its nominal v/I voxels extended by `ghost`
    voxels on each side and clipped to the volume.  Returned as int64 [B, 6] =
    (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z), inclusive, in x-fastest brick order
    (flat index i + I*j + I*J*k)."""
    out = []
    ii, jj, kk = grid
    for k in range(kk):
        for j in range(jj):
            for i in range(ii):
                box = []
                for idx, n in ((i, ii), (j, jj), (k, kk)):
                    w = v // n
                    box.append(max(0, idx * w - ghost))
                lo = box
                hi = []
                for idx, n in ((i, ii), (j, jj), (k, kk)):
                    w = v // n
                    hi.append(min(v - 1, idx * w + w - 1 + ghost))
                out.append(lo + hi)
    return np.array(out, dtype=np.int64)


def uneven_counts(n_bricks: int, lo: int, hi: int, seed: int, multiple: int = 1) -> np.ndarray:
    """Per-brick point counts U[lo, hi], rounded down to a multiple of `multiple`."""
    r = np.random.default_rng(seed)
    c = r.integers(lo, hi + 1, size=n_bricks)
    return (c // multiple * multiple).astype(np.int64)


# --------------------------------------------------------------------------- rendering inputs
def random_lut(seed: int, knots: int = 8, max_opacity: float = 0.01) -> np.ndarray:
    """256 x RGBA float32 transfer function, piecewise linear through `knots` random
    knots (positions U[0,1] plus both ends; colours U[0,1]; opacity U[0, max_opacity])."""
    r = np.random.default_rng(seed)
    pos = np.concatenate([[0.0], np.sort(r.random(knots - 2)), [1.0]])
    val = r.random((knots, 4))
    val[:, 3] *= max_opacity
    t = np.arange(256) / 255.0
    lut = np.stack([np.interp(t, pos, val[:, c]) for c in range(4)], axis=1)
    return lut.astype(np.float32)


def orbit_camera(theta: float, phi: float, ortho: bool, radius: float = 3.0,
                 fov_deg: float = 45.0, ortho_width: float = 2.0 * math.sqrt(3.0)) -> dict:
    """Camera on a sphere of `radius` around the origin, looking at the origin.

    eye = radius*(cos(phi) sin(theta), sin(phi), cos(phi) cos(theta)); the basis is
    forward = -eye/|eye|, right = forward x (0,1,0) normalised, up = right x forward.
    `scale` is tan(fov/2) for a perspective camera and half the view width for an
    orthographic one."""
    eye = radius * np.array([math.cos(phi) * math.sin(theta), math.sin(phi),
                             math.cos(phi) * math.cos(theta)])
    fwd = -eye / np.linalg.norm(eye)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    scale = ortho_width / 2.0 if ortho else math.tan(math.radians(fov_deg) / 2.0)
    return {"eye": eye.astype(np.float32), "forward": fwd.astype(np.float32),
            "right": right.astype(np.float32), "up": up.astype(np.float32),
            "scale": np.float32(scale), "ortho": bool(ortho)}


def random_views(n: int, seed: int):
    """n (theta, phi) view angles: theta U[0, 2pi), phi U[-0.6, 0.6]."""
    r = np.random.default_rng(seed)
    return [(float(r.uniform(0, 2 * np.pi)), float(r.uniform(-0.6, 0.6))) for _ in range(n)]
