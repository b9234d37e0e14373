"""FP64 CPU oracle of the headless neural volume renderer (Sec. 6) and of the
domain-decomposition query (Sec. 5.3).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
baseline of ``bench.py``; never by the product path.

The paper renders with nerfacc's ray marching and front-to-back compositing but
does not spell out the sampling or opacity model, so this oracle fixes one
reading, stated here and shared (by specification, not by code) with the
kernel:
  * rays: pixel centres (i + 0.5); perspective rays leave the eye through
    forward + ndc_x*scale*aspect*right + ndc_y*scale*up (normalised); orthographic
    rays leave eye + ndc_x*scale*aspect*right + ndc_y*scale*up along forward,
    with ndc_x = 2(px+0.5)/W - 1 and ndc_y = 1 - 2(py+0.5)/H;
  * each ray is clipped to the box [-1, 1]^3 (slab test, t >= 0) and sampled at
    n midpoints t_j = t0 + (j + 0.5) dt with dt = (t1 - t0)/n;
  * the value f at a sample maps to s = clamp((f - vmin)/(vmax - vmin), 0, 1),
    the 256-entry RGBA transfer function is read with linear interpolation at
    255 s, and opacity is alpha = 1 - exp(-a dt / dt_ref) with dt_ref = 2/512;
  * compositing is front to back: C += T alpha rgb, T *= 1 - alpha; the pixel is
    (C, 1 - T); rays that miss the box give (0, 0, 0, 0).
"""
from __future__ import annotations

import numpy as np

from . import apmgsrn as ap

DT_REF = 2.0 / 512.0


def camera_rays(cam: dict, width: int, height: int):
    """Ray origins and unit directions [H*W, 3] for the camera dict of
    ``synth.orbit_camera`` (eye, forward, right, up, scale, ortho)."""
    eye = np.asarray(cam["eye"], dtype=np.float64)
    fwd = np.asarray(cam["forward"], dtype=np.float64)
    right = np.asarray(cam["right"], dtype=np.float64)
    up = np.asarray(cam["up"], dtype=np.float64)
    scale = float(cam["scale"])
    aspect = width / height
    py, px = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    nx = (2.0 * (px.ravel() + 0.5) / width - 1.0) * scale * aspect
    ny = (1.0 - 2.0 * (py.ravel() + 0.5) / height) * scale
    off = nx[:, None] * right[None, :] + ny[:, None] * up[None, :]
    if cam["ortho"]:
        org = eye[None, :] + off
        d = np.repeat(fwd[None, :], org.shape[0], axis=0)
    else:
        org = np.repeat(eye[None, :], off.shape[0], axis=0)
        d = fwd[None, :] + off
        d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return org, d


def box_interval(org, d):
    """Slab test against [-1, 1]^3: (t0, t1, hit) with t0 clamped to >= 0."""
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        ta = (-1.0 - org) * inv
        tb = (1.0 - org) * inv
    tmin = np.minimum(ta, tb)
    tmax = np.maximum(ta, tb)
    t0 = np.max(tmin, axis=1)
    t1 = np.min(tmax, axis=1)
    t0 = np.maximum(t0, 0.0)
    return t0, t1, t1 > t0


def lut_lookup(lut, s):
    """Linear interpolation of the [256, 4] transfer function at 255*s, s in [0, 1]."""
    lut = np.asarray(lut, dtype=np.float64)
    pos = np.clip(s, 0.0, 1.0) * 255.0
    i0 = np.minimum(np.floor(pos), 254).astype(np.int64)
    fr = (pos - i0)[:, None]
    return lut[i0] * (1.0 - fr) + lut[i0 + 1] * fr


def dd_query(models, boxes, grid, vox: int, p, rnd=None):
    """Query a domain-decomposed set of models at global points p [N, 3]:
    the Sec. 5.3 hash picks the brick, p is mapped into that brick's local
    domain, and that brick's model answers.  A single model is the case
    grid = (1, 1, 1) with the whole volume as its box.  rnd is the decoder's
    operand rounding (see apmgsrn.mlp_forward)."""
    p = np.asarray(p, dtype=np.float64)
    b = ap.brick_index(p, grid)
    out = np.zeros(p.shape[0])
    for k, params in enumerate(models):
        sel = b == k
        if np.any(sel):
            loc = ap.global_to_brick_local(p[sel], boxes[k], vox)
            out[sel] = ap.query(params, loc, rnd)
    return out


def render(models, boxes, grid, vox, cam, lut, vmin, vmax, width, height, n_samples,
           pixels=None, rnd=None):
    """RGBA image [H, W, 4] (or [len(pixels), 4] for a list of flat pixel indices);
    rnd as in dd_query."""
    org, d = camera_rays(cam, width, height)
    if pixels is not None:
        org, d = org[pixels], d[pixels]
    t0, t1, hit = box_interval(org, d)
    n_rays = org.shape[0]
    color = np.zeros((n_rays, 3))
    trans = np.ones(n_rays)
    dt = np.where(hit, (t1 - t0) / n_samples, 0.0)
    rays = np.nonzero(hit)[0]
    for j in range(n_samples):
        t = t0[rays] + (j + 0.5) * dt[rays]
        p = org[rays] + t[:, None] * d[rays]
        f = dd_query(models, boxes, grid, vox, p, rnd)
        rgba = lut_lookup(lut, (f - vmin) / (vmax - vmin))
        alpha = 1.0 - np.exp(-rgba[:, 3] * dt[rays] / DT_REF)
        color[rays] += (trans[rays] * alpha)[:, None] * rgba[:, :3]
        trans[rays] *= 1.0 - alpha
    out = np.concatenate([color, (1.0 - trans)[:, None]], axis=1)
    if pixels is None:
        return out.reshape(height, width, 4)
    return out


# ----------------------------------------------------------------------------- progressive rendering
# Sec. 6 renders progressively: pixels are evaluated in the order of an image
# hierarchy, in checkerboard fashion, and the image shown after each pass is a
# bilinear upscale of the finest level evaluated so far, with the pixels already
# evaluated shown as they are.  The paper gives no formulas; the reading taken:
#   * level l of the hierarchy holds the pixels (a 2^l, b 2^l), a < ceil(W / 2^l),
#     b < ceil(H / 2^l); the coarsest level L is the first with 2^L >= max(W, H)
#     (the single pixel (0, 0));
#   * the order is level L, then each finer level's pixels that no coarser level
#     holds (three of every 2 x 2 block: the checkerboard), row by row, left to right;
#   * after k pixels, the finest complete level l is the finest whose whole grid is
#     among them; a pixel not yet evaluated takes the bilinear blend of the four
#     level-l samples around (x / 2^l, y / 2^l), the index clamped to the grid
#     (constant beyond its last row or column); nothing evaluated gives 0.


def hierarchy_levels(width: int, height: int) -> int:
    """The coarsest level L: the smallest with 2^L >= max(W, H)."""
    L = 0
    while (1 << L) < max(width, height):
        L += 1
    return L


def level_dims(width: int, height: int, l: int):
    """Columns and rows of level l's grid."""
    s = 1 << l
    return -(-width // s), -(-height // s)


def hierarchy_order(width: int, height: int) -> list:
    """Flat pixel indices (y W + x) in progressive order, written from the definition."""
    L = hierarchy_levels(width, height)
    order = [0]
    for l in range(L - 1, -1, -1):
        s = 1 << l
        for y in range(0, height, s):
            for x in range(0, width, s):
                coarser = (x % (2 * s) == 0) and (y % (2 * s) == 0)
                if not coarser:
                    order.append(y * width + x)
    return order


def progressive_preview(rgba, done: int):
    """In-progress image after the first `done` pixels of hierarchy_order:
    rgba [H, W, 4] holds the evaluated pixels (other entries are ignored)."""
    rgba = np.asarray(rgba, dtype=np.float64)
    H, W = rgba.shape[:2]
    order = hierarchy_order(W, H)
    evaluated = np.zeros(W * H, dtype=bool)
    evaluated[order[:done]] = True
    evaluated = evaluated.reshape(H, W)
    out = np.zeros_like(rgba)
    if done <= 0:
        return out
    L = hierarchy_levels(W, H)
    lvl = L
    for l in range(L, -1, -1):
        nx, ny = level_dims(W, H, l)
        if all(evaluated[b << l, a << l] for b in range(ny) for a in range(nx)):
            lvl = l
    nx, ny = level_dims(W, H, lvl)
    s = float(1 << lvl)
    for y in range(H):
        for x in range(W):
            if evaluated[y, x]:
                out[y, x] = rgba[y, x]
                continue
            fx, fy = x / s, y / s
            a0, b0 = min(int(np.floor(fx)), nx - 1), min(int(np.floor(fy)), ny - 1)
            a1, b1 = min(a0 + 1, nx - 1), min(b0 + 1, ny - 1)
            tx, ty = fx - a0, fy - b0
            if a1 == a0:
                tx = 0.0
            if b1 == b0:
                ty = 0.0
            p00 = rgba[b0 << lvl, a0 << lvl]
            p10 = rgba[b0 << lvl, a1 << lvl]
            p01 = rgba[b1 << lvl, a0 << lvl]
            p11 = rgba[b1 << lvl, a1 << lvl]
            out[y, x] = (1 - ty) * ((1 - tx) * p00 + tx * p10) + ty * ((1 - tx) * p01 + tx * p11)
    return out
