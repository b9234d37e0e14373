"""Pins of the oracle's data side: target lookup v(x), the spatial hash (Sec. 5.3),
the renderer (Sec. 6), the batch sampler, and the synthetic input recipes."""
import math

import numpy as np
import pytest

from oracle import apmgsrn as ap
from oracle import render as orr
from oracle import sampler as osp
from paper_2308_02494_gb300 import synth

from golden import philox_kat


# ----------------------------------------------------------------------------- v(x)
def test_volume_sample_exact_at_voxels_and_linear_fields():
    V = 9
    ax = synth.voxel_coords(V)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    vol = 0.3 + 1.1 * x - 0.7 * y + 2.0 * z
    pts = np.random.default_rng(0).uniform(-1, 1, size=(200, 3))
    np.testing.assert_allclose(ap.volume_sample(vol, pts),
                               0.3 + 1.1 * pts[:, 0] - 0.7 * pts[:, 1] + 2.0 * pts[:, 2], atol=1e-12)
    nodes = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    np.testing.assert_allclose(ap.volume_sample(vol, nodes), vol.ravel(), atol=1e-12)


def test_brick_local_lookup_equals_global_lookup():
    # A brick's local [-1,1]^3 is corner-aligned to its voxel box (Sec. 5.1), so
    # sampling the brick at local(p) must give the global sample at p.
    V = 33
    vol = np.random.default_rng(1).normal(size=(V, V, V))
    boxes = synth.brick_boxes(V, (2, 2, 2), ghost=2)
    r = np.random.default_rng(2)
    for b, box in enumerate(boxes):
        lo = -1 + 2 * box[:3] / (V - 1)
        hi = -1 + 2 * box[3:] / (V - 1)
        p = r.uniform(lo, hi, size=(50, 3))
        loc = ap.global_to_brick_local(p, box, V)
        assert np.all(np.abs(loc) <= 1 + 1e-12)
        np.testing.assert_allclose(ap.volume_sample(vol, np.clip(loc, -1, 1), box),
                                   ap.volume_sample(vol, p), atol=1e-12)


def test_brick_boxes_cover_with_ghost_cells():
    boxes = synth.brick_boxes(1024, (2, 2, 2), ghost=2)
    assert boxes.shape == (8, 6)
    np.testing.assert_array_equal(boxes[0], [0, 0, 0, 513, 513, 513])
    np.testing.assert_array_equal(boxes[7], [510, 510, 510, 1023, 1023, 1023])
    np.testing.assert_array_equal(boxes[1], [510, 0, 0, 1023, 513, 513])   # x fastest


def test_spatial_hash_closed_form():
    # Sec. 5.3: i = floor(I (p+1)/2), clamped at p = 1.0; flat index i + I j + I J k.
    grid = (2, 3, 4)
    p = np.array([[-1.0, -1.0, -1.0], [1.0, 1.0, 1.0], [-1e-9, 0.0, 0.0],
                  [0.0, -1.0 / 3.0 + 1e-9, 0.5 - 1e-9]])
    got = ap.brick_index(p, grid)
    assert got[0] == 0
    assert got[1] == 1 + 2 * 2 + 6 * 3
    assert got[2] == 0 + 2 * 1 + 6 * 2
    assert got[3] == 1 + 2 * 1 + 6 * 2


# ----------------------------------------------------------------------------- render
def _zero_model(M=2, R=3, C=2, H=4):
    shape = synth.ModelShape(M, R, C, H)
    p = synth.init_model(shape, 0)
    p["w3"] = np.zeros(H)            # m == 0 everywhere, f == vmin
    return p


def test_render_constant_field_closed_form():
    # A constant field gives a constant alpha, so along any ray of n samples
    # C = rgb (1 - (1 - alpha)^n) and T = (1 - alpha)^n; with an orthographic view
    # down an axis every ray crosses exactly the box side (length 2).
    lut = np.zeros((256, 4), dtype=np.float32)
    lut[0] = [0.2, 0.5, 0.9, 0.002]
    c = lut[0].astype(np.float64)
    cam = {"eye": np.array([0, 0, 3.0]), "forward": np.array([0, 0, -1.0]),
           "right": np.array([1.0, 0, 0]), "up": np.array([0, 1.0, 0]), "scale": 0.9, "ortho": True}
    n = 16
    img = orr.render([_zero_model()], [[0, 0, 0, 8, 8, 8]], (1, 1, 1), 9, cam, lut, 0.0, 1.0, 8, 8, n)
    alpha = 1 - math.exp(-c[3] * (2.0 / n) / orr.DT_REF)
    T = (1 - alpha) ** n
    assert 0.2 < T < 0.9
    np.testing.assert_allclose(img[..., 3], 1 - T, rtol=1e-12)
    np.testing.assert_allclose(img[..., 0], c[0] * (1 - T), rtol=1e-12)
    np.testing.assert_allclose(img[..., 2], c[2] * (1 - T), rtol=1e-12)


def test_ortho_centre_ray_length_and_misses():
    cam = synth.orbit_camera(0.0, 0.0, ortho=True)
    org, d = orr.camera_rays(cam, 2, 2)
    t0, t1, hit = orr.box_interval(org, d)
    assert np.all(hit)
    np.testing.assert_allclose(t1 - t0, 2.0, atol=1e-6)
    # a camera whose view is far off the box misses it everywhere
    far = {"eye": np.array([5.0, 5.0, 3.0]), "forward": np.array([0, 0, -1.0]),
           "right": np.array([1.0, 0, 0]), "up": np.array([0, 1.0, 0]), "scale": 0.5, "ortho": True}
    lut = np.ones((256, 4), dtype=np.float32)
    img = orr.render([_zero_model()], [[0, 0, 0, 8, 8, 8]], (1, 1, 1), 9, far, lut, 0, 1, 4, 4, 8)
    assert np.all(img == 0.0)


def test_perspective_render_of_a_constant_field_depends_only_on_each_chord():
    # Perspective rays all leave the eye.  With a constant field every sample has the
    # same alpha, and n samples of a chord L give 1 - prod(1 - alpha) = 1 - exp(-a L /
    # dt_ref) whatever n is.  The camera on the z axis at distance 3 sends its centre
    # ray through the box on the axis (in at t = 2, out at t = 4), and the image of this
    # mirror-symmetric scene is mirror-symmetric.
    cam = synth.orbit_camera(0.0, 0.0, ortho=False)
    W = H = 5
    org, d = orr.camera_rays(cam, W, H)
    np.testing.assert_allclose(org, np.broadcast_to(cam["eye"], org.shape), atol=0)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    centre = (H // 2) * W + W // 2
    np.testing.assert_allclose(d[centre], cam["forward"], atol=1e-7)
    t0, t1, hit = orr.box_interval(org, d)
    assert hit[centre]
    np.testing.assert_allclose([t0[centre], t1[centre]], [2.0, 4.0], atol=1e-6)
    lut = np.zeros((256, 4), dtype=np.float32)
    lut[0] = [0.3, 0.6, 0.1, 0.004]
    a = float(lut[0, 3])
    for n in (7, 32):
        img = orr.render([_zero_model()], [[0, 0, 0, 8, 8, 8]], (1, 1, 1), 9, cam, lut, 0.0, 1.0, W, H, n)
        want = np.where(hit, 1.0 - np.exp(-a * (t1 - t0) / orr.DT_REF), 0.0).reshape(H, W)
        np.testing.assert_allclose(img[..., 3], want, rtol=1e-9, atol=1e-15)
        np.testing.assert_allclose(img[..., 1], float(lut[0, 1]) * want, rtol=1e-9, atol=1e-15)
        np.testing.assert_allclose(img, img[:, ::-1], atol=1e-12)
        np.testing.assert_allclose(img, img[::-1, :], atol=1e-12)


def test_lut_linear_interpolation():
    lut = np.zeros((256, 4))
    lut[:, 0] = np.arange(256) / 255.0
    s = np.array([0.0, 0.1234, 0.5, 1.0, -3.0, 7.0])
    np.testing.assert_allclose(orr.lut_lookup(lut, s)[:, 0], np.clip(s, 0, 1), atol=1e-14)


# ----------------------------------------------------------------------------- sampler
def test_philox_known_answer_vectors():
    for ctr, key, out in philox_kat():
        np.testing.assert_array_equal(osp.philox4x32_10(ctr, key), out)


def test_sampler_range_and_uniformity():
    pts = osp.sample_points(seed=7, step=3, brick=1, n=1 << 16)
    assert pts.dtype == np.float32 and pts.min() >= -1.0 and pts.max() < 1.0
    # 8 octants equally likely: chi-square with 7 dof well inside its 99.9% bound (24.3)
    oct_ = ((pts > 0) * np.array([1, 2, 4])).sum(1)
    cnt = np.bincount(oct_, minlength=8)
    chi2 = ((cnt - cnt.mean()) ** 2 / cnt.mean()).sum()
    assert chi2 < 24.3
    assert not np.array_equal(pts, osp.sample_points(seed=7, step=4, brick=1, n=1 << 16))


# ----------------------------------------------------------------------------- recipes
def test_gaussian_volume_recipe_closed_form():
    vol, prm = synth.gaussian_volume(16, 16, seed=3)
    ax = synth.voxel_coords(16)
    for (k, j, i) in [(0, 0, 0), (5, 9, 2), (15, 15, 15)]:
        p = np.array([ax[i], ax[j], ax[k]])
        ref = sum(a * math.exp(-np.sum((p - c) ** 2) / (2 * s * s))
                  for a, c, s in zip(prm["amp"], prm["centre"], prm["sigma"]))
        assert abs(vol[k, j, i] - ref) < 1e-6


def test_fourier_volume_recipe_matches_direct_mode_sum():
    torch = pytest.importorskip("torch")
    modes = synth.fourier_modes(32, 1, 8, seed=4)
    ks = np.linalg.norm(modes["k"], axis=1)
    assert ks.min() >= 1 and ks.max() <= 8
    vol, lo, hi = synth.fourier_volume(20, modes, device="cpu", z_chunk=7)
    assert abs(float(vol.min())) < 1e-7 and abs(float(vol.max()) - 1) < 1e-6
    ax = synth.voxel_coords(20)
    for (k, j, i) in [(0, 0, 0), (3, 17, 8), (19, 2, 11)]:
        ref = synth.fourier_value(modes, [[ax[i], ax[j], ax[k]]])[0]
        assert abs(float(vol[k, j, i]) - (ref - lo) / (hi - lo)) < 2e-5


# ----------------------------------------------------------------------------- progressive rendering
def test_hierarchy_order_of_a_4x4_image_by_hand():
    # level 2: (0,0); level 1: (2,0), (0,2), (2,2); level 0: the rest, row by row
    assert orr.hierarchy_order(4, 4) == [0, 2, 8, 10, 1, 3, 4, 5, 6, 7, 9, 11, 12, 13, 14, 15]


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (7, 5), (33, 17), (16, 16), (64, 3)])
def test_hierarchy_order_is_a_coarse_to_fine_permutation(W, H):
    order = orr.hierarchy_order(W, H)
    assert sorted(order) == list(range(W * H))
    L = orr.hierarchy_levels(W, H)
    assert (1 << L) >= max(W, H) and (L == 0 or (1 << (L - 1)) < max(W, H))

    def level(p):
        x, y = p % W, p // W
        l = 0
        while l < L and x % (2 << l) == 0 and y % (2 << l) == 0:
            l += 1
        return l
    lv = [level(p) for p in order]
    assert all(a >= b for a, b in zip(lv, lv[1:]))
    # after the pixels of levels >= l, exactly level l's grid has been evaluated
    for l in range(L + 1):
        nx, ny = orr.level_dims(W, H, l)
        grid = {(b << l) * W + (a << l) for b in range(ny) for a in range(nx)}
        assert set(order[:nx * ny]) == grid


def test_progressive_preview_upscales_bilinear_images_exactly_and_keeps_evaluated_pixels():
    W, H = 9, 17
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.stack([0.1 + 0.02 * x + 0.01 * y + 0.003 * x * y, 0.5 - 0.03 * y, 0.2 + 0.04 * x,
                    0.9 - 0.001 * x * y], axis=-1)
    # levels 5, 4 and 3 (a 2 x 3 grid) complete after 6 pixels; W-1, H-1 are multiples of 8
    assert orr.level_dims(W, H, 3) == (2, 3)
    np.testing.assert_allclose(orr.progressive_preview(img, 6), img, rtol=0, atol=1e-14)
    assert np.all(orr.progressive_preview(img, 0) == 0.0)
    noise = np.random.default_rng(3).uniform(size=img.shape)
    full = orr.progressive_preview(noise, W * H)
    assert np.array_equal(full, noise)
    part = orr.progressive_preview(noise, 40)
    done = orr.hierarchy_order(W, H)[:40]
    flat_p, flat_n = part.reshape(-1, 4), noise.reshape(-1, 4)
    assert np.array_equal(flat_p[done], flat_n[done])


def test_progressive_preview_holds_the_last_coarse_column_and_row():
    W, H = 11, 6     # level 2 grid: columns 0, 4, 8 and rows 0, 4
    img = np.zeros((H, W, 4))
    img[0, 0], img[0, 4], img[0, 8] = 1.0, 2.0, 3.0
    img[4, 0], img[4, 4], img[4, 8] = 4.0, 5.0, 6.0
    nx, ny = orr.level_dims(W, H, 2)
    assert (nx, ny) == (3, 2)
    pv = orr.progressive_preview(img, nx * ny)
    assert np.allclose(pv[0, 10], 3.0) and np.allclose(pv[5, 10], 6.0) and np.allclose(pv[5, 0], 4.0)
    assert np.allclose(pv[2, 6], 0.25 * (2 + 3 + 5 + 6))
