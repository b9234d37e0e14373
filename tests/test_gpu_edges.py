"""GPU parity on the edges of Eq. 2 and at the sizes the other parity files leave out.

* Eq. 2's inclusive bounds -1 <= u <= 1: grids whose nodes, faces and corners the
  points hit exactly (identity, doubled, translated and axis-permuted transforms, so
  u = +-1 falls inside the domain as well as on its faces), including the upper cell
  c = R - 2 with weight 1 and points just past a face (feature exactly 0).  With
  R - 1 a power of two every node, u and s is exact in float32, so the FP32 path is
  held to the FP32 bar point by point.
* R = 64 grids (the largest the library accepts): forward and backward against the
  oracle in both precisions, M = 32 (K = 64) and M = 64 (K = 128).
* The 2^20-point BF16 batch of the paper-scale model: f at sampled points, and the
  training pass's losses and gradients tied to the oracle through linearity (the
  full batch equals the mean of its four 2^18-point quarters, one of which is checked
  against the oracle).
* The renderer at the benchmark's frame size (1024^2, 512 samples per ray, 8 bricks
  of the paper-scale model): sampled pixels against the oracle renderer in FP32 and
  BF16, and the BF16 frame against the FP32 frame.
"""
import numpy as np
import pytest

from oracle import apmgsrn as ap
from oracle import render as orr
from oracle import sampler as osp
from paper_2308_02494_gb300 import synth
from gpu_util import (RND, TOL, as_stored, ensure_built, make_model, morton_order, morton_sorted,
                      points_off_bf16_midpoints, points_off_faces, points_off_kinks, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


# ------------------------------------------------------------------ Eq. 2 edges
EDGE_SHAPES = {"m8r17c2": synth.ModelShape(8, 17, 2, 64), "m64r33c2": synth.ModelShape(64, 33, 2, 64)}


def _edge_params(shape, seed):
    p = synth.parity_model(shape, seed, shrink=0.0)
    G = np.zeros((shape.n_grids, 3, 4))
    for i in range(shape.n_grids):
        kind = i % 4
        if kind == 0:     # u = x: the grid is the domain, faces at x = +-1
            G[i, :, :3] = np.eye(3)
        elif kind == 1:   # u = 2x: faces at +-1/2 inside the domain, points beyond them outside
            G[i, :, :3] = 2.0 * np.eye(3)
        elif kind == 2:   # u = x + t: faces at x = 3/4 and z = -3/4
            G[i, :, :3] = np.eye(3)
            G[i, :, 3] = (0.25, 0.0, -0.25)
        else:             # u = (y, z, x)
            G[i, :, :3] = np.eye(3)[[1, 2, 0]]
    p["G"] = G
    return p


def _edge_points():
    a = -1.0 + np.arange(17) / 8.0          # nodes of R = 17 (and every other node of R = 33)
    X, Y, Z = np.meshgrid(a, a, a, indexing="ij")
    pts = [np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)]
    r = np.random.default_rng(0)
    for d in range(3):                        # one coordinate on a face value, the others anywhere
        for v in (-1.0, 1.0, -0.5, 0.5, 0.75, -0.75, 0.625, -0.875):
            q = r.uniform(-1.0, 1.0, size=(48, 3))
            q[:, d] = v
            pts.append(q)
    pts.append(np.array([[s0, s1, s2] for s0 in (-1.0, 1.0) for s1 in (-1.0, 1.0) for s2 in (-1.0, 1.0)]))
    return np.concatenate(pts).astype(np.float32)


def _edge_case(shape_name, precision, layout):
    import torch
    from paper_2308_02494_gb300.model import SRN
    shape = EDGE_SHAPES[shape_name]
    p = _edge_params(shape, 5)
    ref = as_stored(p, precision)
    x = _edge_points()
    if precision == "bf16":
        x = points_off_kinks(ref, x, RND[precision])
    if layout == "morton":
        x = morton_sorted(x)
    u = ap.local_coords(ref["G"], x.astype(np.float64))
    on_face = np.any(np.abs(np.abs(u) - 1.0) == 0.0, axis=(1, 2))
    past_face = np.any(np.abs(u) > 1.0, axis=(1, 2))
    assert on_face.sum() > 500 and past_face.sum() > 500
    n = len(x)
    m = SRN(shape, 1, precision=precision, max_points=n)
    m.set_params([p])
    return m, ref, x, torch.as_tensor(x, device="cuda")


@pytest.mark.parametrize("layout", ["given", "morton"])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("shape_name", list(EDGE_SHAPES))
def test_points_on_nodes_faces_and_past_faces(shape_name, precision, layout):
    import torch
    m, ref, x, xt = _edge_case(shape_name, precision, layout)
    n = len(x)
    f = m.forward(xt, [0, n]).cpu().numpy()
    want = ap.query(ref, x.astype(np.float64), rnd=RND[precision])
    rms = np.sqrt(np.mean(want ** 2))
    # point by point: one grid taking the wrong cell or the wrong side of Eq. 2's mask
    # moves f by a sizeable fraction of its RMS
    per_point = {"fp32": 1e-5, "bf16": 1e-2}[precision]
    assert np.max(np.abs(f - want)) <= per_point * rms, np.max(np.abs(f - want)) / rms
    assert rel_l2(f, want) <= TOL[precision]
    v = np.random.default_rng(9).uniform(-0.5, 1.5, n).astype(np.float32)
    m.backward(xt, torch.as_tensor(v, device="cuda"), [0, n])
    g = m.get("grads")[0]
    o = ap.grad_rec(ref, x.astype(np.float64), v.astype(np.float64), rnd=RND[precision])
    for k, w in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
        assert rel_l2(g[k], o[w]) <= TOL[precision], (k, rel_l2(g[k], o[w]))
    # the upper face's nodes (index R - 1) of the identity grids receive the gradient
    # of the points on x = 1 through cell R - 2 with weight 1
    assert np.abs(o["dF"][0, :, :, -1]).max() > 0
    np.testing.assert_allclose(g["F"][0, :, :, -1], o["dF"][0, :, :, -1],
                               atol=TOL[precision] * np.abs(o["dF"][0]).max())


# ------------------------------------------------------------------ R = 64
R64 = {"m32r64c2": synth.ModelShape(32, 64, 2, 64), "m64r64c2": synth.ModelShape(64, 64, 2, 64)}


@pytest.mark.parametrize("layout", ["random", "dense"])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("shape_name", list(R64))
def test_r64_grids_match_oracle(shape_name, precision, layout):
    import torch
    n = 1500
    m, refs = make_model(R64[shape_name], 1, precision, 4096, seed=71)
    ref = refs[0]
    lo, hi = (-1.0, 1.0) if layout == "random" else (-0.2, 0.1)
    x = points_off_kinks(ref, points_off_faces(ref["G"], 2 * n + 64, 72, lo=lo, hi=hi), RND[precision])
    if precision == "bf16":
        # O(1) features on 64^3 nodes: a few points per thousand otherwise have an operand
        # that float32 and float64 round to neighbouring bfloat16 numbers
        x = points_off_bf16_midpoints(ref, x)
    x = x[:n]
    assert len(x) == n
    if layout == "dense":
        x = morton_sorted(x)
    xt = torch.as_tensor(x, device="cuda")
    f = m.forward(xt, [0, n]).cpu().numpy()
    assert rel_l2(f, ap.query(ref, x.astype(np.float64), rnd=RND[precision])) <= TOL[precision]
    v = np.random.default_rng(73).uniform(-0.5, 1.5, n).astype(np.float32)
    losses = m.backward(xt, torch.as_tensor(v, device="cuda"), [0, n], density=True).cpu().numpy()
    g = m.get("grads")[0]
    o = ap.grad_rec(ref, x.astype(np.float64), v.astype(np.float64), rnd=RND[precision])
    d = ap.grad_density(ref["G"], x.astype(np.float64), o["h"])
    assert abs(losses[0, 0] - o["L_rec"]) <= TOL[precision] * o["L_rec"]
    assert abs(losses[0, 1] - d["L_den"]) <= TOL[precision] * abs(d["L_den"])
    for k, w in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
        assert rel_l2(g[k], o[w]) <= TOL[precision], (k, rel_l2(g[k], o[w]))


# ------------------------------------------------------------------ 2^20 points, BF16
def test_bf16_paper_scale_batch_of_2_20_points():
    import torch
    shape = synth.ModelShape(64, 32, 2, 64)
    n, q = 1 << 20, 1 << 18
    m, refs = make_model(shape, 1, "bf16", n, seed=81, shrink=0.3)
    ref = refs[0]
    # quarter 0 is kept off faces and ReLU kinks (it is checked against the oracle);
    # the other three are the sampler's points as they come
    x0 = osp.sample_points(83, 0, 0, q + q // 2)
    u = ap.local_coords(ref["G"], x0.astype(np.float64))
    x0 = points_off_kinks(ref, x0[np.all(np.abs(np.abs(u) - 1.0) > 1e-5, axis=(1, 2))], RND["bf16"])[:q]
    assert len(x0) == q
    quarters = [morton_sorted(x0)] + [morton_sorted(osp.sample_points(83, k, 0, q)) for k in (1, 2, 3)]
    r = np.random.default_rng(84)
    vs = [r.uniform(-0.5, 1.5, q).astype(np.float32) for _ in range(4)]
    xq = torch.as_tensor(np.concatenate(quarters), device="cuda")
    vq = torch.as_tensor(np.concatenate(vs), device="cuda")
    # the whole batch in the sampler's Morton order, as training runs it
    perm = morton_order(np.concatenate(quarters))
    xa = np.concatenate(quarters)[perm]
    xt = torch.as_tensor(xa, device="cuda")
    vt = torch.as_tensor(np.concatenate(vs)[perm], device="cuda")
    # forward values of the whole batch at 2000 sampled points, one by one
    f = m.forward(xt, [0, n]).cpu().numpy()
    pick = r.choice(n, size=2000, replace=False)
    xs = xa[pick].astype(np.float64)
    keep = np.all(np.abs(np.abs(ap.local_coords(ref["G"], xs)) - 1.0) > 1e-5, axis=(1, 2))
    assert rel_l2(f[pick][keep], ap.query(ref, xs[keep], rnd=RND["bf16"])) <= TOL["bf16"]
    # the training pass over 2^20 points, then over each quarter alone
    full = m.backward(xt, vt, [0, n]).cpu().numpy().copy()
    g_full = m.grads.clone()
    acc = torch.zeros_like(g_full)
    lq = []
    for k in range(4):
        lq.append(m.backward(xq[k * q:(k + 1) * q], vq[k * q:(k + 1) * q], [0, q]).cpu().numpy().copy())
        acc += m.grads / 4.0           # dL/dm carries 1/N: a quarter's gradient is 4x its share
        if k == 0:
            g0 = m.get("grads")[0]
    L = m.lay
    assert full[0, 3] == n
    assert abs(full[0, 0] - np.mean([a[0, 0] for a in lq])) <= 1e-5 * full[0, 0]
    # per-point terms are identical in both runs (the 1/N scale is a power of two, so
    # every BF16 rounding commutes with it); only the fixed-point quantisation of the
    # scatter's tiles and the order of float sums differ
    for name, a, b in (("F", L.off_F, L.off_F + L.size_F), ("W1", L.off_W1, L.off_W1 + L.size_W1),
                       ("W2", L.off_W2, L.off_W2 + L.size_W2), ("w3", L.off_w3, L.off_w3 + L.size_w3)):
        e = float(torch.linalg.norm(g_full[a:b] - acc[a:b]) / torch.linalg.norm(acc[a:b]))
        assert e <= 1e-4, (name, e)
    o = ap.grad_rec(ref, quarters[0].astype(np.float64), vs[0].astype(np.float64), rnd=RND["bf16"])
    assert abs(lq[0][0, 0] - o["L_rec"]) <= TOL["bf16"] * o["L_rec"]
    for k, w in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
        assert rel_l2(g0[k], o[w]) <= TOL["bf16"], (k, rel_l2(g0[k], o[w]))


# ------------------------------------------------------------------ full-size frames
def test_full_frame_render_sampled_pixels():
    import torch
    shape = synth.ModelShape(64, 32, 2, 64)
    V, W, H, S = 1024, 1024, 1024, 512
    boxes = synth.brick_boxes(V, (2, 2, 2), ghost=2)
    lut = synth.random_lut(3)
    cams = [synth.orbit_camera(0.9, 0.25, ortho=True), synth.orbit_camera(4.1, -0.35, ortho=False)]
    r = np.random.default_rng(91)
    frames = {}
    refs = {}
    for precision in ("fp32", "bf16"):
        m, refs[precision] = make_model(shape, 8, precision, 1 << 21, seed=93, shrink=0.3)
        lt = torch.as_tensor(lut, device="cuda")
        frames[precision] = [m.render(cam, lt, -0.5, 1.5, W, H, S, (2, 2, 2), boxes, V).cpu().numpy()
                             for cam in cams]
        del m
    for c, cam in enumerate(cams):
        img32, img16 = frames["fp32"][c].reshape(-1, 4), frames["bf16"][c].reshape(-1, 4)
        assert img32[:, 3].max() > 0.05
        hit = np.nonzero(img32[:, 3] > 0)[0]
        pix = np.concatenate([r.choice(hit, size=40, replace=False), r.choice(W * H, size=8, replace=False)])
        want = orr.render(refs["fp32"], boxes, (2, 2, 2), V, cam, lut, -0.5, 1.5, W, H, S, pixels=pix)
        assert rel_l2(img32[pix], want) <= 1e-4, rel_l2(img32[pix], want)
        want16 = orr.render(refs["bf16"], boxes, (2, 2, 2), V, cam, lut, -0.5, 1.5, W, H, S, pixels=pix,
                            rnd=RND["bf16"])
        assert rel_l2(img16[pix], want16) <= TOL["bf16"], rel_l2(img16[pix], want16)
        # the whole BF16 frame against the whole FP32 frame (the FP32 path stands for the
        # exact values here: it meets the oracle at 1e-4 on the sampled pixels)
        assert rel_l2(img16, img32) <= 5 * TOL["bf16"], rel_l2(img16, img32)
