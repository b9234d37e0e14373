"""GPU parity: libsrn (through its C ABI) against the FP64 oracle, element by element,
on seeded inputs that span several tiles and a ragged tail."""
import numpy as np
import pytest

from oracle import apmgsrn as ap
from oracle import render as orr
from oracle import sampler as osp
from paper_2308_02494_gb300 import synth
from gpu_util import (EXACT, RND, TOL, as_stored, dG_error, density_grad_scale, ensure_built,
                      make_model, morton_sorted, points_off_faces, points_off_kinks, rel_l2)

pytestmark = pytest.mark.gpu

SHAPES = {
    "m8r16c2": synth.ModelShape(8, 16, 2, 64),     # the 16 -> 64 -> 64 -> 1 model
    "m16r9c1": synth.ModelShape(16, 9, 1, 64),
    "m32r20c2": synth.ModelShape(32, 20, 2, 64),
    "m64r32c2": synth.ModelShape(64, 32, 2, 64),   # the 128 -> 64 -> 64 -> 1 model
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _torch():
    import torch
    return torch


def _points_for(models, counts, seed, rnd=None, layout="random"):
    """Seeded points per brick, off every grid face and off every ReLU kink.

    layout "random": uniform in [-1,1]^3, unordered (tiles span the domain, so the
    kernel takes its per-corner path); "dense": uniform in a 0.3-wide cube and
    Morton-ordered like the sampler's batches (tiles are compact, so the kernel
    stages and scatters through its per-tile node boxes)."""
    xs = []
    for b, (p, n) in enumerate(zip(models, counts)):
        if not n:
            xs.append(np.zeros((0, 3), np.float32))
            continue
        lo, hi = (-1.0, 1.0) if layout == "random" else (-0.2 + 0.05 * b, 0.1 + 0.05 * b)
        x = points_off_kinks(p, points_off_faces(p["G"], 2 * n + 64, seed + 7 * b, lo=lo, hi=hi), rnd)
        assert len(x) >= n
        x = x[:n]
        xs.append(morton_sorted(x) if layout == "dense" else x)
    return xs


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", list(SHAPES))
def test_forward_matches_oracle(shape, precision):
    torch = _torch()
    counts = [1000]
    m, ref = make_model(SHAPES[shape], 1, precision, 4096, seed=11)
    x = _points_for(ref, counts, 3, RND[precision])[0]
    f = m.forward(torch.as_tensor(x, device="cuda"), [0, 1000]).cpu().numpy()
    fo = ap.query(ref[0], x.astype(np.float64), rnd=RND[precision])
    assert rel_l2(f, fo) <= TOL[precision], rel_l2(f, fo)
    fx = ap.query(ref[0], x.astype(np.float64))
    assert rel_l2(f, fx) <= EXACT[precision]["value"], rel_l2(f, fx)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_forward_uneven_bricks_with_an_empty_brick(precision):
    torch = _torch()
    counts = [0, 300, 7, 129]
    m, ref = make_model(SHAPES["m8r16c2"], 4, precision, 1024, seed=12)
    xs = _points_for(ref, counts, 4, RND[precision])
    off = m.offsets_of(counts)
    f = m.forward(torch.as_tensor(np.concatenate(xs), device="cuda"), off).cpu().numpy()
    for b in range(4):
        if counts[b]:
            fo = ap.query(ref[b], xs[b].astype(np.float64), rnd=RND[precision])
            assert rel_l2(f[off[b]:off[b + 1]], fo) <= TOL[precision], b


def test_forward_of_nothing_is_a_no_op():
    torch = _torch()
    m, _ = make_model(SHAPES["m8r16c2"], 1, "fp32", 64, seed=13)
    out = torch.full((4,), 7.0, device="cuda")
    m.forward(torch.zeros((0, 3), device="cuda"), [0, 0], out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)


def _oracle_backward(ref, x, v, density, rnd=None):
    g = ap.grad_rec(ref, x.astype(np.float64), v.astype(np.float64), rnd=rnd)
    out = dict(g)
    if density:
        d = ap.grad_density(ref["G"], x.astype(np.float64), g["h"])
        out["L_den"], out["dG"], out["S"] = d["L_den"], d["dG"], d["terms"]["S"]
    return out


@pytest.mark.parametrize("layout", ["random", "dense"])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", ["m8r16c2", "m16r9c1", "m32r20c2", "m64r32c2"])
def test_backward_matches_oracle(shape, precision, layout):
    torch = _torch()
    n = 1500
    m, ref = make_model(SHAPES[shape], 1, precision, 4096, seed=21)
    x = _points_for(ref, [n], 5, RND[precision], layout)[0]
    v = np.random.default_rng(6).uniform(-0.5, 1.5, n).astype(np.float32)
    losses = m.backward(torch.as_tensor(x, device="cuda"), torch.as_tensor(v, device="cuda"),
                        [0, n], density=True).cpu().numpy()
    gr = m.get("grads")[0]
    o = _oracle_backward(ref[0], x, v, True, RND[precision])
    tol = TOL[precision]
    assert abs(losses[0, 0] - o["L_rec"]) <= tol * abs(o["L_rec"])
    assert abs(losses[0, 1] - o["L_den"]) <= tol * abs(o["L_den"]) + 1e-12
    assert abs(losses[0, 2] - o["S"]) <= tol * o["S"]
    assert losses[0, 3] == n
    for k, ok in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
        e = rel_l2(gr[k], o[ok])
        assert e <= tol, (k, e)
    scale = density_grad_scale(ref[0]["G"], x, o["h"])
    assert dG_error(gr["G"], o["dG"], scale) <= tol, dG_error(gr["G"], o["dG"], scale)
    if precision == "bf16":   # against the exact (unrounded) oracle: the stated looser bounds
        ox = _oracle_backward(ref[0], x, v, True)
        assert abs(losses[0, 0] - ox["L_rec"]) <= EXACT["bf16"]["value"] * ox["L_rec"]
        for k, ok in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
            assert rel_l2(gr[k], ox[ok]) <= EXACT["bf16"]["grad"], (k, rel_l2(gr[k], ox[ok]))
        assert dG_error(gr["G"], ox["dG"], scale) <= EXACT["bf16"]["grad"]


@pytest.mark.parametrize("layout", ["random", "dense"])
@pytest.mark.parametrize("precision,shape", [("fp32", "m8r16c2"), ("bf16", "m8r16c2"), ("bf16", "m64r32c2")])
def test_backward_uneven_bricks(precision, shape, layout):
    _uneven_backward_case(precision, layout, shape, [257, 31, 140], 1024, seed=22)


def test_backward_bricks_shared_by_one_cta():
    """More decoder tiles than resident CTAs: CTAs of the BF16 training pass start in
    one brick and finish in the next (weight reloads and weight-gradient flushes
    inside a CTA)."""
    _uneven_backward_case("bf16", "dense", "m64r32c2", [23000, 300, 17000], 41000, seed=30)


def _uneven_backward_case(precision, layout, shape, counts, max_points, seed):
    torch = _torch()
    m, ref = make_model(SHAPES[shape], len(counts), precision, max_points, seed=seed)
    xs = _points_for(ref, counts, 8, RND[precision], layout)
    counts = [len(x) for x in xs]
    r = np.random.default_rng(9)
    vs = [r.uniform(0, 1, c).astype(np.float32) for c in counts]
    off = m.offsets_of(counts)
    losses = m.backward(torch.as_tensor(np.concatenate(xs), device="cuda"),
                        torch.as_tensor(np.concatenate(vs), device="cuda"), off, density=True).cpu().numpy()
    grads = m.get("grads")
    tol = TOL[precision]
    for b in range(len(counts)):
        o = _oracle_backward(ref[b], xs[b], vs[b], True, RND[precision])
        assert abs(losses[b, 0] - o["L_rec"]) <= tol * o["L_rec"], b
        assert abs(losses[b, 1] - o["L_den"]) <= tol * abs(o["L_den"]) + 1e-12, b
        for k, ok in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
            assert rel_l2(grads[b][k], o[ok]) <= tol, (b, k, rel_l2(grads[b][k], o[ok]))
        scale = density_grad_scale(ref[b]["G"], xs[b], o["h"])
        assert dG_error(grads[b]["G"], o["dG"], scale) <= tol, b


def test_backward_without_density_leaves_G_gradient_zero_and_rejects_empty_bricks():
    torch = _torch()
    from paper_2308_02494_gb300.srn import SrnError
    m, ref = make_model(SHAPES["m8r16c2"], 2, "fp32", 512, seed=23)
    xs = _points_for(ref, [100, 50], 10)
    x = torch.as_tensor(np.concatenate(xs), device="cuda")
    v = torch.rand(150, device="cuda")
    m.backward(x, v, [0, 100, 150], density=False)
    for b in range(2):
        assert np.all(m.get("grads")[b]["G"] == 0.0)
    with pytest.raises(SrnError):
        m.backward(x, v, [0, 0, 150])


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_adam_step_matches_oracle(precision):
    torch = _torch()
    n = 700
    m, ref = make_model(SHAPES["m8r16c2"], 1, precision, 1024, seed=24)
    x = _points_for(ref, [n], 11)[0]
    v = np.random.default_rng(12).uniform(0, 1, n).astype(np.float32)
    xt, vt = torch.as_tensor(x, device="cuda"), torch.as_tensor(v, device="cuda")
    for density in (False, True):
        p0 = m.get("params")[0]
        m0, v0 = m.get("m")[0], m.get("v")[0]
        m.backward(xt, vt, [0, n], density=density)
        g = m.get("grads")[0]
        m.step(density=density)
        p1 = m.get("params")[0]
        t_a = 1 if not density else 2
        for k in ("F", "W1", "W2", "w3"):
            want, _, _ = ap.adam_update(p0[k], g[k], m0[k], v0[k], t_a, lr=1e-2)
            assert np.max(np.abs(p1[k] - want)) <= 1e-6 * max(1.0, np.max(np.abs(want))), k
        if density:
            want, _, _ = ap.adam_update(p0["G"], g["G"], m0["G"], v0["G"], 1, lr=1e-3)
            assert np.max(np.abs(p1["G"] - want)) <= 1e-6
        else:
            assert np.array_equal(p1["G"], p0["G"])
    if precision == "bf16":   # the shadow the kernels read follows the master
        sh = m.shadow.view(torch.bfloat16).float().cpu().numpy()
        L = m.lay
        np.testing.assert_array_equal(sh[L.off_W1:L.off_W1 + 64 * 16],
                                      synth.round_bf16(m.params[L.off_W1:L.off_W1 + 64 * 16].cpu().numpy()))


def test_sampler_is_the_philox_batch_reordered_by_morton_bin():
    torch = _torch()
    counts = [5000, 0, 1234]
    m, _ = make_model(SHAPES["m8r16c2"], 3, "fp32", 8192, seed=25)
    off = m.offsets_of(counts)
    xyz = m.sample_points(seed=0x1234567890ABCDEF, step=17, offsets=off).cpu().numpy()
    for b, n in enumerate(counts):
        got = xyz[off[b]:off[b + 1]]
        want = osp.sample_points(0x1234567890ABCDEF, 17, b, n)
        key = lambda a: np.lexsort((a[:, 2], a[:, 1], a[:, 0]))
        np.testing.assert_array_equal(got[key(got)], want[key(want)])
        if n:
            cell = np.minimum(((got.astype(np.float64) + 1) * 16).astype(int), 31)
            code = np.zeros(n, dtype=np.int64)
            for bit in range(5):
                for a in range(3):
                    code |= ((cell[:, a] >> bit) & 1) << (3 * bit + a)
            assert np.all(np.diff(code) >= 0)


def test_target_lookup_matches_oracle():
    torch = _torch()
    V = 33
    vol = np.random.default_rng(13).normal(size=(V, V, V)).astype(np.float32)
    boxes = synth.brick_boxes(V, (2, 2, 2), ghost=2)
    counts = [100, 3, 0, 57, 200, 1, 64, 65]
    m, _ = make_model(SHAPES["m8r16c2"], 8, "fp32", 1024, seed=26)
    r = np.random.default_rng(14)
    xs = [r.uniform(-1, 1, size=(c, 3)).astype(np.float32) for c in counts]
    xs[0][:4] = [[-1, -1, -1], [1, 1, 1], [1, -1, 0.5], [0, 0, 0]]
    off = m.offsets_of(counts)
    t = m.sample_target(torch.as_tensor(vol, device="cuda"), boxes,
                        torch.as_tensor(np.concatenate(xs), device="cuda"), off).cpu().numpy()
    for b in range(8):
        if counts[b]:
            want = ap.volume_sample(vol, xs[b].astype(np.float64), boxes[b])
            assert np.max(np.abs(t[off[b]:off[b + 1]] - want)) <= 1e-5 * np.max(np.abs(vol)), b


@pytest.mark.parametrize("ortho", [True, False])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_render_single_model_matches_oracle(ortho, precision):
    torch = _torch()
    shape = synth.ModelShape(8, 6, 2, 64)
    m, ref = make_model(shape, 1, precision, 4096, seed=27, shrink=0.2)
    lut = synth.random_lut(3, max_opacity=0.01)
    cam = synth.orbit_camera(0.7, 0.3, ortho=ortho)
    W, H, S = 20, 14, 24
    img = m.render(cam, torch.as_tensor(lut, device="cuda"), -0.5, 1.5, W, H, S, (1, 1, 1),
                   [[0, 0, 0, 63, 63, 63]], 64).cpu().numpy()
    want = orr.render(ref, [[0, 0, 0, 63, 63, 63]], (1, 1, 1), 64, cam, lut, -0.5, 1.5, W, H, S)
    assert np.any(want[..., 3] > 0.05) and np.any(want[..., 3] == 0.0)
    assert rel_l2(img, want) <= TOL[precision] * 5, rel_l2(img, want)


def test_render_bricks_matches_oracle():
    torch = _torch()
    shape = synth.ModelShape(8, 6, 2, 64)
    m, ref = make_model(shape, 8, "fp32", 2048, seed=28, shrink=0.2)
    V = 65
    boxes = synth.brick_boxes(V, (2, 2, 2), ghost=2)
    lut = synth.random_lut(4, max_opacity=0.01)
    cam = synth.orbit_camera(2.1, -0.4, ortho=False)
    W, H, S = 16, 16, 40
    img = m.render(cam, torch.as_tensor(lut, device="cuda"), -0.5, 1.5, W, H, S, (2, 2, 2), boxes, V).cpu().numpy()
    want = orr.render(ref, boxes, (2, 2, 2), V, cam, lut, -0.5, 1.5, W, H, S)
    assert rel_l2(img, want) <= 1e-4, rel_l2(img, want)


@pytest.mark.parametrize("precision,shape", [("fp32", "m8r16c2"), ("bf16", "m64r32c2")])
def test_autograd_function_equals_the_mse_backward(precision, shape):
    torch = _torch()
    from paper_2308_02494_gb300.model import APMGSRNFunction
    n = 900
    m, ref = make_model(SHAPES[shape], 1, precision, 2048, seed=29)
    x = torch.as_tensor(_points_for(ref, [n], 15)[0], device="cuda")
    v = torch.rand(n, device="cuda")
    params = m.params.clone().requires_grad_(True)
    f = APMGSRNFunction.apply(x, params, m, [0, n])
    loss = ((f - v) ** 2).mean()
    loss.backward()
    g_auto = params.grad.clone()
    m.backward(x, v, [0, n])
    g_mse = m.grads.clone()
    # BF16: the upstream dL/df comes from the forward kernel's f, whose last bits may
    # differ from the training pass's, and BF16 operand rounding can amplify that
    assert torch.linalg.norm(g_auto - g_mse) <= TOL[precision] * torch.linalg.norm(g_mse)
