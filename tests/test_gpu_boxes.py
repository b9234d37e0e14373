"""GPU parity of the BF16 path's shared-memory node boxes (encoder and scatter) at their
edges: grids zoomed in so far that some boxes exceed the shared-memory capacity and take
the direct path beside boxed grids of the same warp; dL/dy spanning seven orders of
magnitude inside every tile (the fixed-point sums resolve each (tile, grid) relative to
its largest |dL/dy|); and a one-cell cluster of equal-sign gradients that drives the
node sums to their bound."""
import numpy as np
import pytest

from oracle import apmgsrn as ap
from gpu_util import (RND, TOL, dG_error, density_grad_scale, ensure_built, make_model, morton_sorted,
                      points_off_faces, points_off_kinks, rel_l2)
from test_gpu_parity import SHAPES, _oracle_backward

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _torch():
    import torch
    return torch


def _dense_points(ref, n, seed, lo, hi):
    x = points_off_kinks(ref, points_off_faces(ref["G"], 3 * n + 64, seed, lo=lo, hi=hi), RND["bf16"])
    assert len(x) >= n
    return morton_sorted(x[:n])


def _scatter(ref, x, dy, absolute=False):
    """Adjoint of Eq. 2 for given dL/dy [N, M*C]: per node the sum of w * dL/dy (or of
    |w * dL/dy|), and the number of (point, grid) corner contributions it receives."""
    F = np.asarray(ref["F"])
    M, R, C = F.shape[0], F.shape[1], F.shape[4]
    u = ap.local_coords(ref["G"], x.astype(np.float64))
    out = np.zeros((M, R * R * R, C))
    cnt = np.zeros((M, R * R * R))
    for i in range(M):
        ins = ap.inside_mask(u[:, i, :])
        cc, w = ap.cell_and_weights(u[:, i, :], R)
        g = dy[:, i * C:(i + 1) * C]
        if absolute:
            g = np.abs(g)
        for dx, dyy, dz in ap.corner_offsets():
            wt = ap.corner_weight(w, dx, dyy, dz) * ins
            node = ((cc[:, 2] + dz) * R + (cc[:, 1] + dyy)) * R + (cc[:, 0] + dx)
            cnt[i] += np.bincount(node, weights=ins.astype(np.float64), minlength=R ** 3)
            for ch in range(C):
                out[i, :, ch] += np.bincount(node, weights=wt * g[:, ch], minlength=R ** 3)
    return out.reshape(F.shape), cnt.reshape(F.shape[:4])


def _upstream_case(ref, x, g, m):
    """The GPU's dF for the upstream gradient dL/df = g, and the oracle's dF from the same
    dL/dy rounded to bfloat16 as the kernels store it (so the comparison isolates the
    scatter's fixed-point sums), with the bound those sums promise per node."""
    torch = _torch()
    n = len(x)
    m.backward(torch.as_tensor(x, device="cuda"), torch.as_tensor(g.astype(np.float32), device="cuda"),
               [0, n], upstream=True)
    got = m.get("grads")[0]["F"]
    f = ap.query(ref, x.astype(np.float64), rnd=RND["bf16"])
    v = f - g.astype(np.float32).astype(np.float64) * n / 2.0   # 2 (f - v) / N = g
    o = ap.grad_rec(ref, x.astype(np.float64), v, rnd=RND["bf16"])
    dy = ap.bf16(o["dy"])
    want, cnt = _scatter(ref, x, dy)
    scale, _ = _scatter(ref, x, dy, absolute=True)
    # per node: each contribution rounds to within half a quantum of its (tile, grid),
    # and the quantum is at most 2^-19 of the tile's largest |dL/dy| (<= the batch's);
    # plus one bfloat16 step of a dL/dy whose float32 and float64 values round apart
    # (2^-8 of that contribution) and float32 rounding of the products and the sum
    bound = cnt[..., None] * 2.0 ** -20 * np.max(np.abs(dy)) + 2.0 ** -7 * scale + 1e-30
    return got, want, bound


def test_zoomed_grids_mix_boxed_and_direct_grids():
    torch = _torch()
    n = 1500
    m, ref = make_model(SHAPES["m64r32c2"], 1, "bf16", 4096, seed=41, shrink=2.0)   # zoom up to 3x
    x = _dense_points(ref[0], n, 42, -0.2, 0.1)
    v = np.random.default_rng(43).uniform(-0.5, 1.5, n).astype(np.float32)
    losses = m.backward(torch.as_tensor(x, device="cuda"), torch.as_tensor(v, device="cuda"),
                        [0, n], density=True).cpu().numpy()
    f = m.forward(torch.as_tensor(x, device="cuda"), [0, n]).cpu().numpy()
    gr = m.get("grads")[0]
    o = _oracle_backward(ref[0], x, v, True, RND["bf16"])
    tol = TOL["bf16"]
    assert rel_l2(f, ap.query(ref[0], x.astype(np.float64), rnd=RND["bf16"])) <= tol
    assert abs(losses[0, 0] - o["L_rec"]) <= tol * abs(o["L_rec"])
    assert abs(losses[0, 1] - o["L_den"]) <= tol * abs(o["L_den"]) + 1e-12
    for k, ok in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
        assert rel_l2(gr[k], o[ok]) <= tol, (k, rel_l2(gr[k], o[ok]))
    scale = density_grad_scale(ref[0]["G"], x, o["h"])
    assert dG_error(gr["G"], o["dG"], scale) <= tol


def test_scatter_resolves_gradients_of_seven_orders_of_magnitude():
    n = 2000
    m, ref = make_model(SHAPES["m64r32c2"], 1, "bf16", 4096, seed=44)
    x = _dense_points(ref[0], n, 45, -0.2, 0.1)
    r = np.random.default_rng(46)
    g = np.sign(r.uniform(-1, 1, n)) * 10.0 ** r.uniform(-5, 2, n)
    got, want, bound = _upstream_case(ref[0], x, g, m)
    assert rel_l2(got, want) <= 1e-3, rel_l2(got, want)
    err = np.abs(got - want)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_one_cell_cluster_of_equal_sign_gradients_does_not_overflow():
    n = 1024   # one scatter tile: every point in the same cell of most grids
    m, ref = make_model(SHAPES["m64r32c2"], 1, "bf16", 4096, seed=47, shrink=0.0)
    x = _dense_points(ref[0], n, 48, 0.301, 0.311)
    g = np.full(n, 100.0)
    got, want, bound = _upstream_case(ref[0], x, g, m)
    assert rel_l2(got, want) <= 1e-3, rel_l2(got, want)
    assert np.all(np.abs(got - want) <= bound)
