"""GPU parity of SRN_REC_DG: the gradient of L_rec (or of an upstream loss) into the
transforms G through Eq. 1-2, against the oracle, in both precisions, alone, added to
the density gradient, over uneven bricks, and through the autograd function."""
import numpy as np
import pytest

from oracle import apmgsrn as ap
from gpu_util import (RND, TOL, density_grad_scale, ensure_built, make_model, morton_sorted,
                      points_off_faces, points_off_kinks)
from test_gpu_parity import SHAPES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _points(params, n, seed, rnd, dense=False, margin=2e-4):
    """Seeded points off every grid face, off every ReLU kink and `margin` (in cells)
    away from every cell face of every grid: the interpolant's derivative jumps across
    a cell face, so the cell must be the same in float32 and float64."""
    lo, hi = (-0.25, 0.15) if dense else (-1.0, 1.0)
    x = points_off_kinks(params, points_off_faces(params["G"], 3 * n + 64, seed, lo=lo, hi=hi), rnd)
    R = params["F"].shape[1]
    u = ap.local_coords(params["G"], x.astype(np.float64))
    s = (np.clip(u, -1, 1) + 1) / 2 * (R - 1)
    off_face = np.all(np.abs(s - np.round(s)) > margin, axis=2) | ~ap.inside_mask(u)   # [N, M]
    x = x[np.all(off_face, axis=1)]
    assert len(x) >= n
    x = x[:n]
    return morton_sorted(x) if dense else x


def _want(params, x, v, precision):
    """Oracle dG through the features, and its summation scale: the same sum with
    every term replaced by its absolute value (float summation errs relative to it).
    On the BF16 path the oracle's dL/dy is rounded to bfloat16, as the kernels store it."""
    g = ap.grad_rec(params, x.astype(np.float64), v.astype(np.float64), rnd=RND[precision])
    dy = g["dy"]
    want = ap.grad_transform_through_features(params, x, dy)
    xt = np.concatenate([np.abs(x.astype(np.float64)), np.ones((len(x), 1))], axis=1)
    u = ap.local_coords(params["G"], x.astype(np.float64))
    C = params["F"].shape[4]
    scale = np.zeros_like(want)
    for i in range(want.shape[0]):
        J = np.abs(ap.interp_grid_du(params["F"][i], u[:, i, :]))          # [N, C, 3]
        t = np.einsum("nc,ncd->nd", np.abs(dy[:, i * C:(i + 1) * C]), J)
        scale[i] = t.T @ xt
    return want, scale, g


def _err(got, want, scale):
    return float(np.max(np.abs(np.asarray(got) - want) / (scale + 1e-30)))


@pytest.mark.parametrize("precision,shape", [("fp32", "m8r16c2"), ("fp32", "m16r9c1"), ("bf16", "m8r16c2"),
                                             ("bf16", "m16r9c1"), ("bf16", "m64r32c2")])
@pytest.mark.parametrize("dense", [False, True])
def test_rec_dg_matches_oracle(precision, shape, dense):
    import torch
    n = 1300
    m, ref = make_model(SHAPES[shape], 1, precision, 4096, seed=51)
    x = _points(ref[0], n, 52, RND[precision], dense)
    v = np.random.default_rng(53).uniform(-0.5, 1.5, n).astype(np.float32)
    xt, vt = torch.as_tensor(x, device="cuda"), torch.as_tensor(v, device="cuda")
    m.backward(xt, vt, [0, n], rec_dg=True)
    got = m.get("grads")[0]["G"]
    want, scale, _ = _want(ref[0], x, v, precision)
    assert np.abs(want).max() > 0
    assert _err(got, want, scale) <= TOL[precision], _err(got, want, scale)
    # the flag touches G's gradient only
    g_rec = m.grads.clone()
    m.backward(xt, vt, [0, n])
    L = m.lay
    # (float atomics make the sums' order, not their terms, differ between runs)
    assert torch.linalg.norm(g_rec[:L.off_G] - m.grads[:L.off_G]) <= 1e-6 * torch.linalg.norm(m.grads[:L.off_G])
    assert torch.all(m.grads[L.off_G:] == 0)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rec_dg_adds_to_the_density_gradient_over_uneven_bricks(precision):
    import torch
    counts = [700, 45, 1200]
    m, ref = make_model(SHAPES["m8r16c2"], len(counts), precision, 4096, seed=55)
    xs = [_points(ref[b], c, 56 + b, RND[precision]) for b, c in enumerate(counts)]
    r = np.random.default_rng(57)
    vs = [r.uniform(0, 1, c).astype(np.float32) for c in counts]
    off = m.offsets_of(counts)
    m.backward(torch.as_tensor(np.concatenate(xs), device="cuda"),
               torch.as_tensor(np.concatenate(vs), device="cuda"), off, density=True, rec_dg=True)
    grads = m.get("grads")
    for b in range(len(counts)):
        want, scale, g = _want(ref[b], xs[b], vs[b], precision)
        d = ap.grad_density(ref[b]["G"], xs[b].astype(np.float64), g["h"])
        dscale = density_grad_scale(ref[b]["G"], xs[b], g["h"])
        e = _err(grads[b]["G"], want + d["dG"], scale + dscale)
        assert e <= TOL[precision], (b, e)


@pytest.mark.parametrize("precision,shape", [("fp32", "m8r16c2"), ("bf16", "m64r32c2")])
def test_autograd_with_transforms_equals_the_mse_backward_with_rec_dg(precision, shape):
    import torch
    from paper_2308_02494_gb300.model import APMGSRNFunction
    n = 900
    m, ref = make_model(SHAPES[shape], 1, precision, 2048, seed=59)
    x = torch.as_tensor(_points(ref[0], n, 60, RND[precision]), device="cuda")
    v = torch.rand(n, device="cuda")
    params = m.params.clone().requires_grad_(True)
    f = APMGSRNFunction.apply(x, params, m, [0, n], True)
    ((f - v) ** 2).mean().backward()
    g_auto = params.grad.clone()
    m.backward(x, v, [0, n], rec_dg=True)
    g_mse = m.grads.clone()
    L = m.lay
    gA, gM = g_auto[L.off_G:L.off_G + L.size_G], g_mse[L.off_G:L.off_G + L.size_G]
    assert torch.linalg.norm(gM) > 0
    assert torch.linalg.norm(gA - gM) <= 5 * TOL[precision] * torch.linalg.norm(gM)


@pytest.mark.parametrize("precision,shape", [("fp32", "m8r16c2"), ("bf16", "m64r32c2")])
def test_autograd_function_differentiates_at_its_params_input(precision, shape):
    # The model is created with one parameter set; the function is given another (only
    # as its input).  f and every gradient must be the oracle's at the input's values.
    import torch
    from paper_2308_02494_gb300 import synth
    from gpu_util import as_stored, rel_l2
    from paper_2308_02494_gb300.model import APMGSRNFunction
    n = 900
    m, ref_a = make_model(SHAPES[shape], 1, precision, 2048, seed=61)
    other = synth.parity_model(SHAPES[shape], 62, shrink=0.4)
    other["vmin"], other["vmax"] = ref_a[0]["vmin"], ref_a[0]["vmax"]   # the range is not a parameter
    ref_b = as_stored(other, precision)
    x = _points(ref_b, n, 63, RND[precision])
    v = np.random.default_rng(64).uniform(-0.5, 1.5, n).astype(np.float32)
    xt, vt = torch.as_tensor(x, device="cuda"), torch.as_tensor(v, device="cuda")
    params = m.pack(other).requires_grad_(True)
    assert not torch.equal(params.detach(), m.params)
    f = APMGSRNFunction.apply(xt, params, m, [0, n], True)
    ((f - vt) ** 2).mean().backward()
    want, scale, g = _want(ref_b, x, v, precision)
    assert rel_l2(f.detach().cpu().numpy(), g["f"]) <= TOL[precision]
    got = m._views(params.grad, 0)
    for k, w in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
        e = rel_l2(got[k].cpu().numpy(), g[w])
        assert e <= TOL[precision], (k, e)
    assert _err(got["G"].cpu().numpy(), want, scale) <= TOL[precision]
    # the model now holds the input's values (and its BF16 shadow follows them)
    assert torch.equal(m.params, params.detach())
    with pytest.raises(ValueError):
        APMGSRNFunction.apply(xt, params.detach()[:-1], m, [0, n])
